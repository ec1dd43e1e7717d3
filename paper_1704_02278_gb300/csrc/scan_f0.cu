// scan_f0.cu -- instantiations of the scan kernel for automata without a start filter (some pattern shorter than 4 bytes).
#include "scan_kernel.cuh"

namespace glop {
namespace kern {

int launch_f0(KParams &kp, uint32_t smem, uint32_t grid, cudaStream_t st, bool batch, bool r16, bool deep, uint32_t ksub,
              bool multi) {
    if (multi)  // several automata: batches, 31 KiB chunks
        return deep ? (r16 ? launch_t<0, true, true, true, 1, true>(kp, smem, grid, st) : launch_t<0, true, false, true, 1, true>(kp, smem, grid, st))
                    : (r16 ? launch_t<0, true, true, false, 1, true>(kp, smem, grid, st) : launch_t<0, true, false, false, 1, true>(kp, smem, grid, st));
    if (deep)
        return batch ? (r16 ? launch_t<0, true, true, true, 1>(kp, smem, grid, st) : launch_t<0, true, false, true, 1>(kp, smem, grid, st))
                     : (r16 ? launch_t<0, false, true, true, 1>(kp, smem, grid, st) : launch_t<0, false, false, true, 1>(kp, smem, grid, st));
    if (ksub == 2)
        return batch ? (r16 ? launch_t<0, true, true, false, 2>(kp, smem, grid, st) : launch_t<0, true, false, false, 2>(kp, smem, grid, st))
                     : (r16 ? launch_t<0, false, true, false, 2>(kp, smem, grid, st) : launch_t<0, false, false, false, 2>(kp, smem, grid, st));
    return batch ? (r16 ? launch_t<0, true, true, false, 1>(kp, smem, grid, st) : launch_t<0, true, false, false, 1>(kp, smem, grid, st))
                 : (r16 ? launch_t<0, false, true, false, 1>(kp, smem, grid, st) : launch_t<0, false, false, false, 1>(kp, smem, grid, st));
}

}  // namespace kern
}  // namespace glop
