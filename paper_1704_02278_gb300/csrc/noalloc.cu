// noalloc.cu -- glop_scan_noalloc: the single-buffer scan with its scratch
// memory in a fixed device array instead of a caller-provided workspace.
//
// Some callers cannot allocate device memory when they scan: a host program
// whose device memory is owned by another allocator (a framework's memory
// pool sized at start-up), a latency-critical loop that must not pay for
// cudaMalloc's implicit synchronisation, or a plug-in that is forbidden to
// grow its memory footprint after initialisation.  For them this entry point
// uses a file-scope device array that the CUDA runtime reserves when the
// library's module is loaded on a device; the array stays reserved on every
// device that loaded the library until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "glop.h"
#include "scan.h"

namespace {

// Scratch of one scan of up to kNoAllocMaxLen bytes (sub-tile descriptors,
// block sums and match records); 25 MiB.
constexpr uint64_t kNoAllocMaxLen = 16ull << 20;
constexpr uint64_t kNoAllocScratchBytes = 25ull << 20;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// The device address of the array on the current device, looked up once per
// device (the host-side symbol is only a stand-in and must never be passed to
// a kernel).  nullptr when the lookup fails.
void *scratch_of_current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_scratch_ptr[dev] = p;
    }
    return g_scratch_ptr[dev];
}

}  // namespace

extern "C" glop_status glop_scan_noalloc(glop_handle h, const uint8_t *d_text, uint64_t len, glop_match *d_matches,
                                         uint64_t capacity, uint64_t *d_count, glop_stream_t stream) {
    if (len > kNoAllocMaxLen) return GLOP_EINVAL;
    if (glop::workspace_bytes(len, false) > kNoAllocScratchBytes) return GLOP_EINVAL;
    void *ws = scratch_of_current_device();
    if (!ws) return GLOP_ECUDA;
    // The header of the scratch is cleared by the scan itself on the stream
    // before any kernel reads it; everything else is written before it is read.
    return glop_scan(h, d_text, len, d_matches, capacity, d_count, ws, kNoAllocScratchBytes, stream);
}
