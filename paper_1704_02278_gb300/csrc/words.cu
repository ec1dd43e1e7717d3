// words.cu -- glop_scan_words: a scan's match count and status written into
// pinned host memory by a one-thread kernel.
//
// A host that overlaps scans with copies (one piece's matches copied back while
// the next piece is scanned) needs each scan's count before it can size that
// piece's copy.  A device-to-host memcpy of those few bytes queues on the copy
// engine behind the large copy already in flight, and every later launch on its
// stream waits for it.  A kernel's stores reach host memory without the copy
// engine.
#include <cuda_runtime.h>

#include <cstdint>

#include "glop.h"
#include "scan.h"

namespace {

// h_words[0] = the match count the scan recorded in its workspace header,
// h_words[1] = its status, with the precedence of glop_scan_status.
__global__ void words_kernel(const uint32_t *hdr, unsigned long long *h_words) {
    const uint32_t f = hdr[0];
    const unsigned long long total = (unsigned long long)hdr[4] | ((unsigned long long)hdr[5] << 32);
    uint32_t st = GLOP_OK;
    if (f & glop::WS_TIMEOUT) st = GLOP_ETIMEOUT;  // (as glop_scan_status: a timeout explains later checks)
    else if (f & glop::WS_INTERNAL) st = GLOP_EINTERNAL;
    else if (f & glop::WS_EINVAL) st = GLOP_EINVAL;
    else if (f & glop::WS_OVERFLOW) st = GLOP_EOVERFLOW;
    h_words[0] = total;
    h_words[1] = st;
    __threadfence_system();
}

}  // namespace

namespace glop {

int launch_words(const void *d_workspace, unsigned long long *h_words_dev, cudaStream_t stream) {
    words_kernel<<<1, 1, 0, stream>>>(static_cast<const uint32_t *>(d_workspace), h_words_dev);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

}  // namespace glop

extern "C" glop_status glop_scan_words(const void *d_workspace, uint64_t *h_words, glop_stream_t stream) {
    if (!d_workspace || !h_words) return GLOP_EINVAL;
    void *dev = nullptr;
    if (cudaHostGetDevicePointer(&dev, h_words, 0) != cudaSuccess) {
        (void)cudaGetLastError();
        return GLOP_EINVAL;  // not addressable by the device (or no device)
    }
    return glop::launch_words(d_workspace, static_cast<unsigned long long *>(dev), reinterpret_cast<cudaStream_t>(stream))
               ? GLOP_ECUDA
               : GLOP_OK;
}
