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
struct Cached {
    unsigned long long ctx_id = 0;  // the CUDA context the address belongs to (0 = none yet)
    void *ptr = nullptr;
};
Cached g_scratch[kMaxDevices];

// The process-unique id of the calling thread's current CUDA context, or 0
// when there is none (or the driver cannot tell).  Read through the driver's
// cuCtxGetId, reached by the runtime's entry-point query so that the library
// does not link the driver library itself.
unsigned long long current_context_id() {
    using CtxGetId = int (*)(void *, unsigned long long *);
    static const CtxGetId fn = []() -> CtxGetId {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<CtxGetId>(f);
    }();
    unsigned long long id = 0;
    if (!fn || fn(nullptr, &id) != 0) return 0;
    return id;
}

}  // namespace

namespace glop {

// The device address of the array in the current device's context, with that
// device current.  The host-side symbol is only a stand-in and must never be
// passed to a kernel.  The address is looked up once per device and context:
// the first call on a device loads the module and reserves the array; after
// a cudaDeviceReset the next call finds a new context and looks it up again.
// nullptr when the lookup fails.
void *noalloc_scratch_of_current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    Cached &c = g_scratch[dev];
    const unsigned long long id = current_context_id();
    if (!c.ptr || !id || id != c.ctx_id) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        c.ptr = p;
        c.ctx_id = current_context_id();  // the lookup made the device's context current if it was not
    }
    return c.ptr;
}

}  // namespace glop


extern "C" glop_status glop_scan_noalloc(glop_handle h, const uint8_t *d_text, uint64_t len, glop_match *d_matches,
                                         uint64_t capacity, uint64_t *d_count, glop_stream_t stream) {
    if (len > kNoAllocMaxLen) return GLOP_EINVAL;
    if (glop::workspace_bytes(len, false) > kNoAllocScratchBytes) return GLOP_EINVAL;
    void *ws = glop::noalloc_scratch_of_current_device();
    if (!ws) return GLOP_ECUDA;
    // The header of the scratch (status flags, ticket, total, barrier counters)
    // is cleared by the scan itself on the stream before any kernel reads it;
    // everything else is written before it is read.  The header then holds this
    // call's outcome until the next call: glop_scan_status(NULL, ...) reads it.
    return glop_scan(h, d_text, len, d_matches, capacity, d_count, ws, kNoAllocScratchBytes, stream);
}
