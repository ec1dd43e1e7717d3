// split.cu -- glop_batch_split: a batch scan's (segment, offset, pattern_id)
// matches rewritten as (offset, pattern_id) pairs plus the index of each
// segment's first match.
//
// A server that batches many requests into one glop_scan_batch launch (one
// segment per request) hands every request its own matches.  The batch output
// is sorted by segment, so each request's matches are one run of it; copying
// back 8-byte pairs and n_segments + 1 run starts instead of the 12-byte
// triples moves a third fewer bytes over the host link, which is what a
// serving loop spends its time on.
#include <cuda_runtime.h>

#include <cstdint>

#include "glop.h"

namespace {

constexpr uint32_t kThreads = 256;
constexpr uint32_t kBlocks = 152 * 8;

// Thread i (grid-stride) writes pair i and, where the segment changes between
// match i - 1 and match i, the first-match index of every segment in between;
// the thread of the last match fills the segments after it.  n = 0 fills
// every entry with 0.  Segment values at or past n_segments (not produced by
// a valid batch scan) are clamped, so no write leaves seg_first[0..n_segments].
__global__ void __launch_bounds__(kThreads) split_kernel(const glop_batch_match *in, const uint64_t *d_count,
                                                         uint64_t capacity, uint32_t n_segments,
                                                         glop_match *pairs, uint64_t *seg_first) {
    const uint64_t total = *d_count;
    const uint64_t n = total < capacity ? total : capacity;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n == 0) {
        for (uint64_t s = t0; s <= n_segments; s += stride) seg_first[s] = 0;
        return;
    }
    for (uint64_t i = t0; i < n; i += stride) {
        const glop_batch_match m = in[i];
        pairs[i] = glop_match{m.offset, m.pattern_id};
        const uint32_t s = m.segment < n_segments ? m.segment : n_segments;
        const uint32_t prev = i ? (in[i - 1].segment < n_segments ? in[i - 1].segment : n_segments) : 0u;
        // segments (prev, s] start at i (with segment 0 as well when i == 0)
        for (uint32_t q = i ? prev + 1 : 0u; q <= s; ++q) seg_first[q] = i;
        if (i == n - 1)
            for (uint32_t q = s + 1; q <= n_segments; ++q) seg_first[q] = n;
    }
}

}  // namespace

extern "C" glop_status glop_batch_split(const glop_batch_match *d_matches, const uint64_t *d_count,
                                        uint64_t capacity, uint32_t n_segments, glop_match *d_pairs,
                                        uint64_t *d_seg_first, glop_stream_t stream) {
    if (!d_count || !d_seg_first || (capacity && (!d_matches || !d_pairs)) || n_segments == UINT32_MAX)
        return GLOP_EINVAL;
    const uint64_t want = capacity / kThreads + 1;
    const uint32_t blocks = (uint32_t)(want < kBlocks ? want : kBlocks);
    split_kernel<<<blocks, kThreads, 0, (cudaStream_t)stream>>>(d_matches, d_count, capacity, n_segments, d_pairs,
                                                               d_seg_first);
    return cudaGetLastError() == cudaSuccess ? GLOP_OK : GLOP_ECUDA;
}
