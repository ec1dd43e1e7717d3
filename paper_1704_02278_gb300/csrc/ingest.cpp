// ingest.cpp -- glop_ingest_*: a byte stream scanned chunk by chunk as it
// arrives, the uploads, scans and copy-backs of consecutive chunks overlapped
// (the paper streams the next batch to the GPU while the current one is
// scanned, Sec. 6; chunked scanning carries the longest pattern - 1 bytes of
// overlap, Sec. 4).
//
// Built on the public entry points alone (glop_scan, glop_scan_words).
// depth + 1 slots rotate, each with its own CUDA stream, device text, output,
// count and workspace, and pinned result rows and words.  feed(k):
//  * the carried tail of chunk k-1 is copied device to device into slot k's
//    buffer (after the previous slot's upload), chunk k is uploaded behind it
//    and scanned, and the scan's count and status go to the slot's pinned
//    words (a kernel's stores, not a memcpy queued behind copy-backs);
//  * the copy-back of chunk k-1's matches is queued once its count is known;
//  * the owned matches of chunk k-depth are handed out.
// A scan owns the match starts in [buffer start, buffer end - halo) (every
// remaining one for the last scan); the next buffer starts at the first
// unowned byte.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <deque>
#include <new>
#include <vector>

#include "glop.h"

namespace {

struct Slot {
    cudaStream_t stream = nullptr;
    uint8_t *d_text = nullptr;  // carried tail + chunk
    glop_match *d_out = nullptr;
    uint64_t rows = 0;
    uint64_t *d_count = nullptr;
    void *d_ws = nullptr;
    uint64_t ws_bytes = 0;
    uint64_t *h_words = nullptr;  // pinned: match count, status (glop_scan_words)
    glop_match *h_out = nullptr;  // pinned result rows
    uint64_t h_rows = 0;
    cudaEvent_t uploaded = nullptr, done = nullptr, copied = nullptr;
    uint64_t last_len = 0;  // bytes in d_text for the slot's latest chunk
};

// a queued scan whose results are not handed out yet: stream bytes [b0, b1) in slot `slot`
struct Pending {
    uint32_t slot;
    uint64_t b0, b1;
    int64_t n;  // match count once the copy-back is queued, -1 before
};

// end (exclusive) of the match starts a scan of stream bytes [b0, b1) owns
uint64_t owned_end(uint64_t b0, uint64_t b1, uint64_t halo, bool final) {
    if (final) return b1;
    return b1 > b0 + halo ? b1 - halo : b0;
}

}  // namespace

struct glop_ingest_s {
    glop_handle h = nullptr;
    int device = 0;
    uint64_t chunk_bytes = 0, halo = 0, cap = 0;
    uint32_t depth = 0;
    std::vector<Slot> slots;
    std::deque<Pending> pending;
    uint64_t buf_start = 0;  // stream offset of the next scan's buffer
    uint64_t k = 0;          // chunks fed in this stream
    uint64_t tail_len = 0;   // carried bytes at the end of slot tail_slot's buffer
    uint32_t tail_slot = 0;
    uint64_t chunks = 0, rescans = 0;  // totals over the object's life
};

namespace {

void free_slots(glop_ingest s) {
    for (Slot &x : s->slots) {
        if (x.stream) cudaStreamSynchronize(x.stream);
        cudaFree(x.d_text);
        cudaFree(x.d_out);
        cudaFree(x.d_count);
        cudaFree(x.d_ws);
        cudaFreeHost(x.h_words);
        cudaFreeHost(x.h_out);
        if (x.uploaded) cudaEventDestroy(x.uploaded);
        if (x.done) cudaEventDestroy(x.done);
        if (x.copied) cudaEventDestroy(x.copied);
        if (x.stream) cudaStreamDestroy(x.stream);
    }
    s->slots.clear();
}

// queue the scan of the slot's first len bytes, then its count and status into the pinned words
glop_status scan_slot(glop_ingest s, Slot &x, uint64_t len) {
    glop_status st = glop_scan(s->h, len ? x.d_text : nullptr, len, x.d_out, x.rows, x.d_count, x.d_ws, x.ws_bytes,
                               x.stream);
    if (st != GLOP_OK) return st;
    st = glop_scan_words(x.d_ws, x.h_words, x.stream);
    if (st != GLOP_OK) return st;
    return cudaEventRecord(x.done, x.stream) == cudaSuccess ? GLOP_OK : GLOP_ECUDA;
}

// wait for p's scan, then queue the copy-back of exactly its matches
glop_status start_copy(glop_ingest s, Pending &p) {
    Slot &x = s->slots[p.slot];
    if (cudaEventSynchronize(x.done) != cudaSuccess) return GLOP_ECUDA;
    uint64_t n = x.h_words[0];
    const uint64_t status = x.h_words[1];
    if (status != GLOP_OK && status != GLOP_EOVERFLOW) return (glop_status)status;
    if (n > x.rows) {
        // more matches than the output holds: scan the same buffer again into a larger one
        ++s->rescans;
        cudaFree(x.d_out);
        x.d_out = nullptr;
        x.rows = 0;
        if (cudaMalloc(&x.d_out, n * sizeof(glop_match)) != cudaSuccess) return GLOP_ENOMEM;
        x.rows = n;
        const glop_status st = scan_slot(s, x, p.b1 - p.b0);
        if (st != GLOP_OK) return st;
        if (cudaEventSynchronize(x.done) != cudaSuccess) return GLOP_ECUDA;
        if (x.h_words[1] != GLOP_OK) return x.h_words[1] == GLOP_EOVERFLOW ? GLOP_EINTERNAL : (glop_status)x.h_words[1];
        n = x.h_words[0];
    }
    if (x.h_rows < n) {
        // (the rows handed out from this slot's previous chunk are no longer valid once this copy is queued)
        cudaFreeHost(x.h_out);
        x.h_out = nullptr;
        x.h_rows = 0;
        if (cudaMallocHost(&x.h_out, n * sizeof(glop_match)) != cudaSuccess) return GLOP_ENOMEM;
        x.h_rows = n;
    }
    if (n && cudaMemcpyAsync(x.h_out, x.d_out, n * sizeof(glop_match), cudaMemcpyDeviceToHost, x.stream) != cudaSuccess)
        return GLOP_ECUDA;
    if (cudaEventRecord(x.copied, x.stream) != cudaSuccess) return GLOP_ECUDA;
    p.n = (int64_t)n;
    return GLOP_OK;
}

// wait for p's copy-back and describe its owned matches (a prefix of its sorted matches)
glop_status finish(glop_ingest s, Pending &p, bool final, glop_ingest_result *res) {
    if (p.n < 0) {
        const glop_status st = start_copy(s, p);
        if (st != GLOP_OK) return st;
    }
    Slot &x = s->slots[p.slot];
    if (cudaEventSynchronize(x.copied) != cudaSuccess) return GLOP_ECUDA;
    const uint64_t end = owned_end(p.b0, p.b1, s->halo, final) - p.b0;
    const glop_match *m = x.h_out;
    const uint64_t n = (uint64_t)p.n;
    const glop_match *e =
        n ? std::lower_bound(m, m + n, end, [](const glop_match &a, uint64_t v) { return a.offset < v; }) : m;
    res->base = p.b0;
    res->matches = n ? m : nullptr;
    res->count = (uint64_t)(e - m);
    return GLOP_OK;
}

}  // namespace

extern "C" {

glop_status glop_ingest_create(glop_handle h, uint64_t chunk_bytes, uint64_t out_rows, uint32_t depth,
                               glop_ingest *out) {
    if (!out) return GLOP_EINVAL;
    *out = nullptr;
    if (!h || chunk_bytes == 0 || depth == 0 || depth > GLOP_INGEST_MAX_DEPTH) return GLOP_EINVAL;
    const uint32_t maxlen = glop_max_pattern_len(h);
    const uint64_t halo = maxlen ? maxlen - 1 : 0;
    if (chunk_bytes + halo > 0xFFFFFFFFull) return GLOP_EINVAL;
    glop_ingest s = new (std::nothrow) glop_ingest_s;
    if (!s) return GLOP_ENOMEM;
    s->h = h;
    s->halo = halo;
    s->chunk_bytes = chunk_bytes;
    s->cap = chunk_bytes + halo;
    s->depth = depth;
    const uint64_t rows = out_rows ? out_rows : std::max<uint64_t>(1u << 16, s->cap / 4);
    uint64_t ws = 0;
    glop_status st = cudaGetDevice(&s->device) == cudaSuccess ? glop_scan_workspace_size(h, s->cap, &ws) : GLOP_ECUDA;
    if (st == GLOP_OK) {
        s->slots.resize(depth + 1);
        for (Slot &x : s->slots) {
            x.rows = x.h_rows = rows;
            x.ws_bytes = ws;
            if (cudaStreamCreateWithFlags(&x.stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&x.uploaded, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&x.done, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&x.copied, cudaEventDisableTiming) != cudaSuccess) {
                st = GLOP_ECUDA;
                break;
            }
            if (cudaMalloc(&x.d_text, s->cap) != cudaSuccess ||
                cudaMalloc(&x.d_out, rows * sizeof(glop_match)) != cudaSuccess ||
                cudaMalloc(&x.d_count, sizeof(uint64_t)) != cudaSuccess || cudaMalloc(&x.d_ws, ws) != cudaSuccess ||
                cudaMallocHost(&x.h_words, 2 * sizeof(uint64_t)) != cudaSuccess ||
                cudaMallocHost(&x.h_out, rows * sizeof(glop_match)) != cudaSuccess) {
                st = GLOP_ENOMEM;
                break;
            }
        }
    }
    if (st != GLOP_OK) {
        (void)cudaGetLastError();
        free_slots(s);
        delete s;
        return st;
    }
    *out = s;
    return GLOP_OK;
}

glop_status glop_ingest_feed(glop_ingest s, const uint8_t *h_chunk, uint64_t n, glop_ingest_result *res) {
    if (!s || !res || (n && !h_chunk) || n > s->chunk_bytes) return GLOP_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != s->device) return GLOP_EINVAL;
    const uint32_t ns = (uint32_t)s->slots.size();
    const uint32_t si = (uint32_t)(s->k % ns);
    Slot &x = s->slots[si];
    const uint64_t h = s->tail_len;
    // every earlier upload, and the tail copy that read this slot's old bytes, come first (each upload waits
    // for the one before it)
    if (s->k && cudaStreamWaitEvent(x.stream, s->slots[(s->k - 1) % ns].uploaded, 0) != cudaSuccess)
        return GLOP_ECUDA;
    if (h) {
        const Slot &t = s->slots[s->tail_slot];
        if (cudaMemcpyAsync(x.d_text, t.d_text + (t.last_len - h), h, cudaMemcpyDeviceToDevice, x.stream) !=
            cudaSuccess)
            return GLOP_ECUDA;
    }
    if (n && cudaMemcpyAsync(x.d_text + h, h_chunk, n, cudaMemcpyHostToDevice, x.stream) != cudaSuccess)
        return GLOP_ECUDA;
    if (cudaEventRecord(x.uploaded, x.stream) != cudaSuccess) return GLOP_ECUDA;
    x.last_len = h + n;
    const uint64_t b0 = s->buf_start, b1 = b0 + h + n;
    glop_status st = scan_slot(s, x, h + n);
    if (st != GLOP_OK) return st;
    s->pending.push_back(Pending{si, b0, b1, -1});
    // while this chunk uploads and scans: the previous chunk's copy-back, then the results of the chunk fed
    // depth calls ago
    if (s->pending.size() >= 2 && s->pending[s->pending.size() - 2].n < 0) {
        st = start_copy(s, s->pending[s->pending.size() - 2]);
        if (st != GLOP_OK) return st;
    }
    *res = glop_ingest_result{0, nullptr, 0};
    if (s->pending.size() > s->depth) {
        Pending p = s->pending.front();
        s->pending.pop_front();
        st = finish(s, p, false, res);
        if (st != GLOP_OK) return st;
    }
    const uint64_t nxt = owned_end(b0, b1, s->halo, false);
    s->tail_len = b1 - nxt;
    s->tail_slot = si;
    s->buf_start = nxt;
    ++s->k;
    ++s->chunks;
    return GLOP_OK;
}

glop_status glop_ingest_flush(glop_ingest s, glop_ingest_result *res, uint32_t max_res, uint32_t *n_res) {
    if (!s || !n_res || (max_res && !res)) return GLOP_EINVAL;
    *n_res = (uint32_t)s->pending.size();
    if (max_res < s->pending.size()) return GLOP_EINVAL;
    for (Pending &p : s->pending)
        if (p.n < 0) {
            const glop_status st = start_copy(s, p);
            if (st != GLOP_OK) return st;
        }
    for (uint32_t i = 0; !s->pending.empty(); ++i) {
        Pending p = s->pending.front();
        s->pending.pop_front();
        const glop_status st = finish(s, p, s->pending.empty(), res + i);
        if (st != GLOP_OK) return st;
    }
    return GLOP_OK;
}

glop_status glop_ingest_reset(glop_ingest s) {
    if (!s || !s->pending.empty()) return GLOP_EINVAL;
    s->buf_start = s->k = s->tail_len = 0;
    s->tail_slot = 0;
    return GLOP_OK;
}

glop_status glop_ingest_info(glop_ingest s, uint64_t *chunks, uint64_t *rescans) {
    if (!s) return GLOP_EINVAL;
    if (chunks) *chunks = s->chunks;
    if (rescans) *rescans = s->rescans;
    return GLOP_OK;
}

glop_status glop_ingest_destroy(glop_ingest s) {
    if (!s) return GLOP_EINVAL;
    free_slots(s);
    delete s;
    return GLOP_OK;
}

}  // extern "C"
