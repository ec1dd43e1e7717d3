// api.cpp -- the C ABI of include/glop.h.
#include <cuda_runtime.h>

#include <chrono>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "compile.h"
#include "glop.h"
#include "scan.h"

struct glop_automaton {
    GlopDevAutomaton dev;  // descriptor with device pointers
    void *blob = nullptr;  // one device allocation holding every table
    uint64_t blob_bytes = 0;
    int device = 0;
    glop_info info{};
    uint32_t smem_budget = 0;
    uint32_t ksub = 1;  // sub-tiles per consumer warp and staged chunk (chunks of 31 or 62 KiB)
    uint32_t ksub_used = 1;  // what the last scan launch used (62 KiB chunks fall back to 31 when they do not fit)
};

namespace {

uint64_t al(uint64_t x) { return (x + 255) / 256 * 256; }

template <class T>
uint64_t bytes_of(const std::vector<T> &v) {
    return (uint64_t)v.size() * sizeof(T);
}

glop_status cuda_ok(cudaError_t e) { return e == cudaSuccess ? GLOP_OK : GLOP_ECUDA; }

}  // namespace

extern "C" {

const char *glop_status_str(glop_status s) {
    switch (s) {
        case GLOP_OK: return "ok";
        case GLOP_EINVAL: return "invalid argument";
        case GLOP_ENOMEM: return "out of memory";
        case GLOP_EOVERFLOW: return "match capacity exceeded";
        case GLOP_ECUDA: return "CUDA error";
        case GLOP_ETIMEOUT: return "bounded wait timed out";
        case GLOP_EBUSY: return "busy";
        case GLOP_EINTERNAL: return "internal error";
    }
    return "unknown status";
}

glop_status glop_compile(const uint8_t *pattern_bytes, const uint64_t *pattern_offsets, uint32_t n_patterns,
                         const glop_compile_opts *opts, glop_handle *out) {
    if (!out || !pattern_offsets || (n_patterns && !pattern_bytes)) return GLOP_EINVAL;
    if (opts && opts->flags) return GLOP_EINVAL;
    auto t0 = std::chrono::steady_clock::now();
    glop::HostAutomaton H;
    std::string err;
    int rc;
    try {
        rc = glop::compile_host(pattern_bytes, pattern_offsets, n_patterns, opts ? opts->prefix_len : 0, &H, &err,
                                opts ? opts->gram_len : 0, opts ? opts->filter_bits_log2 : 0);
    } catch (const std::bad_alloc &) {
        return GLOP_ENOMEM;
    }
    if (rc) return (glop_status)rc;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GLOP_ECUDA;

    // dense rows as uint16 (state | 0x8000 when terminal) when every state id fits in 15 bits
    const bool row16 = H.n_states <= 0x7FFF;
    std::vector<uint16_t> rows16;
    if (row16) {
        rows16.resize(H.rows.size());
        for (size_t i = 0; i < H.rows.size(); ++i) {
            const uint32_t e = (uint32_t)H.rows[i];
            rows16[i] = (uint16_t)((e & GLOP_STATE_MASK) | ((e & GLOP_TERM) ? 0x8000u : 0u));
        }
    }
    const uint64_t rows_bytes = row16 ? bytes_of(rows16) : bytes_of(H.rows);
    // one device blob; every array 256-byte aligned and followed by at least 16 spare bytes
    uint64_t o_cls = 0;
    uint64_t o_rows = al(o_cls + 256);
    uint64_t o_chain = al(o_rows + rows_bytes + 16);
    uint64_t o_cum = al(o_chain + bytes_of(H.chain) + 16);
    uint64_t o_outl = al(o_cum + bytes_of(H.cum_off));
    uint64_t o_ids = al(o_outl + 8ull * H.n_states);
    uint64_t o_bm = al(o_ids + bytes_of(H.cum_ids) + 16);
    uint64_t o_gr = al(o_bm + bytes_of(H.bitmap) + 16);
    uint64_t total = al(o_gr + bytes_of(H.grams) + 16);
    std::vector<uint8_t> host;
    try {
        host.assign(total, 0);
    } catch (const std::bad_alloc &) {
        return GLOP_ENOMEM;
    }
    std::memcpy(host.data() + o_cls, H.cls.data(), 256);
    if (rows_bytes) std::memcpy(host.data() + o_rows, row16 ? (const void *)rows16.data() : (const void *)H.rows.data(),
                                rows_bytes);
    if (!H.chain.empty()) std::memcpy(host.data() + o_chain, H.chain.data(), bytes_of(H.chain));
    std::memcpy(host.data() + o_cum, H.cum_off.data(), bytes_of(H.cum_off));
    {
        uint32_t *ol = reinterpret_cast<uint32_t *>(host.data() + o_outl);
        for (uint32_t t = 0; t < H.n_states; ++t) {
            ol[2 * t] = H.cum_off[t];
            ol[2 * t + 1] = H.cum_off[t + 1] - H.cum_off[t];
        }
    }
    if (!H.cum_ids.empty()) std::memcpy(host.data() + o_ids, H.cum_ids.data(), bytes_of(H.cum_ids));
    if (!H.bitmap.empty()) std::memcpy(host.data() + o_bm, H.bitmap.data(), bytes_of(H.bitmap));
    if (!H.grams.empty()) std::memcpy(host.data() + o_gr, H.grams.data(), bytes_of(H.grams));

    glop_automaton *h = new (std::nothrow) glop_automaton();
    if (!h) return GLOP_ENOMEM;
    if (cudaMalloc(&h->blob, total) != cudaSuccess) {
        delete h;
        cudaGetLastError();
        return GLOP_ENOMEM;
    }
    if (cudaMemcpy(h->blob, host.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(h->blob);
        delete h;
        return GLOP_ECUDA;
    }
    uint8_t *base = reinterpret_cast<uint8_t *>(h->blob);
    GlopDevAutomaton &D = h->dev;
    D.n_states = H.n_states;
    D.n_dense = H.n_dense;
    D.n_classes = H.n_classes;
    D.n_patterns = H.n_patterns;
    D.min_len = H.min_len;
    D.max_len = H.max_len;
    D.gram_len = H.gram_len;
    D.bm_log2 = H.bm_log2;
    D.ht_log2 = H.ht_log2;
    D.hot_lo = H.hot_lo;
    D.cls = base + o_cls;
    D.rows = base + o_rows;
    D.row16 = row16 ? 1u : 0u;
    D.chain = reinterpret_cast<const GlopChain *>(base + o_chain);
    D.cum_off = reinterpret_cast<const uint32_t *>(base + o_cum);
    D.outl = reinterpret_cast<const uint32_t *>(base + o_outl);
    D.cum_ids = reinterpret_cast<const uint32_t *>(base + o_ids);
    D.n_cum_ids = (uint32_t)H.cum_ids.size();
    D.bitmap = reinterpret_cast<const uint32_t *>(base + o_bm);
    D.grams = reinterpret_cast<const GlopGramSlot *>(base + o_gr);
    h->blob_bytes = total;
    h->device = dev;
    h->smem_budget = opts ? opts->smem_budget_bytes : 0;
    h->ksub = (opts && opts->chunk_subtiles == 2) ? 2u : 1u;
    glop_info &I = h->info;
    I.n_patterns = H.n_patterns;
    I.min_pattern_len = H.min_len;
    I.max_pattern_len = H.max_len;
    I.n_states = H.n_states;
    I.n_dense_states = H.n_dense;
    I.n_chain_states = H.n_states - H.n_dense;
    I.n_classes = H.n_classes;
    I.gram_len = H.gram_len;
    I.n_grams = H.n_grams;
    I.cum_ids = (uint32_t)H.cum_ids.size();
    I.device_bytes = total;
    I.compile_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return GLOP_OK;
}

glop_status glop_info_get(glop_handle h, glop_info *info) {
    if (!h || !info) return GLOP_EINVAL;
    *info = h->info;
    return GLOP_OK;
}

uint32_t glop_max_pattern_len(glop_handle h) { return h ? h->info.max_pattern_len : 0; }

glop_status glop_scan_workspace_size(glop_handle h, uint64_t text_len, uint64_t *bytes) {
    if (!h || !bytes) return GLOP_EINVAL;
    *bytes = glop::workspace_bytes(text_len, false);
    return GLOP_OK;
}

glop_status glop_batch_workspace_size(glop_handle h, uint64_t text_len, uint32_t n_segments, uint64_t *bytes) {
    (void)n_segments;
    if (!h || !bytes) return GLOP_EINVAL;
    *bytes = glop::workspace_bytes(text_len, true);
    return GLOP_OK;
}

static glop_status do_scan(glop_handle h, const uint8_t *d_text, uint64_t len, const uint64_t *seg, uint32_t n_seg,
                           void *out, uint64_t capacity, uint64_t *d_count, void *ws, uint64_t ws_bytes,
                           glop_stream_t stream) {
    if (!h || !d_count || !ws || (len && !d_text) || (capacity && !out)) return GLOP_EINVAL;
    if ((reinterpret_cast<uintptr_t>(ws) & 15) || (reinterpret_cast<uintptr_t>(d_count) & 7)) return GLOP_EINVAL;
    if (ws_bytes < glop::workspace_bytes(len, seg != nullptr)) return GLOP_ENOMEM;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GLOP_ECUDA;
    if (dev != h->device) return GLOP_EINVAL;
    glop::ScanLaunch L;
    L.A = &h->dev;
    L.text = d_text;
    L.len = len;
    L.seg = seg;
    L.n_seg = n_seg;
    L.out = out;
    L.capacity = capacity;
    L.d_count = d_count;
    L.ws = ws;
    L.ws_bytes = ws_bytes;
    L.stream = reinterpret_cast<cudaStream_t>(stream);
    L.smem_budget = h->smem_budget;
    L.ksub = h->ksub;
    L.ksub_used = &h->ksub_used;
    return (glop_status)glop::launch_scan(L);
}

glop_status glop_scan(glop_handle h, const uint8_t *d_text, uint64_t len, glop_match *d_matches, uint64_t capacity,
                      uint64_t *d_count, void *d_workspace, uint64_t workspace_bytes, glop_stream_t stream) {
    if (len > 0xFFFFFFFFull) return GLOP_EINVAL;
    if (d_matches && (reinterpret_cast<uintptr_t>(d_matches) & 7)) return GLOP_EINVAL;
    return do_scan(h, d_text, len, nullptr, 0, d_matches, capacity, d_count, d_workspace, workspace_bytes, stream);
}

glop_status glop_count_workspace_size(glop_handle h, uint64_t text_len, uint64_t *bytes) {
    (void)text_len;
    if (!h || !bytes) return GLOP_EINVAL;
    *bytes = glop::count_workspace_bytes(h->dev.n_states);
    return GLOP_OK;
}

glop_status glop_scan_count(glop_handle h, const uint8_t *d_text, uint64_t len, uint64_t *d_hist, uint64_t *d_total,
                            void *d_workspace, uint64_t workspace_bytes, glop_stream_t stream) {
    if (!h || !d_total || !d_workspace || (len && !d_text) || (h->dev.n_patterns && !d_hist)) return GLOP_EINVAL;
    if (len > 0xFFFFFFFFull) return GLOP_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_workspace) & 255) || (reinterpret_cast<uintptr_t>(d_total) & 7) ||
        (reinterpret_cast<uintptr_t>(d_hist) & 7))
        return GLOP_EINVAL;
    if (workspace_bytes < glop::count_workspace_bytes(h->dev.n_states)) return GLOP_ENOMEM;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GLOP_ECUDA;
    if (dev != h->device) return GLOP_EINVAL;
    glop::ScanLaunch L;
    L.A = &h->dev;
    L.text = d_text;
    L.len = len;
    L.seg = nullptr;
    L.n_seg = 0;
    L.out = nullptr;
    L.capacity = 0;
    L.d_count = d_total;
    L.ws = d_workspace;
    L.ws_bytes = workspace_bytes;
    L.stream = reinterpret_cast<cudaStream_t>(stream);
    L.smem_budget = h->smem_budget;
    L.ksub = h->ksub;
    L.ksub_used = &h->ksub_used;
    L.hist = reinterpret_cast<unsigned long long *>(d_hist);
    return (glop_status)glop::launch_scan(L);
}

glop_status glop_scan_batch(glop_handle h, const uint8_t *d_text, uint64_t text_len, const uint64_t *d_seg_offsets,
                            uint32_t n_segments, glop_batch_match *d_matches, uint64_t capacity, uint64_t *d_count,
                            void *d_workspace, uint64_t workspace_bytes, glop_stream_t stream) {
    if (!d_seg_offsets || (reinterpret_cast<uintptr_t>(d_seg_offsets) & 7)) return GLOP_EINVAL;
    if (d_matches && (reinterpret_cast<uintptr_t>(d_matches) & 3)) return GLOP_EINVAL;
    return do_scan(h, d_text, text_len, d_seg_offsets, n_segments, d_matches, capacity, d_count, d_workspace,
                   workspace_bytes, stream);
}

static_assert(GLOP_BATCH_MAX_GROUPS == glop::kMaxBatchGroups, "one limit for the header and the kernel");

glop_status glop_scan_batch_multi(const glop_handle *handles, uint32_t n_groups, const uint64_t *group_start,
                                  const uint8_t *d_text, uint64_t text_len, const uint64_t *d_seg_offsets,
                                  uint32_t n_segments, glop_batch_match *d_matches, uint64_t capacity,
                                  uint64_t *d_count, void *d_workspace, uint64_t workspace_bytes,
                                  glop_stream_t stream) {
    if (!handles || !group_start || n_groups == 0 || n_groups > GLOP_BATCH_MAX_GROUPS) return GLOP_EINVAL;
    if (!d_seg_offsets || (reinterpret_cast<uintptr_t>(d_seg_offsets) & 7)) return GLOP_EINVAL;
    if (d_matches && (reinterpret_cast<uintptr_t>(d_matches) & 3)) return GLOP_EINVAL;
    if (!d_count || !d_workspace || (text_len && !d_text) || (capacity && !d_matches)) return GLOP_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_workspace) & 15) || (reinterpret_cast<uintptr_t>(d_count) & 7)) return GLOP_EINVAL;
    if (workspace_bytes < glop::workspace_bytes(text_len, true)) return GLOP_ENOMEM;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GLOP_ECUDA;
    // group bytes: from 0 to text_len, non-decreasing, every start on a sub-tile boundary
    if (group_start[0] != 0 || group_start[n_groups] != text_len) return GLOP_EINVAL;
    GlopDevAutomaton as[GLOP_BATCH_MAX_GROUPS];
    for (uint32_t g = 0; g < n_groups; ++g) {
        const glop_handle h = handles[g];
        if (!h || h->device != dev || h->dev.n_patterns == 0) return GLOP_EINVAL;
        if (group_start[g + 1] < group_start[g] || group_start[g] % glop::kSubTile) return GLOP_EINVAL;
        // one kernel variant for every group: the start filter's kind and the row width
        const GlopDevAutomaton &a = h->dev, &a0 = handles[0]->dev;
        auto kind = [](uint32_t gram) { return gram == 0 ? 0u : gram == 4 ? 4u : 8u; };
        if (kind(a.gram_len) != kind(a0.gram_len) || a.row16 != a0.row16) return GLOP_EINVAL;
        as[g] = a;
    }
    glop::ScanLaunch L;
    L.A = &as[0];
    L.text = d_text;
    L.len = text_len;
    L.seg = d_seg_offsets;
    L.n_seg = n_segments;
    L.out = d_matches;
    L.capacity = capacity;
    L.d_count = d_count;
    L.ws = d_workspace;
    L.ws_bytes = workspace_bytes;
    L.stream = reinterpret_cast<cudaStream_t>(stream);
    L.smem_budget = handles[0]->smem_budget;
    L.n_groups = n_groups;
    L.group_A = as;
    L.group_start = group_start;
    return (glop_status)glop::launch_scan(L);
}

glop_status glop_batch_multi_kind(glop_handle h, uint32_t *kind) {
    if (!h || !kind) return GLOP_EINVAL;
    const uint32_t g = h->dev.gram_len;
    *kind = (g == 0 ? 0u : g == 4 ? 4u : 8u) | (h->dev.row16 ? 0x100u : 0u);
    return GLOP_OK;
}

glop_status glop_scan_status(const void *d_workspace, glop_stream_t stream, uint64_t *count) {
    // NULL: the scratch array of glop_scan_noalloc on the current device
    if (!d_workspace) d_workspace = glop::noalloc_scratch_of_current_device();
    if (!d_workspace) return GLOP_ECUDA;
    uint32_t hdr[16];
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return GLOP_ECUDA;
    if (cudaMemcpy(hdr, d_workspace, sizeof hdr, cudaMemcpyDeviceToHost) != cudaSuccess) return GLOP_ECUDA;
    uint64_t total;
    std::memcpy(&total, hdr + 4, 8);
    if (count) *count = total;
    // a bounded wait that ran out comes first: phase B may then have met data phase A never wrote, and
    // the checks that caught it are its consequence, not a separate fault
    if (hdr[0] & glop::WS_TIMEOUT) return GLOP_ETIMEOUT;
    if (hdr[0] & glop::WS_INTERNAL) {
        std::fprintf(stderr, "glop: internal check failed at site %u (value %u)\n", hdr[11], hdr[12]);
        return GLOP_EINTERNAL;
    }
    if (hdr[0] & glop::WS_EINVAL) return GLOP_EINVAL;
    if (hdr[0] & glop::WS_TIMEOUT) return GLOP_ETIMEOUT;
    if (hdr[0] & glop::WS_OVERFLOW) return GLOP_EOVERFLOW;
    return GLOP_OK;
}

// staging: text | matches | count area (the count, or per piece counts and output bases) | workspace
constexpr uint64_t kCountArea = 512;

glop_status glop_scan_host_staging_size(glop_handle h, uint64_t len, uint64_t capacity, uint64_t *bytes) {
    if (!h || !bytes) return GLOP_EINVAL;
    *bytes = al(len) + al(capacity * sizeof(glop_match)) + kCountArea + glop::workspace_bytes(len, false);
    return GLOP_OK;
}

namespace {

// glop_scan_host on long texts: pieces uploaded on one stream, scanned in order on the caller's stream (each
// scan places its matches after the previous piece's, from a device word, and covers the next
// longest-pattern - 1 bytes as look-ahead), and copied back on a third stream as soon as each piece's count is
// known -- uploads, scans and copy-backs of different pieces overlap.  A first piece of 1/kHeadDiv of a full
// one (the copy-back of the first matches starts after a short upload and scan), then up to kMidPieces equal
// full pieces, at most one per kPieceMin bytes.  kTailDiv > 0 would end on a short piece as well; on GB300 that
// measured no faster (the copy-back, not the last scan, ends the call).
constexpr uint64_t kPieceMin = 8ull << 20;
constexpr uint32_t kMidPieces = 8;
constexpr uint32_t kHeadDiv = 4, kTailDiv = 0;  // 0: no short piece at that end
constexpr uint32_t kMaxPieces = kMidPieces + 2;
constexpr uint64_t kCopyAlign = 4096;

uint64_t round_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// Piece boundaries of a len-byte text (len >= 2 * kPieceMin): bnd[0] = 0 < bnd[1] < ... < bnd[P] = len, every
// inner boundary a multiple of kCopyAlign.  Returns P.
uint32_t piece_plan(uint64_t len, uint64_t *bnd) {
    const uint32_t M = (uint32_t)std::min<uint64_t>(kMidPieces, len / kPieceMin);
    const double w = M + (kHeadDiv ? 1.0 / kHeadDiv : 0.0) + (kTailDiv ? 1.0 / kTailDiv : 0.0);
    const uint64_t ps = round_up((uint64_t)((double)len / w) + 1, kCopyAlign);
    uint32_t P = 0;
    uint64_t b = 0;
    bnd[0] = 0;
    if constexpr (kHeadDiv != 0) bnd[++P] = b = std::min(len, round_up(ps / kHeadDiv, kCopyAlign));
    for (uint32_t i = 0; i < M && b < len; ++i) bnd[++P] = b = std::min(len, b + ps);
    if (b < len) bnd[++P] = len;
    return P;
}

static_assert((2 * kMaxPieces + 1) * 8 <= 512, "per-piece counts and bases fit the count area");

struct HostPipe {
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t uploaded[kMaxPieces] = {}, scanned[kMaxPieces] = {};
    uint64_t *pinned = nullptr;  // per piece: match count, status (written by the words kernel)
    unsigned long long *pinned_dev = nullptr;  // the same words as the device addresses them
    bool ok = false;
};

// Streams, events and pinned words of this host thread on device dev (created once, kept for the process).
HostPipe *host_pipe(int dev) {
    thread_local HostPipe pipes[64];
    if (dev < 0 || dev >= 64) return nullptr;
    HostPipe &hp = pipes[dev];
    if (hp.ok) return &hp;
    if (cudaStreamCreateWithFlags(&hp.up, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&hp.down, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost(&hp.pinned, 2 * kMaxPieces * sizeof(uint64_t)) != cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void **>(&hp.pinned_dev), hp.pinned, 0) != cudaSuccess)
        return nullptr;
    for (uint32_t k = 0; k < kMaxPieces; ++k)
        if (cudaEventCreateWithFlags(&hp.uploaded[k], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&hp.scanned[k], cudaEventDisableTiming) != cudaSuccess)
            return nullptr;
    hp.ok = true;
    return &hp;
}

glop_status scan_host_pieces(glop_handle h, const uint8_t *h_text, uint64_t len, glop_match *h_matches,
                             uint64_t capacity, uint64_t *h_count, uint8_t *d_text, glop_match *d_m, uint64_t *d_c,
                             void *ws, uint64_t ws_bytes, cudaStream_t st) {
    HostPipe *hp = host_pipe(h->device);
    if (!hp) return GLOP_ECUDA;
    uint64_t bnd[kMaxPieces + 1];
    const uint32_t P = piece_plan(len, bnd);
    const uint64_t halo = h->dev.max_len ? h->dev.max_len - 1 : 0;
    uint64_t *d_counts = d_c, *d_bases = d_c + kMaxPieces;  // count area: P counts, P + 1 bases
    auto lo = [&](uint32_t k) { return bnd[k]; };
    // upload k covers [up_lo(k), up_lo(k + 1)): piece k's bytes from the end of the previous piece's look-ahead
    // through its own look-ahead, so scan k waits for upload k alone (earlier uploads precede it on `up`).
    // The look-ahead end is rounded up to kCopyAlign bytes, so every copy starts aligned.
    auto up_lo = [&](uint32_t k) -> uint64_t {
        if (k == 0) return 0;
        if (k >= P) return len;
        return std::min(len, round_up(lo(k) + halo, kCopyAlign));
    };
    if (cudaMemsetAsync(d_bases, 0, 8, st) != cudaSuccess) return GLOP_ECUDA;
    for (uint32_t k = 0; k < P; ++k) {
        const uint64_t a = up_lo(k), b = up_lo(k + 1);
        if (b > a && cudaMemcpyAsync(d_text + a, h_text + a, b - a, cudaMemcpyHostToDevice, hp->up) != cudaSuccess)
            return GLOP_ECUDA;
        if (cudaEventRecord(hp->uploaded[k], hp->up) != cudaSuccess) return GLOP_ECUDA;
    }
    for (uint32_t k = 0; k < P; ++k) {
        const uint64_t a = lo(k), b = lo(k + 1), e = std::min(len, b + halo);
        if (cudaStreamWaitEvent(st, hp->uploaded[k], 0) != cudaSuccess) return GLOP_ECUDA;
        glop::ScanLaunch L;
        L.A = &h->dev;
        L.text = d_text + a;
        L.len = e - a;
        L.seg = nullptr;
        L.n_seg = 0;
        L.out = d_m;
        L.capacity = capacity;
        L.d_count = d_counts + k;
        L.ws = ws;
        L.ws_bytes = ws_bytes;
        L.stream = st;
        L.smem_budget = h->smem_budget;
        L.ksub = h->ksub;
        L.ksub_used = &h->ksub_used;
        L.own_len = b - a;
        L.base_off = (uint32_t)a;
        L.d_obase = reinterpret_cast<const unsigned long long *>(d_bases + k);
        L.d_next_base = reinterpret_cast<unsigned long long *>(d_bases + k + 1);
        if (b == a) {  // an empty piece: its base passes on unchanged
            if (cudaMemcpyAsync(d_bases + k + 1, d_bases + k, 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return GLOP_ECUDA;
            continue;
        }
        const int rc = glop::launch_scan(L);
        if (rc) return (glop_status)rc;
        // the count and status reach the host through a kernel's stores: a memcpy would wait behind the
        // previous piece's copy-back on the copy engine and hold up the next scan
        if (glop::launch_words(ws, hp->pinned_dev + 2 * k, st) || cudaEventRecord(hp->scanned[k], st) != cudaSuccess)
            return GLOP_ECUDA;
    }
    uint64_t base = 0;
    bool internal = false, timeout = false;
    for (uint32_t k = 0; k < P; ++k) {
        if (lo(k + 1) == lo(k)) continue;
        if (cudaEventSynchronize(hp->scanned[k]) != cudaSuccess) return GLOP_ECUDA;
        const uint64_t c = hp->pinned[2 * k];
        // (a piece's own overflow status is not used: the whole text's overflow is base > capacity below)
        internal |= hp->pinned[2 * k + 1] == GLOP_EINTERNAL;
        timeout |= hp->pinned[2 * k + 1] == GLOP_ETIMEOUT;
        const uint64_t n = base < capacity ? std::min(c, capacity - base) : 0;
        // the copy starts on a kCopyAlign boundary of the output: the bytes before this piece's first match are
        // earlier pieces' matches, final on the device and copied again unchanged after their own copy
        const uint64_t c0 = base * sizeof(glop_match) / kCopyAlign * kCopyAlign;
        const uint64_t c1 = (base + n) * sizeof(glop_match);
        if (n && (cudaStreamWaitEvent(hp->down, hp->scanned[k], 0) != cudaSuccess ||
                  cudaMemcpyAsync(reinterpret_cast<uint8_t *>(h_matches) + c0,
                                  reinterpret_cast<const uint8_t *>(d_m) + c0, c1 - c0, cudaMemcpyDeviceToHost,
                                  hp->down) != cudaSuccess))
            return GLOP_ECUDA;
        base += c;
    }
    if (cudaStreamSynchronize(hp->down) != cudaSuccess) return GLOP_ECUDA;
    *h_count = base;
    if (internal) return GLOP_EINTERNAL;
    if (timeout) return GLOP_ETIMEOUT;
    if (base > capacity) return GLOP_EOVERFLOW;
    return GLOP_OK;
}

}  // namespace

glop_status glop_scan_host_plan(uint64_t len, uint64_t *bounds, uint32_t max_bounds, uint32_t *n_pieces) {
    if (!n_pieces) return GLOP_EINVAL;
    uint64_t bnd[kMaxPieces + 1] = {0, len};
    const uint32_t P = len >= 2 * kPieceMin ? piece_plan(len, bnd) : 1;
    *n_pieces = P;
    if (!bounds) return GLOP_OK;
    if (max_bounds < P + 1) return GLOP_EINVAL;
    for (uint32_t k = 0; k <= P; ++k) bounds[k] = bnd[k];
    return GLOP_OK;
}

glop_status glop_scan_host(glop_handle h, const uint8_t *h_text, uint64_t len, glop_match *h_matches,
                           uint64_t capacity, uint64_t *h_count, void *d_staging, uint64_t staging_bytes,
                           glop_stream_t stream) {
    if (!h || !h_count || !d_staging || (len && !h_text) || (capacity && !h_matches)) return GLOP_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_staging) & 255) return GLOP_EINVAL;
    if (len > 0xFFFFFFFFull) return GLOP_EINVAL;
    uint64_t need = 0;
    glop_scan_host_staging_size(h, len, capacity, &need);
    if (staging_bytes < need) return GLOP_ENOMEM;
    uint8_t *p = reinterpret_cast<uint8_t *>(d_staging);
    uint8_t *d_text = p;
    glop_match *d_m = reinterpret_cast<glop_match *>(p + al(len));
    uint64_t *d_c = reinterpret_cast<uint64_t *>(p + al(len) + al(capacity * sizeof(glop_match)));
    void *ws = p + al(len) + al(capacity * sizeof(glop_match)) + kCountArea;
    uint64_t ws_bytes = glop::workspace_bytes(len, false);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GLOP_ECUDA;
    if (dev != h->device) return GLOP_EINVAL;
    if (len >= 2 * kPieceMin && h->dev.n_patterns)
        return scan_host_pieces(h, h_text, len, h_matches, capacity, h_count, d_text, d_m, d_c, ws, ws_bytes, st);
    if (len && cudaMemcpyAsync(d_text, h_text, len, cudaMemcpyHostToDevice, st) != cudaSuccess) return GLOP_ECUDA;
    glop_status s = glop_scan(h, d_text, len, d_m, capacity, d_c, ws, ws_bytes, stream);
    if (s != GLOP_OK) return s;
    // the count and the status come back together in the thread's pinned words (written by a kernel)
    HostPipe *hp = host_pipe(dev);
    if (!hp) return GLOP_ECUDA;
    if (glop::launch_words(ws, hp->pinned_dev, st) || cudaStreamSynchronize(st) != cudaSuccess) return GLOP_ECUDA;
    const uint64_t total = hp->pinned[0];
    const uint64_t status = hp->pinned[1];
    *h_count = total;
    uint64_t n = total < capacity ? total : capacity;
    if (n && (cudaMemcpyAsync(h_matches, d_m, n * sizeof(glop_match), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
              cudaStreamSynchronize(st) != cudaSuccess))
        return GLOP_ECUDA;
    if (status == GLOP_EINTERNAL || status == GLOP_ETIMEOUT) return (glop_status)status;
    if (total > capacity) return GLOP_EOVERFLOW;
    return GLOP_OK;
}

glop_status glop_tune(const uint8_t *pattern_bytes, const uint64_t *pattern_offsets, uint32_t n_patterns,
                      uint32_t prefix_len, const uint8_t *d_sample, uint64_t sample_len,
                      const uint64_t *d_seg_offsets, uint32_t n_segments, uint32_t repeats, glop_tune_point *points,
                      uint32_t max_points, uint32_t *n_points, glop_compile_opts *best, glop_stream_t stream) {
    if (!best || !n_points || (sample_len && !d_sample)) return GLOP_EINVAL;
    if (repeats < 1) repeats = 1;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // the automatic choice first: its gram length and bitmap size span the grid
    glop_compile_opts base{};
    base.prefix_len = prefix_len;
    glop_handle h0 = nullptr;
    glop_status s = glop_compile(pattern_bytes, pattern_offsets, n_patterns, &base, &h0);
    if (s != GLOP_OK) return s;
    const uint32_t gmax = h0->info.gram_len, bm0 = h0->dev.bm_log2;
    glop_destroy(h0);
    std::vector<uint32_t> grams, bits;
    if (gmax == 0) grams.push_back(0);
    else for (uint32_t g = 4; g <= gmax; ++g) grams.push_back(g);
    if (gmax == 0) bits.push_back(0);
    else for (int d = -2; d <= 2; d += 2) {
        const int b = (int)bm0 + d;
        if (b >= 13 && b <= 19) bits.push_back((uint32_t)b);
    }
    const uint32_t budgets[2] = {0u, 16384u};
    const bool batch = d_seg_offsets != nullptr;
    void *ws = nullptr, *out = nullptr, *cnt = nullptr;
    uint64_t ws_bytes = glop::workspace_bytes(sample_len, batch), out_cap = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (ws) cudaFree(ws);
        if (out) cudaFree(out);
        if (cnt) cudaFree(cnt);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (cudaMalloc(&ws, ws_bytes) != cudaSuccess || cudaMalloc(&cnt, 8) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        cudaGetLastError();
        return GLOP_ENOMEM;
    }
    const uint32_t rec = batch ? (uint32_t)sizeof(glop_batch_match) : (uint32_t)sizeof(glop_match);
    auto scan_once = [&](glop_handle h) -> glop_status {
        return batch ? glop_scan_batch(h, d_sample, sample_len, d_seg_offsets, n_segments,
                                       reinterpret_cast<glop_batch_match *>(out), out_cap, reinterpret_cast<uint64_t *>(cnt),
                                       ws, ws_bytes, stream)
                     : glop_scan(h, d_sample, sample_len, reinterpret_cast<glop_match *>(out), out_cap,
                                 reinterpret_cast<uint64_t *>(cnt), ws, ws_bytes, stream);
    };
    uint32_t np = 0;
    double best_gbps = -1;
    for (uint32_t g : grams) {
        for (uint32_t b : bits) {
            glop_compile_opts o{};
            o.prefix_len = prefix_len;
            o.gram_len = g;
            o.filter_bits_log2 = b;
            glop_handle h = nullptr;
            s = glop_compile(pattern_bytes, pattern_offsets, n_patterns, &o, &h);
            if (s != GLOP_OK) { cleanup(); return s; }
            for (uint32_t budget : budgets)
            for (uint32_t ks : {1u, 2u}) {
                h->smem_budget = budget;
                o.smem_budget_bytes = budget;
                h->ksub = ks;
                // size the output once (identical for every candidate), then warm up and time
                if (!out) {
                    s = scan_once(h);
                    uint64_t total = 0;
                    if (s == GLOP_OK) s = glop_scan_status(ws, stream, &total);
                    if (s != GLOP_OK && s != GLOP_EOVERFLOW) { glop_destroy(h); cleanup(); return s; }
                    out_cap = total ? total : 1;
                    if (cudaMalloc(&out, out_cap * rec) != cudaSuccess) { glop_destroy(h); cleanup(); return GLOP_ENOMEM; }
                }
                s = scan_once(h);
                if (s != GLOP_OK) { glop_destroy(h); cleanup(); return s; }
                o.chunk_subtiles = h->ksub_used;  // (62 KiB chunks run as 31 KiB ones where two slots do not fit)
                if (ks == 2 && h->ksub_used != 2) continue;
                cudaEventRecord(e0, st);
                for (uint32_t r = 0; r < repeats && s == GLOP_OK; ++r) s = scan_once(h);
                cudaEventRecord(e1, st);
                if (s != GLOP_OK || cudaEventSynchronize(e1) != cudaSuccess) { glop_destroy(h); cleanup(); return GLOP_ECUDA; }
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                const double gbps = ms > 0 ? 8.0 * (double)sample_len * repeats / (ms * 1e-3) / 1e9 : 0.0;
                if (points && np < max_points) points[np] = glop_tune_point{o, gbps};
                ++np;
                if (gbps > best_gbps) { best_gbps = gbps; *best = o; }
            }
            glop_destroy(h);
        }
    }
    *n_points = np;
    cleanup();
    return GLOP_OK;
}

struct glop_plan_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

glop_status glop_plan_create(glop_handle h, const uint8_t *d_text, uint64_t text_len, const uint64_t *d_seg_offsets,
                             uint32_t n_segments, void *d_matches, uint64_t capacity, uint64_t *d_count,
                             void *d_workspace, uint64_t workspace_bytes, glop_stream_t stream, glop_plan *out) {
    if (!out || !stream) return GLOP_EINVAL;  // capture needs a real stream, not the legacy default stream
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    glop_plan p = new (std::nothrow) glop_plan_s();
    if (!p) return GLOP_ENOMEM;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        delete p;
        return GLOP_ECUDA;
    }
    glop_status s = d_seg_offsets
                        ? glop_scan_batch(h, d_text, text_len, d_seg_offsets, n_segments,
                                          reinterpret_cast<glop_batch_match *>(d_matches), capacity, d_count,
                                          d_workspace, workspace_bytes, stream)
                        : glop_scan(h, d_text, text_len, reinterpret_cast<glop_match *>(d_matches), capacity, d_count,
                                    d_workspace, workspace_bytes, stream);
    cudaError_t e = cudaStreamEndCapture(st, &p->graph);
    if (s != GLOP_OK || e != cudaSuccess) {
        if (p->graph) cudaGraphDestroy(p->graph);
        delete p;
        cudaGetLastError();
        return s != GLOP_OK ? s : GLOP_ECUDA;
    }
    if (cudaGraphInstantiate(&p->exec, p->graph, 0) != cudaSuccess) {
        cudaGraphDestroy(p->graph);
        delete p;
        cudaGetLastError();
        return GLOP_ECUDA;
    }
    *out = p;
    return GLOP_OK;
}

glop_status glop_plan_launch(glop_plan plan, glop_stream_t stream) {
    if (!plan) return GLOP_EINVAL;
    return cuda_ok(cudaGraphLaunch(plan->exec, reinterpret_cast<cudaStream_t>(stream)));
}

glop_status glop_plan_destroy(glop_plan plan) {
    if (!plan) return GLOP_OK;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    delete plan;
    return GLOP_OK;
}

glop_status glop_destroy(glop_handle h) {
    if (!h) return GLOP_OK;
    glop_status s = GLOP_OK;
    if (h->blob) s = cuda_ok(cudaFree(h->blob));
    delete h;
    return s;
}

}  // extern "C"
