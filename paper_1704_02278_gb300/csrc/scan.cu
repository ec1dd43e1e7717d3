// scan.cu -- host side of the scan: workspace layout, shared-memory carve,
// launch of the scan kernel (device code in scan_kernel.cuh, instantiated in
// scan_f0.cu / scan_f4.cu / scan_f8.cu), and the two small kernels (workspace
// header clear and batch segment check; count-only list spreading).
#include "scan_kernel.cuh"

namespace glop {
namespace kern {

// ---------------------------------------------------------------- kernels
// Zero the workspace header; for batches also check the segment table and
// find, for every sub-tile, the last segment starting at or before it.
// Several automata in one batch: the byte where each group starts.
struct GroupStarts {
    uint32_t n;
    uint64_t start[kMaxBatchGroups + 1];
};

__global__ void init_kernel(uint32_t *hdr, uint32_t *tile_seg, uint64_t n_sub, const uint64_t *seg, uint32_t n_seg,
                            uint64_t len, unsigned long long *d_count, int zero_header, int nothing, GroupStarts gs) {
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    if (zero_header && tid < kHeaderBytes / 4) hdr[tid] = 0;
    if (nothing && tid == 0) *d_count = 0ull;
    if (!seg) return;
    bool bad = false;
    for (uint64_t s = tid; s < n_seg; s += nthr) {
        const uint64_t a = seg[s], b = seg[s + 1];
        if (b < a || b - a > 0xFFFFFFFFull || b > len) bad = true;
    }
    // several automata: every group after the first must start where a segment starts (no segment
    // straddles two groups)
    if (tid >= 1 && tid < gs.n) {
        const uint64_t x = gs.start[tid];
        uint32_t lo = 0, hi = n_seg;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (seg[mid] < x) lo = mid + 1; else hi = mid;
        }
        if (seg[lo] != x) bad = true;
    }
    if (bad) {
        atomicOr(hdr, WS_EINVAL);
        *d_count = 0ull;
    }
    for (uint64_t k = tid; k <= n_sub; k += nthr) {
        const uint64_t x = k * SUB;
        uint32_t lo = 0, hi = n_seg;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (seg[mid] <= x) lo = mid; else hi = mid - 1;
        }
        tile_seg[k] = lo;
    }
}

// Count-only mode, after the scan: every pattern in a state's output list
// occurs once per hit on the state.  hist and total are zero on entry.
__global__ void count_lists_kernel(const uint32_t *hits, const uint32_t *cum_off, const uint32_t *cum_ids,
                                   uint32_t n_states, unsigned long long *hist, unsigned long long *total) {
    unsigned long long sum = 0;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n_states; t += gridDim.x * blockDim.x) {
        const uint32_t h = hits[t];
        if (!h) continue;
        const uint32_t lo = cum_off[t], hi = cum_off[t + 1];
        for (uint32_t q = lo; q < hi; ++q) atomicAdd(hist + cum_ids[q], (unsigned long long)h);
        sum += (unsigned long long)h * (hi - lo);
    }
    for (int d = 16; d; d >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, d);
    if ((threadIdx.x & 31) == 0 && sum) atomicAdd(total, sum);
}

// ---------------------------------------------------------------- host side
struct DevProps {
    int sms = 0, smem_optin = 0, coop = 0;
};

DevProps props_of(int dev) {
    static std::mutex mu;
    static DevProps cache[64];
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) return DevProps{};
    if (!cache[dev].sms) {
        cudaDeviceGetAttribute(&cache[dev].sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&cache[dev].smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&cache[dev].coop, cudaDevAttrCooperativeLaunch, dev);
    }
    return cache[dev];
}

uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

struct WsLayout {
    uint64_t desc, sums, tile_seg, records, total;
    uint64_t rec_slots;
};

WsLayout layout_of(uint64_t len, bool batch) {
    const uint64_t n_sub = (len + SUB - 1) / SUB;
    WsLayout w;
    w.desc = kHeaderBytes;
    w.sums = w.desc + 16 * n_sub;
    w.tile_seg = w.sums + 8ull * kMaxGrid;
    uint64_t after = w.tile_seg + (batch ? 4 * (n_sub + 1) : 0);
    w.records = (after + 255) / 256 * 256;
    w.rec_slots = std::max<uint64_t>(len / 8, 4096);
    const uint64_t rec_bytes = batch ? 16 : 4;
    w.total = (w.records + w.rec_slots * rec_bytes + 255) / 256 * 256;
    return w;
}

}  // namespace kern

using namespace kern;


uint64_t workspace_bytes(uint64_t len, bool batch) { return layout_of(len, batch).total; }

uint64_t count_workspace_bytes(uint32_t n_states) { return kHeaderBytes + (4ull * n_states + 255) / 256 * 256; }

int launch_scan(const ScanLaunch &L) {
    const GlopDevAutomaton &A = *L.A;
    const bool batch = L.seg != nullptr;
    const bool count = L.hist != nullptr;  // count-only mode (single buffer): hits per state, no records
    if (count && batch) return 1;
    // several automata (batches only): na groups, automaton ga(g) for group g
    const uint32_t ng = L.n_groups;
    if (ng && (!batch || ng > kMaxBatchGroups || !L.group_A || !L.group_start)) return 1;
    const uint32_t na = ng ? ng : 1;
    auto ga = [&](uint32_t g) -> const GlopDevAutomaton & { return ng ? L.group_A[g] : A; };
    const uint64_t own_len = L.own_len ? std::min(L.own_len, L.len) : L.len;
    if (batch && own_len != L.len) return 1;
    const uint64_t n_sub = (own_len + SUB - 1) / SUB;
    const WsLayout W = layout_of(L.len, batch);
    if (L.ws_bytes < (count ? count_workspace_bytes(A.n_states) : W.total)) return 2;
    uint8_t *ws = reinterpret_cast<uint8_t *>(L.ws);
    uint32_t *hdr = reinterpret_cast<uint32_t *>(ws);
    uint32_t *hits = count ? reinterpret_cast<uint32_t *>(ws + kHeaderBytes) : nullptr;
    if (count && (cudaMemsetAsync(L.hist, 0, 8ull * A.n_patterns, L.stream) != cudaSuccess ||
                  cudaMemsetAsync(L.d_count, 0, 8, L.stream) != cudaSuccess ||
                  cudaMemsetAsync(hits, 0, 4ull * A.n_states, L.stream) != cudaSuccess))
        return 4;
    uint32_t all_patterns = 0;
    for (uint32_t g = 0; g < na; ++g) all_patterns += ga(g).n_patterns ? 1u : 0u;
    const bool nothing = all_patterns == 0 || n_sub == 0 || (batch && L.n_seg == 0);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 4;
    const DevProps pr = props_of(dev);
    if (!pr.sms || !pr.coop) return 4;

    // header: cleared first when the segment check below sets flags in it
    if (batch && cudaMemsetAsync(hdr, 0, kHeaderBytes, L.stream) != cudaSuccess) return 4;
    {
        const uint64_t work = std::max<uint64_t>(n_sub + 1, batch ? L.n_seg : 0);
        uint32_t blocks = (uint32_t)std::min<uint64_t>((work + 255) / 256, (uint64_t)pr.sms * 8);
        if (blocks == 0) blocks = 1;
        GroupStarts gs{};
        gs.n = ng;
        for (uint32_t g = 0; g <= ng && ng; ++g) gs.start[g] = L.group_start[g];
        init_kernel<<<blocks, 256, 0, L.stream>>>(hdr, reinterpret_cast<uint32_t *>(ws + W.tile_seg), nothing ? 0 : n_sub,
                                                   batch ? L.seg : nullptr, batch ? L.n_seg : 0, L.len,
                                                   reinterpret_cast<unsigned long long *>(L.d_count), batch ? 0 : 1,
                                                   nothing ? 1 : 0, gs);
        if (cudaGetLastError() != cudaSuccess) return 4;
    }
    if (nothing) {
        // a piece with nothing to scan still passes its output base on
        if (L.d_next_base) {
            const cudaError_t e = L.d_obase ? cudaMemcpyAsync(L.d_next_base, L.d_obase, 8, cudaMemcpyDeviceToDevice, L.stream)
                                            : cudaMemsetAsync(L.d_next_base, 0, 8, L.stream);
            if (e != cudaSuccess) return 4;
        }
        return 0;
    }

    KParams kp;
    kp.A = A;
    kp.text = L.text;
    kp.len = L.len;
    kp.own_len = own_len;
    kp.base_off = L.base_off;
    kp.d_obase = L.d_obase;
    kp.d_next_base = L.d_next_base;
    kp.seg = L.seg;
    kp.n_seg = L.n_seg;
    kp.out = L.out;
    kp.cap = L.capacity;
    kp.d_count = reinterpret_cast<unsigned long long *>(L.d_count);
    kp.hdr = hdr;
    // (count-only mode uses none of the descriptors, sums or records: its workspace is the header and hits)
    kp.desc = count ? nullptr : reinterpret_cast<SubDesc *>(ws + W.desc);
    kp.sums = count ? nullptr : reinterpret_cast<unsigned long long *>(ws + W.sums);
    kp.tile_seg = count ? nullptr : reinterpret_cast<const uint32_t *>(ws + W.tile_seg);
    kp.records = count ? nullptr : reinterpret_cast<uint32_t *>(ws + W.records);
    kp.state_hits = hits;
    kp.n_sub = n_sub;
    uint32_t max_len = 0;
    for (uint32_t g = 0; g < na; ++g) max_len = std::max(max_len, ga(g).max_len);
    uint32_t halo = max_len > 1 ? max_len - 1 : 0;
    halo = std::max<uint32_t>(16, align_up(std::min(halo, HALO_CAP), 16));
    kp.halo = halo;
    kp.aligned = (reinterpret_cast<uintptr_t>(L.text) & 15) == 0;
    kp.spin_budget = 4000000000ll;  // about 2 s of SM clock
    // Failure-detection tests make a bounded wait run out on purpose: GLOP_TEST_BARRIER_EXTRA=k makes the
    // grid barriers wait for k blocks that do not exist, GLOP_TEST_SPIN_BUDGET shortens every wait (cycles).
    kp.barrier_extra = 0;
    kp.withhold_chunk = ~0ull;
    if (const char *e = std::getenv("GLOP_TEST_WITHHOLD_CHUNK")) kp.withhold_chunk = std::strtoull(e, nullptr, 10);
    if (const char *e = std::getenv("GLOP_TEST_BARRIER_EXTRA")) kp.barrier_extra = (uint32_t)std::strtoul(e, nullptr, 10);
    if (const char *e = std::getenv("GLOP_TEST_SPIN_BUDGET")) kp.spin_budget = std::strtoll(e, nullptr, 10);

    // shared memory: class map, bitmap, gram table, block state, ring, hot rows.
    // The ring has 3 slots, or 2 when that is what lets every walked dense row stay on chip.
    // (several automata: one layout for every group -- the largest bitmap and gram table -- and each
    // group's hot rows in what is left)
    const uint32_t budget = (uint32_t)pr.smem_optin;
    auto row_bytes_of = [&](uint32_t g) { return ga(g).n_classes * (ga(g).row16 ? 2u : 4u); };
    auto hot_avail_of = [&](uint32_t g) { return ga(g).n_dense > ga(g).hot_lo ? ga(g).n_dense - ga(g).hot_lo : 0u; };
    const uint32_t row_bytes = row_bytes_of(0);
    const uint32_t hot_avail = hot_avail_of(0);
    uint32_t bitmap_bytes = 0, gram_bytes = 0;
    for (uint32_t g = 0; g < na; ++g) {
        const GlopDevAutomaton &B = ga(g);
        if (B.gram_len) {
            bitmap_bytes = std::max(bitmap_bytes, (1u << B.bm_log2) / 8);
            gram_bytes = std::max(gram_bytes, (1u << B.ht_log2) * (B.gram_len == 4 ? 8u : 16u));
        }
    }
    bool rows_short = false;  // some group's walked dense rows do not all fit on chip
    auto carve = [&](uint32_t nstage) -> uint32_t {
        kp.nstage = nstage;
        uint32_t off = 384;
        kp.off_bitmap = off;
        off += bitmap_bytes;
        off = align_up(off, 128);
        kp.off_grams = off;
        const uint32_t fixed_after = align_up((uint32_t)sizeof(CtaMisc), 128) + nstage * kp.slot_bytes + 32 * QBYTES +
                                     (count ? 8 * HCACHE : 0);
        kp.grams_in_smem = (gram_bytes && gram_bytes <= 32768 && off + gram_bytes + fixed_after <= budget) ? 1u : 0u;
        if (kp.grams_in_smem) off += gram_bytes;
        off = align_up(off, 128);
        kp.off_misc = off;
        off += align_up((uint32_t)sizeof(CtaMisc), 128);
        kp.off_ring = off;
        off += nstage * kp.slot_bytes;
        kp.off_q = off;
        off += 32 * QBYTES;
        off = align_up(off, 128);
        kp.off_hc = off;
        if (count) off += 8 * HCACHE;
        kp.off_rows = off;
        uint32_t avail = budget > off + 32 ? budget - off - 32 : 0;
        if (L.smem_budget) avail = std::min(avail, L.smem_budget);
        kp.hot_n = std::min<uint32_t>(hot_avail, row_bytes ? avail / row_bytes : 0);
        uint32_t rows_max = kp.hot_n * row_bytes;
        rows_short = kp.hot_n < hot_avail;
        for (uint32_t g = 0; g < ng; ++g) {
            const uint32_t rb = row_bytes_of(g), h = std::min<uint32_t>(hot_avail_of(g), rb ? avail / rb : 0);
            kp.grp.hot_n[g] = h;
            kp.grp.grams_in_smem[g] = ga(g).gram_len ? kp.grams_in_smem : 0u;
            rows_max = std::max(rows_max, h * rb);
            rows_short = rows_short || h < hot_avail_of(g);
        }
        off += align_up(rows_max + 16, 16);
        return off;
    };
    // (3 slots unless 2 let every walked dense row on chip, or 3 do not fit beside the tables at all)
    auto carve_ring = [&](uint32_t ksub) -> uint32_t {
        kp.ksub = ksub;
        kp.slot_bytes = align_up(CHUNK * ksub + halo + 64, 128);
        uint32_t smem = carve(NSTAGE);
        if ((rows_short && !L.smem_budget) || smem > budget) {
            const uint32_t smem2 = carve(2);
            if ((rows_short || smem2 > budget) && smem <= budget) smem = carve(NSTAGE);
            else smem = smem2;
        }
        return smem;
    };
    // 62 KiB chunks when asked for, the walks stay within the staged halo (no DEEP) and two such ring
    // slots fit beside the tables; else 31 KiB
    const bool deep = max_len > 1 && max_len - 1 > halo;
    uint32_t smem = carve_ring(L.ksub == 2 && !deep && !ng ? 2u : 1u);
    if (smem > budget && kp.ksub == 2) smem = carve_ring(1);
    if (smem > budget) return 7;
    const uint64_t n_chunks = (n_sub + NCONS * kp.ksub - 1) / (NCONS * kp.ksub);
    kp.n_chunks = n_chunks;
    if (L.ksub_used) *L.ksub_used = kp.ksub;
    if (PB * 8 > kp.nstage * kp.slot_bytes) return 7;
    const uint32_t max_grid = (uint32_t)std::min(pr.sms, (int)kMaxGrid);
    uint32_t grid = (uint32_t)std::min<uint64_t>(n_chunks, (uint64_t)max_grid);
    if (grid == 0) grid = 1;
    kp.grp.n = ng;
    if (ng) {
        // group g: sub-tiles [sub[g], sub[g + 1]) and blocks [blk[g], blk[g + 1]), at least one block each,
        // the rest shared in proportion to the groups' chunks
        uint64_t gch[kMaxBatchGroups], tot = 0;
        for (uint32_t g = 0; g < ng; ++g) {
            kp.grp.A[g] = L.group_A[g];
            kp.grp.sub[g] = L.group_start[g] / SUB;
            gch[g] = (L.group_start[g + 1] - L.group_start[g] + CHUNK - 1) / CHUNK;
            tot += gch[g];
        }
        kp.grp.sub[ng] = n_sub;
        grid = (uint32_t)std::max<uint64_t>(ng, std::min<uint64_t>(tot, max_grid));
        if (grid > max_grid) return 1;
        uint32_t extra = grid - ng, given = 0, nb[kMaxBatchGroups];
        for (uint32_t g = 0; g < ng; ++g) {
            nb[g] = 1 + (tot ? (uint32_t)(gch[g] * extra / tot) : 0u);
            given += nb[g];
        }
        for (uint32_t g = 0; given < grid; g = (g + 1) % ng) { ++nb[g]; ++given; }
        kp.grp.blk[0] = 0;
        for (uint32_t g = 0; g < ng; ++g) kp.grp.blk[g + 1] = kp.grp.blk[g] + nb[g];
    }
    kp.rec_cap_cta = (uint32_t)std::min<uint64_t>(W.rec_slots / grid, 0xFFFFFFF0ull / grid);
    // a single-buffer record holds the terminal state in 22 bits: larger automata keep no records (phase B
    // walks every sub-tile again)
    if (!batch && A.n_states >= (1u << 22)) kp.rec_cap_cta = 0;
    kp.rec_slots = W.rec_slots;

    const bool r16 = A.row16 != 0;
    auto dispatch = [&]() -> int {
        const bool multi = ng != 0;
        if (A.gram_len == 0) return launch_f0(kp, smem, grid, L.stream, batch, r16, deep, kp.ksub, multi);
        if (A.gram_len == 4) return launch_f4(kp, smem, grid, L.stream, batch, r16, deep, kp.ksub, multi);
        return launch_f8(kp, smem, grid, L.stream, batch, r16, deep, kp.ksub, multi);
    };
    const int rc = dispatch();
    if (rc || !count) return rc;
    // count-only mode: spread each state's hits over its output list
    const uint32_t cb = (uint32_t)std::min<uint64_t>((A.n_states + 255) / 256, (uint64_t)pr.sms * 8);
    count_lists_kernel<<<cb ? cb : 1, 256, 0, L.stream>>>(kp.state_hits, A.cum_off, A.cum_ids, A.n_states, L.hist,
                                                          reinterpret_cast<unsigned long long *>(L.d_count));
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

}  // namespace glop
