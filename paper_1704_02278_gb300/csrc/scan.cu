// scan.cu -- the GB300 scan kernels.
//
// One walk of the failureless trie starts at every text offset (Sec. 5: one
// thread per character, a mismatch ends the walk).  Here a thread block is a
// persistent set of independent "groups" of 256 threads; a group takes 4 KiB
// tiles of the text from a global ticket counter and, per tile:
//
//  1. the tile plus a halo of at least (longest pattern - 1) bytes arrives in
//     shared memory by a TMA bulk copy issued one tile ahead (double buffer);
//     the halo is the chunk overlap of Sec. 4, so no match is lost at a tile
//     boundary, and a tile only reports matches that start inside it;
//  2. each thread takes 16 consecutive start offsets, reads their bytes from
//     two 16-byte shared-memory vectors and tests the first gram_len bytes of
//     every offset against a bitmap of pattern prefixes (start filter);
//  3. surviving offsets are compacted per warp (ballot-free prefix sums of
//     popc) into a queue in offset order and walked densely: gram table ->
//     state at depth gram_len, then dense rows (hot rows in shared memory,
//     the rest through the read-only path from L2) and unary chains matched
//     by 4-byte comparisons; the deepest terminal state of the walk names the
//     sorted list of every pattern found at that offset (nested patterns);
//  4. per-thread match counts are scanned in the group, the tile's global
//     output position comes from a decoupled look-back over tile order, and
//     every thread writes its matches in (offset, pattern id) order.
//
// There is no failure transition anywhere (Sec. 4 explains why they diverge
// on SIMT hardware) and no floating point.  Every spin wait is bounded by a
// clock budget; running out sets a flag in the workspace header.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "glop_hash.h"
#include "scan.h"

namespace glop {

namespace {

constexpr uint32_t GT = kGroupThreads;
constexpr uint32_t KOFF = kOffsetsPerThread;
constexpr uint32_t TILE = kTile;
constexpr uint32_t WARPS_G = GT / 32;
constexpr uint32_t SEGCAP = 128;
constexpr uint32_t HALO_CAP = 1024;
constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr unsigned long long FLAG_AGG = 1ull << 62, FLAG_PRE = 2ull << 62, VAL_MASK = (1ull << 62) - 1;

struct GroupMisc {
    unsigned long long mbar[2];
    unsigned long long base;
    unsigned long long tick[2];
    uint32_t abort, seg_a, seg_L, seg_fallback;
};

struct KParams {
    GlopDevAutomaton A;
    const uint8_t *text;
    uint64_t len;
    const uint64_t *seg;
    uint32_t n_seg;
    void *out;
    uint64_t cap;
    unsigned long long *d_count;
    uint32_t *hdr;
    unsigned long long *tstat;
    const uint32_t *tile_seg;
    uint64_t n_tiles;
    uint32_t halo, tbuf, hot_n, grams_in_smem, ngroups, aligned;
    uint32_t off_bitmap, off_grams, off_rows, off_groups, group_bytes;
    long long spin_budget;
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// one bulk copy global -> shared completing on bar; bytes multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void tma_load(void *dst, const void *src, uint32_t bytes, unsigned long long *bar) {
    if (bytes) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_addr(dst)),
            "l"(src), "r"(bytes), "r"(smem_addr(bar))
            : "memory");
    } else {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
    }
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; false when the budget ran out
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, long long budget) {
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > budget) return false;
    return true;
}

__device__ __forceinline__ void group_bar(uint32_t id) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(GT) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_relaxed32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long shfl_up64(unsigned long long v, int d) {
    uint32_t lo = __shfl_up_sync(FULL, (uint32_t)v, d), hi = __shfl_up_sync(FULL, (uint32_t)(v >> 32), d);
    return ((unsigned long long)hi << 32) | lo;
}

__device__ __forceinline__ unsigned long long shfl_xor64(unsigned long long v, int d) {
    uint32_t lo = __shfl_xor_sync(FULL, (uint32_t)v, d), hi = __shfl_xor_sync(FULL, (uint32_t)(v >> 32), d);
    return ((unsigned long long)hi << 32) | lo;
}

// largest k in [0, L] with e[k] <= x (e sorted, e[0] <= x assumed by the caller or k = 0)
__device__ __forceinline__ uint32_t seg_find_smem(const unsigned long long *e, uint32_t L, unsigned long long x) {
    uint32_t lo = 0, hi = L;  // invariant: answer in [lo, hi]
    while (lo < hi) {
        uint32_t mid = (lo + hi + 1) >> 1;
        if (e[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ uint32_t seg_find_global(const uint64_t *seg, uint32_t lo, uint32_t hi, uint64_t x) {
    while (lo < hi) {
        uint32_t mid = (lo + hi + 1) >> 1;
        if (__ldg((const unsigned long long *)seg + mid) <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------- the walk
struct TileView {
    const uint8_t *buf;      // staged bytes of the tile (shared memory)
    const uint8_t *gtext;    // the same bytes in global memory (text + tile start)
    uint32_t n_stage;        // staged bytes
};

__device__ __forceinline__ uint32_t tile_byte(const TileView &v, uint32_t pos) {
    return pos < v.n_stage ? (uint32_t)v.buf[pos] : (uint32_t)__ldg(v.gtext + pos);
}

// 4 text bytes starting at pos (little-endian); bytes past the staged region
// come from global memory one by one (patterns longer than the halo)
__device__ __forceinline__ uint32_t tile_word(const TileView &v, uint32_t pos, uint32_t end) {
    if (pos + 8 <= v.n_stage) {
        const uint32_t *b32 = (const uint32_t *)v.buf;
        uint32_t a = pos >> 2;
        return __funnelshift_r(b32[a], b32[a + 1], 8 * (pos & 3));
    }
    uint32_t w = 0;
    for (uint32_t k = 0; k < 4 && pos + k < end; ++k) w |= tile_byte(v, pos + k) << (8 * k);
    return w;
}

// 4 chain bytes starting at chain_bytes[o] (the array is padded by 8 zero bytes)
__device__ __forceinline__ uint32_t chain_word(const uint8_t *cb, uint32_t o) {
    const uint32_t *c32 = (const uint32_t *)cb;
    uint32_t a = o >> 2;
    return __funnelshift_r(__ldg(c32 + a), __ldg(c32 + a + 1), 8 * (o & 3));
}

// Deepest terminal state reached from state s, next text byte at tile position
// pos, walk bounded by end (segment end / text end, tile relative).
__device__ uint32_t walk(const GlopDevAutomaton &A, const uint8_t *cls_s, const int32_t *rows_s, uint32_t hot_n,
                         const TileView &v, uint32_t s, uint32_t pos, uint32_t end, uint32_t t) {
    const uint32_t C = A.n_classes;
    while (true) {
        if (s < A.n_dense) {
            if (pos >= end) return t;
            uint32_t cl = cls_s[tile_byte(v, pos)];
            uint32_t r = s - A.hot_lo;
            int32_t e = (r < hot_n) ? rows_s[r * C + cl] : __ldg(A.rows + (size_t)s * C + cl);
            if (!e) return t;
            s = (uint32_t)e & GLOP_STATE_MASK;
            ++pos;
            if ((uint32_t)e & GLOP_TERM) t = s;
        } else {
            const uint4 ch = __ldg(reinterpret_cast<const uint4 *>(A.chain) + (s - A.n_dense));
            const uint32_t off = ch.x, rem = ch.y, exitv = ch.z;
            const uint32_t lim = min(rem, end - pos);
            uint32_t m = 0;
            while (m < lim) {
                uint32_t x = tile_word(v, pos + m, end) ^ chain_word(A.chain_bytes, off + m);
                if (x) { m += (uint32_t)(__ffs(x) - 1) >> 3; break; }
                m += 4;
            }
            m = min(m, lim);
            const uint32_t nchain = rem - (exitv ? 1u : 0u);
            if (exitv && m == rem) {
                uint32_t tt = __ldg(&A.chain[s + nchain - A.n_dense].term);
                if (tt) t = tt;
                s = exitv & GLOP_STATE_MASK;
                if (exitv & GLOP_TERM) t = s;
                pos += m;
                continue;
            }
            uint32_t tt = __ldg(&A.chain[s + min(m, nchain) - A.n_dense].term);
            return tt ? tt : t;
        }
    }
}

// ---------------------------------------------------------------- look-back
// Exclusive prefix of tile k's match count over all earlier tiles (decoupled
// look-back over tile order; tiles are claimed in increasing order so every
// predecessor is owned by a running group).  Called by one full warp.
__device__ unsigned long long lookback(unsigned long long *tstat, uint64_t k, unsigned long long agg, int lane,
                                       long long budget, uint32_t *hdr) {
    if (k == 0) {
        if (lane == 0) st_relaxed(&tstat[0], FLAG_PRE | agg);
        return 0;
    }
    if (lane == 0) st_relaxed(&tstat[k], FLAG_AGG | agg);
    unsigned long long excl = 0;
    long long j = (long long)k - 1;
    bool timed_out = false;
    while (true) {
        long long idx = j - lane;
        unsigned long long v = FLAG_PRE;  // before tile 0: prefix 0
        if (idx >= 0) {
            long long t0 = clock64();
            while (true) {
                v = ld_relaxed(&tstat[idx]);
                if (v >> 62) break;
                if (clock64() - t0 > budget) { timed_out = true; v = FLAG_PRE; break; }
            }
        }
        unsigned pm = __ballot_sync(FULL, (v >> 62) == 2ull);
        int last = pm ? __ffs(pm) - 1 : 31;
        unsigned long long val = (lane <= last) ? (v & VAL_MASK) : 0ull;
        for (int d = 16; d; d >>= 1) val += shfl_xor64(val, d);
        excl += val;
        if (pm) break;
        j -= 32;
    }
    if (__any_sync(FULL, timed_out) && lane == 0) atomicOr(hdr, WS_TIMEOUT);
    if (lane == 0) st_relaxed(&tstat[k], FLAG_PRE | (excl + agg));
    return excl;
}

// ---------------------------------------------------------------- kernels
// Zero the tile status words and the header; for batches, check the segment
// table and find the first segment of every tile.
__global__ void init_kernel(uint32_t *hdr, unsigned long long *tstat, uint32_t *tile_seg, uint64_t n_tiles,
                            const uint64_t *seg, uint32_t n_seg, uint64_t len, unsigned long long *d_count,
                            int zero_header) {
    uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    if (zero_header && tid < kHeaderBytes / 4) hdr[tid] = 0;
    for (uint64_t k = tid; k < n_tiles; k += nthr) tstat[k] = 0ull;
    if (n_tiles == 0 && tid == 0) *d_count = 0ull;
    if (!seg) return;
    bool bad = false;
    for (uint64_t s = tid; s < n_seg; s += nthr) {
        uint64_t a = seg[s], b = seg[s + 1];
        if (b < a || b - a > 0xFFFFFFFFull || b > len) bad = true;
    }
    if (bad) {
        atomicOr(hdr, WS_EINVAL);
        *d_count = 0ull;
    }
    // tile_seg[k] = last segment whose start <= k * TILE (0 if none), k in [0, n_tiles]
    for (uint64_t k = tid; k <= n_tiles; k += nthr) {
        uint64_t x = k * TILE;
        uint32_t lo = 0, hi = n_seg;  // answer in [lo, hi]
        while (lo < hi) {
            uint32_t mid = (lo + hi + 1) >> 1;
            if (seg[mid] <= x) lo = mid; else hi = mid - 1;
        }
        tile_seg[k] = lo;
    }
}

template <int FILT, bool BATCH>
__global__ void __launch_bounds__(1024, 1) scan_kernel(const KParams p) {
    extern __shared__ __align__(128) uint8_t smem[];
    const GlopDevAutomaton &A = p.A;
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    if (BATCH && (ld_relaxed32(p.hdr) & WS_EINVAL)) return;

    // ---- stage the shared tables (class map, start filter, gram table, hot rows) ----
    uint8_t *cls_s = smem;
    uint32_t *fb_s = reinterpret_cast<uint32_t *>(smem + 256);
    uint32_t *bm_s = reinterpret_cast<uint32_t *>(smem + p.off_bitmap);
    GlopGramSlot *gr_s = reinterpret_cast<GlopGramSlot *>(smem + p.off_grams);
    int32_t *rows_s = reinterpret_cast<int32_t *>(smem + p.off_rows);
    {
        if (tid < 64) reinterpret_cast<uint32_t *>(cls_s)[tid] = __ldg(reinterpret_cast<const uint32_t *>(A.cls) + tid);
        if (tid < 8) fb_s[tid] = 0;
        if (FILT) {
            const uint4 *src = reinterpret_cast<const uint4 *>(A.bitmap);
            uint4 *dst = reinterpret_cast<uint4 *>(bm_s);
            for (uint32_t i = tid; i < (1u << A.bm_log2) / 128; i += nthr) dst[i] = __ldg(src + i);
            if (p.grams_in_smem) {
                const uint4 *gs = reinterpret_cast<const uint4 *>(A.grams);
                uint4 *gd = reinterpret_cast<uint4 *>(gr_s);
                for (uint32_t i = tid; i < (1u << A.ht_log2); i += nthr) gd[i] = __ldg(gs + i);
            }
        }
        const uint32_t nrow = p.hot_n * A.n_classes;
        const int32_t *rsrc = A.rows + (size_t)A.hot_lo * A.n_classes;
        for (uint32_t i = tid; i < nrow; i += nthr) rows_s[i] = __ldg(rsrc + i);
    }
    __syncthreads();
    if (!FILT) {
        // bytes that start some pattern: the initial state has a transition on them
        if (tid < 256) {
            uint32_t e = (uint32_t)__ldg(A.rows + cls_s[tid]);
            if (e) atomicOr(&fb_s[tid >> 5], 1u << (tid & 31));
        }
        __syncthreads();
    }
    const GlopGramSlot *grams = p.grams_in_smem ? gr_s : A.grams;

    // ---- group setup ----
    const uint32_t gid = tid / GT, gtid = tid % GT, lane = tid & 31, warp_g = gtid >> 5;
    const uint32_t bar_id = gid + 1;
    uint8_t *G = smem + p.off_groups + gid * p.group_bytes;
    uint32_t *res = reinterpret_cast<uint32_t *>(G + 2 * p.tbuf);
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(res + TILE);
    unsigned long long *wsum = cnt + GT;
    unsigned long long *segl = wsum + WARPS_G;
    GroupMisc *gm = reinterpret_cast<GroupMisc *>(segl + SEGCAP + 1);

    auto issue = [&](uint64_t k, int bb) {
        uint64_t s0 = k * TILE;
        uint64_t n_stage = min((uint64_t)(TILE + p.halo), p.len - s0);
        uint32_t bytes = p.aligned ? (uint32_t)(n_stage & ~15ull) : 0u;
        tma_load(G + bb * p.tbuf, p.text + s0, bytes, &gm->mbar[bb]);
    };

    if (gtid == 0) {
        mbar_init(&gm->mbar[0], 1);
        mbar_init(&gm->mbar[1], 1);
        fence_barrier_init();
        gm->abort = 0;
        unsigned long long k0 = atomicAdd(reinterpret_cast<unsigned long long *>(p.hdr + 2), 1ull);
        gm->tick[0] = k0;
        if (k0 < p.n_tiles) issue(k0, 0);
    }
    group_bar(bar_id);

    const uint32_t g = A.gram_len;
    const uint32_t w1mask = FILT == 8 ? glop_w1_mask(g) : 0u;
    const uint32_t bsh = 32u - A.bm_log2;
    const uint32_t htmask = (1u << A.ht_log2) - 1u;
    uint32_t phase = 0;
    int b = 0;
    bool pending_other = false;
    while (true) {
        const uint64_t k = gm->tick[b];
        if (k >= p.n_tiles) break;
        if (gtid == 0) {
            unsigned long long k1 = atomicAdd(reinterpret_cast<unsigned long long *>(p.hdr + 2), 1ull);
            gm->tick[b ^ 1] = k1;
            if (k1 < p.n_tiles) issue(k1, b ^ 1);
        }
        pending_other = true;
        const uint64_t s0 = k * TILE;
        const uint32_t n_stage = (uint32_t)min((uint64_t)(TILE + p.halo), p.len - s0);
        const uint32_t tile_len = min(TILE, n_stage);
        uint8_t *buf = G + b * p.tbuf;
        // bytes the bulk copy does not cover (unaligned tail, or everything when the text is unaligned)
        {
            uint32_t done = p.aligned ? (n_stage & ~15u) : 0u;
            for (uint32_t y = done + gtid; y < n_stage; y += GT) buf[y] = __ldg(p.text + s0 + y);
        }
        if (!mbar_wait(&gm->mbar[b], (phase >> b) & 1u, p.spin_budget)) {
            atomicOr(p.hdr, WS_TIMEOUT);
            gm->abort = 1;
        }
        phase ^= 1u << b;
        if (BATCH && gtid == 0) {
            uint32_t a = __ldg(p.tile_seg + k), e = __ldg(p.tile_seg + k + 1) + 1;
            if (e > p.n_seg) e = p.n_seg;
            uint32_t L = e - a;
            gm->seg_a = a;
            gm->seg_L = L;
            gm->seg_fallback = L > SEGCAP;
            if (L <= SEGCAP)
                for (uint32_t x = 0; x <= L; ++x) segl[x] = __ldg((const unsigned long long *)p.seg + a + x);
        }
        group_bar(bar_id);
        if (gm->abort) break;

        // segment of an absolute offset: (index, start, end); false outside every segment
        auto seg_of = [&](uint64_t iabs, uint32_t &si, uint64_t &sstart, uint64_t &send) -> bool {
            if (!BATCH) { si = 0; sstart = 0; send = p.len; return true; }
            const uint32_t a = gm->seg_a, L = gm->seg_L;
            uint32_t kk;
            if (!gm->seg_fallback) {
                if (segl[0] > iabs) return false;
                kk = seg_find_smem(segl, L, iabs);
                if (kk >= L) return false;
                sstart = segl[kk];
                send = segl[kk + 1];
            } else {
                if (__ldg((const unsigned long long *)p.seg + a) > iabs) return false;
                kk = seg_find_global(p.seg, a, a + L, iabs) - a;
                if (kk >= L) return false;
                sstart = __ldg((const unsigned long long *)p.seg + a + kk);
                send = __ldg((const unsigned long long *)p.seg + a + kk + 1);
            }
            si = a + kk;
            return iabs < send;
        };

        // ---- 2. start filter over 16 consecutive offsets ----
        uint32_t mask = 0;
        {
            const uint4 *b4 = reinterpret_cast<const uint4 *>(buf);
            const uint4 v0 = b4[gtid], v1 = b4[gtid + 1];
            const uint32_t x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
            for (int j = 0; j < (int)KOFF; ++j) {
                uint32_t bit;
                if (FILT) {
                    uint32_t w0 = __funnelshift_r(x[j >> 2], x[(j >> 2) + 1], 8 * (j & 3));
                    uint32_t h = w0 * GLOP_HASH_M0;
                    if (FILT == 8) {
                        uint32_t w1 = __funnelshift_r(x[(j >> 2) + 1], x[(j >> 2) + 2], 8 * (j & 3)) & w1mask;
                        h ^= w1 * GLOP_HASH_M1;
                    }
                    uint32_t bi = h >> bsh;
                    bit = (bm_s[bi >> 5] >> (bi & 31)) & 1u;
                } else {
                    uint32_t by = (x[j >> 2] >> (8 * (j & 3))) & 0xFFu;
                    bit = (fb_s[by >> 5] >> (by & 31)) & 1u;
                }
                mask |= bit << j;
            }
            const uint32_t first = gtid * KOFF;
            if (first + KOFF > tile_len) mask &= (first >= tile_len) ? 0u : ((1u << (tile_len - first)) - 1u);
        }

        // ---- 3. per-warp queue of surviving offsets, in offset order ----
        const uint32_t nsurv = __popc(mask);
        uint32_t incl = nsurv;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t vv = __shfl_up_sync(FULL, incl, d);
            if (lane >= (uint32_t)d) incl += vv;
        }
        const uint32_t qpos = incl - nsurv;
        const uint32_t qtotal = __shfl_sync(FULL, incl, 31);
        uint32_t *q = res + warp_g * (32 * KOFF);
        {
            uint32_t m = mask, at = qpos;
            while (m) {
                int bb = __ffs(m) - 1;
                m &= m - 1;
                q[at++] = gtid * KOFF + bb;
            }
        }
        cnt[gtid] = 0ull;
        __syncwarp();

        TileView view{buf, p.text + s0, n_stage};
        for (uint32_t qi = lane; qi < qtotal; qi += 32) {
            const uint32_t off = q[qi];
            uint32_t tres = 0;
            uint32_t si;
            uint64_t sstart, send;
            if (seg_of(s0 + off, si, sstart, send)) {
                uint64_t endr64 = send - s0;
                uint32_t endr = (uint32_t)min(endr64, (uint64_t)0xFFFFFFFFu);
                if (FILT) {
                    if (off + g <= endr) {
                        const uint32_t *b32 = reinterpret_cast<const uint32_t *>(buf);
                        const uint32_t a = off >> 2, sh = 8 * (off & 3);
                        const uint32_t y0 = b32[a], y1 = b32[a + 1];
                        const uint32_t w0 = __funnelshift_r(y0, y1, sh);
                        uint32_t w1 = 0, h = w0 * GLOP_HASH_M0;
                        if (FILT == 8) {
                            w1 = __funnelshift_r(y1, b32[a + 2], sh) & w1mask;
                            h ^= w1 * GLOP_HASH_M1;
                        }
                        uint32_t slot = glop_table_slot(h, A.ht_log2), val = 0;
                        while (true) {
                            const uint4 e = *reinterpret_cast<const uint4 *>(grams + slot);
                            if (!e.z) break;
                            if (e.x == w0 && e.y == w1) { val = e.z; break; }
                            slot = (slot + 1) & htmask;
                        }
                        if (val) {
                            uint32_t s = val & GLOP_STATE_MASK;
                            tres = walk(A, cls_s, rows_s, p.hot_n, view, s, off + g, endr, (val & GLOP_TERM) ? s : 0u);
                        }
                    }
                } else {
                    tres = walk(A, cls_s, rows_s, p.hot_n, view, 0u, off, endr, 0u);
                }
            }
            q[qi] = tres;
            if (tres) {
                unsigned long long c = __ldg(A.cum_off + tres + 1) - __ldg(A.cum_off + tres);
                atomicAdd(&cnt[off / KOFF], c);
            }
        }
        __syncwarp();

        // ---- 4. counts -> group scan -> look-back -> emit ----
        const unsigned long long c = cnt[gtid];
        unsigned long long cincl = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            unsigned long long vv = shfl_up64(cincl, d);
            if (lane >= (uint32_t)d) cincl += vv;
        }
        if (lane == 31) wsum[warp_g] = cincl;
        group_bar(bar_id);
        unsigned long long wpre = 0, ttot = 0;
#pragma unroll
        for (uint32_t w = 0; w < WARPS_G; ++w) {
            unsigned long long vv = wsum[w];
            if (w < warp_g) wpre += vv;
            ttot += vv;
        }
        if (warp_g == 0) {
            unsigned long long ex = lookback(p.tstat, k, ttot, (int)lane, p.spin_budget, p.hdr);
            if (lane == 0) {
                gm->base = ex;
                if (k == p.n_tiles - 1) {
                    unsigned long long total = ex + ttot;
                    *p.d_count = total;
                    *reinterpret_cast<unsigned long long *>(p.hdr + 4) = total;
                    if (total > p.cap) atomicOr(p.hdr, WS_OVERFLOW);
                }
            }
        }
        group_bar(bar_id);
        if (c) {
            unsigned long long o = gm->base + wpre + cincl - c;
            uint32_t m = mask, r = 0;
            while (m && o < p.cap) {
                const int bb = __ffs(m) - 1;
                m &= m - 1;
                const uint32_t tv = q[qpos + r];
                ++r;
                if (!tv) continue;
                const uint32_t lo = __ldg(A.cum_off + tv), hi = __ldg(A.cum_off + tv + 1);
                const uint64_t iabs = s0 + gtid * KOFF + bb;
                if (BATCH) {
                    uint32_t si = 0;
                    uint64_t sstart = 0, send = 0;
                    seg_of(iabs, si, sstart, send);
                    uint32_t *ob = reinterpret_cast<uint32_t *>(p.out);
                    for (uint32_t x = lo; x < hi && o < p.cap; ++x, ++o) {
                        ob[3 * o] = si;
                        ob[3 * o + 1] = (uint32_t)(iabs - sstart);
                        ob[3 * o + 2] = __ldg(A.cum_ids + x);
                    }
                } else {
                    uint2 *ob = reinterpret_cast<uint2 *>(p.out);
                    for (uint32_t x = lo; x < hi && o < p.cap; ++x, ++o)
                        ob[o] = make_uint2((uint32_t)iabs, __ldg(A.cum_ids + x));
                }
            }
        }
        b ^= 1;
        pending_other = false;
    }
    // a bulk copy still in flight into the other buffer (only after an abort): wait for it, bounded
    if (pending_other && gtid == 0 && gm->tick[b ^ 1] < p.n_tiles)
        mbar_wait(&gm->mbar[b ^ 1], (phase >> (b ^ 1)) & 1u, p.spin_budget);
}

// ---------------------------------------------------------------- host side
struct DevProps {
    int sms = 0, smem_optin = 0;
};

DevProps props_of(int dev) {
    static std::mutex mu;
    static DevProps cache[64];
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) return DevProps{};
    if (!cache[dev].sms) {
        cudaDeviceGetAttribute(&cache[dev].sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&cache[dev].smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    }
    return cache[dev];
}

template <int FILT, bool BATCH>
int launch_t(const KParams &kp, uint32_t smem, uint32_t grid, cudaStream_t st) {
    static std::mutex mu;
    static uint32_t set_for[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev >= 0 && dev < 64 && set_for[dev] < smem) {
            if (cudaFuncSetAttribute(scan_kernel<FILT, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem) != cudaSuccess)
                return 4;
            set_for[dev] = smem;
        }
    }
    scan_kernel<FILT, BATCH><<<grid, kp.ngroups * GT, smem, st>>>(kp);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

}  // namespace

uint64_t workspace_bytes(uint64_t len, bool batch) {
    uint64_t n_tiles = (len + TILE - 1) / TILE;
    uint64_t b = kHeaderBytes + 8 * n_tiles;
    if (batch) b += 4 * (n_tiles + 1);
    return (b + 255) / 256 * 256;
}

int launch_scan(const ScanLaunch &L) {
    const GlopDevAutomaton &A = *L.A;
    const bool batch = L.seg != nullptr;
    const uint64_t n_tiles = (L.len + TILE - 1) / TILE;
    if (L.ws_bytes < workspace_bytes(L.len, batch)) return 2;
    uint32_t *hdr = reinterpret_cast<uint32_t *>(L.ws);
    unsigned long long *tstat = reinterpret_cast<unsigned long long *>(reinterpret_cast<uint8_t *>(L.ws) + kHeaderBytes);
    uint32_t *tile_seg = reinterpret_cast<uint32_t *>(tstat + n_tiles);
    const bool nothing = (A.n_patterns == 0) || n_tiles == 0 || (batch && L.n_seg == 0);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 4;
    DevProps pr = props_of(dev);
    if (!pr.sms) return 4;

    // header: cleared first (the segment check below sets flags in it)
    if (batch && cudaMemsetAsync(hdr, 0, kHeaderBytes, L.stream) != cudaSuccess) return 4;
    {
        uint64_t work = std::max<uint64_t>(n_tiles + 1, batch ? L.n_seg : 0);
        uint32_t blocks = (uint32_t)std::min<uint64_t>((work + 255) / 256, (uint64_t)pr.sms * 8);
        if (blocks == 0) blocks = 1;
        init_kernel<<<blocks, 256, 0, L.stream>>>(hdr, tstat, tile_seg, nothing ? 0 : n_tiles,
                                                   batch ? L.seg : nullptr, batch ? L.n_seg : 0, L.len,
                                                   reinterpret_cast<unsigned long long *>(L.d_count), batch ? 0 : 1);
        if (cudaGetLastError() != cudaSuccess) return 4;
    }
    if (nothing) return 0;

    KParams kp;
    kp.A = A;
    kp.text = L.text;
    kp.len = L.len;
    kp.seg = L.seg;
    kp.n_seg = L.n_seg;
    kp.out = L.out;
    kp.cap = L.capacity;
    kp.d_count = reinterpret_cast<unsigned long long *>(L.d_count);
    kp.hdr = hdr;
    kp.tstat = tstat;
    kp.tile_seg = tile_seg;
    kp.n_tiles = n_tiles;
    uint32_t halo = A.max_len > 1 ? A.max_len - 1 : 0;
    halo = std::max<uint32_t>(16, align_up(std::min(halo, HALO_CAP), 16));
    kp.halo = halo;
    kp.tbuf = align_up(TILE + halo, 128);
    kp.aligned = (reinterpret_cast<uintptr_t>(L.text) & 15) == 0;
    kp.spin_budget = 4000000000ll;  // ~2 s of SM clock

    // shared memory: tables first, then the groups
    const uint32_t budget = (uint32_t)pr.smem_optin - 1024;
    uint32_t group_bytes = align_up(2 * kp.tbuf + TILE * 4 + GT * 8 + WARPS_G * 8 + (SEGCAP + 1) * 8 +
                                    (uint32_t)sizeof(GroupMisc), 128);
    uint32_t ngroups = 4;
    uint32_t off = 384;
    kp.off_bitmap = off;
    if (A.gram_len) off += (1u << A.bm_log2) / 8;
    off = align_up(off, 128);
    kp.off_grams = off;
    uint32_t gram_bytes = A.gram_len ? (1u << A.ht_log2) * 16u : 0u;
    const uint32_t groups_total = ngroups * group_bytes;
    kp.grams_in_smem = (A.gram_len && gram_bytes <= 32768 && off + gram_bytes + groups_total <= budget) ? 1u : 0u;
    if (kp.grams_in_smem) off += gram_bytes;
    off = align_up(off, 128);
    kp.off_rows = off;
    const uint32_t row_bytes = A.n_classes * 4;
    uint32_t avail = budget > off + groups_total ? budget - off - groups_total : 0;
    if (L.smem_budget) avail = std::min(avail, L.smem_budget);
    uint32_t hot_avail = A.n_dense > A.hot_lo ? A.n_dense - A.hot_lo : 0;
    kp.hot_n = std::min<uint32_t>(hot_avail, row_bytes ? avail / row_bytes : 0);
    off += kp.hot_n * row_bytes;
    off = align_up(off, 128);
    kp.off_groups = off;
    kp.group_bytes = group_bytes;
    kp.ngroups = ngroups;
    const uint32_t smem = off + groups_total;
    if (smem > (uint32_t)pr.smem_optin) return 7;
    uint64_t want = (n_tiles + ngroups - 1) / ngroups;
    uint32_t grid = (uint32_t)std::min<uint64_t>(want, (uint64_t)pr.sms);
    if (grid == 0) grid = 1;

    if (A.gram_len == 0)
        return batch ? launch_t<0, true>(kp, smem, grid, L.stream) : launch_t<0, false>(kp, smem, grid, L.stream);
    if (A.gram_len == 4)
        return batch ? launch_t<4, true>(kp, smem, grid, L.stream) : launch_t<4, false>(kp, smem, grid, L.stream);
    return batch ? launch_t<8, true>(kp, smem, grid, L.stream) : launch_t<8, false>(kp, smem, grid, L.stream);
}

}  // namespace glop
