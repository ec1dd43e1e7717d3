// scan_kernel.cuh -- the GB300 scan kernel (device code), included by one
// translation unit per start-filter kind (scan_f0.cu, scan_f4.cu, scan_f8.cu)
// so that its instantiations compile in parallel; scan.cu holds the launcher.
//
// One walk of the failureless trie starts at every text offset (Sec. 5: one
// thread per character; a mismatch ends the walk).  The kernel is persistent
// and cooperative (one 1024-thread block per SM) and runs in two phases.
//
// Phase A -- walk.  Warp 0 is a producer: it takes 31 KiB chunks of the text
// (62 KiB when the compile options ask for two sub-tiles per warp) from a
// global ticket counter and brings each, plus a halo of at least (longest
// pattern - 1) bytes, into a 2- or 3-slot shared-memory ring with one TMA bulk
// copy (L2 evict-first: the text is read once).  The halo is the chunk
// overlap of Sec. 4: a chunk reports only matches that start inside it, and
// no match is lost at a boundary.  Warps 1..31 are consumers; consumer w owns
// the w-th 1 KiB sub-tile (or pair of sub-tiles) of every chunk, so consumers
// never wait on each other, only on the ring.  Per sub-tile a lane takes 32 consecutive start
// offsets, reads their bytes from shared memory as 16-byte vectors and tests
// the first gram_len bytes of each against a bitmap of pattern prefixes.
// Survivors are compacted across the warp with shuffles (in offset order) and
// walked 32 at a time: gram table -> state at depth gram_len -> dense rows
// (staged in shared memory when they fit) and unary chains (one 32-byte
// record per step, bytes inline).  The deepest terminal state of a walk names
// the sorted list of all patterns that occur at that offset (nested patterns
// included).  A sub-tile writes 4-byte (state, offset) records into its
// block's scratch slice plus a descriptor (records, match count).
//
// Phase B -- ordered output.  After a grid-wide barrier every block sums the
// match counts of a static range of sub-tiles; after a second barrier each
// block knows where its range starts in the sorted output and expands its
// records into (offset, pattern id) pairs with coalesced warp-wide writes.  A
// sub-tile whose records did not fit the scratch slice is walked again here
// and written directly, so results are exact for any input.
//
// There is no failure transition anywhere (Sec. 4 explains why they diverge
// on SIMT hardware) and no floating point.  Every wait is bounded by a clock
// budget; running out sets a flag in the workspace header.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include "glop_hash.h"
#include "scan.h"

namespace glop {
namespace kern {


constexpr uint32_t SUB = kSubTile;
constexpr uint32_t NCONS = kConsumers;
constexpr uint32_t CHUNK = kChunk;
constexpr uint32_t NSTAGE = 3;  // ring slots at most (a launch uses p.nstage = 2 or 3)
constexpr uint32_t THREADS = 32 * (NCONS + 1);
constexpr uint32_t SEGW = 32;  // segment boundaries kept on chip per sub-tile
constexpr uint32_t HALO_CAP = 1024;
constexpr uint32_t PB = 4096;  // sub-tiles per phase-B piece
constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr unsigned long long END_TICKET = ~0ull;
constexpr uint32_t REC_OVERFLOW = 0xFFFFFFFFu;
constexpr uint32_t QCAP = 128;   // survivors per walk batch of one warp
constexpr uint32_t HCACHE = 1024;  // count-only mode: per-block hit table (state, hits), shared memory
constexpr uint32_t CCAP = 64;    // walks listed for continuation after their first step
// per-warp queue: offsets (u16), states (u32), walk bounds (u32); continuation states (u32), positions (u32), indexes (u8)
constexpr uint32_t QBYTES = QCAP * 10 + CCAP * 9;

struct SubDesc {
    uint32_t rec_start, n_rec;  // absolute record index; n_rec == REC_OVERFLOW: records not stored
    unsigned long long n_match;
};

struct CtaMisc {
    unsigned long long full[NSTAGE], empty[NSTAGE];
    unsigned long long slot_tile[NSTAGE];
    uint32_t slot_nstage[NSTAGE];
    uint32_t rec_cursor;
    uint32_t pad;
    unsigned long long red[32];
    unsigned long long segl[32][SEGW + 1];
    uint32_t seg_a[32], seg_L[32];
    uint32_t slot_seg[NSTAGE][2 * NCONS + 2];  // batches: first segment of each sub-tile of the slot's chunk (+ the next)
    GlopDevAutomaton a_s;  // several automata in one launch: the automaton of this block's group
};

// Several automata in one batch launch (a batch of requests for several
// resident pattern sets): group g is the segments of sub-tiles
// [sub[g], sub[g + 1]) (its bytes start on a sub-tile boundary), scanned with
// automaton A[g] by blocks [blk[g], blk[g + 1]) -- each block stages its own
// group's tables once and takes chunk tickets of that group alone, so no
// block ever switches automata.
constexpr uint32_t kMaxGroups = kMaxBatchGroups;
struct Groups {
    uint32_t n;  // 0: one automaton (KParams::A)
    uint32_t blk[kMaxGroups + 1];
    uint32_t hot_n[kMaxGroups], grams_in_smem[kMaxGroups];
    uint64_t sub[kMaxGroups + 1];
    GlopDevAutomaton A[kMaxGroups];
};

struct KParams {
    GlopDevAutomaton A;
    const uint8_t *text;
    uint64_t len;          // bytes a walk may read
    uint64_t own_len;      // match starts are taken in [0, own_len) (<= len; the rest is look-ahead)
    uint32_t base_off;     // added to every reported offset (single buffer)
    const unsigned long long *d_obase;  // device word: output index of this scan's first match (or null: 0)
    unsigned long long *d_next_base;    // device word: receives that index + this scan's match count (or null)
    const uint64_t *seg;
    uint32_t n_seg;
    void *out;
    uint64_t cap;
    unsigned long long *d_count;
    uint32_t *hdr;
    SubDesc *desc;
    unsigned long long *sums;
    const uint32_t *tile_seg;
    uint32_t *records;
    uint32_t *state_hits;  // count-only mode: matched offsets per terminal state (no records, no phase B)
    uint32_t rec_cap_cta;  // record slots per block
    uint64_t rec_slots;    // record slots in the workspace
    uint64_t n_sub, n_chunks;
    uint32_t ksub;         // sub-tiles each consumer warp takes from a staged chunk (1 or 2): chunks of 31 or 62 KiB
    uint32_t halo, slot_bytes, hot_n, grams_in_smem, aligned, nstage;
    uint32_t off_bitmap, off_grams, off_rows, off_misc, off_ring, off_q, off_hc;
    long long spin_budget;
    uint32_t barrier_extra;  // fault injection for tests: grid barriers wait for this many absent blocks
    unsigned long long withhold_chunk;  // fault injection for tests: this chunk is never staged (~0: none)
    Groups grp;
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// one bulk copy global -> shared completing on bar (16-byte aligned addresses,
// size a multiple of 16); the text is streamed once, so it is evict-first in L2
__device__ __forceinline__ void tma_load(void *dst, const void *src, uint32_t bytes, unsigned long long *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
        "%4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
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

// Wait for the phase with the given parity; false when the clock budget ran out.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, long long budget) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > budget) return false;
    return true;
}

__device__ __forceinline__ uint32_t ld_acquire32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long shfl64(unsigned long long v, int src) {
    uint32_t lo = __shfl_sync(FULL, (uint32_t)v, src), hi = __shfl_sync(FULL, (uint32_t)(v >> 32), src);
    return ((unsigned long long)hi << 32) | lo;
}

__device__ __forceinline__ unsigned long long shfl_up64(unsigned long long v, int d) {
    uint32_t lo = __shfl_up_sync(FULL, (uint32_t)v, d), hi = __shfl_up_sync(FULL, (uint32_t)(v >> 32), d);
    return ((unsigned long long)hi << 32) | lo;
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
    for (int d = 16; d; d >>= 1) {
        uint32_t lo = __shfl_xor_sync(FULL, (uint32_t)v, d), hi = __shfl_xor_sync(FULL, (uint32_t)(v >> 32), d);
        v += ((unsigned long long)hi << 32) | lo;
    }
    return v;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, uint32_t lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t u = __shfl_up_sync(FULL, v, d);
        if (lane >= (uint32_t)d) v += u;
    }
    return v;
}

// the lane holding item i: the largest lane L with excl(L) <= i (excl non-decreasing, excl(0) = 0)
__device__ __forceinline__ uint32_t owner_of(uint32_t excl, uint32_t i) {
    uint32_t o = 0;
#pragma unroll
    for (uint32_t d = 16; d; d >>= 1) {
        const uint32_t e = __shfl_sync(FULL, excl, o + d);
        if (e <= i) o += d;
    }
    return o;
}

// A broken internal invariant: flag it with the site, never touch the memory.
static __device__ __noinline__ void fail_check(uint32_t *hdr, uint32_t site, uint32_t value) {
    if (atomicOr(hdr, WS_INTERNAL) & WS_INTERNAL) return;
    hdr[11] = site;
    hdr[12] = value;
}

// Debug builds (-DGLOP_BOUNDS_CHECK) check every global index against its
// array before the access; a failed check records its site and skips it.
#ifdef GLOP_BOUNDS_CHECK
#define GLOP_CK(hdr, cond, site, val) if (!(cond)) fail_check((hdr), (site), (uint32_t)(val)); else
#define GLOP_BAIL(hdr, cond, site, val, ret) \
    if (!(cond)) { fail_check((hdr), (site), (uint32_t)(val)); return ret; }
#else
#define GLOP_CK(hdr, cond, site, val)
#define GLOP_BAIL(hdr, cond, site, val, ret)
#endif

// bounded grid-wide barrier (the launch is cooperative: every block is resident)
static __device__ void grid_sync(uint32_t *ctr, uint32_t nblocks, long long budget, uint32_t *hdr) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
        long long t0 = clock64();
        while (ld_acquire32(ctr) < nblocks) {
            if (clock64() - t0 > budget) { atomicOr(hdr, WS_TIMEOUT); break; }
            __nanosleep(64);
        }
        __threadfence();
    }
    __syncthreads();
}

// ---------------------------------------------------------------- the walk
struct TextView {
    const uint8_t *buf;    // staged bytes of the sub-tile (shared memory), or nullptr
    const uint8_t *gtext;  // the same bytes in global memory
    uint32_t n_stage;      // bytes available in buf
#ifdef GLOP_BOUNDS_CHECK
    uint64_t avail;        // text bytes from gtext to the end of the text
    uint32_t *hdr;
#endif
};

template <bool DEEP = true>
__device__ __forceinline__ uint32_t tbyte(const TextView &v, uint32_t pos) {
    if (!DEEP || pos < v.n_stage) return v.buf[pos];
    uint32_t r = 0;
    GLOP_CK(v.hdr, pos < v.avail, 20, pos) r = __ldg(v.gtext + pos);
    return r;
}

// 4 text bytes at pos (aligned shared-memory words and a funnel shift)
__device__ __forceinline__ uint32_t tword(const uint32_t *b32, uint32_t pos) {
    const uint32_t a = pos >> 2;
    return __funnelshift_r(b32[a], b32[a + 1], 8 * (pos & 3));
}

// Raw dense-row entry of state s for class cl: uint16 (state | 0x8000 when
// terminal) or int32 (state | GLOP_TERM); 0 when there is no transition.
template <bool ROW16>
__device__ __forceinline__ uint32_t row_entry(const GlopDevAutomaton &A, const void *rows_s, uint32_t hot_n,
                                              uint32_t s, uint32_t cl, uint32_t *hdr) {
    const uint32_t C = A.n_classes;
    (void)hdr;
    GLOP_BAIL(hdr, s < A.n_dense && cl < C, 21, s, 0u)
    const uint32_t r = s - A.hot_lo;
    if (ROW16)
        return (r < hot_n) ? (uint32_t)reinterpret_cast<const uint16_t *>(rows_s)[r * C + cl]
                           : (uint32_t)__ldg(reinterpret_cast<const uint16_t *>(A.rows) + (size_t)s * C + cl);
    return (r < hot_n) ? (uint32_t)reinterpret_cast<const int32_t *>(rows_s)[r * C + cl]
                       : (uint32_t)__ldg(reinterpret_cast<const int32_t *>(A.rows) + (size_t)s * C + cl);
}

// One dense-row transition; returns true when the walk is over.
template <bool ROW16, bool DEEP>
__device__ __forceinline__ bool dense_step(const GlopDevAutomaton &A, const uint8_t *cls_s, const void *rows_s,
                                           uint32_t hot_n, const TextView &v, uint32_t &s, uint32_t &pos,
                                           uint32_t end, uint32_t &t, uint32_t *hdr) {
    if (pos >= end) return true;
    const uint32_t e = row_entry<ROW16>(A, rows_s, hot_n, s, cls_s[tbyte<DEEP>(v, pos)], hdr);
    if (!e) return true;
    constexpr uint32_t TB = ROW16 ? 0x8000u : GLOP_TERM;
    s = e & (TB - 1u);
    ++pos;
    if (e & TB) t = s;
    return false;
}

// One step of a walk from state s with the next text byte at sub-tile
// position pos, never reading at or past end: a dense-row transition when s
// is dense, then one chain piece (up to 16 bytes compared at once) when the
// walk is on a chain, then one more dense transition when the piece exits
// into a dense state.  t is the deepest terminal state passed so far.
// Returns true when the walk is over (t is then final).
template <bool ROW16, bool DEEP>
__device__ __forceinline__ bool step(const GlopDevAutomaton &A, const uint8_t *cls_s, const void *rows_s,
                                     uint32_t hot_n, const TextView &v, uint32_t &s, uint32_t &pos, uint32_t end,
                                     uint32_t &t, uint32_t *hdr) {
#ifdef GLOP_BOUNDS_CHECK
    if (s >= A.n_states) {
        fail_check(hdr, 1, s);
        t = 0;
        return true;
    }
#endif
    if (s < A.n_dense && dense_step<ROW16, DEEP>(A, cls_s, rows_s, hot_n, v, s, pos, end, t, hdr)) return true;
    if (s < A.n_dense) return false;
    const uint4 *rec = reinterpret_cast<const uint4 *>(A.chain) + 2 * (size_t)(s - A.n_dense);
    const uint4 c0 = __ldg(rec), c1 = __ldg(rec + 1);
    const uint32_t exitv = c1.x, term = c1.y, tm = c1.z & 0xFFFFu, rem = (c1.z >> 16) & 0xFFu, nst = c1.z >> 24;
    const uint32_t lim = min(rem, end - pos);
    uint32_t m;
    // Without DEEP every walk stays within its sub-tile's staged bytes plus the
    // halo (longest pattern - 1), and the ring slot has 64 more bytes of room, so
    // the 20 bytes read here are always in the slot; bytes past the text end are
    // stale but never counted (m is capped by end - pos).
    if (!DEEP || pos + 20 <= v.n_stage) {
        const uint32_t *b32 = reinterpret_cast<const uint32_t *>(v.buf) + (pos >> 2);
        const uint32_t sh = 8 * (pos & 3);
        const uint32_t y0 = b32[0], y1 = b32[1], y2 = b32[2], y3 = b32[3], y4 = b32[4];
        // the first differing 32-bit word, then its first differing byte
        uint32_t dw = __funnelshift_r(y0, y1, sh) ^ c0.x, mb = 0;
        if (!dw) { dw = __funnelshift_r(y1, y2, sh) ^ c0.y; mb = 4; }
        if (!dw) { dw = __funnelshift_r(y2, y3, sh) ^ c0.z; mb = 8; }
        if (!dw) { dw = __funnelshift_r(y3, y4, sh) ^ c0.w; mb = 12; }
        m = dw ? mb + ((uint32_t)__clz(__brev(dw)) >> 3) : 16u;
        m = min(m, lim);
    } else {
        m = 0;
        while (m < lim) {
            const uint32_t w = m < 4 ? c0.x : m < 8 ? c0.y : m < 12 ? c0.z : c0.w;
            if (tbyte<DEEP>(v, pos + m) != ((w >> (8 * (m & 3))) & 0xFFu)) break;
            ++m;
        }
    }
    const uint32_t hit = tm & ((2u << min(m, nst)) - 1u);
    if (hit) t = s + 31 - __clz(hit);
    else if (term) t = term;
    if (!exitv || m != rem) return true;
    s = exitv & GLOP_STATE_MASK;
    pos += m;
    if (exitv & GLOP_TERM) t = s;
    if (s < A.n_dense) return dense_step<ROW16, DEEP>(A, cls_s, rows_s, hot_n, v, s, pos, end, t, hdr);
    return false;
}

// (The parameter block is __grid_constant__: with several automata a block
// reads its group's descriptor by address, and that must not copy the
// parameters to local memory.)
template <int FILT, bool BATCH, bool ROW16, bool DEEP, uint32_t KSUB, bool MULTI>
__global__ void __launch_bounds__(THREADS, 1) scan_kernel(const __grid_constant__ KParams p) {
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (BATCH && (ld_acquire32(p.hdr) & WS_EINVAL)) return;
    // this block's automaton: the launch's, or (several automata) its group's, copied to shared memory
    uint32_t grp = 0;
    if (MULTI) {
        while (grp + 1 < p.grp.n && blockIdx.x >= p.grp.blk[grp + 1]) ++grp;
        CtaMisc *m0 = reinterpret_cast<CtaMisc *>(smem + p.off_misc);
        constexpr uint32_t NW = sizeof(GlopDevAutomaton) / 4;
        if (tid < NW) reinterpret_cast<uint32_t *>(&m0->a_s)[tid] = reinterpret_cast<const uint32_t *>(&p.grp.A[grp])[tid];
        __syncthreads();
    }
    const GlopDevAutomaton &A = MULTI ? reinterpret_cast<CtaMisc *>(smem + p.off_misc)->a_s : p.A;
    const uint32_t hot_n = MULTI ? p.grp.hot_n[grp] : p.hot_n;
    const uint32_t grams_in_smem = MULTI ? p.grp.grams_in_smem[grp] : p.grams_in_smem;
    // sub-tiles and chunks of this block's group (the whole text with one automaton)
    const uint64_t sub0 = MULTI ? p.grp.sub[grp] : 0ull, sub_end = MULTI ? p.grp.sub[grp + 1] : p.n_sub;
    const uint64_t n_chunks = MULTI ? (sub_end - sub0 + NCONS * KSUB - 1) / (NCONS * KSUB) : p.n_chunks;
    unsigned long long *ticket = reinterpret_cast<unsigned long long *>(p.hdr + (MULTI ? 16 + 2 * grp : 2));

    uint8_t *cls_s = smem;
    uint32_t *fb_s = reinterpret_cast<uint32_t *>(smem + 256);
    const uint32_t *bm_s = reinterpret_cast<const uint32_t *>(smem + p.off_bitmap);
    // 4-byte grams: the shared-memory copy keeps (key_lo, val) only, 8 bytes a slot
    const GlopGramSlot *grams =
        grams_in_smem ? reinterpret_cast<const GlopGramSlot *>(smem + p.off_grams) : A.grams;
    const uint2 *grams8 = reinterpret_cast<const uint2 *>(smem + p.off_grams);
    const void *rows_s =
        smem + p.off_rows + (((size_t)A.hot_lo * A.n_classes * (ROW16 ? 2u : 4u)) & 15);
    CtaMisc *mc = reinterpret_cast<CtaMisc *>(smem + p.off_misc);
    uint8_t *ring = smem + p.off_ring;

    // ---- stage the tables: class map, start filter, gram table, hot rows ----
    {
        if (tid < 64) reinterpret_cast<uint32_t *>(cls_s)[tid] = __ldg(reinterpret_cast<const uint32_t *>(A.cls) + tid);
        if (p.state_hits)
            for (uint32_t i = tid; i < 2 * HCACHE; i += THREADS) reinterpret_cast<uint32_t *>(smem + p.off_hc)[i] = 0;
        if (tid < 8) fb_s[tid] = 0;
        if (FILT) {
            const uint4 *src = reinterpret_cast<const uint4 *>(A.bitmap);
            uint4 *dst = reinterpret_cast<uint4 *>(smem + p.off_bitmap);
            for (uint32_t i = tid; i < (1u << A.bm_log2) / 128; i += THREADS) dst[i] = __ldg(src + i);
            if (grams_in_smem) {
                const uint4 *gs = reinterpret_cast<const uint4 *>(A.grams);
                if (FILT == 4) {
                    uint2 *gd = reinterpret_cast<uint2 *>(smem + p.off_grams);
                    for (uint32_t i = tid; i < (1u << A.ht_log2); i += THREADS) {
                        const uint4 e = __ldg(gs + i);
                        gd[i] = make_uint2(e.x, e.z);
                    }
                } else {
                    uint4 *gd = reinterpret_cast<uint4 *>(smem + p.off_grams);
                    for (uint32_t i = tid; i < (1u << A.ht_log2); i += THREADS) gd[i] = __ldg(gs + i);
                }
            }
        }
        // hot rows: copied in 16-byte units from the 16-byte boundary at or before their start
        const uint32_t esz = ROW16 ? 2u : 4u;
        const size_t start = (size_t)A.hot_lo * A.n_classes * esz;
        const uint32_t lead = (uint32_t)(start & 15);
        const uint32_t n16 = (lead + hot_n * A.n_classes * esz + 15) / 16;
        const uint4 *rsrc = reinterpret_cast<const uint4 *>(reinterpret_cast<const uint8_t *>(A.rows) + start - lead);
        uint4 *rdst = reinterpret_cast<uint4 *>(smem + p.off_rows);
        for (uint32_t i = tid; i < n16; i += THREADS) rdst[i] = __ldg(rsrc + i);
        if (tid == 0) {
            for (uint32_t s = 0; s < p.nstage; ++s) {
                mbar_init(&mc->full[s], 1);
                mbar_init(&mc->empty[s], NCONS);
            }
            mc->rec_cursor = 0;
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
    }
    __syncthreads();
    if (!FILT) {
        if (tid < 256) {
            const uint32_t e = ROW16 ? (uint32_t)__ldg(reinterpret_cast<const uint16_t *>(A.rows) + cls_s[tid])
                                     : (uint32_t)__ldg(reinterpret_cast<const int32_t *>(A.rows) + cls_s[tid]);
            if (e) atomicOr(&fb_s[tid >> 5], 1u << (tid & 31));
        }
        __syncthreads();
    }

    const uint32_t g = A.gram_len;
    const uint32_t w1mask = FILT == 8 ? glop_w1_mask(g) : 0u;
    const uint32_t wsh = 37u - A.bm_log2, bsh = 32u - A.bm_log2;  // a gram's bitmap word and (longer grams) bit
    const uint32_t htmask = (1u << A.ht_log2) - 1u;
    // Scratch record of a matching offset.  Single buffer: (t << 10) | offset in
    // its sub-tile, t the deepest terminal state (below 2^22: larger automata
    // store no records and phase B walks every sub-tile again).  Batches:
    // (segment, offset in the segment, output-list start, count).
    constexpr uint32_t REC_W = BATCH ? 4u : 1u;  // record size in uint32
    // every output list shorter than 2^22 entries: a sub-tile's match count (at most 1,024 lists) fits 32 bits
    const bool narrow = A.n_cum_ids < (1u << 22);

    // Start of the walk from sub-tile offset off (walk bound endr): the state
    // reached by the first gram_len bytes, | GLOP_TERM when it is terminal;
    // without a start filter the initial state, encoded GLOP_TERM (state 0 is
    // never terminal).  0 when no pattern can start here.
    auto probe = [&](const TextView &v, uint32_t off, uint32_t endr, bool staged) -> uint32_t {
        if (FILT) {
            if (off + g > endr) return 0u;
            uint32_t w0 = 0, w1 = 0;
            // (staged text: the 12 bytes from off < 1 KiB are inside the ring slot, and the gram's own
            // bytes end at or before endr, so they were staged; bytes past them are masked off)
            if (staged || off + 12 <= v.n_stage) {
                const uint32_t *b32 = reinterpret_cast<const uint32_t *>(v.buf);
                const uint32_t a = off >> 2, sh = 8 * (off & 3);
                const uint32_t y1 = b32[a + 1];
                w0 = __funnelshift_r(b32[a], y1, sh);
                if (FILT == 8) w1 = __funnelshift_r(y1, b32[a + 2], sh) & w1mask;
            } else {
                for (uint32_t k = 0; k < 4; ++k) w0 |= tbyte(v, off + k) << (8 * k);
                if (FILT == 8)
                    for (uint32_t k = 4; k < g; ++k) w1 |= tbyte(v, off + k) << (8 * (k - 4));
            }
            uint32_t h = w0 * GLOP_HASH_M0;
            if (FILT == 8) h ^= w1 * GLOP_HASH_M1;
            uint32_t slot = glop_table_slot(h, A.ht_log2);
            if (FILT == 4 && grams_in_smem) {
                while (true) {
                    const uint2 e = grams8[slot];
                    if (!e.y) return 0u;
                    if (e.x == w0) return e.y;
                    slot = (slot + 1) & htmask;
                }
            }
            while (true) {
                const uint4 e = *reinterpret_cast<const uint4 *>(grams + slot);
                if (!e.z) return 0u;
                if (e.x == w0 && e.y == w1) return e.z;
                slot = (slot + 1) & htmask;
            }
        }
        return off < endr ? GLOP_TERM : 0u;
    };

    // start filter: bit j of the result = offset 32*lane + j of the sub-tile may start a match
    auto filter = [&](const TextView &v, uint32_t sub_len, uint64_t avail) -> uint32_t {
        uint32_t x[10];
        const uint32_t o = 32 * lane;
        if (v.n_stage >= SUB + 16) {
            const uint4 v0 = *reinterpret_cast<const uint4 *>(v.buf + o);
            const uint4 v1 = *reinterpret_cast<const uint4 *>(v.buf + o + 16);
            const uint2 v2 = *reinterpret_cast<const uint2 *>(v.buf + o + 32);
            x[0] = v0.x; x[1] = v0.y; x[2] = v0.z; x[3] = v0.w;
            x[4] = v1.x; x[5] = v1.y; x[6] = v1.z; x[7] = v1.w;
            x[8] = v2.x; x[9] = v2.y;
        } else {
#pragma unroll
            for (int k = 0; k < 10; ++k) {
                uint32_t w = 0;
                for (uint32_t b = 0; b < 4; ++b) {
                    const uint32_t pos = o + 4 * k + b;
                    if (pos < avail) w |= tbyte(v, pos) << (8 * b);
                }
                x[k] = w;
            }
        }
        // Offsets are tested from the last to the first; each test rotates its
        // bitmap word so the tested bit (stored bit-reversed) is bit 31 and
        // shifts it into the mask, so offset j ends at bit j.
        uint32_t acc[2] = {0u, 0u};
#pragma unroll
        for (int j = 31; j >= 0; --j) {
            uint32_t rot;
            if (FILT) {
                const uint32_t w0 = __funnelshift_r(x[j >> 2], x[(j >> 2) + 1], 8 * (j & 3));
                if (FILT == 4) {
                    // one wide multiply: the low half picks the word, the high half's low 5 bits the bit
                    const unsigned long long pr = (unsigned long long)w0 * GLOP_HASH_M0;
                    const uint32_t word = bm_s[(uint32_t)pr >> wsh];
                    rot = __funnelshift_l(word, word, (uint32_t)(pr >> 32));
                } else {
                    const uint32_t h =
                        w0 * GLOP_HASH_M0 ^
                        (__funnelshift_r(x[(j >> 2) + 1], x[(j >> 2) + 2], 8 * (j & 3)) & w1mask) * GLOP_HASH_M1;
                    const uint32_t word = bm_s[h >> wsh];
                    rot = __funnelshift_l(word, word, h >> bsh);
                }
            } else {
                const uint32_t by = (x[j >> 2] >> (8 * (j & 3))) & 0xFFu;
                rot = fb_s[by >> 5] << (31 - (by & 31));
            }
            acc[j >> 4] = __funnelshift_l(rot, acc[j >> 4], 1);
        }
        uint32_t mask = (acc[1] << 16) | acc[0];
        if (o + 32 > sub_len) mask &= (o >= sub_len) ? 0u : ((1u << (sub_len - o)) - 1u);
        return mask;
    };

    // segment holding absolute offset iabs (list of warp slot cw): false outside every segment
    auto seg_of = [&](uint32_t cw, bool onchip, uint64_t iabs, uint32_t &si, uint64_t &sstart,
                      uint64_t &send) -> bool {
        const uint32_t a = mc->seg_a[cw], L = mc->seg_L[cw];
        uint32_t lo = 0, hi = L;
        if (onchip) {
            const unsigned long long *e = mc->segl[cw];
            if (e[0] > iabs) return false;
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (e[mid] <= iabs) lo = mid; else hi = mid - 1;
            }
            if (lo >= L) return false;
            sstart = e[lo];
            send = e[lo + 1];
        } else {
            const unsigned long long *e = reinterpret_cast<const unsigned long long *>(p.seg) + a;
            GLOP_BAIL(p.hdr, (uint64_t)a + L <= p.n_seg, 24, a, false)
            if (__ldg(e) > iabs) return false;
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (__ldg(e + mid) <= iabs) lo = mid; else hi = mid - 1;
            }
            if (lo >= L) return false;
            sstart = __ldg(e + lo);
            send = __ldg(e + lo + 1);
        }
        si = a + lo;
        return iabs < send;
    };


    // Phase B copies the first n_ids_s output-list pattern ids into the ring
    // (free once phase A is over), after the scan bases; expand reads them
    // there and the rest from global memory.
    const uint32_t *ids_s = reinterpret_cast<const uint32_t *>(ring + PB * 8);
    uint32_t n_ids_s = 0;

    // Expand up to 32 matching offsets held one per lane (output list lo..lo+c
    // of the deepest terminal state, fields f0/f1) into output slots o, o+1,
    // ...: all patterns of an offset, offsets in lane order.  Returns the
    // number of outputs.
    auto expand = [&](uint32_t lo, uint32_t c, uint32_t f0, uint32_t f1, unsigned long long o) -> uint32_t {
        const uint32_t incl = warp_incl_scan(c, lane), excl = incl - c, tot = __shfl_sync(FULL, incl, 31);
        if (!tot) return 0u;
        // output slot s of the lane that owns it reads list entry base + s
        const uint32_t base = lo - excl;
        // When the lanes with outputs are a prefix of the warp (records fill lanes 0, 1, ...), the owner of
        // slot i is the number of lanes that start at or before i, less one: the lanes that started in
        // earlier rounds plus the starts at or below this lane's slot in a mask of this round's starts.
        const uint32_t nz = __ballot_sync(FULL, c != 0u);
        // (long lists -- 8 or more outputs a record on average -- keep the shuffle search: most rounds then
        // belong to one or two records, and a warp reduction every round costs more than it saves.  In batch
        // mode, a round that one record owns entirely needs no search at all: the owner of each round's first
        // slot is carried from round to round.  The single-buffer kernel keeps the plain search, where that
        // bookkeeping measured slower.)
        const bool pre = (nz & (nz + 1u)) == 0u;
        const bool prefix = pre && tot < 8u * __popc(nz), track = BATCH && pre && !prefix;
        const uint32_t le = (2u << lane) - 1u;
        const uint32_t room = o < p.cap ? (uint32_t)min(p.cap - o, (unsigned long long)tot) : 0u;
        uint32_t before = 0;
        uint32_t cur = 0, cur_end = track ? __shfl_sync(FULL, incl, 0) : 0u;  // owner of slot s0, end of its slots
        for (uint32_t s0 = 0; s0 < tot; s0 += 32) {
            const uint32_t slot = s0 + lane;
            uint32_t ow;
            if (prefix) {
                const uint32_t starts = __reduce_or_sync(FULL, (c && excl - s0 < 32u) ? 1u << (excl - s0) : 0u);
                ow = before + __popc(starts & le) - 1u;
                before += __popc(starts);
            } else if (track && cur_end >= s0 + 32u) {
                ow = cur;
            } else {
                ow = owner_of(excl, slot);
            }
            if (track) {
                // the owner of slot s0 + 32: the last slot's, or the next lane when that one ends here
                if (cur_end < s0 + 32u) {
                    cur = __shfl_sync(FULL, ow, 31);
                    cur_end = __shfl_sync(FULL, incl, cur);
                }
                if (cur_end == s0 + 32u && cur < 31u) {
                    ++cur;
                    cur_end = __shfl_sync(FULL, incl, cur);
                }
            }
            const uint32_t base_o = __shfl_sync(FULL, base, ow), f0_o = __shfl_sync(FULL, f0, ow);
            const uint32_t f1_o = BATCH ? __shfl_sync(FULL, f1, ow) : 0u;
            if (slot < room) {
                uint32_t pid = 0;
                const uint32_t q = base_o + slot;
                const unsigned long long pos = o + slot;
                // (lo + c never passes the end of cum_ids: walks end at valid states, and
                // load_rec bounds what it takes from records)
                GLOP_CK(p.hdr, q < A.n_cum_ids, 25, base_o) pid = q < n_ids_s ? ids_s[q] : __ldg(A.cum_ids + q);
                if (BATCH) {
                    uint32_t *ob = reinterpret_cast<uint32_t *>(p.out) + 3 * pos;
                    __stcs(ob, f0_o);
                    __stcs(ob + 1, f1_o);
                    __stcs(ob + 2, pid);
                } else {
                    __stcs(reinterpret_cast<uint2 *>(p.out) + pos, make_uint2(f0_o, pid));
                }
            }
        }
        return tot;
    };

    // Walk every survivor of sub-tile j, in batches of up to QCAP survivors:
    // (1) survivor offsets into the warp's queue, (2) probe pass: gram table,
    // keeping the survivors a pattern can start at, in offset order, (3) walk
    // pass: each lane takes the next queued walk as soon as its previous one
    // ends, (4) in offset order, record mode writes (offset, output list)
    // records to this block's scratch slice and the sub-tile descriptor;
    // direct mode (output position known) expands straight into the output.
    auto process = [&](uint64_t j, const TextView &v, uint32_t qw, bool direct, unsigned long long obase,
                       const uint32_t *sseg) {
        const uint64_t s0 = j * SUB;
        const uint64_t avail = p.len - s0;
        const uint32_t sub_len = (uint32_t)min((uint64_t)SUB, p.own_len - s0);
        const uint32_t endsub = (uint32_t)min(avail, (uint64_t)0xFFFFFFFFu);
        bool onchip = true;
        // batches: the segment boundaries of the sub-tile load into registers while the start filter runs
        uint32_t sa = 0, sL = 0;
        unsigned long long pb0 = 0, pb1 = 0;
        if (BATCH) {
            uint32_t a = 0, e = 1;
            if (sseg) {
                a = sseg[0];
                e = sseg[1] + 1;
            } else {
                GLOP_CK(p.hdr, j + 1 <= p.n_sub, 22, j) {
                    a = __ldg(p.tile_seg + j);
                    e = __ldg(p.tile_seg + j + 1) + 1;
                }
            }
            if (e > p.n_seg) e = p.n_seg;
            sa = a;
            sL = e - a;
            if (sL <= SEGW) {
                const unsigned long long *sb = reinterpret_cast<const unsigned long long *>(p.seg) + a;
                if (lane <= sL) GLOP_CK(p.hdr, a + lane <= p.n_seg, 23, a + lane) pb0 = __ldg(sb + lane);
                if (lane == 0 && sL == SEGW) GLOP_CK(p.hdr, a + SEGW <= p.n_seg, 23, a + SEGW) pb1 = __ldg(sb + SEGW);
            }
        }
        const uint32_t mask = filter(v, sub_len, avail);
        if (BATCH) {
            if (lane == 0) {
                mc->seg_a[qw] = sa;
                mc->seg_L[qw] = sL;
            }
            if (sL <= SEGW) {
                if (lane <= sL) mc->segl[qw][lane] = pb0;
                if (lane == 0 && sL == SEGW) mc->segl[qw][SEGW] = pb1;
            }
            __syncwarp();
            onchip = sL <= SEGW;
        }
        const uint32_t n = __popc(mask);
        const uint32_t incl = warp_incl_scan(n, lane), excl = incl - n, total = __shfl_sync(FULL, incl, 31);
        uint8_t *qbase = smem + p.off_q + qw * QBYTES;
        uint16_t *qoff = reinterpret_cast<uint16_t *>(qbase);
        uint32_t *qst = reinterpret_cast<uint32_t *>(qbase + QCAP * 2);
        uint32_t *qend = reinterpret_cast<uint32_t *>(qbase + QCAP * 6);
        const uint32_t lt = (1u << lane) - 1u;
        uint32_t rbase = 0;
        bool ovf = false;
        if (!direct && !p.state_hits) {
            if (lane == 0) rbase = atomicAdd(&mc->rec_cursor, total);
            rbase = __shfl_sync(FULL, rbase, 0);
            ovf = (uint64_t)rbase + total > p.rec_cap_cta;
        }
        const uint32_t rabs = blockIdx.x * p.rec_cap_cta + rbase;
        uint32_t *recs = p.records + (size_t)rabs * REC_W;
        uint32_t nrec = 0, nm32 = 0;
        unsigned long long nm64 = 0, o = obase;
        for (uint32_t b0 = 0; b0 < total; b0 += QCAP) {
            const uint32_t nb = min(QCAP, total - b0);
            // (1) survivor offsets
            if (total <= QCAP) {
                // all of them fit (the usual case): each lane writes its own from the highest
                uint32_t m = mask;
                uint16_t *qp = qoff + excl + n;
                while (m) {
                    const uint32_t bit = 31u - __clz(m);
                    m ^= 1u << bit;
                    *--qp = (uint16_t)(32 * lane + bit);
                }
            } else if (excl < b0 + nb && excl + n > b0) {
                uint32_t m = mask, idx = excl;
                while (m) {
                    const uint32_t bit = __ffs(m) - 1;
                    m &= m - 1;
                    const uint32_t rel = idx - b0;
                    if (rel < nb) qoff[rel] = (uint16_t)(32 * lane + bit);
                    ++idx;
                }
            }
            __syncwarp();
            // (2) probe pass (in place: entry i moves to position <= i)
            uint32_t nw = 0;
            for (uint32_t r0 = 0; r0 < nb; r0 += 32) {
                const uint32_t i = r0 + lane;
                uint32_t off = 0, val = 0, endr = endsub;
                if (i < nb) {
                    off = qoff[i];
                    bool in = true;
                    if (BATCH) {
                        uint32_t si;
                        uint64_t sstart, send;
                        in = seg_of(qw, onchip, s0 + off, si, sstart, send);
                        endr = in ? (uint32_t)min(send - s0, (uint64_t)0xFFFFFFFFu) : 0u;
                    }
                    if (in) val = probe(v, off, endr, !direct);
                }
                const uint32_t bm = __ballot_sync(FULL, val != 0);
                __syncwarp();
                if (val) {
                    const uint32_t q = nw + __popc(bm & lt);
                    qoff[q] = (uint16_t)off;
                    qst[q] = val;
                    if (BATCH) qend[q] = endr;
                }
                nw += __popc(bm);
            }
            __syncwarp();
            // (3) walk pass.  (3a) every walk takes its first step in
            // lock-step rounds of 32; the walks that go on are listed
            // (state, position, queue index) and (3b) walked by lanes that
            // refill from that list as their walks end.  qst[i] holds the
            // deepest terminal state of walk i so far.
            uint32_t *cst = reinterpret_cast<uint32_t *>(qbase + QCAP * 10);
            uint32_t *cpos = cst + CCAP;
            uint8_t *cidx = reinterpret_cast<uint8_t *>(cpos + CCAP);
            auto run_cont = [&](uint32_t ncont) {
                uint32_t nxt = 0, qi = 0, st = 0, pos = 0, t = 0, endw = endsub;
                bool have = false;
                while (true) {
                    if (nxt < ncont) {  // (once every listed walk is handed out, lanes only finish theirs)
                        const uint32_t wm = __ballot_sync(FULL, !have);
                        if (!have) {
                            const uint32_t k = nxt + __popc(wm & lt);
                            if (k < ncont) {
                                qi = cidx[k];
                                st = cst[k];
                                pos = cpos[k];
                                t = qst[qi];
                                if (BATCH) endw = qend[qi];
                                have = true;
                            }
                        }
                        nxt += __popc(wm);
                    }
                    if (!__any_sync(FULL, have)) break;
                    // the direct (re-walk) mode reads the text from global memory: no staged bytes
                    const bool fin = have && (direct ? step<ROW16, true>(A, cls_s, rows_s, hot_n, v, st, pos, endw, t, p.hdr)
                                                     : step<ROW16, DEEP>(A, cls_s, rows_s, hot_n, v, st, pos, endw, t, p.hdr));
                    if (fin) {
                        qst[qi] = t;
                        have = false;
                    }
                }
            };
            {
                uint32_t nc = 0;
                for (uint32_t r0 = 0; r0 < nw; r0 += 32) {
                    if (nc > CCAP - 32) {
                        __syncwarp();
                        run_cont(nc);
                        nc = 0;
                        __syncwarp();
                    }
                    const uint32_t i = r0 + lane;
                    bool cont = false;
                    uint32_t st = 0, pos = 0;
                    if (i < nw) {
                        const uint32_t val = qst[i];
                        st = val & GLOP_STATE_MASK;
                        uint32_t t = (val & GLOP_TERM) ? st : 0u;
                        pos = qoff[i] + g;
                        const uint32_t endw = BATCH ? qend[i] : endsub;
                        const bool fin = direct ? step<ROW16, true>(A, cls_s, rows_s, hot_n, v, st, pos, endw, t, p.hdr)
                                                : step<ROW16, DEEP>(A, cls_s, rows_s, hot_n, v, st, pos, endw, t, p.hdr);
                        qst[i] = t;
                        cont = !fin;
                    }
                    const uint32_t bm = __ballot_sync(FULL, cont);
                    if (cont) {
                        const uint32_t k = nc + __popc(bm & lt);
                        cst[k] = st;
                        cpos[k] = pos;
                        cidx[k] = (uint8_t)i;
                    }
                    nc += __popc(bm);
                }
                __syncwarp();
                if (nc) run_cont(nc);
            }
            __syncwarp();
            // (4) records or direct output, in offset order
            for (uint32_t r0 = 0; r0 < nw; r0 += 32) {
                const uint32_t i = r0 + lane;
                uint32_t t = 0, f0 = 0, f1 = 0, lo = 0, c = 0, off_i = 0;
                if (i < nw) {
                    t = qst[i];
                    if (t >= A.n_states) {
                        fail_check(p.hdr, 2, t);
                        t = 0;
                    }
                    if (t) {
                        const uint2 lc = __ldg(reinterpret_cast<const uint2 *>(A.outl) + t);
                        lo = lc.x;
                        c = lc.y;
                        off_i = qoff[i];
                        const uint64_t iabs = s0 + off_i;
                        if (BATCH) {
                            uint32_t si = 0;
                            uint64_t sstart = 0, send = 0;
                            seg_of(qw, onchip, iabs, si, sstart, send);
                            f0 = si;
                            f1 = (uint32_t)(iabs - sstart);
                        } else {
                            f0 = (uint32_t)iabs + p.base_off;
                        }
                    }
                }
                if (direct) {
                    o += expand(lo, c, f0, f1, o);
                } else if (p.state_hits) {
                    // count-only mode: one hit on the offset's deepest terminal state, counted in the
                    // block's table when the state has (or gets) its slot there, else in global memory
                    if (t) {
                        uint32_t *hk = reinterpret_cast<uint32_t *>(smem + p.off_hc);
                        const uint32_t slot = (t * 0x9E3779B1u) >> (32 - 10);
                        uint32_t k = hk[slot];
                        if (k == 0) {
                            const uint32_t old = atomicCAS(hk + slot, 0u, t);
                            k = old ? old : t;
                        }
                        if (k == t) atomicAdd(hk + HCACHE + slot, 1u);
                        else atomicAdd(p.state_hits + t, 1u);
                    }
                } else {
                    const uint32_t b = __ballot_sync(FULL, t != 0);
                    if (t) {
                        const uint32_t q = nrec + __popc(b & lt);
                        if (narrow) nm32 += c;
                        else nm64 += c;
                        GLOP_CK(p.hdr, ovf || (uint64_t)rabs + q < p.rec_slots, 27, rabs + q)
                        if (!ovf) {
                            uint32_t *rp = recs + (size_t)q * REC_W;
                            if (BATCH) *reinterpret_cast<uint4 *>(rp) = make_uint4(f0, f1, lo, c);
                            else *rp = (t << 10) | off_i;
                        }
                    }
                    nrec += __popc(b);
                }
            }
            __syncwarp();
        }
        if (!direct && !p.state_hits) {
            const unsigned long long nmatch = narrow ? (unsigned long long)__reduce_add_sync(FULL, nm32) : warp_sum64(nm64);
            if (lane == 0) {
                SubDesc d;
                d.rec_start = rabs;
                d.n_rec = ovf ? REC_OVERFLOW : nrec;
                d.n_match = nmatch;
                GLOP_CK(p.hdr, j < p.n_sub, 28, j) p.desc[j] = d;
                if (ovf) atomicAdd(p.hdr + 10, 1u);
            }
        }
    };

    // ================= phase A =================
    if (warp == 0) {
        // producer: chunk tickets -> ring slots.  Bit s of issued: slot s has a
        // bulk copy queued that no consumer is known to have waited for; bit s of
        // par: the phase parity that copy completes.  (A slot's bit is cleared when
        // the consumers have released the slot: they waited for its copy.  Only
        // then does the producer arrive on the slot's full barrier again, so the
        // barrier is still in the copy's phase whenever the bit is set.)
        uint32_t issued = 0, par = 0;
        // ring slot and round of step cs (cs % nstage, cs / nstage), kept without a division
        uint32_t slot = 0, rnd = 0;
        for (uint32_t cs = 0;; ++cs) {
            if (cs) {
                if (++slot == p.nstage) {
                    slot = 0;
                    ++rnd;
                }
            }
            if (rnd) {
                uint32_t ok = 1;
                if (lane == 0) ok = mbar_wait(&mc->empty[slot], (rnd - 1) & 1u, p.spin_budget) ? 1u : 0u;
                ok = __shfl_sync(FULL, ok, 0);
                if (!ok) {
                    if (lane == 0) atomicOr(p.hdr, WS_TIMEOUT);
                    break;
                }
                issued &= ~(1u << slot);
            }
            unsigned long long k = 0;
            if (lane == 0) k = atomicAdd(ticket, 1ull);
            k = shfl64(k, 0);
            uint8_t *dst = ring + (size_t)slot * p.slot_bytes;
            if (k >= n_chunks) {
                if (lane == 0) {
                    mc->slot_tile[slot] = END_TICKET;
                    mbar_arrive(&mc->full[slot]);
                }
                break;
            }
            // (test hook: a chunk that is never staged, so every consumer's wait for it runs out)
            if (k == p.withhold_chunk) continue;
            const uint32_t csubs = NCONS * KSUB;  // sub-tiles per chunk
            const uint64_t c0 = (sub0 + k * csubs) * SUB;
            const uint32_t n_stage = (uint32_t)min((uint64_t)(csubs * SUB + p.halo), p.len - c0);
            const uint32_t bulk = p.aligned ? (n_stage & ~15u) : 0u;
            for (uint32_t y = bulk + lane; y < n_stage; y += 32)
                GLOP_CK(p.hdr, c0 + y < p.len && y < p.slot_bytes, 29, y) dst[y] = __ldg(p.text + c0 + y);
            // batches: the first segment of each of the chunk's sub-tiles (and of the one after), so consumers
            // start their segment-boundary loads without a round trip
            if (BATCH)
                for (uint32_t q = lane; q <= csubs; q += 32)
                    mc->slot_seg[slot][q] = __ldg(p.tile_seg + min((uint64_t)(sub0 + k * csubs + q), (uint64_t)p.n_sub));
            __syncwarp();
            if (lane == 0) {
                mc->slot_tile[slot] = k;
                mc->slot_nstage[slot] = n_stage;
                bool tma_ok = true;
                // (a bulk copy is issued only when bulk > 0: misaligned text is copied by the lanes above)
                GLOP_CK(p.hdr, bulk == 0 || (c0 + bulk <= p.len && bulk <= p.slot_bytes &&
                                              !(reinterpret_cast<uintptr_t>(p.text + c0) & 15) &&
                                              !(smem_addr(dst) & 15) && (bulk & 15) == 0), 30, bulk) {}
#ifdef GLOP_BOUNDS_CHECK
                tma_ok = c0 + bulk <= p.len && bulk <= p.slot_bytes && !(reinterpret_cast<uintptr_t>(p.text + c0) & 15) &&
                         !(smem_addr(dst) & 15) && (bulk & 15) == 0;
#endif
                if (bulk && tma_ok) {
                    tma_load(dst, p.text + c0, bulk, &mc->full[slot]);
                    issued |= 1u << slot;
                    par = (par & ~(1u << slot)) | ((rnd & 1u) << slot);
                } else {
                    mbar_arrive(&mc->full[slot]);
                }
            }
        }
        // Leaving early (a wait ran out) can leave bulk copies in flight into
        // the ring: wait, with the same bound, until each slot's last one has
        // landed before the ring is reused or the block exits.
        if (lane == 0)
            for (uint32_t sl = 0; sl < p.nstage; ++sl)
                if ((issued >> sl) & 1u)
                    if (!mbar_wait(&mc->full[sl], (par >> sl) & 1u, p.spin_budget)) atomicOr(p.hdr, WS_TIMEOUT);
        __syncwarp();
    } else {
        const uint32_t cw = warp - 1;
        for (uint32_t slot = 0, ph = 0;;) {
            if (!mbar_wait(&mc->full[slot], ph, p.spin_budget)) {
                if (lane == 0) atomicOr(p.hdr, WS_TIMEOUT);
                break;
            }
            const unsigned long long k = mc->slot_tile[slot];
            if (k == END_TICKET) break;
            // the warp's ksub consecutive sub-tiles of the chunk
            for (uint32_t u = 0; u < KSUB; ++u) {
                const uint32_t w = cw * KSUB + u;  // sub-tile position in the chunk
                const uint64_t j = sub0 + k * NCONS * KSUB + w;
                if (j >= sub_end) break;
                const uint32_t ns = mc->slot_nstage[slot];
                TextView v;
                v.buf = ring + (size_t)slot * p.slot_bytes + w * SUB;
                v.gtext = p.text + j * SUB;
                v.n_stage = ns > w * SUB ? ns - w * SUB : 0u;
#ifdef GLOP_BOUNDS_CHECK
                v.avail = p.len - j * SUB;
                v.hdr = p.hdr;
#endif
                process(j, v, cw, false, 0ull, BATCH ? &mc->slot_seg[slot][w] : nullptr);
                __syncwarp();
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&mc->empty[slot]);
            if (++slot == p.nstage) {
                slot = 0;
                ph ^= 1u;
            }
        }
    }

    // count-only mode ends here (nothing to place, no grid barrier): flush the block's hit table
    if (p.state_hits) {
        __syncthreads();
        const uint32_t *hk = reinterpret_cast<const uint32_t *>(smem + p.off_hc);
        for (uint32_t i = tid; i < HCACHE; i += THREADS)
            if (hk[i]) atomicAdd(p.state_hits + hk[i], hk[HCACHE + i]);
        return;
    }

    // ================= phase B =================
    const uint32_t G = gridDim.x;
    grid_sync(p.hdr + 8, G + p.barrier_extra, p.spin_budget, p.hdr);
    {
        // the ring is free now: stage the output-list ids that fit after the scan bases
        // (the __syncthreads of the block sums below orders these stores before any read)
        n_ids_s = min(A.n_cum_ids, (p.nstage * p.slot_bytes - PB * 8) / 4u);
        uint32_t *dst = reinterpret_cast<uint32_t *>(ring + PB * 8);
        for (uint32_t i = tid; i < n_ids_s; i += THREADS) dst[i] = __ldg(A.cum_ids + i);
    }
    // this block's static range of sub-tiles (several automata: a share of its own group's, so that
    // records, re-walks and output lists use the tables this block staged; blocks and groups are in
    // text order, so block order is still sub-tile order)
    uint64_t ra, rb;
    {
        const uint64_t b0 = MULTI ? p.grp.blk[grp] : 0u, nb = MULTI ? p.grp.blk[grp + 1] - b0 : G;
        const uint64_t R = (sub_end - sub0 + nb - 1) / nb;
        ra = min(sub_end, sub0 + (blockIdx.x - b0) * R);
        rb = min(sub_end, ra + R);
    }
    {
        unsigned long long sum = 0;
        for (uint64_t j = ra + tid; j < rb; j += THREADS)
            GLOP_CK(p.hdr, j < p.n_sub, 31, j) sum += __ldcg(&p.desc[j].n_match);
        sum = warp_sum64(sum);
        if (lane == 0) mc->red[warp] = sum;
        __syncthreads();
        if (warp == 0) {
            const unsigned long long v = warp_sum64(mc->red[lane]);
            if (lane == 0) p.sums[blockIdx.x] = v;
        }
    }
    grid_sync(p.hdr + 9, G + p.barrier_extra, p.spin_budget, p.hdr);
    if (warp == 0) {
        unsigned long long before = 0, all = 0;
        for (uint32_t c = lane; c < G; c += 32) {
            const unsigned long long v = __ldcg(p.sums + c);
            if (c < blockIdx.x) before += v;
            all += v;
        }
        before = warp_sum64(before);
        all = warp_sum64(all);
        if (lane == 0) {
            const unsigned long long obase = p.d_obase ? *p.d_obase : 0ull;
            mc->red[0] = obase + before;
            if (blockIdx.x == 0) {
                *p.d_count = all;
                *reinterpret_cast<unsigned long long *>(p.hdr + 4) = all;
                if (obase + all > p.cap) atomicOr(p.hdr, WS_OVERFLOW);
                if (p.d_next_base) *p.d_next_base = obase + all;
            }
        }
    }
    __syncthreads();
    unsigned long long running = mc->red[0];
    __syncthreads();

    unsigned long long *bases = reinterpret_cast<unsigned long long *>(ring);  // the ring is free now
    for (uint64_t p0 = ra; p0 < rb; p0 += PB) {
        const uint32_t np = (uint32_t)min((uint64_t)PB, rb - p0);
        // exclusive scan of the piece's match counts, 4 per thread
        unsigned long long v[4], s = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t idx = tid * 4 + q;
            v[q] = idx < np ? __ldcg(&p.desc[p0 + idx].n_match) : 0ull;
            s += v[q];
        }
        unsigned long long inc = s;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long u = shfl_up64(inc, d);
            if (lane >= (uint32_t)d) inc += u;
        }
        if (lane == 31) mc->red[warp] = inc;
        __syncthreads();
        unsigned long long wpre = 0, ptot = 0;
        for (uint32_t w = 0; w < 32; ++w) {
            const unsigned long long x = mc->red[w];
            if (w < warp) wpre += x;
            ptot += x;
        }
        unsigned long long e = running + wpre + inc - s;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t idx = tid * 4 + q;
            if (idx < np) bases[idx] = e;
            e += v[q];
        }
        __syncthreads();
        // Software pipeline over this warp's sub-tiles x, x + 32, ...: the
        // descriptor two sub-tiles ahead and the first 32 records one
        // sub-tile ahead load while the current sub-tile expands.
        auto load_desc = [&](uint32_t x) -> uint4 {
            uint4 d = make_uint4(0, 0, 0, 0);
            if (x < np) GLOP_CK(p.hdr, p0 + x < p.n_sub, 32, p0 + x) d = __ldcg(reinterpret_cast<const uint4 *>(p.desc + p0 + x));
            return d;
        };
        // Record r of a sub-tile as loaded (0s past its end).  Nothing here depends
        // on the loaded value, so the load of the next sub-tile's records stays in
        // flight while the current one expands; decode_rec uses it afterwards.
        auto load_rec = [&](const uint4 &d, uint32_t r) -> uint4 {
            uint4 x = make_uint4(0, 0, 0, 0);
            if (d.y != REC_OVERFLOW && (uint64_t)d.x + d.y <= p.rec_slots && r < d.y) {
                const uint32_t *rp = p.records + ((size_t)d.x + r) * REC_W;
                if (BATCH) x = __ldcg(reinterpret_cast<const uint4 *>(rp));
                else x.x = __ldcg(rp);
            }
            return x;
        };
        // A loaded record of sub-tile j as (f0, f1, lo, c): the reported offset
        // (batches: segment, offset in it) and the output list.  Every index taken
        // from a record is checked, in every build: after a bounded wait has run
        // out, phase B can meet records that phase A never wrote.  (A record of a
        // single buffer is never 0: its state is not the initial one.)
        auto decode_rec = [&](uint4 x, uint64_t j) -> uint4 {
            if (BATCH) {
                x.w = min(x.w, A.n_cum_ids - min(x.z, A.n_cum_ids));
                return x;
            }
            uint4 o = make_uint4(0, 0, 0, 0);
            const uint32_t t = x.x >> 10;
            if (x.x) {
                o.x = (uint32_t)j * SUB + (x.x & 1023u) + p.base_off;
                if (t < A.n_states) {
                    const uint2 lc = __ldg(reinterpret_cast<const uint2 *>(A.outl) + t);
                    o.z = lc.x;
                    o.w = lc.y;
                }
            }
            return o;
        };
        // (batch mode, with its wider records, keeps the descriptor one sub-tile ahead only: registers)
        uint4 d1 = load_desc(warp), d2 = BATCH ? make_uint4(0, 0, 0, 0) : load_desc(warp + 32);
        uint4 r1 = load_rec(d1, lane);
        for (uint32_t x = warp; x < np; x += 32) {
            const uint64_t j = p0 + x;
            const uint4 dr = d1, rc = r1;
            if (BATCH) {
                d1 = load_desc(x + 32);
            } else {
                d1 = d2;
                d2 = load_desc(x + 64);
            }
            r1 = load_rec(d1, lane);
            unsigned long long o = bases[x];
            if (dr.y != REC_OVERFLOW && (uint64_t)dr.x + dr.y > p.rec_slots) {
                fail_check(p.hdr, 4, dr.x);
            } else if (dr.y != REC_OVERFLOW) {
                const uint4 e0 = decode_rec(rc, j);
                o += expand(e0.z, e0.w, e0.x, e0.y, o);
                for (uint32_t r0 = 32; r0 < dr.y; r0 += 32) {
                    const uint4 rr = decode_rec(load_rec(dr, r0 + lane), j);
                    o += expand(rr.z, rr.w, rr.x, rr.y, o);
                }
            } else {
                // the records did not fit: walk the sub-tile again from global memory
                TextView gv;
                gv.buf = nullptr;
                gv.gtext = p.text + j * SUB;
                gv.n_stage = 0u;
#ifdef GLOP_BOUNDS_CHECK
                gv.avail = p.len - j * SUB;
                gv.hdr = p.hdr;
#endif
                process(j, gv, warp, true, o, nullptr);
            }
        }
        running += ptot;
        __syncthreads();
    }
}

template <int FILT, bool BATCH, bool ROW16, bool DEEP, uint32_t KSUB, bool MULTI = false>
int launch_t(KParams &kp, uint32_t smem, uint32_t grid, cudaStream_t st) {
    static std::mutex mu;
    static uint32_t set_for[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    auto fn = scan_kernel<FILT, BATCH, ROW16, DEEP, KSUB, MULTI>;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev >= 0 && dev < 64 && set_for[dev] < smem) {
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
                return 4;
            set_for[dev] = smem;
        }
    }
    void *args[] = {&kp};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)fn, dim3(grid), dim3(THREADS), args, smem, st);
    return e == cudaSuccess ? 0 : 4;
}

// One cooperative launch of the scan kernel for the automaton's start-filter
// kind (gram length 0, 4 or 8 bytes), defined in scan_f0.cu / scan_f4.cu /
// scan_f8.cu.  ksub 2 (62 KiB chunks) is instantiated only without DEEP and
// for one automaton; several automata (multi) only for batches with ksub 1.
int launch_f0(KParams &kp, uint32_t smem, uint32_t grid, cudaStream_t st, bool batch, bool r16, bool deep, uint32_t ksub,
              bool multi);
int launch_f4(KParams &kp, uint32_t smem, uint32_t grid, cudaStream_t st, bool batch, bool r16, bool deep, uint32_t ksub,
              bool multi);
int launch_f8(KParams &kp, uint32_t smem, uint32_t grid, cudaStream_t st, bool batch, bool r16, bool deep, uint32_t ksub,
              bool multi);

}  // namespace kern
}  // namespace glop
