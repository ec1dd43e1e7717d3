// server.cpp -- glop_server_*: the serving loop of a scan server in native
// code.  The paper's use case (Sec. 1) sends logs and rules to a GPU that
// answers with the count and locations of suspect events; its library hands
// the GPU the next batch while a kernel runs (Sec. 6) and names real-time
// operation as future work (Sec. 8).  This engine keeps several compiled
// pattern sets resident, admits requests (a payload and the set to scan it
// with) into a device-memory budget, and batches whatever is pending while
// earlier batches are still on the GPU.
//
// Built on the public entry points alone (glop_scan_batch,
// glop_scan_batch_multi, glop_batch_split, glop_scan_host).  One poll of the
// loop, in the caller's thread:
//  * finished batches advance: once a batch's match count is on the host its
//    matches go, request by request, into pinned result rows (a batch whose
//    output bound was too small is scanned again into a larger one first);
//  * a lone small request on an idle server takes one end-to-end
//    glop_scan_host call;
//  * otherwise pending requests become a batch, in arrival order from the
//    oldest, over every set whose automaton shares the oldest request's
//    kernel kind (one group of segments per set, each group on a 1 KiB
//    boundary with a padding segment in the gap), within the batch limits
//    and the largest free block of the device arena;
// and requests of at least big_bytes go to a lane of their own: a worker
// thread scanning them end to end with glop_scan_host, so they neither wait
// for a batch nor hold small requests behind them.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "glop.h"

namespace {

constexpr uint64_t kAlign = 256;
constexpr uint64_t kGroupAlign = 1024;  // each set's group of segments starts on this boundary
constexpr uint64_t kEagerRows = 1 << 16;  // output bounds up to this many rows come back with the count

uint64_t al(uint64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// First-fit allocator over one device allocation (the HBM budget).
struct Arena {
    uint8_t *base = nullptr;
    uint64_t size = 0;
    std::map<uint64_t, uint64_t> free;  // offset -> length
    bool init(uint64_t bytes) {
        if (cudaMalloc(&base, bytes) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        size = bytes;
        free[0] = bytes;
        return true;
    }
    int64_t alloc(uint64_t n) {
        n = al(std::max<uint64_t>(n, 1));
        for (auto it = free.begin(); it != free.end(); ++it) {
            if (it->second < n) continue;
            const uint64_t off = it->first, len = it->second;
            free.erase(it);
            if (len > n) free[off + n] = len - n;
            return (int64_t)off;
        }
        return -1;
    }
    void release(uint64_t off, uint64_t n) {
        n = al(std::max<uint64_t>(n, 1));
        auto it = free.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free.erase(nx);
        }
        if (it != free.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free.erase(it);
            }
        }
    }
    uint64_t largest() const {
        uint64_t m = 0;
        for (auto &kv : free) m = std::max(m, kv.second);
        return m;
    }
    void destroy() {
        if (base) cudaFree(base);
        base = nullptr;
    }
};

// Pinned host blocks for result rows, reused after release.
struct PinnedPool {
    std::mutex mu;
    std::multimap<uint64_t, void *> idle;  // capacity (bytes) -> block
    std::map<void *, uint64_t> cap;
    std::atomic<uint64_t> allocs{0};  // blocks made (cudaHostAlloc calls)
    void *get(uint64_t bytes) {
        bytes = std::max<uint64_t>(bytes, 1 << 16);
        {
            std::lock_guard<std::mutex> lk(mu);
            auto it = idle.lower_bound(bytes);
            if (it != idle.end() && it->first <= 4 * bytes) {
                void *p = it->second;
                idle.erase(it);
                return p;
            }
        }
        // powers of two up to 64 MiB, then multiples of 64 MiB (a batch's block of a few hundred MiB would
        // otherwise take up to twice its size)
        uint64_t c = 1 << 16;
        while (c < bytes && c < (64ull << 20)) c <<= 1;
        if (c < bytes) c = (bytes + (64ull << 20) - 1) & ~((64ull << 20) - 1);
        void *p = nullptr;
        ++allocs;
        if (cudaHostAlloc(&p, c, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        std::lock_guard<std::mutex> lk(mu);
        cap[p] = c;
        return p;
    }
    void put(void *p) {
        if (!p) return;
        std::lock_guard<std::mutex> lk(mu);
        idle.emplace(cap[p], p);
    }
    void destroy() {
        for (auto &kv : cap) cudaFreeHost(kv.first);
        cap.clear();
        idle.clear();
    }
};

// A batch's result rows: one pinned block holding every request's rows, given back to the pool when the
// last of its requests is released.
struct Block {
    void *p = nullptr;
    uint32_t refs = 0;
};

struct Request {
    uint64_t id;
    uint32_t set;
    const uint8_t *payload;
    uint64_t len;
    // results
    glop_status st = GLOP_OK;
    uint64_t count = 0;
    glop_match *rows = nullptr;  // pinned: inside blk, or a block of its own from the pool (or the lane's rows)
    Block *blk = nullptr;
    uint64_t done_ns = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    uint64_t *seg_host = nullptr;    // pinned segment offsets
    uint64_t *first_host = nullptr;  // pinned per-segment first match
    uint64_t *count_host = nullptr;  // pinned match count
    glop_match *eager = nullptr;     // pinned rows for small batches (kEagerRows)
    uint32_t max_seg = 0;
};

struct Batch {
    Slot *slot = nullptr;
    std::vector<std::pair<uint32_t, std::vector<Request *>>> groups;  // (set, requests)
    std::vector<uint64_t> gstart;   // group starts (bytes), n_groups + 1
    std::vector<uint32_t> rseg;     // segment of each request, in group order
    uint64_t nbytes = 0;
    uint32_t nseg = 0;
    uint64_t cap = 0;               // output rows
    // arena regions
    uint64_t off = 0, len = 0;
    uint64_t t_off, s_off, c_off, w_off, m_off, p_off, f_off, ws_bytes;
    void *extra_out = nullptr, *extra_pairs = nullptr;  // rescan outputs (device)
    uint64_t extra_off = 0, extra_len = 0;              // (their arena block, when they came from the budget)
    int stage = 0;                  // 1: count on the host; 2: results copied
    uint64_t total = 0;
    bool eager = false;
};

}  // namespace

struct glop_server_s {
    std::vector<glop_handle> sets;
    std::vector<uint32_t> kind;
    std::vector<double> density;  // matches per payload byte, a slowly decaying maximum
    glop_server_opts o{};
    int device = 0;
    Arena arena;
    PinnedPool pool;
    std::vector<Slot> slots;
    std::vector<Slot *> free_slots;
    std::deque<Request *> pending;  // arrival order
    std::vector<Batch *> inflight;
    std::vector<Request *> finished;
    std::map<uint64_t, Request *> handed;  // results handed out, until released
    std::mutex fin_mu;                     // guards finished (the lane thread adds to it)
    // the idle fast path
    void *fast_staging = nullptr;
    uint64_t fast_staging_bytes = 0, fast_cap = 0;
    glop_match *fast_out = nullptr;
    cudaStream_t fast_stream = nullptr;
    // the large-request lane
    std::thread lane;
    std::mutex lane_mu;
    std::condition_variable lane_cv;
    std::deque<Request *> lane_q;
    bool lane_stop = false;
    void *lane_staging = nullptr;
    uint64_t lane_staging_bytes = 0, lane_rows = 0;
    glop_match *lane_buf = nullptr;         // pinned rows for the lane's results (lane_rows), one request at a time
    std::atomic<bool> lane_buf_busy{false};  // handed out and not yet released
    cudaStream_t lane_stream = nullptr;
    std::atomic<uint64_t> lane_active{0};
    glop_server_stats stats{};
    uint64_t warm_allocs = 0;  // pool blocks made at creation
};

namespace {

uint64_t cap_of(glop_server_s *S, const std::vector<std::pair<uint32_t, std::vector<Request *>>> &groups) {
    double m = 0;
    for (auto &g : groups) {
        uint64_t b = 0;
        for (Request *r : g.second) b += r->len;
        m += S->density[g.first] * (double)b;
    }
    return (uint64_t)(m * 1.25) + 4096;
}

void layout(Batch &b) {
    b.gstart.clear();
    b.rseg.clear();
    uint64_t pos = 0;
    uint32_t nseg = 0;
    std::vector<uint64_t> ends;
    for (size_t gi = 0; gi < b.groups.size(); ++gi) {
        b.gstart.push_back(pos);
        for (Request *r : b.groups[gi].second) {
            pos += r->len;
            b.rseg.push_back(nseg++);
        }
        const uint64_t pad = gi + 1 < b.groups.size() ? (kGroupAlign - pos % kGroupAlign) % kGroupAlign : 0;
        if (pad) {
            pos += pad;
            ++nseg;
        }
    }
    b.gstart.push_back(pos);
    b.nbytes = pos;
    b.nseg = nseg;
}

// arena footprint of a batch with output bound cap; false when it does not fit anywhere
bool regions(glop_server_s *S, Batch &b, uint64_t cap) {
    uint64_t ws = 0;
    glop_batch_workspace_size(S->sets[b.groups[0].first], b.nbytes, b.nseg, &ws);
    b.ws_bytes = ws;
    const uint64_t sz[7] = {al(b.nbytes), al(8ull * (b.nseg + 1)), al(8), al(ws), al(12 * cap), al(8 * cap),
                            al(8ull * (b.nseg + 1))};
    uint64_t tot = 0;
    for (uint64_t z : sz) tot += z;
    const int64_t off = S->arena.alloc(tot);
    if (off < 0) return false;
    b.off = (uint64_t)off;
    b.len = tot;
    uint64_t o = b.off;
    uint64_t *outs[7] = {&b.t_off, &b.s_off, &b.c_off, &b.w_off, &b.m_off, &b.p_off, &b.f_off};
    for (int k = 0; k < 7; ++k) {
        *outs[k] = o;
        o += sz[k];
    }
    b.cap = cap;
    return true;
}

glop_status scan_split(glop_server_s *S, Batch &b, void *out, void *pairs, uint64_t cap) {
    uint8_t *base = S->arena.base;
    cudaStream_t st = b.slot->stream;
    glop_status rc;
    if (b.groups.size() == 1) {
        rc = glop_scan_batch(S->sets[b.groups[0].first], base + b.t_off, b.nbytes,
                             reinterpret_cast<const uint64_t *>(base + b.s_off), b.nseg,
                             reinterpret_cast<glop_batch_match *>(out), cap, reinterpret_cast<uint64_t *>(base + b.c_off),
                             base + b.w_off, b.ws_bytes, st);
    } else {
        glop_handle hs[GLOP_BATCH_MAX_GROUPS];
        for (size_t g = 0; g < b.groups.size(); ++g) hs[g] = S->sets[b.groups[g].first];
        rc = glop_scan_batch_multi(hs, (uint32_t)b.groups.size(), b.gstart.data(), base + b.t_off, b.nbytes,
                                   reinterpret_cast<const uint64_t *>(base + b.s_off), b.nseg,
                                   reinterpret_cast<glop_batch_match *>(out), cap,
                                   reinterpret_cast<uint64_t *>(base + b.c_off), base + b.w_off, b.ws_bytes, st);
    }
    if (rc != GLOP_OK) return rc;
    return glop_batch_split(reinterpret_cast<const glop_batch_match *>(out),
                            reinterpret_cast<const uint64_t *>(base + b.c_off), cap, b.nseg,
                            reinterpret_cast<glop_match *>(pairs), reinterpret_cast<uint64_t *>(base + b.f_off), st);
}

glop_status launch(glop_server_s *S, Batch &b) {
    Slot &sl = *b.slot;
    uint8_t *base = S->arena.base;
    cudaStream_t st = sl.stream;
    // segment offsets (payloads, then the padding segment of every group but the last)
    uint64_t pos = 0;
    uint32_t k = 0;
    sl.seg_host[k++] = 0;
    for (size_t gi = 0; gi < b.groups.size(); ++gi) {
        for (Request *r : b.groups[gi].second) {
            if (r->len && cudaMemcpyAsync(base + b.t_off + pos, r->payload, r->len, cudaMemcpyHostToDevice, st) !=
                              cudaSuccess)
                return GLOP_ECUDA;
            pos += r->len;
            sl.seg_host[k++] = pos;
        }
        if (pos < b.gstart[gi + 1]) {
            if (cudaMemsetAsync(base + b.t_off + pos, 0, b.gstart[gi + 1] - pos, st) != cudaSuccess) return GLOP_ECUDA;
            pos = b.gstart[gi + 1];
            sl.seg_host[k++] = pos;
        }
    }
    if (cudaMemcpyAsync(base + b.s_off, sl.seg_host, 8ull * (b.nseg + 1), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return GLOP_ECUDA;
    glop_status rc = scan_split(S, b, base + b.m_off, base + b.p_off, b.cap);
    if (rc != GLOP_OK) return rc;
    b.eager = b.cap <= kEagerRows;
    if (cudaMemcpyAsync(sl.count_host, base + b.c_off, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(sl.first_host, base + b.f_off, 8ull * (b.nseg + 1), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return GLOP_ECUDA;
    if (b.eager && cudaMemcpyAsync(sl.eager, base + b.p_off, 8 * b.cap, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return GLOP_ECUDA;
    if (cudaEventRecord(sl.ev, st) != cudaSuccess) return GLOP_ECUDA;
    b.stage = 1;
    return GLOP_OK;
}

// stage 1 done: rescan on overflow, then each request's rows into its pinned result block
glop_status advance(glop_server_s *S, Batch &b) {
    Slot &sl = *b.slot;
    cudaStream_t st = sl.stream;
    const uint64_t total = *sl.count_host;
    if (total > b.cap) {
        ++S->stats.rescans;
        // outputs of the true size: from the budget when a block is free, else a device allocation
        const int64_t xo = S->arena.alloc(al(12 * total) + al(8 * total));
        if (xo >= 0) {
            b.extra_off = (uint64_t)xo;
            b.extra_len = al(12 * total) + al(8 * total);
            b.extra_out = S->arena.base + xo;
            b.extra_pairs = S->arena.base + xo + al(12 * total);
        } else if (cudaMalloc(&b.extra_out, 12 * total) != cudaSuccess ||
                   cudaMalloc(&b.extra_pairs, 8 * total) != cudaSuccess) {
            cudaGetLastError();
            return GLOP_ENOMEM;
        }
        glop_status rc = scan_split(S, b, b.extra_out, b.extra_pairs, total);
        if (rc != GLOP_OK) return rc;
        b.cap = total;
        b.eager = false;
        if (cudaMemcpyAsync(sl.first_host, S->arena.base + b.f_off, 8ull * (b.nseg + 1), cudaMemcpyDeviceToHost,
                            st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return GLOP_ECUDA;
    }
    b.total = total;
    const glop_match *dpairs =
        reinterpret_cast<const glop_match *>(b.extra_pairs ? b.extra_pairs : (void *)(S->arena.base + b.p_off));
    // every request's rows in one pinned block, copied back in one piece (or from the eager rows)
    Block *blk = new (std::nothrow) Block();
    if (!blk) return GLOP_ENOMEM;
    blk->p = S->pool.get(8 * (total + 1));
    if (!blk->p) {
        delete blk;
        return GLOP_ENOMEM;
    }
    glop_match *rows = reinterpret_cast<glop_match *>(blk->p);
    if (total) {
        if (b.eager) std::memcpy(rows, sl.eager, 8 * total);
        else if (cudaMemcpyAsync(rows, dpairs, 8 * total, cudaMemcpyDeviceToHost, st) != cudaSuccess) return GLOP_ECUDA;
    }
    size_t k = 0;
    for (auto &g : b.groups) {
        for (Request *r : g.second) {
            const uint32_t si = b.rseg[k++];
            const uint64_t lo = sl.first_host[si], hi = sl.first_host[si + 1];
            r->count = hi - lo;
            r->rows = rows + lo;
            r->blk = blk;
            ++blk->refs;
        }
    }
    if (!blk->refs) {
        S->pool.put(blk->p);
        delete blk;
    }
    if (cudaEventRecord(sl.ev, st) != cudaSuccess) return GLOP_ECUDA;
    b.stage = 2;
    return GLOP_OK;
}

void finish(glop_server_s *S, Batch *b) {
    const uint64_t t = now_ns();
    std::vector<Request *> done;
    std::lock_guard<std::mutex> lk(S->fin_mu);  // (the lane thread reads the densities)
    for (auto &g : b->groups) {
        uint64_t bytes = 0, matches = 0;
        for (Request *r : g.second) {
            r->done_ns = t;
            bytes += r->len;
            matches += r->count;
            done.push_back(r);
        }
        S->density[g.first] = std::max(0.97 * S->density[g.first], (double)matches / (double)std::max<uint64_t>(bytes, 1));
    }
    if (b->extra_len) {
        S->arena.release(b->extra_off, b->extra_len);
    } else {
        if (b->extra_out) cudaFree(b->extra_out);
        if (b->extra_pairs) cudaFree(b->extra_pairs);
    }
    S->arena.release(b->off, b->len);
    S->free_slots.push_back(b->slot);
    ++S->stats.batches;
    S->stats.requests_per_batch_max = std::max<uint64_t>(S->stats.requests_per_batch_max, done.size());
    S->stats.sets_per_batch_max = std::max<uint64_t>(S->stats.sets_per_batch_max, b->groups.size());
    S->finished.insert(S->finished.end(), done.begin(), done.end());
    delete b;
}

// the next batch: pending requests from the oldest, of every set of its kernel kind, within the limits
Batch *form(glop_server_s *S) {
    Request *r0 = S->pending.front();
    const uint32_t kind = S->kind[r0->set];
    std::map<uint32_t, std::vector<Request *>> by_set;
    uint64_t nbytes = 0, nreq = 0;
    double rows = 0;  // the output bound's estimate so far (matches per byte of each request's set)
    for (Request *r : S->pending) {
        if (S->kind[r->set] != kind) continue;
        const double rows2 = rows + S->density[r->set] * (double)r->len;
        const size_t groups2 = by_set.size() + (by_set.count(r->set) ? 0 : 1);
        if (nreq && (nbytes + r->len > S->o.max_batch_bytes || nreq >= S->o.max_batch_requests ||
                     groups2 > GLOP_BATCH_MAX_GROUPS ||
                     (uint64_t)(rows2 * 1.25) + 4096 > S->o.out_rows_per_batch))
            break;
        by_set[r->set].push_back(r);
        rows = rows2;
        nbytes += r->len;
        ++nreq;
    }
    Batch *b = new (std::nothrow) Batch();
    if (!b) return nullptr;
    b->groups.assign(by_set.begin(), by_set.end());
    return b;
}

void take(glop_server_s *S, const Batch &b) {
    std::vector<Request *> keep;
    keep.reserve(S->pending.size());
    std::map<Request *, int> in;
    for (auto &g : b.groups)
        for (Request *r : g.second) in[r] = 1;
    for (Request *r : S->pending)
        if (!in.count(r)) keep.push_back(r);
    S->pending.assign(keep.begin(), keep.end());
}

void lane_main(glop_server_s *S) {
    cudaSetDevice(S->device);
    while (true) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->lane_mu);
            S->lane_cv.wait(lk, [&] { return S->lane_stop || !S->lane_q.empty(); });
            if (S->lane_stop && S->lane_q.empty()) return;
            r = S->lane_q.front();
            S->lane_q.pop_front();
        }
        // results into the lane's pinned rows (two rows per payload byte, sized at creation); while a caller
        // still holds the previous lane result, into a block of the pool sized from the set's matches per
        // byte so far; one rescan into exact rows when a request has more matches than its rows
        double dens;
        {
            std::lock_guard<std::mutex> lk(S->fin_mu);
            dens = S->density[r->set];
        }
        uint64_t cap = S->lane_rows;
        glop_match *rows = nullptr;
        // (a caller that polls hands the previous lane result back within microseconds: wait up to 20 ms for
        // it rather than make a large pinned block, which can take longer than the scan)
        bool got = false;
        const uint64_t t_wait = now_ns() + 20000000ull;
        while (!(got = !S->lane_buf_busy.exchange(true)) && now_ns() < t_wait) std::this_thread::yield();
        if (got) rows = S->lane_buf;
        else cap = std::min<uint64_t>(S->lane_rows, (uint64_t)(2.5 * dens * (double)r->len) + 65536);
        while (true) {
            uint64_t need = 0;
            glop_scan_host_staging_size(S->sets[r->set], r->len, cap, &need);
            if (need > S->lane_staging_bytes) {  // (rare: a device allocation waits for the device)
                if (S->lane_staging) cudaFree(S->lane_staging);
                S->lane_staging = nullptr;
                S->lane_staging_bytes = 0;
                if (cudaMalloc(&S->lane_staging, need) != cudaSuccess) {
                    cudaGetLastError();
                    r->st = GLOP_ENOMEM;
                    break;
                }
                S->lane_staging_bytes = need;
            }
            if (!rows) {
                rows = reinterpret_cast<glop_match *>(S->pool.get(8 * (cap + 1)));
                if (!rows) {
                    r->st = GLOP_ENOMEM;
                    break;
                }
            }
            uint64_t cnt = 0;
            const glop_status rc = glop_scan_host(S->sets[r->set], r->payload, r->len, rows, cap, &cnt,
                                                  S->lane_staging, S->lane_staging_bytes, S->lane_stream);
            r->count = cnt;
            if (rc == GLOP_EOVERFLOW) {
                if (rows != S->lane_buf) S->pool.put(rows);
                else S->lane_buf_busy = false;
                rows = nullptr;
                cap = cnt + 65536;
                continue;
            }
            r->st = rc;
            break;
        }
        r->rows = rows;
        if (r->st == GLOP_OK) {
            std::lock_guard<std::mutex> lk(S->fin_mu);
            S->density[r->set] = std::max(0.97 * S->density[r->set], (double)r->count / (double)std::max<uint64_t>(r->len, 1));
        }
        r->done_ns = now_ns();
        std::lock_guard<std::mutex> lk(S->fin_mu);
        S->finished.push_back(r);
        --S->lane_active;
    }
}

}  // namespace

extern "C" {

glop_status glop_server_create(const glop_handle *sets, uint32_t n_sets, const glop_server_opts *opts,
                               glop_server *out) {
    if (!sets || !n_sets || !opts || !out) return GLOP_EINVAL;
    if (opts->max_inflight < 1 || opts->max_inflight > 16 || !opts->hbm_budget || !opts->max_batch_requests)
        return GLOP_EINVAL;
    glop_server_s *S = new (std::nothrow) glop_server_s();
    if (!S) return GLOP_ENOMEM;
    S->o = *opts;
    if (!S->o.out_rows_per_batch) S->o.out_rows_per_batch = std::max<uint64_t>(1 << 16, S->o.max_batch_bytes / 16);
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        return GLOP_ECUDA;
    }
    auto fail = [&](glop_status st) {
        glop_server_destroy(S);
        return st;
    };
    for (uint32_t i = 0; i < n_sets; ++i) {
        uint32_t k = 0;
        if (!sets[i] || glop_batch_multi_kind(sets[i], &k) != GLOP_OK) return fail(GLOP_EINVAL);
        S->sets.push_back(sets[i]);
        S->kind.push_back(k);
        S->density.push_back(0.25);
    }
    if (!S->arena.init(S->o.hbm_budget)) return fail(GLOP_ENOMEM);
    S->slots.resize(S->o.max_inflight);
    for (Slot &sl : S->slots) {
        sl.max_seg = S->o.max_batch_requests + GLOP_BATCH_MAX_GROUPS + 1;
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaHostAlloc(&sl.seg_host, 8ull * sl.max_seg, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc(&sl.first_host, 8ull * sl.max_seg, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc(&sl.count_host, 8, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc(&sl.eager, 8 * kEagerRows, cudaHostAllocDefault) != cudaSuccess)
            return fail(GLOP_ENOMEM);
        S->free_slots.push_back(&sl);
    }
    // result blocks made ahead of time (a pinned allocation in the loop stalls it for as long as the
    // allocation takes, ~0.1 s for a few hundred MiB): for every stream slot, blocks of 64 KiB to 16 MiB,
    // of 64 and 256 MiB, and of the largest batch's rows (one more of those than there are slots, for the
    // block whose requests the caller has not released yet)
    {
        std::vector<void *> warm;
        for (uint64_t sz = 1 << 16; sz <= (16ull << 20); sz <<= 2)
            for (uint32_t k = 0; k < 4 * S->o.max_inflight; ++k) warm.push_back(S->pool.get(sz));
        for (uint64_t sz = 64ull << 20; sz <= (256ull << 20); sz <<= 2)
            for (uint32_t k = 0; k < S->o.max_inflight; ++k) warm.push_back(S->pool.get(sz));
        const uint64_t top = 8 * (S->o.out_rows_per_batch + 1);
        if (top > (256ull << 20))
            for (uint32_t k = 0; k <= S->o.max_inflight; ++k) warm.push_back(S->pool.get(top));
        for (void *p : warm) {
            if (!p) return fail(GLOP_ENOMEM);
            S->pool.put(p);
        }
        S->warm_allocs = S->pool.allocs;
    }
    // latency first: the idle path and the lane run on the device's highest-priority streams, so their
    // kernels are scheduled ahead of a batch's when both wait for the SMs
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (S->o.fast_bytes) {
        S->fast_cap = std::max<uint64_t>(1 << 16, S->o.fast_bytes);
        glop_scan_host_staging_size(sets[0], S->o.fast_bytes, S->fast_cap, &S->fast_staging_bytes);
        if (cudaMalloc(&S->fast_staging, S->fast_staging_bytes) != cudaSuccess ||
            cudaHostAlloc(reinterpret_cast<void **>(&S->fast_out), 8 * S->fast_cap, cudaHostAllocDefault) != cudaSuccess ||
            cudaStreamCreateWithPriority(&S->fast_stream, cudaStreamNonBlocking, prio_hi) != cudaSuccess)
            return fail(GLOP_ENOMEM);
    }
    if (S->o.big_bytes) {
        if (cudaStreamCreateWithPriority(&S->lane_stream, cudaStreamNonBlocking, prio_hi) != cudaSuccess)
            return fail(GLOP_ECUDA);
        // device staging for the largest request with two result rows a byte, allocated up front
        const uint64_t mx = std::max(S->o.max_request_bytes, S->o.big_bytes);
        S->lane_rows = 2 * mx + 65536;
        glop_scan_host_staging_size(sets[0], mx, S->lane_rows, &S->lane_staging_bytes);
        if (cudaMalloc(&S->lane_staging, S->lane_staging_bytes) != cudaSuccess ||
            cudaHostAlloc(reinterpret_cast<void **>(&S->lane_buf), 8 * S->lane_rows, cudaHostAllocDefault) !=
                cudaSuccess)
            return fail(GLOP_ENOMEM);
        try {
            S->lane = std::thread(lane_main, S);
        } catch (...) {
            return fail(GLOP_ENOMEM);
        }
    }
    *out = S;
    return GLOP_OK;
}

glop_status glop_server_submit(glop_server S, uint64_t id, uint32_t set, const uint8_t *h_payload, uint64_t len) {
    if (!S || set >= S->sets.size() || (len && !h_payload) || len > 0xFFFFFFFFull) return GLOP_EINVAL;
    Request *r = new (std::nothrow) Request();
    if (!r) return GLOP_ENOMEM;
    r->id = id;
    r->set = set;
    r->payload = h_payload;
    r->len = len;
    ++S->stats.submitted;
    if (S->o.big_bytes && len >= S->o.big_bytes) {
        ++S->stats.big;
        ++S->lane_active;
        {
            std::lock_guard<std::mutex> lk(S->lane_mu);
            S->lane_q.push_back(r);
        }
        S->lane_cv.notify_one();
        return GLOP_OK;
    }
    S->pending.push_back(r);
    return GLOP_OK;
}

glop_status glop_server_poll(glop_server S, glop_server_result *res, uint32_t max_res, uint32_t *n_res,
                             uint32_t wait_us) {
    if (!S || !n_res || (max_res && !res)) return GLOP_EINVAL;
    *n_res = 0;
    const uint64_t t_end = now_ns() + 1000ull * wait_us;
    uint32_t idle = 0;  // loop iterations since the last completion or launch
    while (true) {
        const size_t n_inflight = S->inflight.size(), n_pending = S->pending.size();
        // completions
        for (size_t i = 0; i < S->inflight.size();) {
            Batch *b = S->inflight[i];
            const cudaError_t q = cudaEventQuery(b->slot->ev);
            if (q == cudaErrorNotReady) {
                ++i;
                continue;
            }
            if (q != cudaSuccess) return GLOP_ECUDA;
            idle = 0;
            if (b->stage == 1) {
                const glop_status rc = advance(S, *b);
                if (rc != GLOP_OK) return rc;
                ++i;
                continue;
            }
            S->inflight.erase(S->inflight.begin() + i);
            finish(S, b);
        }
        // new work while stream slots allow
        while (!S->pending.empty() && !S->free_slots.empty()) {
            Request *r0 = S->pending.front();
            if (S->inflight.empty() && S->pending.size() == 1 && S->o.fast_bytes && r0->len <= S->o.fast_bytes) {
                // rows for this request from the set's matches per byte so far (a block sized for the
                // largest fast request would drain the pool's large blocks and make new ones in the loop);
                // more matches than that: once more with the exact count, while it fits the fast path
                double dens;
                {
                    std::lock_guard<std::mutex> lk(S->fin_mu);
                    dens = S->density[r0->set];
                }
                uint64_t fcap = std::min<uint64_t>(S->fast_cap, (uint64_t)(2.5 * dens * (double)r0->len) + 65536);
                glop_status rc = GLOP_EOVERFLOW;
                uint64_t cnt = 0;
                for (int pass = 0; pass < 2 && rc == GLOP_EOVERFLOW; ++pass) {
                    if (pass) {
                        if (cnt > S->fast_cap) break;
                        fcap = cnt;
                        ++S->stats.rescans;
                    }
                    r0->rows = reinterpret_cast<glop_match *>(S->pool.get(8 * (fcap + 1)));
                    if (!r0->rows) return GLOP_ENOMEM;
                    rc = glop_scan_host(S->sets[r0->set], r0->payload, r0->len, r0->rows, fcap, &cnt, S->fast_staging,
                                        S->fast_staging_bytes, S->fast_stream);
                    if (rc != GLOP_OK) {
                        S->pool.put(r0->rows);
                        r0->rows = nullptr;
                    }
                }
                if (rc == GLOP_OK) {
                    r0->count = cnt;
                    r0->done_ns = now_ns();
                    S->pending.pop_front();
                    ++S->stats.fast;
                    std::lock_guard<std::mutex> lk(S->fin_mu);
                    if (r0->len >= (1u << 20))  // (a small request's density says little about the set's)
                        S->density[r0->set] = std::max(0.97 * S->density[r0->set], (double)cnt / (double)r0->len);
                    S->finished.push_back(r0);
                    continue;
                }
                if (rc != GLOP_EOVERFLOW) return rc;
                // more matches than the fast path holds: scan it as a batch
            }
            Batch *b = form(S);
            if (!b) return GLOP_ENOMEM;
            bool placed = false;
            while (true) {
                layout(*b);
                const uint64_t cap = cap_of(S, b->groups);
                if (regions(S, *b, cap)) {
                    placed = true;
                    break;
                }
                size_t nr = 0;
                for (auto &g : b->groups) nr += g.second.size();
                if (nr <= 1) {
                    // one request: try the smallest output bound (a rescan makes a larger one)
                    if (S->inflight.empty() && regions(S, *b, 4096)) placed = true;
                    break;
                }
                // keep the older half of the batch
                std::vector<Request *> all;
                for (auto &g : b->groups) all.insert(all.end(), g.second.begin(), g.second.end());
                std::map<Request *, size_t> order;
                for (size_t i = 0; i < S->pending.size(); ++i) order[S->pending[i]] = i;
                std::sort(all.begin(), all.end(), [&](Request *x, Request *y) { return order[x] < order[y]; });
                all.resize((all.size() + 1) / 2);
                std::map<uint32_t, std::vector<Request *>> by;
                for (Request *r : all) by[r->set].push_back(r);
                b->groups.assign(by.begin(), by.end());
            }
            if (!placed) {
                delete b;
                ++S->stats.admission_waits;
                if (S->inflight.empty()) return GLOP_ENOMEM;  // a request larger than the whole budget
                break;
            }
            b->slot = S->free_slots.back();
            if (b->nseg + 1 > b->slot->max_seg) {
                S->arena.release(b->off, b->len);
                delete b;
                return GLOP_EINVAL;
            }
            S->free_slots.pop_back();
            take(S, *b);
            const glop_status rc = launch(S, *b);
            if (rc != GLOP_OK) return rc;
            S->inflight.push_back(b);
        }
        // hand out finished requests
        {
            std::lock_guard<std::mutex> lk(S->fin_mu);
            while (*n_res < max_res && !S->finished.empty()) {
                Request *r = S->finished.front();
                S->finished.erase(S->finished.begin());
                glop_server_result &o = res[(*n_res)++];
                o.id = r->id;
                o.status = r->st;
                o.matches = r->rows;
                o.count = r->count;
                o.done_ns = r->done_ns;
                S->handed[r->id] = r;
            }
        }
        if (*n_res || now_ns() >= t_end) break;
        if (S->inflight.empty() && S->pending.empty() && !S->lane_active) break;
        // Waiting: after a few idle turns the loop sleeps between rounds of event queries instead of spinning
        // on them, leaving the core (and the driver) to the lane's thread and the caller.
        if (S->inflight.size() != n_inflight || S->pending.size() != n_pending) idle = 0;
        if (++idle > 16) std::this_thread::sleep_for(std::chrono::microseconds(10));
        else std::this_thread::yield();
    }
    return GLOP_OK;
}

glop_status glop_server_release(glop_server S, uint64_t id) {
    if (!S) return GLOP_EINVAL;
    auto it = S->handed.find(id);
    if (it == S->handed.end()) return GLOP_EINVAL;
    Request *r = it->second;
    if (r->blk) {
        if (--r->blk->refs == 0) {
            S->pool.put(r->blk->p);
            delete r->blk;
        }
    } else if (r->rows && r->rows == S->lane_buf) {
        S->lane_buf_busy = false;
    } else {
        S->pool.put(r->rows);
    }
    delete it->second;
    S->handed.erase(it);
    return GLOP_OK;
}

glop_status glop_server_stats_get(glop_server S, glop_server_stats *st) {
    if (!S || !st) return GLOP_EINVAL;
    *st = S->stats;
    st->pending = S->pending.size();
    st->inflight = S->inflight.size();
    st->pinned_allocs = S->pool.allocs - S->warm_allocs;
    return GLOP_OK;
}

glop_status glop_server_destroy(glop_server S) {
    if (!S) return GLOP_OK;
    if (S->lane.joinable()) {
        {
            std::lock_guard<std::mutex> lk(S->lane_mu);
            S->lane_stop = true;
        }
        S->lane_cv.notify_one();
        S->lane.join();
    }
    for (Slot &sl : S->slots)
        if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (S->lane_stream) cudaStreamSynchronize(S->lane_stream);
    std::vector<Block *> blocks;  // (shared by several requests: deleted once)
    auto drop = [&](Request *r) {
        if (r->blk && std::find(blocks.begin(), blocks.end(), r->blk) == blocks.end()) blocks.push_back(r->blk);
        delete r;
    };
    for (Batch *b : S->inflight) {
        if (!b->extra_len && b->extra_out) cudaFree(b->extra_out);
        if (!b->extra_len && b->extra_pairs) cudaFree(b->extra_pairs);
        for (auto &g : b->groups)
            for (Request *r : g.second) drop(r);
        delete b;
    }
    for (Request *r : S->pending) drop(r);
    for (Request *r : S->finished) drop(r);
    for (auto &kv : S->handed) drop(kv.second);
    for (Block *b : blocks) delete b;
    for (Slot &sl : S->slots) {
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.seg_host) cudaFreeHost(sl.seg_host);
        if (sl.first_host) cudaFreeHost(sl.first_host);
        if (sl.count_host) cudaFreeHost(sl.count_host);
        if (sl.eager) cudaFreeHost(sl.eager);
    }
    if (S->fast_staging) cudaFree(S->fast_staging);
    if (S->fast_out) cudaFreeHost(S->fast_out);
    if (S->fast_stream) cudaStreamDestroy(S->fast_stream);
    if (S->lane_staging) cudaFree(S->lane_staging);
    if (S->lane_buf) cudaFreeHost(S->lane_buf);
    if (S->lane_stream) cudaStreamDestroy(S->lane_stream);
    S->arena.destroy();
    S->pool.destroy();
    delete S;
    return GLOP_OK;
}

}  // extern "C"
