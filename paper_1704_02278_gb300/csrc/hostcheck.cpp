// hostcheck.cpp -- test-only host check of the compiled tables.
//
// Built into a separate library (libglop_hostcheck.so) that the CPU test
// suite loads; libglop.so does not contain it and no scan entry point calls
// it.  It runs the GPU walk's decision rules (start filter, gram table,
// dense rows, chain comparison, per-state output lists) sequentially over
// the compiler's host tables, so that the compiler can be checked against the
// oracle on a machine without a GPU.  It is not a scan path of the library.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "compile.h"
#include "glop_hash.h"

using glop::HostAutomaton;

static uint32_t g_gram_len = 0, g_bm_log2 = 0;  // compile options of the next host checks

namespace {

uint32_t rd32(const uint8_t *p, uint64_t avail) {
    uint32_t w = 0;
    for (uint64_t k = 0; k < 4 && k < avail; ++k) w |= (uint32_t)p[k] << (8 * k);
    return w;
}

struct WalkStats {
    uint64_t dense_steps = 0, chain_entries = 0, chain_bytes = 0, hot_steps = 0;
    uint32_t iters = 0;  // loop iterations of the last walk
};

// deepest terminal state reached from state s with the next text byte at pos
uint32_t walk(const HostAutomaton &A, const uint8_t *text, uint32_t s, uint64_t pos, uint64_t end, uint32_t t,
              WalkStats &ws) {
    const uint32_t C = A.n_classes;
    ws.iters = 0;
    while (true) {
        ++ws.iters;
        if (s < A.n_dense) {
            if (pos >= end) return t;
            ++ws.dense_steps;
            int32_t e = A.rows[(size_t)s * C + A.cls[text[pos]]];
            if (!e) return t;
            s = (uint32_t)e & GLOP_STATE_MASK;
            ++pos;
            if ((uint32_t)e & GLOP_TERM) t = s;
        } else {
            const GlopChain &ch = A.chain[s - A.n_dense];
            ++ws.chain_entries;
            uint8_t inl[16];
            std::memcpy(inl, ch.inl, 16);
            uint64_t lim = std::min<uint64_t>(ch.rem, end - pos);
            uint64_t m = 0;
            while (m < lim && text[pos + m] == inl[m]) ++m;
            ws.chain_bytes += m + (m < lim ? 1 : 0);
            uint32_t r = (uint32_t)std::min<uint64_t>(m, ch.nst);
            uint32_t tm = ch.termmask & ((2u << r) - 1u);
            if (tm) {
                uint32_t hb = 31;
                while (!((tm >> hb) & 1u)) --hb;
                t = s + hb;
            } else if (ch.term) {
                t = ch.term;
            }
            if (ch.exit && m == ch.rem) {
                s = ch.exit & GLOP_STATE_MASK;
                if (ch.exit & GLOP_TERM) t = s;
                pos += m;
                continue;
            }
            return t;
        }
    }
}

}  // namespace

extern "C" {

// Compile the pattern set, then report every (segment, offset, pattern_id)
// of text by the GPU's decision rules.  stats[0..3] = n_states, n_dense,
// n_classes, gram_len; stats[4] = offsets passing the start filter;
// stats[5] = offsets found in the gram table; stats[6..8] = dense-row steps,
// chain entries and chain bytes compared by all walks; stats[9] = offsets
// with at least one match.  Returns a glop_status value.
int glop_hostcheck_scan_iters(const uint8_t *pat, const uint64_t *poff, uint32_t npat, uint32_t prefix_len,
                              const uint8_t *text, const uint64_t *seg, uint32_t nseg, uint32_t **out,
                              uint64_t *count, uint64_t *stats, uint8_t *iters);

int glop_hostcheck_scan(const uint8_t *pat, const uint64_t *poff, uint32_t npat, uint32_t prefix_len,
                        const uint8_t *text, const uint64_t *seg, uint32_t nseg, uint32_t **out, uint64_t *count,
                        uint64_t *stats) {
    return glop_hostcheck_scan_iters(pat, poff, npat, prefix_len, text, seg, nseg, out, count, stats, nullptr);
}

// As glop_hostcheck_scan; iters (one byte per text byte, may be NULL) receives
// 255 for offsets that fail the start filter, else the walk's loop iterations
// (0 when the gram table has no entry).
int glop_hostcheck_scan_iters(const uint8_t *pat, const uint64_t *poff, uint32_t npat, uint32_t prefix_len,
                              const uint8_t *text, const uint64_t *seg, uint32_t nseg, uint32_t **out,
                              uint64_t *count, uint64_t *stats, uint8_t *iters) {
    *out = nullptr;
    *count = 0;
    HostAutomaton A;
    std::string err;
    int rc = glop::compile_host(pat, poff, npat, prefix_len, &A, &err, g_gram_len, g_bm_log2);
    if (rc) return rc;
    std::vector<uint32_t> res;
    uint64_t passed = 0, found = 0, matched = 0;
    WalkStats wst;
    const uint32_t g = A.gram_len;
    for (uint32_t sg = 0; sg < nseg && npat; ++sg) {
        uint64_t lo = seg[sg], hi = seg[sg + 1];
        for (uint64_t i = lo; i < hi; ++i) {
            uint32_t s, t = 0;
            uint64_t pos;
            if (g) {
                if (i + g > hi) continue;
                uint32_t w0 = rd32(text + i, hi - i);
                uint32_t w1 = rd32(text + i + 4, hi - i - 4) & glop_w1_mask(g);
                uint32_t h = glop_gram_hash(w0, w1);
                const uint32_t bw = glop_bitmap_word(h, A.bm_log2), bb = glop_bitmap_bit(h, w0, g, A.bm_log2);
                if (iters) iters[i] = 255;
                if (!((A.bitmap[bw] << bb) & 0x80000000u)) continue;
                if (iters) iters[i] = 0;
                ++passed;
                uint32_t m = (1u << A.ht_log2) - 1, slot = glop_table_slot(h, A.ht_log2), v = 0;
                while (A.grams[slot].val) {
                    if (A.grams[slot].key_lo == w0 && A.grams[slot].key_hi == w1) { v = A.grams[slot].val; break; }
                    slot = (slot + 1) & m;
                }
                if (!v) continue;
                ++found;
                s = v & GLOP_STATE_MASK;
                if (v & GLOP_TERM) t = s;
                pos = i + g;
            } else {
                s = 0;
                pos = i;
            }
            t = walk(A, text, s, pos, hi, t, wst);
            if (iters) iters[i] = (uint8_t)std::min<uint32_t>(wst.iters, 254);
            if (t) ++matched;
            for (uint32_t k = A.cum_off[t]; t && k < A.cum_off[t + 1]; ++k) {
                res.push_back(sg);
                res.push_back((uint32_t)(i - lo));
                res.push_back(A.cum_ids[k]);
            }
        }
    }
    if (stats) {
        stats[0] = A.n_states; stats[1] = A.n_dense; stats[2] = A.n_classes; stats[3] = A.gram_len;
        stats[4] = passed; stats[5] = found;
        stats[6] = wst.dense_steps; stats[7] = wst.chain_entries; stats[8] = wst.chain_bytes; stats[9] = matched;
    }
    *count = res.size() / 3;
    if (!res.empty()) {
        *out = (uint32_t *)std::malloc(res.size() * sizeof(uint32_t));
        if (!*out) return 2;
        std::memcpy(*out, res.data(), res.size() * sizeof(uint32_t));
    }
    return 0;
}

void glop_hostcheck_free(void *p) { std::free(p); }

// Start-filter options (gram length, bitmap bits) for the following checks; 0 = automatic.
void glop_hostcheck_set_options(uint32_t gram_len, uint32_t bm_log2) {
    g_gram_len = gram_len;
    g_bm_log2 = bm_log2;
}

}  // extern "C"
