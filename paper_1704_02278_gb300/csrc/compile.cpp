// compile.cpp -- build the failureless trie of a pattern set and lay it out
// for the scan kernels.
//
// Sec. 4 builds the Aho-Corasick state machine from the patterns in a first
// phase; Sec. 5 removes its failure transitions (the failureless trie of
// PFAC) so that one walk can start at every text byte.  Sec. 5 also notes
// that truncating the trie to a prefix depth (prefix matching) shrinks the
// state machine; prefix_len implements that cut.  The layout below is this
// library's own (see glop_layout.h): breadth-first dense rows over a
// compressed alphabet for branching states, byte strings for unary chains,
// per-state sorted output lists, and a start filter over the first gram_len
// bytes.
#include "compile.h"

#include <algorithm>
#include <cstring>
#include <map>

#include "glop_hash.h"

namespace glop {

namespace {

constexpr uint32_t NIL = 0xFFFFFFFFu;

uint32_t ceil_log2(uint64_t x) {
    uint32_t k = 0;
    while ((1ull << k) < x) ++k;
    return k;
}

}  // namespace

int compile_host(const uint8_t *bytes, const uint64_t *offs, uint32_t n, uint32_t prefix_len, HostAutomaton *out,
                 std::string *err, uint32_t want_gram, uint32_t want_bm_log2) {
    HostAutomaton &A = *out;
    A = HostAutomaton();
    if (!offs || (n && !bytes)) { if (err) *err = "null pointer"; return 1; }
    if (n > 0x80000000u) { if (err) *err = "too many patterns"; return 1; }

    // ---- effective patterns (prefix cut) ----
    std::vector<uint32_t> len(n);
    uint64_t total = 0;
    uint32_t minlen = 0xFFFFFFFFu, maxlen = 0;
    for (uint32_t j = 0; j < n; ++j) {
        if (offs[j + 1] < offs[j]) { if (err) *err = "decreasing pattern offsets"; return 1; }
        uint64_t L = offs[j + 1] - offs[j];
        if (prefix_len && L > prefix_len) L = prefix_len;
        if (L == 0) { if (err) *err = "zero-length pattern " + std::to_string(j); return 1; }
        if (L > 0x7FFFFFFFull) { if (err) *err = "pattern too long"; return 1; }
        len[j] = (uint32_t)L;
        total += L;
        minlen = std::min(minlen, (uint32_t)L);
        maxlen = std::max(maxlen, (uint32_t)L);
    }
    if (total + 1 > 0x7FFFFFFFull) { if (err) *err = "pattern set too large"; return 1; }
    A.n_patterns = n;
    A.min_len = n ? minlen : 0;
    A.max_len = maxlen;

    // ---- trie (goto graph) from the patterns in lexicographic order ----
    std::vector<uint32_t> order(n);
    for (uint32_t j = 0; j < n; ++j) order[j] = j;
    auto pbytes = [&](uint32_t j) { return bytes + offs[j]; };
    std::sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
        uint32_t m = std::min(len[a], len[b]);
        int c = std::memcmp(pbytes(a), pbytes(b), m);
        if (c) return c < 0;
        if (len[a] != len[b]) return len[a] < len[b];
        return a < b;
    });
    size_t cap = (size_t)total + 1;
    std::vector<uint32_t> parent, first_child, last_child, next_sib, nchild, depth;
    std::vector<uint8_t> ebyte;
    parent.reserve(cap); first_child.reserve(cap); last_child.reserve(cap); next_sib.reserve(cap);
    nchild.reserve(cap); depth.reserve(cap); ebyte.reserve(cap);
    auto new_node = [&](uint32_t par, uint8_t b, uint32_t d) {
        uint32_t id = (uint32_t)parent.size();
        parent.push_back(par); ebyte.push_back(b); depth.push_back(d);
        first_child.push_back(NIL); last_child.push_back(NIL); next_sib.push_back(NIL); nchild.push_back(0);
        if (par != NIL) {
            if (last_child[par] == NIL) first_child[par] = id; else next_sib[last_child[par]] = id;
            last_child[par] = id;
            ++nchild[par];
        }
        return id;
    };
    new_node(NIL, 0, 0);  // initial state
    std::vector<uint32_t> path((size_t)maxlen + 1, 0);
    std::vector<std::pair<uint32_t, uint32_t>> own;  // (node, pattern id)
    own.reserve(n);
    int64_t prev = -1;
    for (uint32_t k = 0; k < n; ++k) {
        uint32_t j = order[k];
        const uint8_t *p = pbytes(j);
        uint32_t l = 0;
        if (prev >= 0) {
            uint32_t pj = (uint32_t)prev, m = std::min(len[pj], len[j]);
            const uint8_t *q = pbytes(pj);
            while (l < m && q[l] == p[l]) ++l;
        }
        for (uint32_t d = l; d < len[j]; ++d) path[d + 1] = new_node(path[d], p[d], d + 1);
        own.emplace_back(path[len[j]], j);
        prev = j;
    }
    const uint32_t N = (uint32_t)parent.size();
    std::sort(own.begin(), own.end());
    std::vector<uint32_t> own_start(N + 1, 0);
    for (auto &o : own) ++own_start[o.first + 1];
    for (uint32_t v = 0; v < N; ++v) own_start[v + 1] += own_start[v];
    auto terminal = [&](uint32_t v) { return own_start[v + 1] > own_start[v]; };

    // ---- numbering: dense states in BFS order, then chains ----
    std::vector<uint32_t> bfs;
    bfs.reserve(N);
    bfs.push_back(0);
    for (size_t h = 0; h < bfs.size(); ++h)
        for (uint32_t c = first_child[bfs[h]]; c != NIL; c = next_sib[c]) bfs.push_back(c);
    auto is_dense = [&](uint32_t v) { return v == 0 || nchild[v] >= 2; };
    std::vector<uint32_t> nid(N, NIL);
    uint32_t next_id = 0;
    for (uint32_t v : bfs) if (is_dense(v)) nid[v] = next_id++;
    A.n_dense = next_id;
    std::vector<std::vector<uint32_t>> chains;  // node lists, in head BFS order
    for (uint32_t v : bfs) {
        if (is_dense(v) || !is_dense(parent[v])) continue;
        std::vector<uint32_t> ch;
        uint32_t u = v;
        while (true) {
            ch.push_back(u);
            nid[u] = next_id++;
            uint32_t c = first_child[u];
            if (c == NIL || is_dense(c)) break;
            u = c;
        }
        chains.push_back(std::move(ch));
    }
    if (next_id != N) { if (err) *err = "internal: numbering"; return 7; }
    A.n_states = N;
    A.depth.assign(N, 0);
    for (uint32_t v = 0; v < N; ++v) A.depth[nid[v]] = depth[v];
    auto enc = [&](uint32_t v) { return nid[v] | (terminal(v) ? GLOP_TERM : 0u); };

    // ---- alphabet classes: bytes with identical dense-row columns share a class ----
    std::vector<std::vector<uint64_t>> col(256);
    std::vector<uint32_t> dense_nodes(A.n_dense);
    for (uint32_t v = 0; v < N; ++v) if (is_dense(v)) dense_nodes[nid[v]] = v;
    for (uint32_t d = 0; d < A.n_dense; ++d)
        for (uint32_t c = first_child[dense_nodes[d]]; c != NIL; c = next_sib[c])
            col[ebyte[c]].push_back(((uint64_t)d << 32) | enc(c));
    std::map<std::vector<uint64_t>, uint32_t> classes;
    A.cls.assign(256, 0);
    // the class of bytes with no transition anywhere gets number 0 when it exists
    std::vector<uint64_t> empty;
    for (int b = 0; b < 256; ++b) if (col[b].empty()) { classes.emplace(empty, 0u); break; }
    for (int b = 0; b < 256; ++b) {
        auto it = classes.find(col[b]);
        if (it == classes.end()) it = classes.emplace(col[b], (uint32_t)classes.size()).first;
        A.cls[b] = (uint8_t)it->second;
    }
    A.n_classes = (uint32_t)classes.size();
    const uint32_t C = A.n_classes;
    A.rows.assign((size_t)A.n_dense * C, 0);
    for (uint32_t d = 0; d < A.n_dense; ++d)
        for (uint32_t c = first_child[dense_nodes[d]]; c != NIL; c = next_sib[c])
            A.rows[(size_t)d * C + A.cls[ebyte[c]]] = (int32_t)enc(c);

    // ---- chains, cut into pieces of at most 16 states ----
    A.chain.resize(N - A.n_dense);
    for (auto &ch : chains) {
        const uint32_t L = (uint32_t)ch.size();
        const uint32_t last = ch[L - 1];
        const uint32_t dense_child = first_child[last];  // NIL or a dense state
        uint32_t term = 0;
        for (uint32_t k = 0; k < L; ++k) {
            if (terminal(ch[k])) term = nid[ch[k]];
            const uint32_t p0 = k / 16 * 16, p1 = std::min(L, p0 + 16);  // piece [p0, p1)
            const bool final_piece = (p1 == L);
            uint32_t exit = 0, exit_byte = 0, has_exit = 0;
            if (!final_piece) { exit = enc(ch[p1]); exit_byte = ebyte[ch[p1]]; has_exit = 1; }
            else if (dense_child != NIL) { exit = enc(dense_child); exit_byte = ebyte[dense_child]; has_exit = 1; }
            GlopChain g;
            std::memset(&g, 0, sizeof g);
            uint8_t b[16] = {0};
            uint32_t nb = 0;
            for (uint32_t x = k + 1; x < p1; ++x) b[nb++] = ebyte[ch[x]];
            if (has_exit) b[nb++] = (uint8_t)exit_byte;
            std::memcpy(g.inl, b, 16);
            g.exit = exit;
            g.term = term;
            uint16_t tm = 0;
            for (uint32_t x = k; x < p1; ++x) if (terminal(ch[x])) tm |= (uint16_t)(1u << (x - k));
            g.termmask = tm;
            g.nst = (uint8_t)(p1 - 1 - k);
            g.rem = (uint8_t)(p1 - 1 - k + has_exit);
            A.chain[nid[ch[k]] - A.n_dense] = g;
        }
    }

    // ---- per-state output lists: own ids merged with the nearest terminal ancestor's list ----
    std::vector<uint64_t> lst_start(N, 0), lst_len(N, 0);
    std::vector<uint32_t> pool;
    std::vector<uint32_t> nta(N, NIL);  // nearest terminal ancestor-or-self
    for (uint32_t v : bfs) {
        uint32_t up = (v == 0) ? NIL : nta[parent[v]];
        if (!terminal(v)) { nta[v] = up; continue; }
        nta[v] = v;
        size_t s = pool.size();
        const uint32_t *a = (up == NIL) ? nullptr : pool.data() + lst_start[up];
        size_t na = (up == NIL) ? 0 : lst_len[up];
        std::vector<uint32_t> merged;
        merged.reserve(na + own_start[v + 1] - own_start[v]);
        std::vector<uint32_t> mine;
        for (uint32_t k = own_start[v]; k < own_start[v + 1]; ++k) mine.push_back(own[k].second);
        std::merge(a, a + na, mine.begin(), mine.end(), std::back_inserter(merged));
        if (pool.size() + merged.size() > 0xFFFFFFF0ull) { if (err) *err = "output lists too large"; return 1; }
        pool.insert(pool.end(), merged.begin(), merged.end());
        lst_start[v] = s;
        lst_len[v] = merged.size();
    }
    A.cum_off.assign((size_t)N + 1, 0);
    std::vector<uint32_t> by_id(N);
    for (uint32_t v = 0; v < N; ++v) by_id[nid[v]] = v;
    for (uint32_t s = 0; s < N; ++s) A.cum_off[s + 1] = A.cum_off[s] + (uint32_t)lst_len[by_id[s]];
    A.cum_ids.resize(A.cum_off[N]);
    for (uint32_t s = 0; s < N; ++s) {
        uint32_t v = by_id[s];
        std::copy(pool.begin() + lst_start[v], pool.begin() + lst_start[v] + lst_len[v],
                  A.cum_ids.begin() + A.cum_off[s]);
    }

    // ---- start filter over the first gram_len bytes (all patterns >= 4 bytes) ----
    if (n && A.min_len >= 4) {
        uint32_t g = std::min<uint32_t>(A.min_len, 8);
        if (want_gram) g = std::max<uint32_t>(4, std::min(g, want_gram));
        A.gram_len = g;
        std::vector<uint32_t> keys;
        for (uint32_t v : bfs) if (depth[v] == g) keys.push_back(v);
        A.n_grams = (uint32_t)keys.size();
        A.bm_log2 = std::min<uint32_t>(19, std::max<uint32_t>(13, ceil_log2((uint64_t)keys.size() * 64)));
        if (want_bm_log2) A.bm_log2 = std::min<uint32_t>(19, std::max<uint32_t>(13, want_bm_log2));
        A.ht_log2 = std::max<uint32_t>(6, ceil_log2((uint64_t)keys.size() * 2));
        A.bitmap.assign((1u << A.bm_log2) / 32, 0);
        A.grams.assign(1u << A.ht_log2, GlopGramSlot{0, 0, 0, 0});
        const uint32_t mask1 = glop_w1_mask(g);
        for (uint32_t v : keys) {
            uint8_t gb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            uint32_t u = v;
            for (int k = (int)g - 1; k >= 0; --k) { gb[k] = ebyte[u]; u = parent[u]; }
            uint32_t w0 = (uint32_t)gb[0] | ((uint32_t)gb[1] << 8) | ((uint32_t)gb[2] << 16) | ((uint32_t)gb[3] << 24);
            uint32_t w1 = ((uint32_t)gb[4] | ((uint32_t)gb[5] << 8) | ((uint32_t)gb[6] << 16) | ((uint32_t)gb[7] << 24)) & mask1;
            uint32_t h = glop_gram_hash(w0, w1);
            A.bitmap[glop_bitmap_word(h, A.bm_log2)] |= 0x80000000u >> glop_bitmap_bit(h, w0, g, A.bm_log2);
            uint32_t slot = glop_table_slot(h, A.ht_log2), m = (1u << A.ht_log2) - 1;
            while (A.grams[slot].val) slot = (slot + 1) & m;
            A.grams[slot] = GlopGramSlot{w0, w1, enc(v), 0};
        }
        uint32_t lo = 0;
        while (lo < A.n_dense && A.depth[lo] < g) ++lo;
        A.hot_lo = lo;
    } else {
        A.gram_len = 0;
        A.hot_lo = 0;
    }
    return 0;
}

}  // namespace glop
