// synth.cpp -- seeded synthetic inputs shaped like the paper's workloads.
//
// This module only draws random inputs (texts, packet payloads, pattern sets,
// sizes).  It holds none of the search arithmetic and is shared by the GPU
// tests, the oracle tests and the benchmark as the single source of inputs.
//
// The paper generated its logs with the Mersenne Twister uniform generator
// (Sec. 6); every stream here is a std::mt19937_64 seeded by the caller.
// Vocabulary words, host/process names and HTTP-like tokens are random
// strings drawn from the seed: no real word list, rule set or corpus is used.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <random>
#include <string>
#include <thread>
#include <vector>

namespace {

using Rng = std::mt19937_64;

static uint64_t uni(Rng& r, uint64_t lo, uint64_t hi) {  // inclusive
    return lo + (r() % (hi - lo + 1));
}
static double unif01(Rng& r) { return (double)(r() >> 11) * (1.0 / 9007199254740992.0); }

static std::string rand_lower(Rng& r, int lo, int hi) {
    int L = (int)uni(r, lo, hi);
    std::string s(L, 'a');
    for (auto& c : s) c = (char)('a' + uni(r, 0, 25));
    return s;
}

static std::string rand_alnum(Rng& r, int lo, int hi) {
    static const char A[] = "abcdefghijklmnopqrstuvwxyz0123456789";
    int L = (int)uni(r, lo, hi);
    std::string s(L, 'a');
    for (auto& c : s) c = A[uni(r, 0, 35)];
    return s;
}

// 2,000-word vocabulary with a Zipf(1.1) rank distribution, 50 host names and
// 30 process names, all drawn from one seed.
struct Vocab {
    std::vector<std::string> words;   // by rank (rank 0 = most frequent)
    std::vector<double> cdf;          // Zipf cumulative distribution over ranks
    std::vector<std::string> hosts, procs;

    explicit Vocab(uint64_t seed, int nwords = 2000, double s = 1.1) {
        Rng r(seed);
        words.reserve(nwords);
        for (int i = 0; i < nwords; ++i) words.push_back(rand_lower(r, 2, 12));
        cdf.resize(nwords);
        double acc = 0;
        for (int i = 0; i < nwords; ++i) { acc += std::pow((double)(i + 1), -s); cdf[i] = acc; }
        for (auto& c : cdf) c /= acc;
        for (int i = 0; i < 50; ++i) hosts.push_back(rand_alnum(r, 4, 12));
        for (int i = 0; i < 30; ++i) procs.push_back(rand_lower(r, 3, 10));
    }
    const std::string& zipf_word(Rng& r) const {
        double u = unif01(r);
        size_t k = std::lower_bound(cdf.begin(), cdf.end(), u) - cdf.begin();
        if (k >= words.size()) k = words.size() - 1;
        return words[k];
    }
};

struct PatternView {
    const uint8_t* bytes;
    const uint64_t* offs;
    uint32_t n;
};

// syslog-style lines: "YYYY-MM-DDThh:mm:ss.mmmZ host proc[pid]: msg\n", msg =
// 4..20 Zipf words; with probability plant_rate a line's message carries one
// uniformly chosen pattern as an extra word.  Fills exactly nbytes (the last
// line is cut).  Returns the number of planted patterns.
static uint64_t gen_syslog(const Vocab& V, uint64_t seed, uint8_t* out, uint64_t nbytes, double plant_rate,
                           const PatternView& P) {
    Rng r(seed);
    uint64_t at = 0, planted = 0;
    int year = 2016 + (int)uni(r, 0, 2), mon = 1 + (int)uni(r, 0, 11), day = 1 + (int)uni(r, 0, 27);
    int64_t ms = (int64_t)uni(r, 0, 86399999);
    std::string line;
    line.reserve(512);
    char ts[64];
    while (at < nbytes) {
        ms += (int64_t)uni(r, 0, 50);
        if (ms >= 86400000) {
            ms -= 86400000;
            if (++day > 28) { day = 1; if (++mon > 12) { mon = 1; ++year; } }
        }
        int h = (int)(ms / 3600000), mi = (int)(ms / 60000 % 60), se = (int)(ms / 1000 % 60), mm = (int)(ms % 1000);
        std::snprintf(ts, sizeof ts, "%04d-%02d-%02dT%02d:%02d:%02d.%03dZ ", year, mon, day, h, mi, se, mm);
        line.assign(ts);
        line += V.hosts[uni(r, 0, V.hosts.size() - 1)];
        line += ' ';
        line += V.procs[uni(r, 0, V.procs.size() - 1)];
        line += '[';
        line += std::to_string(uni(r, 1, 65535));
        line += "]: ";
        int nw = (int)uni(r, 4, 20);
        int plant_at = -1;
        if (P.n && unif01(r) < plant_rate) plant_at = (int)uni(r, 0, nw);
        for (int w = 0; w <= nw; ++w) {
            if (w == plant_at) {
                uint32_t j = (uint32_t)uni(r, 0, P.n - 1);
                if (w == nw && nw > 0) line += ' ';
                line.append((const char*)P.bytes + P.offs[j], (size_t)(P.offs[j + 1] - P.offs[j]));
                ++planted;
                if (w < nw) line += ' ';
            }
            if (w == nw) break;
            line += V.zipf_word(r);
            if (w + 1 < nw) line += ' ';
        }
        line += '\n';
        uint64_t take = std::min<uint64_t>(line.size(), nbytes - at);
        std::memcpy(out + at, line.data(), (size_t)take);
        at += take;
    }
    return planted;
}

// HTTP-like token alphabet: methods, path segments, header names and values.
struct HttpTokens {
    std::vector<std::string> methods, segs, hnames, hvals;
    explicit HttpTokens(uint64_t seed) {
        Rng r(seed);
        for (int i = 0; i < 8; ++i) {
            std::string m = rand_lower(r, 3, 7);
            for (auto& c : m) c = (char)(c - 'a' + 'A');
            methods.push_back(m);
        }
        for (int i = 0; i < 300; ++i) segs.push_back(rand_alnum(r, 2, 10));
        for (int i = 0; i < 40; ++i) {
            std::string h;
            int parts = (int)uni(r, 1, 3);
            for (int p = 0; p < parts; ++p) {
                std::string w = rand_lower(r, 2, 8);
                w[0] = (char)(w[0] - 'a' + 'A');
                if (p) h += '-';
                h += w;
            }
            hnames.push_back(h);
        }
        static const char VA[] = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ0123456789/.=;, -_";
        for (int i = 0; i < 200; ++i) {
            int L = (int)uni(r, 2, 24);
            std::string v(L, 'a');
            for (auto& c : v) c = VA[uni(r, 0, sizeof(VA) - 2)];
            hvals.push_back(v);
        }
    }
    std::string request_line(Rng& r) const {
        std::string s = methods[uni(r, 0, methods.size() - 1)];
        s += ' ';
        int depth = (int)uni(r, 1, 5);
        for (int d = 0; d < depth; ++d) { s += '/'; s += segs[uni(r, 0, segs.size() - 1)]; }
        s += " HTTP/1.1\r\n";
        return s;
    }
    std::string header(Rng& r) const {
        return hnames[uni(r, 0, hnames.size() - 1)] + ": " + hvals[uni(r, 0, hvals.size() - 1)] + "\r\n";
    }
    // an HTTP-like fragment of at least L bytes
    std::string fragment(Rng& r, size_t L) const {
        std::string s;
        int kind = (int)uni(r, 0, 2);
        if (kind == 0) s = request_line(r);
        else if (kind == 1) s = header(r);
        else { int d = (int)uni(r, 1, 4); for (int k = 0; k < d; ++k) { s += '/'; s += segs[uni(r, 0, segs.size() - 1)]; } }
        while (s.size() < L) s += (uni(r, 0, 1) ? header(r) : request_line(r));
        return s;
    }
};

static void fill_http(const HttpTokens& T, Rng& r, uint8_t* out, uint64_t n) {
    std::string s = T.request_line(r);
    while (s.size() < n) {
        if (uni(r, 0, 5) == 0) s += "\r\n";
        s += T.header(r);
    }
    std::memcpy(out, s.data(), (size_t)n);
}

static void fill_random(Rng& r, uint8_t* out, uint64_t n) {
    uint64_t k = 0;
    for (; k + 8 <= n; k += 8) { uint64_t v = r(); std::memcpy(out + k, &v, 8); }
    if (k < n) { uint64_t v = r(); std::memcpy(out + k, &v, (size_t)(n - k)); }
}

}  // namespace

extern "C" {

// Fill out[0..nbytes) with syslog lines (see gen_syslog); vocabulary from
// vocab_seed, lines from text_seed.  Returns the number of planted patterns.
uint64_t synth_syslog(uint64_t vocab_seed, uint64_t text_seed, uint8_t* out, uint64_t nbytes, double plant_rate,
                      const uint8_t* pat, const uint64_t* poff, uint32_t npat) {
    Vocab V(vocab_seed);
    return gen_syslog(V, text_seed, out, nbytes, plant_rate, PatternView{pat, poff, npat});
}

// Syslog files: file f occupies out[seg[f]..seg[f+1]) and is generated from
// seed (base_seed + f) with its own fresh lines.  Threads only split the work;
// the bytes do not depend on the thread count.
uint64_t synth_syslog_files(uint64_t vocab_seed, uint64_t base_seed, uint8_t* out, const uint64_t* seg, uint32_t nseg,
                            double plant_rate, const uint8_t* pat, const uint64_t* poff, uint32_t npat,
                            uint32_t nthreads) {
    Vocab V(vocab_seed);
    PatternView P{pat, poff, npat};
    if (nthreads < 1) nthreads = 1;
    std::vector<uint64_t> planted(nthreads, 0);
    std::vector<std::thread> th;
    for (uint32_t t = 0; t < nthreads; ++t)
        th.emplace_back([&, t] {
            for (uint32_t f = t; f < nseg; f += nthreads)
                planted[t] += gen_syslog(V, base_seed + f, out + seg[f], seg[f + 1] - seg[f], plant_rate, P);
        });
    for (auto& x : th) x.join();
    uint64_t s = 0;
    for (auto v : planted) s += v;
    return s;
}

// Syslog-style pattern set: n patterns with lengths U[minlen, maxlen];
// prefix_frac of them are prefixes (length U[minlen, len-1]) of other
// patterns with len > minlen; the rest are vocabulary phrases (consecutive
// Zipf words joined by a space, cut to length) with probability vocab_frac,
// else uniform printable bytes 0x20..0x7E.  Returns 0, or -1 on bad args.
// *out_bytes / *out_offs are malloc'd (free with synth_free).
int synth_patterns_syslog(uint64_t vocab_seed, uint64_t seed, uint32_t n, uint32_t minlen, uint32_t maxlen,
                          double prefix_frac, double vocab_frac, uint8_t** out_bytes, uint64_t** out_offs) {
    if (minlen < 1 || maxlen < minlen) return -1;
    Vocab V(vocab_seed);
    Rng r(seed);
    uint32_t nprefix = (uint32_t)std::floor(prefix_frac * n + 0.5);
    if (nprefix > n) nprefix = n;
    uint32_t nbase = n - nprefix;
    std::vector<std::string> pats;
    pats.reserve(n);
    for (uint32_t i = 0; i < nbase; ++i) {
        size_t L = (size_t)uni(r, minlen, maxlen);
        std::string s;
        if (unif01(r) < vocab_frac) {
            while (s.size() < L) { if (!s.empty()) s += ' '; s += V.zipf_word(r); }
            s.resize(L);
        } else {
            s.resize(L);
            for (auto& c : s) c = (char)uni(r, 0x20, 0x7E);
        }
        pats.push_back(s);
    }
    std::vector<uint32_t> longer;
    for (uint32_t i = 0; i < nbase; ++i) if (pats[i].size() > minlen) longer.push_back(i);
    for (uint32_t i = 0; i < nprefix; ++i) {
        if (longer.empty()) { pats.push_back(pats.empty() ? std::string(minlen, 'a') : pats[uni(r, 0, pats.size() - 1)]); continue; }
        const std::string& b = pats[longer[uni(r, 0, longer.size() - 1)]];
        size_t L = (size_t)uni(r, minlen, b.size() - 1);
        pats.push_back(b.substr(0, L));
    }
    // shuffle so that prefixes are not all at the end of the id space
    for (size_t i = pats.size(); i > 1; --i) std::swap(pats[i - 1], pats[uni(r, 0, i - 1)]);
    size_t tot = 0;
    for (auto& p : pats) tot += p.size();
    *out_bytes = (uint8_t*)std::malloc(tot ? tot : 1);
    *out_offs = (uint64_t*)std::malloc(sizeof(uint64_t) * (pats.size() + 1));
    if (!*out_bytes || !*out_offs) return -2;
    size_t at = 0;
    (*out_offs)[0] = 0;
    for (size_t i = 0; i < pats.size(); ++i) {
        std::memcpy(*out_bytes + at, pats[i].data(), pats[i].size());
        at += pats[i].size();
        (*out_offs)[i + 1] = at;
    }
    return 0;
}

// DPI signatures: n with lengths U[minlen, maxlen]; http_frac of them are
// HTTP-like token fragments cut to length, the rest have every byte printable
// (0x20..0x7E) or uniform 0..255 with probability 1/2 each.
int synth_signatures_dpi(uint64_t tok_seed, uint64_t seed, uint32_t n, uint32_t minlen, uint32_t maxlen,
                         double http_frac, uint8_t** out_bytes, uint64_t** out_offs) {
    if (minlen < 1 || maxlen < minlen) return -1;
    HttpTokens T(tok_seed);
    Rng r(seed);
    std::vector<std::string> pats;
    pats.reserve(n);
    for (uint32_t i = 0; i < n; ++i) {
        size_t L = (size_t)uni(r, minlen, maxlen);
        std::string s;
        if (unif01(r) < http_frac) {
            s = T.fragment(r, L);
            s.resize(L);
        } else {
            s.resize(L);
            for (auto& c : s) c = (char)(uni(r, 0, 1) ? uni(r, 0x20, 0x7E) : uni(r, 0, 255));
        }
        pats.push_back(s);
    }
    size_t tot = 0;
    for (auto& p : pats) tot += p.size();
    *out_bytes = (uint8_t*)std::malloc(tot ? tot : 1);
    *out_offs = (uint64_t*)std::malloc(sizeof(uint64_t) * (pats.size() + 1));
    if (!*out_bytes || !*out_offs) return -2;
    size_t at = 0;
    (*out_offs)[0] = 0;
    for (size_t i = 0; i < pats.size(); ++i) {
        std::memcpy(*out_bytes + at, pats[i].data(), pats[i].size());
        at += pats[i].size();
        (*out_offs)[i + 1] = at;
    }
    return 0;
}

// Packet sizes drawn uniformly from {64, 576, 1500} until nbytes is reached;
// the last packet is cut so the total is exactly nbytes.  Writes the segment
// offsets (count+1 entries) when seg != NULL and cap > count; returns count.
uint64_t synth_packet_sizes(uint64_t seed, uint64_t nbytes, uint64_t* seg, uint64_t cap) {
    static const uint64_t S[3] = {64, 576, 1500};
    Rng r(seed);
    uint64_t at = 0, k = 0;
    if (seg && cap > 0) seg[0] = 0;
    while (at < nbytes) {
        uint64_t s = std::min<uint64_t>(S[uni(r, 0, 2)], nbytes - at);
        at += s;
        ++k;
        if (seg && k < cap) seg[k] = at;
    }
    return k;
}

// Packet payloads: packet p (bytes out[seg[p]..seg[p+1])) is drawn from its
// block's generator (blocks of 4096 packets, seed base_seed + block): with
// probability http_frac HTTP-like text, else uniform bytes; with probability
// plant_rate one pattern that fits is copied in at a random position.
uint64_t synth_packets_fill(uint64_t tok_seed, uint64_t base_seed, uint8_t* out, const uint64_t* seg, uint64_t nseg,
                            double http_frac, double plant_rate, const uint8_t* pat, const uint64_t* poff,
                            uint32_t npat, uint32_t nthreads) {
    HttpTokens T(tok_seed);
    const uint64_t B = 4096;
    uint64_t nblocks = (nseg + B - 1) / B;
    if (nthreads < 1) nthreads = 1;
    std::vector<uint64_t> planted(nthreads, 0);
    std::vector<std::thread> th;
    for (uint32_t t = 0; t < nthreads; ++t)
        th.emplace_back([&, t] {
            for (uint64_t b = t; b < nblocks; b += nthreads) {
                Rng r(base_seed + b);
                for (uint64_t p = b * B; p < std::min(nseg, (b + 1) * B); ++p) {
                    uint8_t* dst = out + seg[p];
                    uint64_t n = seg[p + 1] - seg[p];
                    if (unif01(r) < http_frac) fill_http(T, r, dst, n); else fill_random(r, dst, n);
                    if (npat && unif01(r) < plant_rate) {
                        for (int tries = 0; tries < 8; ++tries) {
                            uint32_t j = (uint32_t)uni(r, 0, npat - 1);
                            uint64_t L = poff[j + 1] - poff[j];
                            if (L > n) continue;
                            uint64_t at = uni(r, 0, n - L);
                            std::memcpy(dst + at, pat + poff[j], (size_t)L);
                            ++planted[t];
                            break;
                        }
                    }
                }
            }
        });
    for (auto& x : th) x.join();
    uint64_t s = 0;
    for (auto v : planted) s += v;
    return s;
}

// n log-normal sizes with the given median and sigma, clipped to [lo, hi].
void synth_lognormal_sizes(uint64_t seed, uint64_t n, double median, double sigma, uint64_t lo, uint64_t hi,
                           uint64_t* out) {
    Rng r(seed);
    std::normal_distribution<double> N(0.0, 1.0);
    double mu = std::log(median);
    for (uint64_t i = 0; i < n; ++i) {
        double v = std::exp(mu + sigma * N(r));
        uint64_t s = (uint64_t)std::llround(v);
        if (s < lo) s = lo;
        if (s > hi) s = hi;
        out[i] = s;
    }
}

// Uniform random bytes (fixtures for edge-case tests).
void synth_random_bytes(uint64_t seed, uint8_t* out, uint64_t n) {
    Rng r(seed);
    fill_random(r, out, n);
}

void synth_free(void* p) { std::free(p); }

}  // extern "C"
