// compile.h -- host-side automaton compiler (no CUDA dependency).
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "glop_layout.h"

namespace glop {

// The compiled automaton in host memory, laid out exactly as the device copy
// (see glop_layout.h for the meaning of every array).
struct HostAutomaton {
    uint32_t n_patterns = 0, min_len = 0, max_len = 0;
    uint32_t n_states = 0, n_dense = 0, n_classes = 0;
    uint32_t gram_len = 0, bm_log2 = 0, ht_log2 = 0, hot_lo = 0, n_grams = 0;
    std::vector<uint8_t> cls;             // 256
    std::vector<int32_t> rows;            // n_dense * n_classes
    std::vector<GlopChain> chain;         // n_states - n_dense
    std::vector<uint32_t> cum_off;        // n_states + 1
    std::vector<uint32_t> cum_ids;
    std::vector<uint32_t> bitmap;         // (1 << bm_log2) / 32 words
    std::vector<GlopGramSlot> grams;      // 1 << ht_log2 slots
    std::vector<uint32_t> depth;          // per state
};

// Status codes use the values of glop_status.
// prefix_len 0 = exact patterns; K > 0 cuts every pattern to K bytes.
// gram_len / bm_log2: start-filter gram length and bitmap size; 0 = automatic.
int compile_host(const uint8_t *bytes, const uint64_t *offs, uint32_t n, uint32_t prefix_len, HostAutomaton *out,
                 std::string *err, uint32_t gram_len = 0, uint32_t bm_log2 = 0);

}  // namespace glop
