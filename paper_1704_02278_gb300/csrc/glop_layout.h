// glop_layout.h -- the compiled automaton as the scan kernels read it.
//
// Shared by the host compiler (compile.cpp) and the kernels (scan.cu).
//
// The automaton is the failureless trie of Sec. 5: the goto graph of the
// Aho-Corasick machine (Sec. 4) with no failure transitions.  A walk that
// starts at text offset i follows goto transitions until one is missing; every
// terminal state it passes marks a pattern occurrence starting at i.
//
// State numbering.  States [0, n_dense) are "dense": the initial state (0)
// and every state with two or more children, in breadth-first order.  Each
// has a row of n_classes int32 entries, one per alphabet class.  States
// [n_dense, n_states) lie on unary chains (one child or none); the states of
// one chain are numbered consecutively from the chain's first state, and the
// chain is matched by comparing text bytes with the chain's bytes instead of
// one table lookup per byte.  A chain ends at a leaf or exits into a dense
// state.
//
// Row entry / chain exit / gram-table value encoding: target state id in bits
// 0..30, bit 31 set when the target is terminal (some pattern ends there);
// 0 means "no transition" (no edge enters the initial state).
#pragma once
#include <stdint.h>

#define GLOP_TERM 0x80000000u
#define GLOP_STATE_MASK 0x7FFFFFFFu

// per chain state: remaining chain bytes after this state, the exit into a
// dense state, and the deepest terminal state of the chain up to this state
struct GlopChain {
    uint32_t off;   // index into chain_bytes of the byte that follows this state
    uint32_t rem;   // remaining bytes: chain bytes after this state, plus 1 if the chain exits
    uint32_t exit;  // dense state entered after the last chain byte (| GLOP_TERM), 0 = leaf-ended chain
    uint32_t term;  // deepest terminal state among the chain's states up to this one, 0 = none
};

// slot of the gram table: the state reached from the initial state by the
// first gram_len bytes of some pattern
struct GlopGramSlot {
    uint32_t key_lo, key_hi;  // the gram_len bytes, little-endian, zero padded
    uint32_t val;             // state | GLOP_TERM, 0 = empty slot
    uint32_t pad;
};

// Offsets (bytes) of the arrays inside one device allocation, and sizes.
struct GlopDevAutomaton {
    uint32_t n_states, n_dense, n_classes;
    uint32_t n_patterns, min_len, max_len;
    uint32_t gram_len;     // 0: no start filter (some pattern shorter than 4 bytes)
    uint32_t bm_log2;      // start-filter bitmap has 1 << bm_log2 bits
    uint32_t ht_log2;      // gram table has 1 << ht_log2 slots
    uint32_t hot_lo;       // first dense state worth staging on chip (depth >= gram_len)
    const uint8_t *cls;            // [256] byte -> class
    const int32_t *rows;           // [n_dense * n_classes]
    const GlopChain *chain;        // [n_states - n_dense]
    const uint8_t *chain_bytes;
    const uint32_t *cum_off;       // [n_states + 1] output list of each state
    const uint32_t *cum_ids;       // pattern ids, ascending within a list
    const uint32_t *bitmap;        // [(1 << bm_log2) / 32]
    const GlopGramSlot *grams;     // [1 << ht_log2]
};
