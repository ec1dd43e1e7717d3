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

// Per chain state (32 bytes, one sector).  A chain is cut into pieces of at
// most 16 states; the record of a state holds, inline, every byte still to be
// compared in its piece (the bytes leading to the later states of the piece,
// then the byte of the exit), so one load resolves a chain step.
struct GlopChain {
    uint32_t inl[4];    // bytes to compare after this state, little-endian, zero padded
    uint32_t exit;      // state entered after the piece (| GLOP_TERM): next piece or a dense state; 0 = none
    uint32_t term;      // deepest terminal state of the chain from its first state up to this one, 0 = none
    uint16_t termmask;  // bit k: the state k places after this one in the piece is terminal (bit 0: this state)
    uint8_t rem;        // bytes to compare: states after this one in the piece, plus 1 if there is an exit
    uint8_t nst;        // states after this one in the piece
    uint32_t pad;
};
static_assert(sizeof(GlopChain) == 32, "a chain record is one 32-byte sector");

// slot of the gram table: the state reached from the initial state by the
// first gram_len bytes of some pattern
struct GlopGramSlot {
    uint32_t key_lo, key_hi;  // the gram_len bytes, little-endian, zero padded
    uint32_t val;             // state | GLOP_TERM, 0 = empty slot
    uint32_t pad;
};
static_assert(sizeof(GlopGramSlot) == 16, "a gram slot is one 16-byte load");

// Offsets (bytes) of the arrays inside one device allocation, and sizes.
struct GlopDevAutomaton {
    uint32_t n_states, n_dense, n_classes;
    uint32_t n_patterns, min_len, max_len;
    uint32_t gram_len;     // 0: no start filter (some pattern shorter than 4 bytes)
    uint32_t bm_log2;      // start-filter bitmap has 1 << bm_log2 bits
    uint32_t ht_log2;      // gram table has 1 << ht_log2 slots
    uint32_t hot_lo;       // first dense state worth staging on chip (depth >= gram_len)
    const uint8_t *cls;            // [256] byte -> class
    const void *rows;              // [n_dense * n_classes], see row16
    const GlopChain *chain;        // [n_states - n_dense]
    uint32_t row16;                // 1: rows are uint16 (state | 0x8000 when terminal), else int32
    const uint32_t *cum_off;       // [n_states + 1] output list of each state
    const uint32_t *outl;          // [2 * n_states] the same lists as (start, count) pairs, one 8-byte load each
    const uint32_t *cum_ids;       // pattern ids, ascending within a list
    uint32_t n_cum_ids;            // entries of cum_ids
    const uint32_t *bitmap;        // [(1 << bm_log2) / 32]; a gram's word and bit as glop_hash.h places them
    const GlopGramSlot *grams;     // [1 << ht_log2]
};
