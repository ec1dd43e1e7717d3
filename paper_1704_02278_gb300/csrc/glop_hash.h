// glop_hash.h -- the start-filter hash, identical on host (compiler) and device.
//
// The start filter looks at the first gram_len (4..8) bytes at a text offset.
// Every pattern is at least gram_len bytes long, so an offset can only start a
// match if those bytes equal the first gram_len bytes of some pattern.  The
// bytes are read as two little-endian words w0 (bytes 0..3) and w1 (bytes
// 4..7, masked to gram_len - 4 bytes) and mixed multiplicatively.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define GLOP_HD __host__ __device__ __forceinline__
#else
#define GLOP_HD static inline
#endif

#define GLOP_HASH_M0 0x9E3779B1u
#define GLOP_HASH_M1 0x85EBCA77u
#define GLOP_HASH_M2 0x2C1B3C6Du

// mask keeping the bytes of w1 that belong to a gram of gram_len bytes
GLOP_HD uint32_t glop_w1_mask(uint32_t gram_len) {
    return gram_len >= 8 ? 0xFFFFFFFFu : ((1u << (8u * (gram_len - 4u))) - 1u);
}

GLOP_HD uint32_t glop_gram_hash(uint32_t w0, uint32_t w1_masked) {
    return (w0 * GLOP_HASH_M0) ^ (w1_masked * GLOP_HASH_M1);
}

// Position of a gram in the start-filter bitmap (1 << bm_log2 bits in 32-bit
// words), the bit stored reversed (bit b of the gram is bit 31 - b of its word,
// so a rotate left by b brings it to bit 31).  The word is the top bm_log2 - 5
// bits of glop_gram_hash.  The bit: for 4-byte grams, the low 5 bits of the high
// half of the 64-bit product w0 * M0 -- the device then needs one wide multiply,
// one shift for the word and none for the bit; for longer grams (two products),
// the next 5 bits of glop_gram_hash below the word's.
GLOP_HD uint32_t glop_bitmap_word(uint32_t h, uint32_t bm_log2) { return h >> (37u - bm_log2); }

GLOP_HD uint32_t glop_bitmap_bit(uint32_t h, uint32_t w0, uint32_t gram_len, uint32_t bm_log2) {
    return gram_len == 4 ? (uint32_t)(((uint64_t)w0 * GLOP_HASH_M0) >> 32) & 31u : (h >> (32u - bm_log2)) & 31u;
}

// first probe of the gram table (linear probing)
GLOP_HD uint32_t glop_table_slot(uint32_t h, uint32_t ht_log2) {
    return ((h ^ (h >> 15)) * GLOP_HASH_M2) >> (32u - ht_log2);
}
