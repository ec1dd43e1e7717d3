// scan.h -- launchers of the scan kernels (internal to libglop.so).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "glop_layout.h"

namespace glop {

// workspace header flags (uint32 at offset 0 of the workspace)
enum : uint32_t { WS_TIMEOUT = 1u, WS_OVERFLOW = 2u, WS_EINVAL = 4u };

// Geometry of one scan tile: 256 threads x 16 start offsets.
constexpr uint32_t kGroupThreads = 256;
constexpr uint32_t kOffsetsPerThread = 16;
constexpr uint32_t kTile = kGroupThreads * kOffsetsPerThread;  // 4096 bytes
constexpr uint32_t kHeaderBytes = 256;

struct ScanLaunch {
    const GlopDevAutomaton *A;  // descriptor with device pointers (host copy)
    const uint8_t *text;
    uint64_t len;
    const uint64_t *seg;  // device segment offsets, nullptr for one buffer
    uint32_t n_seg;
    void *out;
    uint64_t capacity;
    uint64_t *d_count;
    void *ws;
    uint64_t ws_bytes;
    cudaStream_t stream;
    uint32_t smem_budget;  // 0 = library default
};

uint64_t workspace_bytes(uint64_t len, bool batch);
// returns a glop_status value
int launch_scan(const ScanLaunch &L);

}  // namespace glop
