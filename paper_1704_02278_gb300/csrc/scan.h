// scan.h -- launcher of the scan kernel (internal to libglop.so).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "glop_layout.h"

namespace glop {

// workspace header flags (uint32 at offset 0 of the workspace)
// header word 11/12 hold the site and value of the first broken internal check
enum : uint32_t { WS_TIMEOUT = 1u, WS_OVERFLOW = 2u, WS_EINVAL = 4u, WS_INTERNAL = 8u };

// Geometry: a consumer warp scans 1 KiB sub-tiles (32 lanes x 32 start
// offsets); 31 consumer warps share 31 KiB chunks brought in by one producer.
constexpr uint32_t kSubTile = 1024;
constexpr uint32_t kConsumers = 31;
constexpr uint32_t kChunk = kSubTile * kConsumers;
constexpr uint32_t kHeaderBytes = 256;
constexpr uint32_t kMaxGrid = 1024;
constexpr uint32_t kMaxBatchGroups = 8;  // automata in one batch launch

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
    uint32_t ksub = 1;     // sub-tiles each consumer warp takes from a staged chunk: 1 (31 KiB chunks) or 2 (62 KiB)
    uint32_t *ksub_used = nullptr;  // if set: receives the ksub the launch used (2 falls back to 1 when it does not fit)
    // Several automata in one batch launch: n_groups > 0 groups of segments, group g starting at byte
    // group_start[g] (a multiple of kSubTile; group_start[n_groups] = len) and scanned with group_A[g]
    // (host arrays).  A then points at group_A[0]; every group must share its start-filter kind and row
    // width (the kernel variant).
    uint32_t n_groups = 0;
    const GlopDevAutomaton *group_A = nullptr;
    const uint64_t *group_start = nullptr;
    unsigned long long *hist = nullptr;  // count-only mode: per-pattern counts (n_patterns); d_count = their sum
    // Pieces of a longer buffer (single buffer only): match starts in [0, own_len) (0 = len; bytes up to
    // len are look-ahead for walks), reported offsets + base_off, the first match written at output index
    // *d_obase (null: 0), and *d_next_base = that index + this piece's match count (null: not written).
    uint64_t own_len = 0;
    uint32_t base_off = 0;
    const unsigned long long *d_obase = nullptr;
    unsigned long long *d_next_base = nullptr;
};

// Workspace: header, one descriptor per sub-tile, block sums, (batch) the
// first segment of every sub-tile, then scratch records of walked offsets
// with a match -- room for one record per 8 text bytes.  A sub-tile whose
// records do not fit is walked a second time instead; results stay exact.
uint64_t workspace_bytes(uint64_t len, bool batch);
// Count-only mode: the header, then one uint32 hit counter per automaton state.
uint64_t count_workspace_bytes(uint32_t n_states);
// returns a glop_status value
int launch_scan(const ScanLaunch &L);
// The scratch array of glop_scan_noalloc on the current device (its workspace), or nullptr.
void *noalloc_scratch_of_current_device();
// Queue a one-thread kernel writing the scan's count and status (as glop_scan_words) to h_words_dev, a
// device-side address of pinned host memory.  Returns a glop_status value.
int launch_words(const void *d_workspace, unsigned long long *h_words_dev, cudaStream_t stream);

}  // namespace glop
