/*
 * glop.h -- C ABI of the GB300 multi-pattern scan library (libglop.so).
 *
 * The library finds every occurrence of every pattern of a signature set in
 * a byte buffer: the result is the set of (offset, pattern_id) pairs with
 * pattern j equal to text[offset .. offset + |p_j|), sorted by offset then
 * pattern id.  It is the first searching stage of the paper's log-processing
 * library (Sec. 1, use case: rules in, logs in, the number of suspect
 * events and their locations out) done by a failureless trie walked from
 * every byte offset (Sec. 5), completed on the GPU so that results are exact.
 *
 * Conventions for every entry point:
 *  - Pointers named d_* are CUDA device pointers; all others are host
 *    pointers.  Sizes are in bytes unless stated.
 *  - The caller owns every buffer it passes (text, matches, count,
 *    workspace); the library never frees them.  The library owns the
 *    compiled automaton until glop_destroy().
 *  - stream is a cudaStream_t (cast to void*); 0 is the legacy default stream.
 *  - Argument errors are returned synchronously, before any work is queued.
 *    Conditions found by the GPU (match overflow, a bounded wait that ran
 *    out) are reported through *d_count and the workspace status word, read
 *    with glop_scan_status().
 *  - A handle is immutable after glop_compile() and may be scanned
 *    concurrently from several streams, each with its own workspace.
 *  - Every call on a machine without a usable CUDA device returns
 *    GLOP_ECUDA; there is no CPU fallback.
 */
#ifndef GLOP_H
#define GLOP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct glop_automaton *glop_handle; /* opaque */
typedef void *glop_stream_t;                /* a cudaStream_t */

typedef enum {
    GLOP_OK = 0,
    GLOP_EINVAL = 1,    /* bad argument (null pointer, zero-length pattern, size limits, ...) */
    GLOP_ENOMEM = 2,    /* host or device allocation failed, or workspace too small */
    GLOP_EOVERFLOW = 3, /* more matches than the capacity given; *d_count holds the true total */
    GLOP_ECUDA = 4,     /* a CUDA runtime call failed or no device is usable */
    GLOP_ETIMEOUT = 5,  /* a bounded wait inside a kernel ran out; results are incomplete */
    GLOP_EBUSY = 6,     /* resource in use */
    GLOP_EINTERNAL = 7  /* an internal consistency check failed */
} glop_status;

/* One match of glop_scan(): pattern pattern_id occurs at text[offset ...]. */
typedef struct {
    uint32_t offset;
    uint32_t pattern_id;
} glop_match;

/* One match of glop_scan_batch(): offset is relative to the segment start. */
typedef struct {
    uint32_t segment;
    uint32_t offset;
    uint32_t pattern_id;
} glop_batch_match;

/* Compile options; a NULL pointer means all zero. */
typedef struct {
    /* 0: exact full-pattern matching.  K > 0: every pattern is cut to its
     * first min(|p|, K) bytes before compiling -- the prefix (partial)
     * matching of Sec. 1 and Sec. 5, whose paper setting is K = 8. */
    uint32_t prefix_len;
    /* Shared memory per thread block for transition rows staged on chip;
     * 0 lets the library choose. */
    uint32_t smem_budget_bytes;
    uint32_t flags; /* reserved, must be 0 */
    /* Start filter: bytes hashed at every offset (4..8, at most the shortest
     * pattern; 0 = the library's choice, min(shortest pattern, 8)). */
    uint32_t gram_len;
    /* Start filter bitmap of 2^filter_bits_log2 bits (13..19; 0 = the
     * library's choice from the number of distinct grams). */
    uint32_t filter_bits_log2;
    /* Text staged per bulk copy: every consumer warp of a thread block takes
     * chunk_subtiles consecutive 1 KiB sub-tiles (32 start offsets per lane)
     * of each staged chunk.  0 or 1: 31 KiB chunks; 2: 62 KiB chunks (in two
     * ring slots, when they fit in shared memory beside the tables; else 31
     * KiB).  Other values are taken as 1. */
    uint32_t chunk_subtiles;
} glop_compile_opts;

/* Facts about a compiled automaton (glop_info_get). */
typedef struct {
    uint32_t n_patterns;
    uint32_t min_pattern_len, max_pattern_len; /* after prefix cut */
    uint32_t n_states;        /* trie states including the initial state */
    uint32_t n_dense_states;  /* states with a full transition row (initial + branching) */
    uint32_t n_chain_states;  /* states on unary chains, matched by byte comparison */
    uint32_t n_classes;       /* alphabet classes of the transition rows */
    uint32_t gram_len;        /* bytes hashed by the start filter; 0 = no filter */
    uint32_t n_grams;         /* distinct gram_len-byte pattern prefixes */
    uint32_t cum_ids;         /* pattern ids stored in per-state output lists */
    uint64_t device_bytes;    /* device memory held by the handle */
    double compile_ms;        /* host time of glop_compile */
} glop_info;

/*
 * glop_compile -- build the automaton of a pattern set (Sec. 4, first phase;
 * Sec. 5, failure transitions removed) and copy it to the current device.
 *
 * pattern_bytes   host, concatenated pattern bytes (any of the 256 values).
 * pattern_offsets host, n_patterns + 1 non-decreasing offsets into
 *                 pattern_bytes; pattern j is bytes [off[j], off[j+1]).
 *                 Its id is j.  Duplicates are allowed and all reported.
 * n_patterns      0 is valid (every scan then finds nothing); at most 2^31.
 * opts            may be NULL.
 * out             receives the handle; unchanged on error.
 *
 * Errors: GLOP_EINVAL for a zero-length pattern (after the prefix cut),
 * decreasing offsets, a null pointer, or tables beyond 2^31 states;
 * GLOP_ENOMEM; GLOP_ECUDA.  Synchronous: the handle is ready on return.
 */
glop_status glop_compile(const uint8_t *pattern_bytes, const uint64_t *pattern_offsets, uint32_t n_patterns,
                         const glop_compile_opts *opts, glop_handle *out);

/* glop_info_get -- fill *info for handle h.  GLOP_EINVAL on null arguments. */
glop_status glop_info_get(glop_handle h, glop_info *info);

/* Longest pattern after the prefix cut: the overlap a caller needs between
 * consecutive chunks of a stream (Sec. 4: at least the longest pattern - 1). */
uint32_t glop_max_pattern_len(glop_handle h);

/* glop_scan_workspace_size -- device workspace bytes glop_scan() needs for a
 * text of text_len bytes (a few bytes per 4 KiB tile). */
glop_status glop_scan_workspace_size(glop_handle h, uint64_t text_len, uint64_t *bytes);

/*
 * glop_scan -- every (offset, pattern_id) match in d_text[0, len), sorted by
 * (offset, pattern_id), written to d_matches[0, min(count, capacity)).
 *
 * This is the searching phase of Sec. 5: the failureless trie is walked from
 * every byte offset (one walk per offset, a missing transition ends it), and
 * every pattern that ends on the walk is reported at the walk's start -- the
 * count and locations of the suspect events of the use case in Sec. 1.  With
 * prefix_len = 0 the second stage of Sec. 2 and Sec. 5 (completing a prefix
 * hit into a full match) is done in the same walk, so results are exact.
 *
 * d_text       device, len bytes; any alignment (16-byte aligned is fastest).
 * len          at most 2^32 - 1 (offsets are 32-bit).  0 is valid.
 * d_matches    device, capacity entries (may be NULL when capacity is 0).
 * d_count      device, one uint64_t: receives the total number of matches,
 *              also when it exceeds capacity (then only the first capacity
 *              matches in sorted order are written).
 * d_workspace  device, at least glop_scan_workspace_size() bytes, 16-byte
 *              aligned.  Must not be used by another scan until this one
 *              has finished on the stream.
 *
 * Asynchronous on stream.  Returns GLOP_EINVAL / GLOP_ENOMEM (workspace too
 * small) / GLOP_ECUDA synchronously; GPU-side conditions via
 * glop_scan_status().
 */
glop_status glop_scan(glop_handle h, const uint8_t *d_text, uint64_t len, glop_match *d_matches, uint64_t capacity,
                      uint64_t *d_count, void *d_workspace, uint64_t workspace_bytes, glop_stream_t stream);

/* glop_batch_workspace_size -- device workspace bytes for glop_scan_batch()
 * over text_len bytes cut into n_segments segments. */
glop_status glop_batch_workspace_size(glop_handle h, uint64_t text_len, uint32_t n_segments, uint64_t *bytes);

/*
 * glop_scan_batch -- the definition of glop_scan applied to every segment of
 * one buffer (log files, packet payloads) -- the batches of logs that the
 * paper's library hands to the GPU (Sec. 6), each searched as in Sec. 5:
 * segment s is
 * d_text[d_seg_offsets[s], d_seg_offsets[s+1]); matches never cross a segment
 * end; offsets are relative to the segment start; output sorted by
 * (segment, offset, pattern_id).  One persistent launch covers all segments.
 *
 * d_seg_offsets device, n_segments + 1 non-decreasing values, the last at
 *               most text_len; each segment at most 2^32 - 1 bytes.  Checked
 *               on the GPU: malformed offsets make glop_scan_status() return
 *               GLOP_EINVAL and write *d_count = 0.
 * text_len      bytes of d_text covered by the segments.
 * Other arguments as for glop_scan().
 */
glop_status glop_scan_batch(glop_handle h, const uint8_t *d_text, uint64_t text_len, const uint64_t *d_seg_offsets,
                            uint32_t n_segments, glop_batch_match *d_matches, uint64_t capacity, uint64_t *d_count,
                            void *d_workspace, uint64_t workspace_bytes, glop_stream_t stream);

/*
 * glop_scan_batch_multi -- glop_scan_batch over segments that are scanned
 * with different automata, in one persistent launch: a batch of requests for
 * several resident pattern sets (the serving loop's continuous batching;
 * the paper's library hands batches of logs to the GPU, Sec. 6, each searched
 * as in Sec. 5 -- here with the rule set of its own request).
 *
 * handles       host, n_groups automata (1 .. GLOP_BATCH_MAX_GROUPS) of the
 *               current device, each with at least one pattern, all of one
 *               kernel kind (equal glop_batch_multi_kind values).
 * group_start   host, n_groups + 1 byte offsets: group g is the text
 *               [group_start[g], group_start[g + 1]), scanned with handles[g].
 *               group_start[0] = 0, group_start[n_groups] = text_len,
 *               non-decreasing, every group_start[g] a multiple of 1024 (the
 *               scan's sub-tile) and, on the device, equal to some
 *               d_seg_offsets value, so that no segment straddles two groups
 *               (else glop_scan_status returns GLOP_EINVAL and *d_count = 0).
 *               Bytes between segments are not possible (segments are
 *               contiguous): a caller that pads a group to 1024 bytes gives
 *               the padding a segment of its own and ignores its matches.
 * Other arguments, results, ordering (by segment, offset, pattern id; pattern
 * ids of the segment's own automaton) and errors as for glop_scan_batch; the
 * workspace size is glop_batch_workspace_size's.  Each thread block of the
 * launch serves one group and stages that group's tables once.
 */
#define GLOP_BATCH_MAX_GROUPS 8
glop_status glop_scan_batch_multi(const glop_handle *handles, uint32_t n_groups, const uint64_t *group_start,
                                  const uint8_t *d_text, uint64_t text_len, const uint64_t *d_seg_offsets,
                                  uint32_t n_segments, glop_batch_match *d_matches, uint64_t capacity,
                                  uint64_t *d_count, void *d_workspace, uint64_t workspace_bytes,
                                  glop_stream_t stream);
/* The kernel kind of an automaton (its start filter's gram class and row
 * width): handles can share one glop_scan_batch_multi launch when their kinds
 * are equal.  Host only. */
glop_status glop_batch_multi_kind(glop_handle h, uint32_t *kind);

/*
 * glop_scan_status -- wait for stream, then report the outcome of the last
 * scan that used d_workspace: GLOP_OK, GLOP_EOVERFLOW (more matches than
 * capacity), GLOP_ETIMEOUT (a bounded in-kernel wait ran out), GLOP_EINVAL
 * (malformed batch offsets), GLOP_EINTERNAL or GLOP_ECUDA.  If count is not
 * NULL it receives the total match count -- the number of suspect events of
 * Sec. 1; the status codes themselves have no counterpart in the paper.
 * When several conditions were raised, GLOP_ETIMEOUT is reported first: after
 * a wait ran out the rest of the scan may meet scratch data that was never
 * written, and the checks that catch it (GLOP_EINTERNAL) are its consequence.
 *
 * d_workspace NULL means the scratch array of glop_scan_noalloc on the
 * current device: the outcome of the last glop_scan_noalloc call there
 * (GLOP_OK before any such call).  GLOP_ECUDA when that array cannot be
 * reached.
 */
glop_status glop_scan_status(const void *d_workspace, glop_stream_t stream, uint64_t *count);

/*
 * glop_scan_words -- queue, on stream, the copy of a finished scan's match
 * count and status into pinned host memory, made by a one-thread kernel and
 * not by the copy engine (a small device-to-host memcpy waits behind any
 * large copy already in flight and holds up its stream).  d_workspace is the
 * workspace of a glop_scan or glop_scan_batch queued earlier on stream;
 * h_words (caller-owned, two uint64_t host words the device can address:
 * pinned by cudaMallocHost / cudaHostAlloc / cudaHostRegister; on systems
 * whose GPU reads host page tables, any host memory) receives [total match
 * count, glop_status of the scan as glop_scan_status maps it].  The values
 * are there once the stream has passed this point (an event or a
 * synchronize).  GLOP_EINVAL when a pointer is NULL or the driver reports
 * h_words as not addressable by the device.
 */
glop_status glop_scan_words(const void *d_workspace, uint64_t *h_words, glop_stream_t stream);

/*
 * glop_ingest_* -- a byte stream scanned chunk by chunk as it arrives (the
 * paper streams the next batch to the GPU while the current one is scanned,
 * Sec. 6), with the uploads, scans and copy-backs of consecutive chunks
 * overlapped.  Each scan covers the carried last longest-pattern - 1 bytes of
 * the previous buffer (kept on the device) plus the new chunk, and owns the
 * match starts before its last longest-pattern - 1 bytes (the final scan owns
 * all of them); in order, the results are exactly the matches of the whole
 * stream, with offsets relative to each result's base.
 *
 * glop_ingest_create: chunks of at most chunk_bytes; out_rows the initial
 * match rows per chunk (0: a quarter of the chunk; more matches are handled
 * by scanning the chunk again into a larger output); depth (1 ..
 * GLOP_INGEST_MAX_DEPTH) the number of chunks whose results are not handed
 * out yet.  Allocates depth + 1 slots (device buffers, pinned host rows,
 * CUDA streams) on the current device, which must stay current for every
 * call.  The handle h must outlive the object.
 * glop_ingest_feed: queues n bytes of h_chunk (host memory; pinned is
 * fastest; it must stay unchanged until the next feed or flush returns) and
 * sets *res to the owned matches of the chunk fed depth calls before (count
 * 0 while fewer were fed).  res->matches points into the object's pinned
 * memory and stays valid until the second feed after the one that returned
 * it.  Blocks until the previous chunk's scan has finished.
 * glop_ingest_flush: ends the stream; res[0 .. *n_res) receive the results
 * not handed out yet, in order (at most depth; max_res smaller returns
 * GLOP_EINVAL with *n_res set).  glop_ingest_reset then starts a new stream.
 * Errors from the scans (GLOP_ETIMEOUT, GLOP_EINTERNAL, GLOP_ECUDA) leave the
 * object unusable: destroy it.  Not thread-safe: one thread per object.
 */
#define GLOP_INGEST_MAX_DEPTH 8
typedef struct glop_ingest_s *glop_ingest; /* opaque */
typedef struct {
    uint64_t base;              /* stream offset that match offsets are relative to */
    const glop_match *matches;  /* count rows, sorted by (offset, pattern_id) */
    uint64_t count;
} glop_ingest_result;
glop_status glop_ingest_create(glop_handle h, uint64_t chunk_bytes, uint64_t out_rows, uint32_t depth,
                               glop_ingest *out);
glop_status glop_ingest_feed(glop_ingest s, const uint8_t *h_chunk, uint64_t n, glop_ingest_result *res);
glop_status glop_ingest_flush(glop_ingest s, glop_ingest_result *res, uint32_t max_res, uint32_t *n_res);
glop_status glop_ingest_reset(glop_ingest s);
glop_status glop_ingest_info(glop_ingest s, uint64_t *chunks, uint64_t *rescans);
glop_status glop_ingest_destroy(glop_ingest s);

/*
 * glop_scan_host -- glop_scan on HOST buffers, end to end: copies text to the
 * device, scans, copies the count and the matches back, and waits for
 * completion.  Device buffers come from d_staging (at least
 * glop_scan_host_staging_size() bytes, caller-owned, 256-byte aligned).
 * h_matches receives min(count, capacity) matches; *h_count the total.
 * Pinned host memory gives the fastest copies.  Returns GLOP_EOVERFLOW when
 * count > capacity (the first capacity matches are still delivered).
 */
glop_status glop_scan_host_staging_size(glop_handle h, uint64_t len, uint64_t capacity, uint64_t *bytes);
glop_status glop_scan_host(glop_handle h, const uint8_t *h_text, uint64_t len, glop_match *h_matches,
                           uint64_t capacity, uint64_t *h_count, void *d_staging, uint64_t staging_bytes,
                           glop_stream_t stream);

/*
 * glop_scan_host_plan -- the pieces glop_scan_host splits a len-byte text
 * into (the paper's overlap of the next batch's transfer with the current
 * scan, Sec. 6): piece k is bytes [bounds[k], bounds[k + 1]) for
 * k < *n_pieces, with bounds[0] = 0, bounds[*n_pieces] = len, strictly
 * increasing, inner bounds multiples of 4096.  Texts under 16 MiB go in one
 * piece; longer ones in at most 9: a short first piece, then equal full
 * pieces (8 at most, and at most one per 8 MiB of text).
 * (glop_scan_host scans an automaton without patterns in one piece whatever
 * the length.)  Each piece's scan also reads the next longest-pattern - 1
 * bytes; its upload is issued with them.  Host only, no device work.
 * bounds (caller-owned, may be NULL to query *n_pieces alone) must hold
 * *n_pieces + 1 entries: max_bounds smaller returns GLOP_EINVAL with
 * *n_pieces set.
 */
glop_status glop_scan_host_plan(uint64_t len, uint64_t *bounds, uint32_t max_bounds, uint32_t *n_pieces);

/*
 * glop_tune -- pick compile options for a pattern set by timing scans of a
 * sample on the current device: the start filter's gram length and bitmap
 * size, the shared-memory budget of on-chip transition rows and the text
 * staged per bulk copy (31 or 62 KiB chunks; a 62 KiB candidate that does not
 * fit in shared memory is not timed).  Every
 * candidate is compiled, warmed up and timed over `repeats` scans of the
 * sample (d_sample, sample_len; a batch when d_seg_offsets is not NULL) with
 * CUDA events on stream.  points[0 .. *n_points) receive every candidate and
 * its Gbit/s (at most max_points are stored); *best the fastest options.
 * Allocates its own scratch; synchronous.  Errors as for glop_compile and
 * glop_scan.
 */
typedef struct {
    glop_compile_opts opts;
    double gbps;
} glop_tune_point;
glop_status glop_tune(const uint8_t *pattern_bytes, const uint64_t *pattern_offsets, uint32_t n_patterns,
                      uint32_t prefix_len, const uint8_t *d_sample, uint64_t sample_len,
                      const uint64_t *d_seg_offsets, uint32_t n_segments, uint32_t repeats, glop_tune_point *points,
                      uint32_t max_points, uint32_t *n_points, glop_compile_opts *best, glop_stream_t stream);

/*
 * Plans: a whole scan (glop_scan, or glop_scan_batch when d_seg_offsets is
 * not NULL) captured once into a CUDA graph for fixed buffers, then replayed
 * with a single graph launch -- the batched form of the paper's streamed
 * kernels (Sec. 6: the CPU streams the next batch while a kernel runs).
 *
 * glop_plan_create captures the scan's work on stream (nothing runs) and
 * instantiates the graph; every argument is as for glop_scan /
 * glop_scan_batch and must stay valid for the plan's lifetime.  Errors as
 * for those calls; GLOP_ECUDA if capture or instantiation fails.
 * glop_plan_launch queues one replay on stream (any stream of the device).
 * glop_plan_destroy frees the graph (NULL accepted); no replay may be in
 * flight.
 */
typedef struct glop_plan_s *glop_plan;
glop_status glop_plan_create(glop_handle h, const uint8_t *d_text, uint64_t text_len, const uint64_t *d_seg_offsets,
                             uint32_t n_segments, void *d_matches, uint64_t capacity, uint64_t *d_count,
                             void *d_workspace, uint64_t workspace_bytes, glop_stream_t stream, glop_plan *out);
glop_status glop_plan_launch(glop_plan plan, glop_stream_t stream);
glop_status glop_plan_destroy(glop_plan plan);

/*
 * glop_scan_noalloc -- glop_scan for callers that cannot allocate device
 * memory at scan time (their device memory belongs to another allocator, or
 * their loop must not pay for an allocation's implicit synchronisation).  The
 * paper has no counterpart for this entry point.
 *
 * Arguments and results are those of glop_scan, without the workspace: the
 * scratch memory is a 25 MiB device array in the library.  len must be at
 * most 16 MiB (16777216); longer texts return GLOP_EINVAL before anything is
 * queued.  The call allocates nothing.  Conditions found on the GPU (a
 * bounded wait that ran out, an internal check) are read with
 * glop_scan_status(NULL, stream, &count), which reports the last
 * glop_scan_noalloc call on the current device; an overflow also shows as
 * *d_count > capacity.
 *
 * The first call on a device (and the first after a cudaDeviceReset) loads
 * the library's device module there, which reserves the 25 MiB, and looks up
 * the array's device address with that device current: make that first call
 * at start-up, before another allocator takes the device's memory and before
 * any stream capture.  The array stays reserved on that device until the
 * process exits.  Every call uses the same array and leaves its contents
 * behind: two calls whose work overlaps on the GPU (different streams, or
 * different host threads) race on it and give wrong results.  Serialise
 * them, e.g. on one stream.  Per-call state in the array is reset by the
 * call itself.
 */
glop_status glop_scan_noalloc(glop_handle h, const uint8_t *d_text, uint64_t len, glop_match *d_matches,
                              uint64_t capacity, uint64_t *d_count, glop_stream_t stream);

/*
 * Count-only alert mode: how often each pattern occurs in a buffer, without
 * the list of locations -- the paper's use case reports the number of
 * suspect events as well as where they are (Sec. 1); this is the first half
 * alone, and it writes no match list at all.
 *
 * glop_count_workspace_size: device workspace bytes glop_scan_count needs on
 * this handle (a header plus one counter per automaton state; text_len does
 * not change it).
 *
 * glop_scan_count: d_hist[j] = the number of offsets i with
 * d_text[i, i + |p_j|) = p_j (n_patterns uint64, device, 8-byte aligned,
 * overwritten), *d_total = their sum (device uint64) -- the same counts a
 * glop_scan of d_text would report.  d_workspace is 256-byte aligned and
 * caller-owned; len at most 2^32 - 1.  Queued on stream; errors as for
 * glop_scan (GLOP_EINVAL for a NULL or misaligned pointer or a handle of
 * another device, GLOP_ENOMEM for a small workspace, GLOP_ECUDA); device
 * conditions (a timeout) through glop_scan_status on d_workspace.
 */
glop_status glop_count_workspace_size(glop_handle h, uint64_t text_len, uint64_t *bytes);
glop_status glop_scan_count(glop_handle h, const uint8_t *d_text, uint64_t len, uint64_t *d_hist, uint64_t *d_total,
                            void *d_workspace, uint64_t workspace_bytes, glop_stream_t stream);

/*
 * glop_batch_split -- a batch scan's matches as (offset, pattern_id) pairs
 * plus the run of each segment.  The paper has no counterpart: it serves a
 * server that batches one request per segment and returns each request its
 * own matches (8 bytes a match over the host link instead of 12).
 *
 * d_matches: the glop_scan_batch output (capacity entries, sorted by
 * segment); d_count: its device match count (only min(*d_count, capacity)
 * entries are read).  Writes d_pairs[i] = (offset, pattern_id) of match i
 * (capacity entries of room) and d_seg_first[s] = the index of the first
 * match of segment s, for s = 0 .. n_segments (d_seg_first[n_segments] =
 * the number of matches read), so segment s owns pairs
 * [d_seg_first[s], d_seg_first[s + 1]).  All pointers are device pointers
 * owned by the caller; d_pairs must not overlap d_matches.  Queued on stream
 * after the scan; GLOP_EINVAL for a NULL pointer or n_segments = UINT32_MAX.
 */
glop_status glop_batch_split(const glop_batch_match *d_matches, const uint64_t *d_count, uint64_t capacity,
                             uint32_t n_segments, glop_match *d_pairs, uint64_t *d_seg_first, glop_stream_t stream);

/* glop_destroy -- free the device memory of the automaton that
 * glop_compile built (the goto graph of Sec. 4 without failure transitions,
 * Sec. 5).  No scan using h may still be in flight.  NULL is accepted. */
glop_status glop_destroy(glop_handle h);

/*
 * glop_server_* -- a scan server's serving loop in native code: several
 * compiled pattern sets stay resident, requests (a host payload and the set to
 * scan it with) are admitted into a device-memory budget and batched while
 * earlier batches are still on the GPU -- the paper's use case (Sec. 1: logs
 * and rules in, the count and locations of suspect events out) with its
 * library's overlap of the next batch with the current scan (Sec. 6) and the
 * real-time operation it leaves for future work (Sec. 8).
 *
 * glop_server_create: sets[0 .. n_sets) stay owned by the caller and must
 * outlive the server; the server allocates hbm_budget bytes of device memory
 * (payloads, scratch and results of the batches in flight), max_inflight CUDA
 * streams with pinned buffers, the idle path's staging (fast_bytes) and, when
 * big_bytes > 0, a large-request lane: a worker thread with device staging for
 * requests of up to max_request_bytes.  The current device must stay current
 * for every call.
 * glop_server_submit: queues request `id` (caller-chosen, unique among
 * requests not yet released) of `len` bytes at h_payload (host memory; pinned
 * is fastest), scanned with sets[set].  The payload must stay unchanged until
 * the request's result is handed out.  Requests of at least big_bytes go to
 * the lane; the rest wait for a batch.
 * glop_server_poll: runs the loop -- finished batches advance, a lone request
 * of at most fast_bytes on an idle server takes one glop_scan_host call, and
 * pending requests become batches: in arrival order from the oldest, over
 * every set whose automaton shares the oldest one's kernel kind (one
 * glop_scan_batch_multi launch), within max_batch_bytes,
 * max_batch_requests, out_rows_per_batch (the output bound from each set's
 * matches per byte so far) and the largest free block of the budget.  Stores
 * up to max_res finished results in res and their number in *n_res; waits up
 * to wait_us microseconds for one (0: one pass).  A result's matches (count
 * rows, sorted by offset then pattern id) are pinned host memory owned by the
 * server until glop_server_release(id).  done_ns is the host's monotonic clock
 * (CLOCK_MONOTONIC) when the result was complete.  GLOP_ENOMEM when a request
 * cannot fit the budget even alone; device errors as for the scans.
 * Not thread-safe: one thread per server (the lane's thread is internal).
 */
typedef struct glop_server_s *glop_server; /* opaque */
typedef struct {
    uint64_t hbm_budget;         /* device bytes for the batches in flight */
    uint32_t max_inflight;       /* batches in flight, 1 .. 16 */
    uint32_t max_batch_requests; /* requests per batch */
    uint64_t max_batch_bytes;    /* payload bytes per batch */
    uint64_t out_rows_per_batch; /* largest output bound of a batch, rows (0: max_batch_bytes / 16) */
    uint64_t fast_bytes;         /* idle path for lone requests up to this size (0: none) */
    uint64_t big_bytes;          /* requests of at least this size take the lane (0: no lane) */
    uint64_t max_request_bytes;  /* the largest request the lane must take */
} glop_server_opts;
typedef struct {
    uint64_t id;
    glop_status status;
    const glop_match *matches;   /* count rows, pinned, valid until glop_server_release(id) */
    uint64_t count;
    uint64_t done_ns;            /* CLOCK_MONOTONIC nanoseconds at completion */
} glop_server_result;
typedef struct {
    uint64_t submitted, batches, fast, big, rescans, admission_waits;
    uint64_t requests_per_batch_max, sets_per_batch_max;
    uint64_t pending, inflight;
    uint64_t pinned_allocs;  /* pinned result blocks made after creation (the pool had none of the size) */
} glop_server_stats;
glop_status glop_server_create(const glop_handle *sets, uint32_t n_sets, const glop_server_opts *opts,
                               glop_server *out);
glop_status glop_server_submit(glop_server s, uint64_t id, uint32_t set, const uint8_t *h_payload, uint64_t len);
glop_status glop_server_poll(glop_server s, glop_server_result *res, uint32_t max_res, uint32_t *n_res,
                             uint32_t wait_us);
glop_status glop_server_release(glop_server s, uint64_t id);
glop_status glop_server_stats_get(glop_server s, glop_server_stats *stats);
glop_status glop_server_destroy(glop_server s);

/* Static description of a status code. */
const char *glop_status_str(glop_status s);

#ifdef __cplusplus
}
#endif

#endif /* GLOP_H */
