/*
 * bsort.h -- C ABI of the GB300 (sm_103a) bsort library.
 *
 * Sorts arrays of 8..64-bit unsigned and signed integers and IEEE floats into
 * the order defined by the bsort paper (Guzman, "bsort: a theoretically
 * efficient non-comparison-based sorting algorithm for integer and
 * floating-point numbers"):
 *   - integers: numeric order (Sec. II, Alg. 2 for unsigned keys; Sec. III-A,
 *     Alg. 3 for two's-complement keys);
 *   - floats: sign, then exponent, then mantissa, with the negative half in
 *     the inverted direction (Sec. III-B, Thms. 2/3, Algs. 4/5, Fig. 4), which
 *     places -NaN < -inf < negatives < -0 < +0 < positives < +inf < +NaN, NaNs
 *     ordered by their mantissa field (Sec. III-C, special values).
 * A descending sort is the exact reverse of the ascending one.  Keys are
 * moved as raw bit patterns: no NaN canonicalisation, no flushing of
 * subnormals, signalling NaNs keep their bits.
 *
 * Every call sorts in place: the result is written back into the caller's
 * array, as the paper's functions hand back their input array sorted
 * (outputs of Algs. 3/4).
 *
 * Conventions shared by all entry points
 *   - `keys` / offsets are DEVICE pointers unless the name says host; the
 *     caller owns them.  Pointers must be aligned to the key size; 16-byte
 *     alignment is a fast path, not a requirement.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is asynchronous on `stream` unless stated.
 *   - Arguments are validated before any launch; a rejected call launches
 *     nothing and leaves the keys untouched.
 *   - Errors detected on the device (a work list exceeding its planned
 *     capacity, an expired bounded wait) set a device error word that
 *     bsort_get_error() returns; device code never traps or spins forever.
 *   - No entry point prints or aborts.
 */
#ifndef BSORT_H_
#define BSORT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BSORT_U8 = 0,
    BSORT_I8 = 1,
    BSORT_U16 = 2,
    BSORT_I16 = 3,
    BSORT_F16 = 4,  /* IEEE binary16: 1 sign, 5 exponent, 10 mantissa bits */
    BSORT_U32 = 5,
    BSORT_I32 = 6,
    BSORT_F32 = 7,
    BSORT_U64 = 8,
    BSORT_I64 = 9,
    BSORT_F64 = 10,
    BSORT_BF16 = 11, /* bfloat16: 1 sign, 8 exponent, 7 mantissa bits (the high half of a binary32) */
    /* 128-bit integers (Sec. III-C: the method holds for any word size): a key
     * is 16 bytes, little-endian -- the low 64 bits first -- and the buffer is
     * aligned to 16 bytes.  Ping-pong and segmented sorts; the in-place mode,
     * the key-value sort and the serving loop take keys of up to 8 bytes. */
    BSORT_U128 = 12,
    BSORT_I128 = 13
} bsort_dtype;

typedef enum {
    BSORT_OK = 0,
    BSORT_ERR_INVALID_ARG = 1,          /* NULL pointer, bad dtype/mode, bad handle */
    BSORT_ERR_UNSUPPORTED = 2,          /* valid request the library does not support */
    BSORT_ERR_MISALIGNED = 3,           /* pointer not aligned to the key size */
    BSORT_ERR_NO_MEMORY = 4,            /* device allocation failed */
    BSORT_ERR_WORKSPACE_TOO_SMALL = 5,  /* ws_bytes < bsort_workspace_bytes() */
    BSORT_ERR_CUDA = 6,                 /* a CUDA runtime call failed */
    BSORT_ERR_TIMEOUT = 7,              /* a bounded device wait expired */
    BSORT_ERR_CAPACITY = 8,             /* a device work list outgrew its plan */
    BSORT_ERR_INTERNAL = 9              /* a device-side bounds check refused a store */
} bsort_status;

typedef enum {
    BSORT_MODE_PINGPONG = 0,  /* default: an n-key alternate buffer in the workspace */
    BSORT_MODE_INPLACE = 1    /* digit permutation inside the caller's array (no alternate buffer) */
} bsort_mode;

typedef struct bsort_handle bsort_handle;

/* Human-readable name of a status code; never NULL. */
const char *bsort_status_string(bsort_status status);

/*
 * Sorts keys[0, n) of type `dt` in place on `stream` (ascending if
 * `descending` == 0).  Uses a per-device default handle whose workspace is
 * allocated with cudaMalloc on first use and grown when a larger n arrives
 * (growth synchronises the device).  n == 0 or 1: returns BSORT_OK with no
 * launch.  keys == NULL with n > 1: BSORT_ERR_INVALID_ARG.
 */
bsort_status bsort_keys(void *keys, size_t n, bsort_dtype dt, int descending, void *stream);

/*
 * Bytes of device workspace bsort_keys_ws() needs for n keys of `dt` in
 * `mode` (host-only computation, no CUDA call).  Ping-pong mode needs the
 * n-key alternate buffer plus metadata bounded by n / (finish-threshold).
 * In-place mode needs no alternate buffer: its worst-case reservation is the
 * metadata plus one 32 KB partial-block buffer per 1 MB stripe and per bucket
 * larger than 192 KB, and one state word per 128-byte block; what a call
 * really used is reported by bsort_last_aux_bytes().
 */
bsort_status bsort_workspace_bytes(size_t n, bsort_dtype dt, bsort_mode mode, size_t *bytes);

/* Creates / destroys an explicit handle (profiling state, device error word,
 * statistics of the last call).  A handle must not be used by two host
 * threads at once. */
bsort_status bsort_handle_create(bsort_handle **handle);
bsort_status bsort_handle_destroy(bsort_handle *handle);

/*
 * bsort_keys with a caller-provided workspace: no allocation, no host
 * synchronisation, so the call can be captured in a CUDA graph.  `workspace`
 * is a device pointer, 256-byte aligned, of at least
 * bsort_workspace_bytes(n, dt, mode) bytes; its contents need no
 * initialisation and are scratch after the call.
 *
 * mode BSORT_MODE_INPLACE: every digit pass permutes the keys inside `keys`
 * instead of moving them to an alternate buffer (the paper sorts in place
 * with O(w) extra memory, Sec. III; the GPU keeps counters and block buffers,
 * see bsort_last_aux_bytes).  A bucket of at most 192 KB is read whole into
 * shared memory and written back in digit order; a larger one is classified
 * stripe by stripe into 128-byte blocks of one digit each, the blocks are
 * carried to their digit's block slots, and partial blocks fill the rest.
 * The result is bit-identical to ping-pong mode.
 */
bsort_status bsort_keys_ws(bsort_handle *handle, void *keys, size_t n, bsort_dtype dt, int descending,
                           bsort_mode mode, void *workspace, size_t ws_bytes, void *stream);

/*
 * Runtime tuning of the MSD path of a handle (used by bsort_keys_ws on that
 * handle), per key width (key_bytes 4 or 8); 1- and 2-byte keys take the
 * counting path and have nothing to tune.  Zero fields keep the defaults:
 *   radix_bits  digit width of the MSD levels, 1..11 (default 8): r binary
 *               partitions of Alg. 1 fused per pass; ceil(w / r) levels
 *               (r = 1: one partition per bit, as the paper's recursion).
 *               Widths above 8 use 2048-entry digit tables; the in-place
 *               mode runs widths above 8 as 8;
 *   unit_keys   largest bucket the shared-memory finish takes, 256..default
 *               (5104 for 4-byte keys, 2544 for 8-byte keys);
 *   merge_keys  adjacent small buckets merge up to this many keys, 64..4/5 of
 *               unit_keys (default 4/5 of unit_keys, rounded down to 64);
 *   chunk_tiles keys one CTA histograms and scatters at a time, in scatter
 *               tiles: 1 or 2 (default 2; a tile is 8192 4-byte or 4096
 *               8-byte keys).
 * The result never depends on the tuning, only the speed.  The tuning applies
 * to bsort_keys_ws and to the segmented calls on that handle.  A workspace
 * for a tuned handle must be sized with bsort_workspace_bytes_tuned or
 * bsort_segmented_workspace_bytes_tuned (a smaller finish threshold, a
 * narrower digit or a smaller chunk needs longer work lists, a wider digit
 * larger tables).  NULL restores the defaults.  Invalid fields:
 * BSORT_ERR_INVALID_ARG, nothing changed.
 */
typedef struct {
    int32_t radix_bits;
    int32_t unit_keys;
    int32_t merge_keys;
    int32_t chunk_tiles;
} bsort_tuning;
bsort_status bsort_handle_set_tuning(bsort_handle *handle, int key_bytes, const bsort_tuning *tuning);
bsort_status bsort_workspace_bytes_tuned(size_t n, bsort_dtype dt, bsort_mode mode, const bsort_tuning *tuning,
                                         size_t *bytes);

/*
 * Intermediate state, for checking the digit passes on their own: runs only
 * the first `levels` MSD levels (r bits each, r = the handle's digit width)
 * of bsort_keys_ws, finishes the shared-memory units and constant runs they
 * produced, and leaves every bucket still open unsorted in place (decoded).
 * The result is partitioned by the top levels * r bits of the key order --
 * invariants (i)/(ii) of Alg. 1 at each of those bits (Sec. II) -- with the
 * same bucket boundaries as any such partition; the order inside an open
 * bucket is unspecified (the digit pass is not stable; keys are bit-identical
 * when equal, so the final result is unique).  4- and 8-byte keys, ping-pong
 * workspace.  levels >= the full count: the complete sort.
 */
bsort_status bsort_keys_partial_ws(bsort_handle *handle, void *keys, size_t n, bsort_dtype dt, int descending,
                                   int levels, void *workspace, size_t ws_bytes, void *stream);

/*
 * Counts of the keys by the top `bits` bits of their position in the sorted
 * order, for ranks that sort one array together (each holding a shard): the
 * key is mapped by the library's order-preserving encoding (unsigned: as
 * is; signed: sign bit inverted, Alg. 3's inverted sign pass; float: the sign
 * pass inverted and the negative half's other bits inverted, Algs. 4/5 as
 * Sec. III-B requires; descending: all bits inverted) and its top `bits`
 * bits form digit d.  Digit d's keys precede digit d + 1's in the sorted
 * output, so prefix sums of the counts, summed over the shards, are output
 * positions -- the split that the method's first `bits` MSB partitions make
 * (Thm. 3's refinement).
 *   keys      device pointer, n keys of dtype dt (read only, any alignment
 *             that dt itself needs)
 *   bits      1 .. min(12, key bits)
 *   d_counts  device array of 2^bits uint64 words, owned by the caller,
 *             overwritten: d_counts[d] = keys of digit d
 * Asynchronous on `stream`.  Errors: BSORT_ERR_INVALID_ARG (bits out of
 * range, NULL pointers with n > 0), BSORT_ERR_MISALIGNED, BSORT_ERR_CUDA.
 * n == 0 writes zeros.
 */
bsort_status bsort_top_digit_counts(const void *keys, size_t n, bsort_dtype dt, int descending, int bits,
                                    uint64_t *d_counts, void *stream);

/*
 * Failure-detection self-test: launches one device wait of the kind the
 * library uses (a bounded poll, a fraction of a second) on a flag that nothing
 * sets, on `stream`, and synchronises.  Returns BSORT_ERR_TIMEOUT when the
 * wait gave up and reported it as designed (the context stays usable);
 * BSORT_OK would mean the flag was seen set.  Allocates 8 bytes of device
 * memory for the call.  The paper has no counterpart.
 */
bsort_status bsort_selftest_bounded_wait(void *stream);

/*
 * Auxiliary device bytes the last call on `handle` used beyond the keys:
 * ping-pong mode, its whole workspace (the alternate buffer included);
 * in-place mode, the metadata plus the largest block buffers, slot states
 * and per-digit counters any level used (read from the device: synchronises
 * with the last call's stream); 1- and 2-byte keys, the histogram.  Compare
 * with the paper's O(w) bound for its sequential in-place partition.
 */
bsort_status bsort_last_aux_bytes(bsort_handle *handle, size_t *bytes);

/*
 * End-to-end sort of a HOST array: copies host_keys[0, n) to the device,
 * sorts it and copies the result back into host_keys.  Uses the per-device
 * default handle and a cached device buffer.  Synchronous: returns after the
 * result is in host memory.  Pinned host memory gives the fastest copies.
 */
bsort_status bsort_keys_host(void *host_keys, size_t n, bsort_dtype dt, int descending, void *stream);

/* ---- key-value sorting ----------------------------------------------------
 *
 * Stable key-value sort (the paper sorts keys only; here equal keys -- they
 * are bit-identical -- keep their input order, ascending and descending
 * alike, so the permutation is unique).  keys: n keys of dtype dt (device),
 * sorted in place exactly as bsort_keys sorts them; values: NULL, or n
 * device elements of value_bytes (1, 2, 4 or 8) bytes, any content, permuted
 * in place along with their keys; indices: NULL, or n device int64 outputs,
 * the input position of each output element (an argsort).  keys, values and
 * indices must not overlap each other or the workspace.  n < 2^32 (else
 * BSORT_ERR_UNSUPPORTED); pointers aligned to their element size
 * (BSORT_ERR_MISALIGNED); workspace: bsort_pairs_workspace_bytes, 256-byte
 * aligned, owned by the caller.  Asynchronous on `stream`; device-side
 * failures land in the handle's error word (bsort_get_error).
 * Method, 4- and 8-byte keys: the MSD levels of bsort_keys with a stable
 * scatter (ties keep their order inside every tile, tiles and chunks in
 * buffer order) and a stable LSD finish, the values travelling with their
 * keys through every level.  Values of 4 or 8 bytes travel themselves when
 * no indices are asked for; otherwise 32-bit input positions travel (made
 * when a key is first read), the int64 indices are written beside the sorted
 * keys and values of any width follow by one gather along the positions.
 * With neither values nor indices the keys-only sort runs.  1- and 2-byte
 * keys: each key's order-preserving code is widened to a 32-bit word, the
 * words are sorted so (unsigned, ascending) and narrowed back to keys.  The
 * value-carrying levels have a fixed shape: no handle tuning applies, and
 * bsort_pairs_workspace_bytes_tuned (kept for callers of earlier versions;
 * it validates the tuning) returns the same bytes as
 * bsort_pairs_workspace_bytes.
 */
bsort_status bsort_pairs_workspace_bytes(size_t n, bsort_dtype dt, size_t *bytes);
bsort_status bsort_pairs_workspace_bytes_tuned(size_t n, bsort_dtype dt, const bsort_tuning *tuning8, size_t *bytes);
bsort_status bsort_pairs_ws(bsort_handle *handle, void *keys, void *values, size_t value_bytes, int64_t *indices,
                            size_t n, bsort_dtype dt, int descending, void *workspace, size_t ws_bytes,
                            void *stream);

/* ---- segmented and graph forms -------------------------------------------
 *
 * Segmented sort: the segments [d_offsets[s], d_offsets[s+1]), s <
 * num_segments, of one keys buffer of n keys are each sorted in place and
 * independently (the paper's functions applied to every segment).  d_offsets
 * is a DEVICE array of num_segments + 1 uint64 offsets, non-decreasing, the
 * last <= n; it is read on the device, and a decreasing or out-of-range
 * offset sets the device error word (BSORT_ERR_INTERNAL via
 * bsort_get_error), after which the call's remaining device work stops and
 * the keys are left partly unsorted (never written outside [0, n)).  4- and
 * 8-byte keys
 * (1/2-byte keys: BSORT_ERR_UNSUPPORTED).  All segments run in one fixed
 * launch sequence: segments become the initial buckets (or, up to the
 * shared-memory finish size, finish units) of the MSD levels.
 */
bsort_status bsort_segmented_workspace_bytes(size_t n, size_t num_segments, bsort_dtype dt, size_t *bytes);
/* Workspace of a segmented sort on a handle tuned with `tuning` (NULL: defaults). */
bsort_status bsort_segmented_workspace_bytes_tuned(size_t n, size_t num_segments, bsort_dtype dt,
                                                   const bsort_tuning *tuning, size_t *bytes);
bsort_status bsort_keys_segmented_ws(bsort_handle *handle, void *keys, size_t n, const uint64_t *d_offsets,
                                     size_t num_segments, bsort_dtype dt, int descending, void *workspace,
                                     size_t ws_bytes, void *stream);
/* As above with the per-device default handle (workspace cached, grown with cudaMalloc). */
bsort_status bsort_keys_segmented(void *keys, size_t n, const uint64_t *d_offsets, size_t num_segments,
                                  bsort_dtype dt, int descending, void *stream);

/*
 * CUDA graphs of a whole sort, for callers that repeat the same sort on the
 * same buffers: the launch sequence (with its device-side work lists) is
 * captured once and replayed with one cudaGraphLaunch.  The graph is bound
 * to keys / offsets / workspace; their contents may change between launches.
 * bsort_graph_error waits for `stream` and reads the device error word of the
 * graph's last run.
 */
typedef struct bsort_graph bsort_graph;
bsort_status bsort_graph_create(bsort_handle *handle, void *keys, size_t n, bsort_dtype dt, int descending,
                                void *workspace, size_t ws_bytes, bsort_graph **graph);
bsort_status bsort_graph_create_segmented(bsort_handle *handle, void *keys, size_t n, const uint64_t *d_offsets,
                                          size_t num_segments, bsort_dtype dt, int descending, void *workspace,
                                          size_t ws_bytes, bsort_graph **graph);
bsort_status bsort_graph_launch(bsort_graph *graph, void *stream);
bsort_status bsort_graph_error(bsort_graph *graph, void *stream);
bsort_status bsort_graph_destroy(bsort_graph *graph);

/* ---- serving: continuous batching of sort requests ------------------------
 *
 * A server owns lanes, one per entry of its device list, and a scheduler
 * thread.  A lane has num_slots slots (a CUDA stream, a handle, a workspace
 * of the largest request, and a staging buffer plus segmented workspace of
 * batch_keys keys) and its own HBM budget.  A request joins the queue of the
 * least-loaded lane of the device its buffer lives on (in-flight plus queued
 * bytes over the lane's budget; ties: the lower lane); a device listed twice
 * is two lanes sharing one GPU.  In each lane, the oldest waiting request is
 * admitted when a slot is free and the lane's budget -- payload bytes plus
 * the workspace a standalone sort of the request needs, summed over the
 * lane's admitted requests -- has room (a request is always admitted when
 * nothing else is in flight on its lane).  The budget covers the requests'
 * own footprints; the slots' workspaces (slot_workspace_bytes each, reported
 * by bsort_server_stats) are held on top of it from creation on.  A slot
 * takes up to max_batch requests at once while their keys stay <=
 * batch_keys; those of one 4- or 8-byte dtype and direction are gathered into
 * the slot's staging buffer and sorted by one segmented sort (one launch
 * sequence), the rest by the plain sort.  Requests in different slots
 * overlap on the device.  A segment is sorted exactly as a plain array, so a
 * request's result is the same alone and in the mix.  Timestamps are host
 * steady-clock nanoseconds.  The caller keeps each request's device buffer
 * alive, and does not touch it, until its completion is polled.
 */
#define BSORT_SERVER_MAX_LANES 64
typedef struct bsort_server bsort_server;
typedef struct {
    int32_t num_slots;          /* 1..64 */
    int32_t max_batch;          /* requests a slot takes at once, 1..4096 */
    size_t hbm_budget_bytes;    /* admission budget */
    size_t max_request_keys;    /* largest request accepted (sizes the slot workspaces) */
    size_t batch_keys;          /* a slot batches requests while their total keys stay <= this */
    int32_t mode;               /* bsort_mode of every sort (in-place: smaller workspaces) */
    int32_t pad;
} bsort_server_config;
typedef struct {
    uint64_t tag;
    int32_t status;             /* bsort_status of this request's sort */
    int32_t slot;               /* server-wide slot index: lane * num_slots + slot of the lane */
    int32_t lane;               /* lane that sorted it */
    int32_t pad;
    uint64_t t_submit_ns, t_admit_ns, t_done_ns;
} bsort_completion;
typedef struct {
    uint64_t submitted, completed, batches, pending;
    size_t in_flight_bytes, peak_in_flight_bytes;  /* summed over the lanes */
    int32_t max_concurrent_slots;
    int32_t num_lanes;
    size_t slot_workspace_bytes;  /* device bytes each slot holds: plain and segmented workspaces, staging */
    uint64_t launches;          /* kernel launches (and memsets) enqueued so far */
    uint64_t grouped_sorts;     /* segmented sorts that took several requests at once */
} bsort_server_info;
typedef struct {
    int32_t device;
    int32_t num_slots;
    size_t budget_bytes;
    size_t in_flight_bytes, peak_in_flight_bytes, queued_bytes;
    uint64_t admitted, completed;
} bsort_server_lane_info;
/* One lane on the current device. */
bsort_status bsort_server_create(const bsort_server_config *cfg, bsort_server **server);
/* One lane per entry of devices[0, num_devices) (CUDA device ordinals,
 * 1..BSORT_SERVER_MAX_LANES entries, repeats allowed), each with cfg's slots
 * and budget.  Bad ordinals or config: BSORT_ERR_INVALID_ARG. */
bsort_status bsort_server_create_multi(const bsort_server_config *cfg, const int32_t *devices, int32_t num_devices,
                                       bsort_server **server);
/* The device of the least-loaded lane: where to put the next request. */
bsort_status bsort_server_pick_device(bsort_server *server, int32_t *device);
/* Queues a request (non-blocking) on the least-loaded lane of the device
 * holding `keys`.  n > max_request_keys: BSORT_ERR_UNSUPPORTED; keys not in
 * device memory of a served device: BSORT_ERR_INVALID_ARG. */
bsort_status bsort_server_submit(bsort_server *server, void *keys, size_t n, bsort_dtype dt, int descending,
                                 uint64_t tag);
/* Counters of one lane. */
bsort_status bsort_server_lane_stats(bsort_server *server, int32_t lane, bsort_server_lane_info *out);
/* Moves up to max completions into out; *count = how many. */
bsort_status bsort_server_poll(bsort_server *server, bsort_completion *out, size_t max, size_t *count);
bsort_status bsort_server_stats(bsort_server *server, bsort_server_info *out);
/* Waits until every submitted request has completed (BSORT_ERR_TIMEOUT after timeout_s). */
bsort_status bsort_server_drain(bsort_server *server, double timeout_s);
/* paused != 0: admit nothing new (slots in flight still complete); 0: resume. */
bsort_status bsort_server_pause(bsort_server *server, int paused);
bsort_status bsort_server_destroy(bsort_server *server);

/*
 * The paper has no counterpart of this entry point.  bsort_keys() for callers
 * that may not allocate device memory while they run -- code under CUDA
 * graph capture (allocation is not capturable, and cudaMalloc / cudaFree
 * synchronise the device), programs whose device memory belongs to their own
 * pool allocator, plugins whose host engine forbids raw allocations.  The
 * scratch memory is a static device array of BSORT_NOALLOC_SCRATCH_BYTES
 * inside the library; the call allocates and frees nothing.
 *   - Sizes: n is accepted while bsort_workspace_bytes(n, dt, PINGPONG)
 *     fits the array (64 MiB): about 14.5 million 4-byte keys or 7.2 million
 *     8-byte keys; 1- and 2-byte keys need a fixed amount, so any n.  A larger
 *     n returns BSORT_ERR_WORKSPACE_TOO_SMALL before any launch.
 *   - Set-up: the first call on each device looks up the array's device
 *     address (cudaGetSymbolAddress) and loads the module that holds it; make
 *     that first call before any stream capture.  The array then stays
 *     resident on that device until the process exits.
 *   - Sharing: all calls on a device share the one array and leave their
 *     scratch in it.  The sort initialises everything it reads, so stale
 *     contents do no harm, but calls whose device work overlaps in time
 *     (different streams with no ordering between them) race on the array
 *     and give wrong results: order them on one stream or with events.
 *   - The device error word of these calls lives in the shared array and is
 *     not reported; the call returns launch-time errors only.
 */
#define BSORT_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
bsort_status bsort_keys_noalloc(void *keys, size_t n, bsort_dtype dt, int descending, void *stream);

/*
 * Waits for `stream`, then returns (and clears) the device error word of the
 * last call made with `handle` (NULL = the default handle of the current
 * device): BSORT_OK, BSORT_ERR_CAPACITY, BSORT_ERR_TIMEOUT or
 * BSORT_ERR_INTERNAL.
 */
bsort_status bsort_get_error(bsort_handle *handle, void *stream);

/* ---- measurement ------------------------------------------------------- */

enum { BSORT_PROFILE_MAX = 1024, BSORT_PROFILE_MAX_CALLS = 64 };

/* kinds of device launches, used in profile records */
typedef enum {
    BSORT_K_INIT = 0,     /* resets the work lists */
    BSORT_K_HIST = 1,     /* key transform + digit histogram of one level */
    BSORT_K_SCAN = 2,     /* per-digit offsets across chunks */
    BSORT_K_CLASSIFY = 3, /* bucket digit bases, child classification */
    BSORT_K_SCATTER = 4,  /* shared-memory-staged digit scatter */
    BSORT_K_FINISH = 5,   /* per-bucket shared-memory finish + decode */
    BSORT_K_FILL = 6,     /* write-only fill of constant runs */
    BSORT_K_COUNT_HIST = 7,  /* 8/16-bit: histogram of all key bits */
    BSORT_K_COUNT_SCAN = 8,  /* 8/16-bit: bin starts */
    BSORT_K_COUNT_FILL = 9   /* 8/16-bit: counting fill of the output */
} bsort_kernel_kind;

typedef struct {
    int32_t kind;            /* bsort_kernel_kind */
    int32_t level;           /* MSD level for per-level kernels, else -1 */
    int32_t call;            /* index of the call since the records were last read */
    float ms;                /* CUDA-event time of this launch group on the call's stream */
    uint64_t keys;           /* keys this launch processed (device counters) */
    uint64_t counted_bytes;  /* algorithmic HBM bytes of this launch: keys read (histogram),
                              * keys read and written (scatter, finish), keys written (fill);
                              * a key-value call adds the values each key carries and, in the
                              * finish and fills, the values or int64 positions written */
} bsort_profile_record;

typedef struct {
    int32_t num_records;
    int32_t num_calls;       /* calls covered by the records */
    int32_t num_launches;    /* kernels launched by those calls */
    int32_t pad;
    /* shared-memory finish units of those calls, by method: one counting pass,
     * split + comparison ranks, LSD passes */
    uint64_t finish_units_counting, finish_units_compare, finish_units_lsd;
    /* of the counting units, those finished by the vector-load counting pass
     * for keys known to agree above their low 16 bits */
    uint64_t finish_units_counting_fast;
    bsort_profile_record rec[BSORT_PROFILE_MAX];
} bsort_profile;

/* Enables CUDA-event timing of every launch of later calls on `handle`.
 * Records accumulate over up to BSORT_PROFILE_MAX_CALLS calls (each call
 * also copies its work counters into a handle-owned device slot, on its
 * stream, so no call synchronises) until bsort_handle_get_profile(). */
bsort_status bsort_handle_set_profiling(bsort_handle *handle, int enable);

/* Synchronises with the device, returns the records accumulated since the
 * last read (calls beyond BSORT_PROFILE_MAX_CALLS are not recorded) and
 * clears them. */
bsort_status bsort_handle_get_profile(bsort_handle *handle, bsort_profile *out);

/* Number of kernels the last call on `handle` launched (host count). */
bsort_status bsort_last_launch_count(bsort_handle *handle, int *launches);

#ifdef __cplusplus
}
#endif

#endif /* BSORT_H_ */
