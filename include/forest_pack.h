/*
 * forest_pack.h -- C ABI of the GB300 forest-packing classification library.
 *
 * The library classifies batches of observations with a trained decision
 * forest stored in the packed layout of "Forest Packing: Fast, Parallel
 * Decision Forests" (Browne et al.):
 *   - trees are grouped into bins of B trees (Section III, "T/B bins");
 *   - the top of each tree -- its 2^(d+1)-1 most frequently visited nodes,
 *     levels 0..d for a complete tree -- is interleaved with the other trees
 *     of its bin into one contiguous block (Section III-A, Bin layout; d = 0
 *     interleaves the roots only, Fig. 2), staged into shared memory;
 *   - deeper nodes are laid out per tree depth-first with the more frequently
 *     reached child placed next to or first after its parent (Section III-A,
 *     Stat), in super-nodes of two or three tree levels that fill one 32-byte
 *     memory sector (three levels store thresholds as order-preserving keys,
 *     the last level's shortened, with exact tie-breaking from a side table);
 *   - leaves are not stored as nodes: their class is folded into the reference
 *     that leads to them (Section III-A, DF-, which replaces leaves with
 *     per-class nodes);
 * and reduces the per-tree leaf classes to a majority vote.
 *
 * Groups of entry points: packing and upload (fp_pack_forest, fp_upload,
 * fp_configure); classification of device rows (fp_predict,
 * fp_predict_values, fp_predict_leaves, fp_predict_batched,
 * fp_predict_noalloc); classification of host rows with copies pipelined
 * against the kernels (fp_predict_host, fp_predict_values_host); the serving
 * runtime (fp_server_*, fp_request_*); tree-bin sharding over processes
 * (fp_shard_trees, fp_pack_forest_trees, fp_votes_argmax); the plain-layout baseline
 * (fp_plain_*); statistics and probes (fp_count_leaves,
 * fp_cardinality_from_leaf_counts, fp_infer_cardinality, fp_l2_read_probe);
 * status and fault injection (fp_sync_status, fp_inject_fault).
 *
 * Conventions for every entry point:
 *   - Return FP_OK (0) or a negative FP_E* code; no C++ exception crosses the
 *     boundary.  fp_last_error() returns a thread-local message for the last
 *     failing call on the calling thread.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is enqueued asynchronously on it; an argument
 *     error is reported before anything is enqueued.  Errors raised inside a
 *     kernel (a bounded wait that ran out, a corrupt record) are recorded in
 *     the forest's device status word and reported by fp_sync_status().
 *   - Pointers marked "device" must be device (or managed) memory of the
 *     current device; "host" pointers are ordinary host memory.  The caller
 *     owns every buffer it passes; the library owns every object it returns
 *     through an out-pointer until the matching release call.
 *   - n == 0 is valid and enqueues nothing.  A NULL optional output is skipped.
 *   - Split rule: x[feature] <= threshold goes to the left child, otherwise
 *     (including NaN) to the right child, compared in IEEE FP32 without
 *     flushing subnormals.  Vote ties go to the lowest class index.  (The paper
 *     states neither rule.)
 */
#ifndef FOREST_PACK_H
#define FOREST_PACK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FP_OK 0
#define FP_EINVAL (-1)       /* bad argument or malformed forest */
#define FP_ENOMEM (-2)       /* host or device allocation failed */
#define FP_ECUDA (-3)        /* a CUDA runtime call failed */
#define FP_EUNSUPPORTED (-4) /* forest exceeds a field width of the record format */
#define FP_ETIMEOUT (-5)     /* a bounded device wait ran out */
#define FP_EDEVICE (-6)      /* a kernel reported a corrupt record or index */

/* A trained forest (Section III: T binary trees, each internal node a split
 * condition with two children, each leaf one class label).  Host memory,
 * owned by the caller, read only during fp_pack_forest / fp_plain_build.
 * Node arrays are concatenated per tree; node ids are tree-local and node 0
 * of each tree is its root. */
typedef struct fp_forest_desc {
    int32_t n_trees;                /* T >= 1 */
    int32_t n_features;             /* 1 .. 1024 */
    int32_t n_classes;              /* 1 .. 512 */
    const int64_t *tree_node_begin; /* [T+1] offsets into the node arrays */
    const int32_t *left;            /* child id, tree-local; -1 marks a leaf */
    const int32_t *right;           /* child id, tree-local; -1 on leaves */
    const int32_t *feature;         /* split feature (internal nodes) */
    const float *threshold;         /* split threshold (internal nodes) */
    const int32_t *leaf_class;      /* class label (leaves) */
    const int64_t *cardinality;     /* training count reaching the node; used to
                                       order children (Section III-A, Stat).
                                       NULL: children keep left-first order. */
    const float *leaf_value;        /* NULL for a classification forest; else a
                                       forest with real leaf values (regression
                                       or boosted trees): the value of each leaf
                                       (finite; entries of internal nodes are
                                       ignored), evaluated by fp_predict_values */
} fp_forest_desc;

/* Layout and launch parameters; 0 selects the default (for interleave_depth,
 * -1 does, since 0 is a valid depth).  The defaults depend on the row width:
 * for rows of more than 384 features ("wide rows") they are bins of 32 trees,
 * paired level heads 0..3, tiles of up to ~200 KiB of rows and two bin
 * buffers (few rows fit in shared memory, so bins hold many trees); else the
 * values below.
 *   bin_size          B, trees per bin (Section III-A "stripe width"), 1..1024
 *                     (default 3; wide rows 32)
 *   interleave_depth  d: each tree contributes 2^(d+1)-1 nodes (levels 0..d of
 *                     a complete tree) to its bin's interleaved block
 *                     (Section III-A), 0..9 for ranked heads, 0..11 for
 *                     level heads (default 9; wide rows 3)
 *   obs_tile          observations per work item of the traversal kernel,
 *                     a multiple of 32, up to 2048 (default: ~96 KiB of rows,
 *                     wide rows ~200 KiB; shrunk at upload to fit shared
 *                     memory)
 *   warps_per_cta     warps per CTA of the traversal kernel, 1..32
 *   pass_bytes        bins are swept in groups ("passes") whose records fit in
 *                     this many bytes, so a pass stays resident in L2 while
 *                     every observation tile walks it; 0 = default (48 MiB),
 *                     negative = one pass over the whole forest
 *   refill_lanes      a warp hands new (observation, tree) tasks to its idle
 *                     lanes once this many lanes are idle, 1..32
 *   head_select       which 2^(d+1)-1 nodes of a tree form its interleaved head:
 *                     1 = levels 0..d in implicit breadth-first slots (the
 *                     Bin layout's interleaved levels; every walk takes d+1
 *                     steps); 2 = the same levels stored two per 16-byte
 *                     record (a node and its children; d odd), one
 *                     shared-memory load per two levels; 3 = ranked: the
 *                     nodes of highest training cardinality (the popular
 *                     paths of Section III-A), walked by explicit targets;
 *                     0 = default: 2 when d is odd, else 1
 *   bin_buffers       shared-memory buffers that bin blocks stream through,
 *                     2 or 3 (0 = 3; wide rows 2): two leave room for larger
 *                     heads or tiles, three hide copy latency better
 *   deep_levels       tree levels per 32-byte super-node below the head: 2
 *                     (full thresholds), 3 (thresholds as order keys, some
 *                     shortened to key prefixes, ties decided by a side
 *                     table of full keys; the field widths deep_format
 *                     names must fit, classes not counted for forests with
 *                     leaf values), or 0 = default: 3 when
 *                     deep_format 1 or 2 fits (below, within the default
 *                     bounds), else 2
 *   deep_format       the fields of a three-level super-node: 1 = full keys
 *                     for the first two levels, key prefixes for the last
 *                     (needs 2 * ceil(log2 F) + 2 * ceil(log2 C) <= 24;
 *                     default bound 16); 2 = key prefixes in every slot, of
 *                     keys remapped onto the forest's own threshold range
 *                     (needs ceil(log2 F) + 2 * ceil(log2 C) <= 24; default
 *                     bound 20), for forests with many features or classes;
 *                     0 = default: 1 where it fits, else 2.  Both compare
 *                     exactly (a prefix tie is decided by the full key). */
typedef struct fp_pack_params {
    int32_t bin_size;
    int32_t interleave_depth;
    int32_t obs_tile;
    int32_t warps_per_cta;
    int64_t pass_bytes;
    int32_t refill_lanes;
    int32_t head_select;
    int32_t bin_buffers;
    int32_t deep_levels;
    int32_t deep_format;
} fp_pack_params;

typedef struct fp_packed_forest fp_packed_forest; /* host image, opaque */
typedef struct fp_device_forest fp_device_forest; /* resident on one device, opaque */

/* Sizes of a packed image (for tests, memory planning and the roofline). */
typedef struct fp_packed_info {
    int32_t n_trees, n_features, n_classes;
    int32_t bin_size, interleave_depth, n_bins;
    int32_t obs_tile, warps_per_cta;
    int64_t n_internal;       /* internal nodes of the forest */
    int64_t n_super;          /* 32-byte super-nodes below the interleaved levels */
    int64_t head_bytes;       /* all bins' interleaved blocks (+ link rows) */
    int64_t deep_bytes;       /* n_super * 32 */
    int64_t total_bytes;      /* bytes uploaded for classification */
    int64_t parity_bytes;     /* leaf-id side tables, uploaded for fp_predict_leaves */
    int32_t max_head_bytes;   /* largest single bin block (staged in shared memory) */
    int32_t passes;           /* bin groups swept one after another (L2 blocking) */
    int32_t refill_lanes;
    int32_t head_nodes;       /* 2^(d+1)-1: head nodes per tree at most */
    int32_t head_select;
    int32_t bin_buffers;
    int32_t deep_levels;      /* tree levels per super-node (2 or 3) */
    int32_t deep_format;      /* three levels: 1 full keys first, 2 prefixes in every slot; else 0 */
} fp_packed_info;

/* Build the packed host image of a forest (Section III-A: DF-, Stat, Bin).
 * desc: host, caller-owned.  params: may be NULL (all defaults).
 * *out: library-owned until fp_release_packed.
 * Errors: FP_EINVAL (malformed forest: bad child ids, cycles, classes or
 * features out of range, bad params), FP_EUNSUPPORTED (more than 1024
 * features or 512 classes, a bin block over 100 KiB, 2^32 super-nodes or
 * more), FP_ENOMEM. */
int fp_pack_forest(const fp_forest_desc *desc, const fp_pack_params *params, fp_packed_forest **out);

/* Fill *info with the sizes of a packed image.  Host only. */
int fp_packed_info_get(const fp_packed_forest *pf, fp_packed_info *info);

/* The packed host image itself, for host-side decoding tests: the bytes that
 * fp_upload copies (*bytes receives the size).  Library-owned; valid until
 * fp_release_packed.  Returns NULL on bad arguments. */
const void *fp_packed_image(const fp_packed_forest *pf, int64_t *bytes);

/* Copy a packed image to the current device on `stream` and return a
 * resident forest (library-owned until fp_release).  The call waits for the
 * copy to finish on `stream`, so the host image may be released once it
 * returns.  Errors: FP_EINVAL, FP_ENOMEM, FP_ECUDA, FP_EUNSUPPORTED (the
 * launch does not fit shared memory). */
int fp_upload(const fp_packed_forest *pf, void *stream, fp_device_forest **out);

/* Change the launch parameters of a resident forest: obs_tile,
 * warps_per_cta, refill_lanes and bin_buffers of *params (0 keeps the current
 * value); the layout fields (bin_size, interleave_depth, pass_bytes) must be 0
 * or equal to the forest's.  The observation tile is lowered, if needed, to fit shared
 * memory.  Host only; do not call while a launch on this forest is being
 * enqueued from another thread.  Errors: FP_EINVAL, FP_EUNSUPPORTED, FP_ECUDA. */
int fp_configure(fp_device_forest *forest, const fp_pack_params *params);

/* Classify n observations (Section III; Section III-B evaluates a bin's
 * trees together, here a CTA walks a bin's trees for a tile of observations).
 *   X          device, [n][n_features] FP32 row-major, contiguous rows
 *   out_votes  device, [n][n_classes] uint32 per-class leaf counts, or NULL
 *   out_class  device, [n] int32 argmax of the votes (lowest class on ties),
 *              or NULL
 * Asynchronous on `stream`; X must stay valid and the outputs untouched until
 * the stream reaches this work.  Calls on different streams may overlap.
 * Errors: FP_EINVAL, FP_ENOMEM (stream-ordered scratch), FP_ECUDA. */
int fp_predict(const fp_device_forest *forest, const float *X, int64_t n, uint32_t *out_votes, int32_t *out_class,
               void *stream);

/* fp_predict without any device allocation.  The paper has no counterpart:
 * this entry point serves callers that cannot allocate device memory while
 * they classify -- a serving loop that runs under a fixed device-memory
 * budget and must not grow or fragment the heap, code that runs while it
 * holds its own allocator's lock, or code that must not reach the driver's
 * allocation path, which can synchronise the device.
 * Arguments, outputs and errors are those of fp_predict.  A forest swept in
 * several passes needs scratch (a vote accumulator when out_votes is NULL and
 * one counter per observation tile when out_class is given); here it comes
 * from one fixed 16 MiB device array inside the library, which every GPU that
 * loads the library holds until the process exits.  A call whose scratch
 * would exceed 16 MiB returns FP_EINVAL before enqueuing anything (pass
 * out_votes, split the batch, or use fp_predict).  The first call on a device
 * looks up the array's device address, so make it before any CUDA-graph
 * stream capture.  All calls on a device share its one array, which keeps
 * the last call's contents; each call clears the part it uses.  Calls whose
 * work overlaps on the GPU (for instance on two streams) race on the array
 * and must be ordered by the caller.  Nothing is allocated or freed: no
 * cudaMalloc, cudaFree, cudaMallocAsync or library allocator. */
int fp_predict_noalloc(const fp_device_forest *forest, const float *X, int64_t n, uint32_t *out_votes,
                       int32_t *out_class, void *stream);

/* Forests with real leaf values (packed from a descriptor with leaf_value;
 * regression and boosted trees, the forest variants the paper names beside
 * classification): the same traversal as fp_predict, then
 *   out[i] = bias + scale * (sum over trees of the value of the leaf x_i reaches)
 * computed in float32: the leaf values of a tile are added in shared memory
 * with atomics, and across passes in global memory, in no fixed order, so
 * the result is within (T + 2) * 2^-24 * (|bias| + |scale| * sum |value|) of
 * the exact one (recursive summation in any order, then one multiply-add).
 * Use scale = 1/T for a regression forest's mean, scale = 1 and bias = the
 * initial score for a boosted ensemble.
 *   X     device, [n][n_features] FP32 row-major
 *   out   device, [n] float
 * Errors: FP_EINVAL (also for a forest without leaf values), FP_ENOMEM,
 * FP_ECUDA.  fp_predict, fp_predict_noalloc and fp_predict_batched refuse
 * forests with leaf values (FP_EINVAL); fp_predict_leaves accepts them. */
int fp_predict_values(const fp_device_forest *forest, const float *X, int64_t n, float scale, float bias,
                      float *out, void *stream);

/* fp_predict and fp_predict_values for rows and results in host memory: the
 * rows go to the device in chunks of chunk_rows (0: an eighth of n, at least
 * 65,536) through two device buffers; chunk c+1 is copied in on a copy
 * stream the library keeps per device while chunk c is classified.  The
 * chunks of the first buffer are classified on `stream`, those of the second
 * on a second stream the library keeps per device (so a chunk's kernel
 * starts on the SMs the previous one has left); each chunk's outputs are
 * copied back on its kernel's stream, and `stream` waits for the second
 * stream before the call's last work, so completion of `stream` covers
 * everything.  Device memory for the buffers comes from the stream-ordered
 * pool.
 *   X_host          host, [n][n_features] FP32 row-major; page-locked memory
 *                   (cudaHostAlloc, or a pinned torch tensor) lets the copies
 *                   overlap the kernels, ordinary memory works but copies
 *                   synchronously
 *   out_votes_host  host, [n][n_classes] uint32, or NULL
 *   out_class_host  host, [n] int32, or NULL
 *   out_host        host, [n] float (fp_predict_values_host)
 * The calls return once the work is queued; the results are in the host
 * buffers, which must stay valid until then, when `stream` completes.
 * Errors: as fp_predict / fp_predict_values. */
int fp_predict_host(const fp_device_forest *forest, const float *X_host, int64_t n, uint32_t *out_votes_host,
                    int32_t *out_class_host, int64_t chunk_rows, void *stream);
int fp_predict_values_host(const fp_device_forest *forest, const float *X_host, int64_t n, float scale, float bias,
                           float *out_host, int64_t chunk_rows, void *stream);

/* ---- Serving: continuous batching over resident forests (library threads).
 *
 * A server owns `slots` CUDA streams with page-locked staging and device
 * buffers on `device`, a batcher thread and a completion thread.  Requests
 * (rows of one forest in host memory) are submitted from any thread; the
 * batcher takes what has arrived, in arrival order up to max_rows rows (a
 * larger request forms a launch of its own), groups it by forest and issues one
 * fp_predict_batched launch on a free slot once the device reports at least
 * the launch's bytes + mem_margin free (else it waits for launches in
 * flight); with max_wait_s > 0 it first lets a batch grow until the oldest
 * request has waited that long.  The completion thread polls launches in
 * order (at most 60 s each, then FP_ETIMEOUT), copies each request's classes
 * (and votes) into the caller's buffers and wakes its waiters.
 *   fp_server_create        slots 1..64, max_rows >= 1, mem_margin >= 0 bytes;
 *                           return_votes: requests may ask for votes
 *   fp_server_add_forest    before fp_server_start; the forest must stay
 *                           resident until fp_server_release; *out_id names it
 *   fp_server_submit        X_host [n][n_features] FP32, out_class_host [n]
 *                           int32 and/or out_votes_host [n][n_classes] uint32,
 *                           all host, caller-owned, valid until the request
 *                           is answered; *out: the request, library-owned
 *                           until fp_request_release
 *   fp_request_wait         waits up to timeout_s seconds (< 0: no limit);
 *                           returns the request's status, or FP_ETIMEOUT if
 *                           it is not answered yet
 *   fp_request_latency      seconds from submit to answer, or -1 before
 *   fp_request_release      waits for the answer, then frees the request
 *   fp_server_stop          answers every queued request, then joins the
 *                           threads; no submits afterwards
 *   fp_server_stats         launches issued and admission waits so far
 *   fp_server_set_free_bytes  tests: the free device bytes admission sees
 *                           (-1: ask the device)
 *   fp_server_set_launch_timeout  the completion poll's limit per launch in
 *                           seconds (default 60; >= 0)
 *   fp_server_slots_in_service  slots not retired.  A slot returns to service
 *                           only once all work queued on it has finished; a
 *                           launch still running at its limit (or a failed
 *                           launch whose queued copies are still running after
 *                           another such wait) answers its requests with
 *                           FP_ETIMEOUT and retires the slot, whose buffers
 *                           are never reused; with no slot left in service
 *                           every request is answered with FP_ETIMEOUT
 *   fp_server_release       stops if needed and frees the server (a retired
 *                           slot's buffers are freed only if its work has
 *                           finished within one more launch limit)
 * Errors: FP_EINVAL, FP_ENOMEM, FP_ECUDA; a failed launch answers its
 * requests with its status. */
typedef struct fp_server fp_server;
typedef struct fp_request fp_request;
int fp_server_create(int32_t device, int32_t slots, int64_t max_rows, int64_t mem_margin, int32_t return_votes,
                     double max_wait_s, fp_server **out);
int fp_server_add_forest(fp_server *server, const fp_device_forest *forest, int32_t *out_id);
int fp_server_start(fp_server *server);
int fp_server_submit(fp_server *server, int32_t forest_id, const float *X_host, int64_t n, int32_t *out_class_host,
                     uint32_t *out_votes_host, fp_request **out);
int fp_request_wait(fp_request *request, double timeout_s);
double fp_request_latency(const fp_request *request);
void fp_request_release(fp_request *request);
int fp_server_stop(fp_server *server);
int fp_server_stats(const fp_server *server, int64_t *launches, int64_t *rejected_for_memory);
int fp_server_set_free_bytes(fp_server *server, int64_t free_bytes);
int fp_server_set_launch_timeout(fp_server *server, double seconds);
int fp_server_slots_in_service(const fp_server *server, int32_t *out);
void fp_server_release(fp_server *server);

/* Parity mode: the leaf each observation reaches in each tree.
 *   out_leaf   device, [n][n_trees] int32, tree-local node id of the leaf in
 *              the fp_forest_desc the forest was packed from
 * Errors as fp_predict. */
int fp_predict_leaves(const fp_device_forest *forest, const float *X, int64_t n, int32_t *out_leaf, void *stream);

/* One launch over several resident forests and uneven batches (the batching
 * pattern: many forests and observation batches in one persistent kernel,
 * suitable for CUDA-graph capture).  Every element is as in fp_predict. */
typedef struct fp_batch {
    const float *X;      /* device [n][n_features of its forest] */
    int64_t n;
    uint32_t *out_votes; /* device [n][n_classes] or NULL */
    int32_t *out_class;  /* device [n] or NULL */
} fp_batch;
int fp_predict_batched(const fp_device_forest *const *forests, const fp_batch *batches, int32_t k, void *stream);

/* Wait for `stream` and report the forest's device status word: FP_OK, or the
 * first error a kernel recorded since the last call (FP_ETIMEOUT,
 * FP_EDEVICE).  Clears the word.  Blocks the calling host thread. */
int fp_sync_status(const fp_device_forest *forest, void *stream);

/* Fault injection for failure-detection tests (the paper has no counterpart).
 * Nothing it does faults, traps or hangs a GPU: it makes the library's own
 * error paths run.
 *   FP_FAULT_ALLOC           forest ignored (may be NULL); the next `value`
 *                            device allocations made by fp_upload and by the
 *                            scratch of fp_predict / fp_predict_batched fail
 *                            with FP_ENOMEM (0 clears)
 *   FP_FAULT_WAIT_LIMIT      a bin-block wait of this forest's kernels polls its
 *                            barrier at most `value` times (1 .. 2^24; the
 *                            default is 2^24) before recording FP_ETIMEOUT
 *   FP_FAULT_STALL_BIN_COPY  value 1: this forest's bin-block waits ignore
 *                            completed copies, so every launch records
 *                            FP_ETIMEOUT (read by fp_sync_status) and leaves
 *                            its outputs unspecified; the copies still land
 *                            before the kernel exits.  value 0 restores.
 * Not thread-safe against concurrent launches of the same forest.
 * Errors: FP_EINVAL (unknown kind, value out of range, NULL forest). */
#define FP_FAULT_ALLOC 1
#define FP_FAULT_WAIT_LIMIT 2
#define FP_FAULT_STALL_BIN_COPY 3
int fp_inject_fault(fp_device_forest *forest, int32_t kind, int64_t value);

/* Sizes of a resident forest (same fields as fp_packed_info_get). */
int fp_device_info_get(const fp_device_forest *forest, fp_packed_info *info);

void fp_release_packed(fp_packed_forest *pf); /* NULL is a no-op */
void fp_release(fp_device_forest *forest);     /* NULL is a no-op; synchronises the device */

/* Thread-local message describing the last error on this thread ("" if none). */
const char *fp_last_error(void);

/* Statistics inferred from observations (Section III-A allows the leaf
 * cardinalities that drive the Stat ordering to be estimated after training
 * by classifying a large sample of observations).  For the leaf ids that fp_predict_leaves wrote for n
 * observations, add 1 to leaf_count[node_begin[t] + out_leaf[i][t]] for every
 * (i, t).  Summing each leaf's count into its ancestors gives cardinalities to
 * pack the forest with.
 *   out_leaf    device, [n][n_trees] int32 tree-local leaf ids
 *   node_begin  device, [n_trees+1] int64 offsets of the forest's node arrays
 *   leaf_count  device, int64 per node of the forest; zeroed by the caller,
 *               accumulated (so several samples can be added up)
 *   status      device int32, set to FP_EDEVICE if a leaf id is not a node of
 *               its tree (that entry is skipped)
 * Asynchronous on stream.  Errors: FP_EINVAL, FP_ECUDA. */
int fp_count_leaves(const int32_t *out_leaf, int64_t n, int32_t n_trees, const int64_t *node_begin,
                    int64_t *leaf_count, int32_t *status, void *stream);

/* Node cardinalities from leaf counts (Section III-A: the statistics behind
 * the Stat ordering may be measured on observations after training).  For
 * every tree of desc, a leaf's cardinality is its count and an internal
 * node's is the sum of its two children's, so it is the number of counted
 * observations whose path passes through the node; a node that no path from
 * the root reaches gets 0.  Host only.
 *   desc        host, caller-owned; its tree structure is read (and validated
 *               as fp_pack_forest does)
 *   leaf_count  host, int64 per node of desc (tree_node_begin[T] entries);
 *               only the leaves' entries are read
 *   out_card    host, int64 per node, overwritten; may be leaf_count itself
 * Errors: FP_EINVAL (NULL argument, malformed forest), FP_ENOMEM. */
int fp_cardinality_from_leaf_counts(const fp_forest_desc *desc, const int64_t *leaf_count, int64_t *out_card);

/* Statistics inferred from observations, end to end (Section III-A): the
 * resident forest classifies n observations in parity mode, the leaf each
 * reaches in each tree is counted on the device (fp_count_leaves), and
 * fp_cardinality_from_leaf_counts turns the counts into node cardinalities,
 * which can be given to fp_pack_forest as desc->cardinality to order the
 * layout by observed rather than training frequencies.
 *   forest      resident forest packed from desc
 *   desc        host, caller-owned: the same trees (counts of trees, features,
 *               classes and internal nodes must match the forest's)
 *   X           device, [n][n_features] FP32 row-major
 *   chunk_rows  rows classified per parity launch (0: as many as 256 MiB of
 *               leaf ids hold); device scratch for one chunk's leaf ids and
 *               the counters comes from the stream-ordered pool
 *   out_card    host, int64 per node of desc, overwritten
 * Synchronises `stream`; a kernel error is reported (and the forest's status
 * word cleared) as by fp_sync_status.  Errors: FP_EINVAL, FP_ENOMEM, FP_ECUDA,
 * FP_EDEVICE, FP_ETIMEOUT. */
int fp_infer_cardinality(const fp_device_forest *forest, const fp_forest_desc *desc, const float *X, int64_t n,
                         int64_t chunk_rows, int64_t *out_card, void *stream);

/* ---- Tree-bin sharding over processes (Section III: the T/B bins of a
 * forest are bound to processes; Section IV-E scales that over machines).
 * Every process packs the same forest's bins for its shard, classifies the
 * same rows with them (fp_predict with out_votes), the per-class votes are
 * summed over processes by the caller's collective (for example an NCCL
 * all-reduce of the [n][n_classes] uint32 array), and fp_votes_argmax turns
 * the sums into classes.  Because every tree belongs to exactly one shard,
 * the summed votes and the classes equal the whole forest's.
 *
 * fp_shard_trees: the trees of shard `shard` of n_shards, whole bins of
 * bin_size consecutive trees, in contiguous runs cut so that each shard's
 * expected work is as even as the bin boundaries allow.  A tree's work is its
 * expected number of internal nodes visited per observation, the sum of its
 * internal nodes' cardinalities divided by its root's (Section III-A's
 * training statistics), or its internal node count when desc has no
 * cardinalities.  Host only; every process computes the same split.
 *   *tree_begin, *tree_end   trees [begin, end) of desc; an empty range when
 *                            there are fewer bins than shards
 * Errors: FP_EINVAL, FP_ENOMEM. */
int fp_shard_trees(const fp_forest_desc *desc, int32_t bin_size, int32_t n_shards, int32_t shard,
                   int32_t *tree_begin, int32_t *tree_end);

/* fp_pack_forest over the trees [tree_begin, tree_end) of desc alone (a
 * shard), as a forest of tree_end - tree_begin trees; leaf ids stay the
 * trees' own node ids.  Errors: as fp_pack_forest, FP_EINVAL for an empty or
 * out-of-range tree range. */
int fp_pack_forest_trees(const fp_forest_desc *desc, const fp_pack_params *params, int32_t tree_begin,
                         int32_t tree_end, fp_packed_forest **out);

/* The class of each row from its (summed) votes: out_class[i] = the first c
 * with the largest votes[i][c] (lowest class on ties, as fp_predict).
 *   votes      device, [n][n_classes] uint32
 *   out_class  device, [n] int32
 * Asynchronous on `stream`.  Errors: FP_EINVAL, FP_ECUDA. */
int fp_votes_argmax(const uint32_t *votes, int64_t n, int32_t n_classes, int32_t *out_class, void *stream);

/* Measurement helper, no counterpart in the paper: time `iters` passes of
 * 16-byte reads over a device buffer of `bytes` (16-byte aligned; pick a size
 * that stays resident in L2) after one warming pass, and return the
 * milliseconds in *out_ms; bytes * iters / ms is the L2 read bandwidth used
 * as the traversal kernel's roofline.  Synchronises `stream`.
 * Errors: FP_EINVAL, FP_ECUDA. */
int fp_l2_read_probe(const void *buf, int64_t bytes, int32_t iters, void *stream, float *out_ms);

/* ------------------------------------------------------------------------
 * Plain baseline: the breadth-first per-tree layout the paper measures its
 * layouts against (Section III-A, BF; Section IV-B uses BF as the baseline),
 * evaluated the plain GPU way: one thread per (observation, tree), global
 * atomic votes, then a separate argmax kernel.
 * ------------------------------------------------------------------------ */
typedef struct fp_plain_forest fp_plain_forest;

#define FP_PLAIN_OBS_FASTEST 0  /* consecutive threads: same tree, next observation */
#define FP_PLAIN_TREE_FASTEST 1 /* consecutive threads: same observation, next tree */

/* Build the BF layout of desc and copy it to the current device on stream.
 * *out library-owned until fp_plain_release.  Errors: FP_EINVAL, FP_ENOMEM,
 * FP_ECUDA. */
int fp_plain_build(const fp_forest_desc *desc, void *stream, fp_plain_forest **out);

/* Classify with the plain layout.  out_votes (device [n][C] uint32) is
 * required: it is zeroed on the stream and accumulated with atomics;
 * out_class (device [n] int32) may be NULL.  order: FP_PLAIN_*. */
int fp_plain_predict(const fp_plain_forest *pf, const float *X, int64_t n, int32_t order, uint32_t *out_votes,
                     int32_t *out_class, void *stream);

/* The plain layout of a forest with leaf values (the value sits in the leaf's
 * record): out[i] = bias + scale * sum of the reached leaves' values, added
 * with global float atomics in no fixed order (error bound as
 * fp_predict_values).  out: device [n] float, zeroed on the stream here.
 * Errors: FP_EINVAL (also for a forest without leaf values), FP_ECUDA. */
int fp_plain_predict_values(const fp_plain_forest *pf, const float *X, int64_t n, int32_t order, float scale,
                            float bias, float *out, void *stream);

/* Bytes of the plain layout on the device. */
int64_t fp_plain_bytes(const fp_plain_forest *pf);

void fp_plain_release(fp_plain_forest *pf); /* NULL is a no-op */

#ifdef __cplusplus
}
#endif

#endif /* FOREST_PACK_H */
