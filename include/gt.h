/*
 * gt.h - exact range search by adaptive group testing on one GPU (sm_103a).
 *
 * Method: Shah, Mittal, Rajwade, "Group Testing for Accurate and Efficient
 * Range-Based Near Neighbor Search for Plagiarism Detection" (arXiv
 * 2311.02573).  A database of N non-negative, unit-norm vectors f_i in R^d is
 * pooled by summation into a binary tree; a query q with threshold rho tests
 * pools from the root down, pruning every pool y with q.y < rho (exact,
 * because every member scores q.f_i <= q.y when all entries are >= 0), and
 * splitting the survivors until single items are tested (Sec. 2, Algorithm
 * 1; the level-by-level view of the same tree is the "rounds" of Sec. 4).
 * The answer for each query is exactly {i : q.f_i >= rho} (Sec. 1).
 *
 * Tree layout: level h holds the pools of 2^h consecutive tree positions,
 * pool j covering positions [j 2^h, (j+1) 2^h) intersected with [0, N); level
 * 0 holds the items themselves.  Only pools that meet [0, N) are stored
 * (about 2N rows).  The paper's cumulative sums (Eq. 1) describe the same
 * pools; this library stores each pool explicitly.
 *
 * Conventions for every entry point:
 *  - Float inputs are FP32, row-major, rows of d contiguous entries.  Input
 *    pointers may be host or device memory (detected per call); the caller
 *    keeps ownership and the library never writes to them.
 *  - rho is used as the exact FP32 value passed (converted exactly to FP64
 *    where the FP64 recheck compares against it).  Valid thresholds are
 *    0 < rho <= 1 (cosine similarity, Sec. 2).
 *  - Entries must be >= 0 and finite (Sec. 2 assumes non-negative vectors);
 *    otherwise the call returns GT_EDOMAIN and leaves no partial result.
 *  - Work runs on the stream given in the options (NULL: the legacy default
 *    stream).  Calls return after their results are complete.
 *  - On any error the call returns a non-zero gt_status, writes no output,
 *    and gt_last_error() describes the failure (per calling thread).
 *  - Handles are not thread-safe: one call at a time per gt_tree.
 */
#ifndef GT_H
#define GT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gt_status {
  GT_OK = 0,
  GT_EINVAL = 1,    /* bad argument: null pointer, size or option out of range */
  GT_EDOMAIN = 2,   /* an input entry is negative, NaN or infinite */
  GT_ENOMEM = 3,    /* a device or host allocation failed */
  GT_ECUDA = 4,     /* a CUDA runtime or driver call failed */
  GT_ETIMEOUT = 5,  /* a bounded device-side wait ran out */
  GT_EOVERFLOW = 6, /* a single query's work exceeds the scratch budget */
  GT_EBUSY = 7      /* the handle is in use by another call */
} gt_status;

/* Row formats.  Item and pool rows are always kept in FP32 (the masters the
 * FP64 recheck and the inserts read); BF16 and FP8 copies are what the
 * traversal gathers when asked to. */
typedef enum gt_dtype {
  GT_F32 = 0,  /* 4 bytes per entry; the plain form */
  GT_BF16 = 1, /* round-to-nearest bfloat16, 2 bytes per entry */
  GT_FP8 = 2   /* float8 e4m3 with a power-of-two FP32 scale per row */
} gt_dtype;

typedef struct gt_tree gt_tree; /* opaque, library-owned device state */

/* How a pool vector is formed from its members.
 *   GT_POOL_SUM  the sum of the members (Eq. 1; q.y is the sum of the
 *                members' scores, so a pool below rho holds no neighbour and
 *                the left child can be bounded as parent minus right child).
 *   GT_POOL_MAX  the element-wise maximum of the members (Sec. 2, pooling
 *                by maximum; with non-negative entries q.y is at least the
 *                best member's score, so the same pruning holds).  Both
 *                children of every kept pool are tested: no subtraction.
 *   GT_POOL_MAXMIN  for descriptors with negative entries (Sec. 2 pools such
 *                data by element-wise maximum and minimum).  Each row f is
 *                stored split as [max(f, 0), max(-f, 0)] (2d non-negative
 *                entries) and the pools are element-wise maxima of the split
 *                rows, i.e. [max(M, 0), max(-m, 0)] for the members' maximum
 *                M and minimum m; a query q is split the same way.  A pool's
 *                split score q+.max(M, 0) + q-.max(-m, 0) bounds every
 *                member's q.f from above, so the same pruning holds; at an
 *                item the split score exceeds q.f by its cross terms, so
 *                every item it keeps is decided by an FP64 dot product of the
 *                signed q and f (no item is accepted on a bound).  Entries
 *                may be negative (non-finite ones are still GT_EDOMAIN);
 *                d <= 1024; the dense cutover level must be >= 1 and
 *                gt_exhaustive_tree is not available. */
typedef enum gt_pooling { GT_POOL_SUM = 0, GT_POOL_MAX = 1, GT_POOL_MAXMIN = 2 } gt_pooling;

/* How the pools are stored.
 *   GT_LAYOUT_TREE    one row per pool of every level (about 2N rows per
 *                     kept format).
 *   GT_LAYOUT_PREFIX  the cumulative sums of Eq. 1, restarted at every block
 *                     of 2^c consecutive items (c = prefix_level): row i is
 *                     the sum of the items from its block's first one up to
 *                     item i, so a pool inside a block scores as the
 *                     difference of two prefix scores and one split costs one
 *                     gathered row (N prefix rows in all).  The blocks' totals
 *                     (the pools of level c) are kept as BF16 rows and scored
 *                     for every query by the dense GEMM; the items are kept in
 *                     FP32 for the exact decision of doubtful leaves.  The
 *                     restart bounds the cancellation of the differences: a
 *                     prefix score never exceeds its block's score, where
 *                     global sums over 10^6 items would reach 10^4 and leave
 *                     FP32 bounds wider than rho.  Sum pooling only; row
 *                     formats BF16 (required) and FP32 (optional). */
typedef enum gt_layout { GT_LAYOUT_TREE = 0, GT_LAYOUT_PREFIX = 1 } gt_layout;

typedef struct gt_build_opts {
  void *stream;          /* cudaStream_t the build runs on (NULL: default) */
  const int64_t *perm;   /* optional, host: tree position p holds input row
                            perm[p] (a permutation of 0..N-1).  NULL keeps
                            the input order, which the paper takes to be
                            random already (Sec. 2). */
  int64_t capacity;      /* items the tree holds before an insert must grow
                            it (0: N) */
  uint32_t formats;      /* bitmask of (1 << gt_dtype) row formats to keep
                            besides FP32 (0: BF16 and FP8) */
  int32_t pooling;       /* gt_pooling: how a pool's vector is formed from
                            its members (0: GT_POOL_SUM) */
  int32_t layout;        /* gt_layout (0: GT_LAYOUT_TREE).  With
                            GT_LAYOUT_PREFIX, formats selects the prefix
                            rows kept: BF16 always, FP32 when (1 << GT_F32)
                            is set; FP8 is refused (GT_EINVAL) */
  int32_t prefix_level;  /* GT_LAYOUT_PREFIX: c, blocks of 2^c items,
                            1 <= c <= 12 (0: 3) */
} gt_build_opts;

/* Counters of one query call (all micro-batches together). */
typedef struct gt_query_stats {
  int64_t tests;          /* dot products computed: dense + gathered */
  int64_t dense_tests;    /* (query, pool) scores from the dense cutover GEMM */
  int64_t gathered_tests; /* (query, pool or item) tests that gathered a row */
  int64_t rechecks;       /* leaf tests settled by the FP64 recheck */
  int64_t results;        /* neighbours returned */
  int64_t micro_batches;
  int64_t retries;        /* micro-batches re-run smaller after a scratch overflow */
  int32_t cutover;        /* level the dense GEMM ran at (-1: none) */
  int32_t levels;         /* L + 1 */
  int64_t level_tests[64];/* gathered tests per tree level (index = h) */
  double gathered_bytes;  /* algorithmic bytes of gathered rows (d x entry size
                             per test, plus scales) */
  int64_t launches;       /* kernels the call launched */
  int64_t level_launches; /* of which frontier-level kernels (levels >= 1) */
  float kernel_ms[8];     /* with opts->timing: device time per kernel kind,
                             measured with CUDA events on the call's stream:
                             [0] frontier levels >= 1, [1] leaf level,
                             [2] dense GEMM, [3] FP64 recheck, [4] CSR
                             assembly, [5] query preparation, [6] grouping
                             of the GEMM's survivors by query */
  int64_t refines;        /* leaf re-scorings after a low-precision bound
                             straddled rho: from the BF16 row (FP8 leaves,
                             when the tree keeps BF16 rows), then from the
                             FP32 row */
  int64_t graph_captures; /* micro-batches captured into a new CUDA graph */
  int64_t graph_replays;  /* micro-batches run by replaying a captured graph */
} gt_query_stats;

typedef struct gt_query_opts {
  void *stream;          /* cudaStream_t (NULL: default) */
  int32_t dtype;         /* row format gathered by the traversal (gt_dtype) */
  int32_t cutover;       /* level h whose pools a dense tensor-core GEMM
                            scores for every query (levels above h are then
                            not visited: a pool pruned there would have been
                            pruned below too).  -1: choose automatically;
                            -2: none, start at the root (the plain form). */
  int64_t max_batch;     /* queries per micro-batch (0: automatic) */
  int64_t scratch_bytes; /* device scratch budget per call (0: 1/4 of free
                            device memory, at most 16 GiB) */
  int32_t results_on_device; /* 1: return the CSR in device memory */
  int32_t timing;        /* 1: fill stats->kernel_ms (CUDA events per launch) */
  gt_query_stats *stats; /* optional out */
  int32_t no_graph;      /* 1: launch every kernel directly instead of capturing
                            each micro-batch's launches in a CUDA graph (the
                            first call of a shape captures, later ones replay) */
  int32_t subtract;      /* below the dense cutover, gather only the right child
                            of each surviving pool and bound the left one as
                            parent minus right (Sec. 2, Algorithm 1).  1: on,
                            -1: off, 0: the tree's tuned choice (on unless
                            gt_autotune found it slower).  Items are always
                            tested. */
} gt_query_opts;

/* Neighbour lists: query q's ids are ids[offsets[q] .. offsets[q+1]),
 * ascending, as the original input row numbers (tree permutation undone).
 * Library-allocated; release with gt_csr_free. */
typedef struct gt_csr {
  int64_t n_queries;
  int64_t *offsets;  /* [n_queries + 1] */
  int32_t *ids;      /* [offsets[n_queries]] */
  int32_t on_device; /* 1 if offsets/ids are device pointers */
  int32_t reserved;
} gt_csr;

/* Build the pooled tree over F (N x d) - the offline index of Sec. 2: pools
 * made by summing members (Eq. 1 gives the same pools as differences of
 * cumulative sums).  Level 0 is the (optionally permuted) items; level h+1
 * row j is the FP32 sum of level-h rows 2j and 2j+1.  Requires 1 <= N <
 * 2^31 and 1 <= d <= 2048 (d <= 1024 for GT_POOL_MAXMIN).  Entries are
 * checked: GT_EDOMAIN if any is negative (allowed with GT_POOL_MAXMIN) or
 * not finite.  *out receives a new handle (free with gt_free).  The stored
 * rows (gt_read_rows, gt_dense_scores, gt_pair_bounds) of a GT_POOL_MAXMIN
 * tree are the split rows, 2d entries wide. */
gt_status gt_build(const float *F, int64_t N, int32_t d, const gt_build_opts *opts,
                   gt_tree **out);
/* A GT_LAYOUT_PREFIX tree (opts->layout) is queried by gt_query and
 * gt_query_into (dense GEMM at level c, then one prefix split per kept pool
 * down to the items; cutover must be -1 or c, dtype GT_BF16 or, when kept,
 * GT_F32 for the prefix rows; FP32 prefix rows need d <= 1152) and by the
 * server (gt_server_*), grown by gt_insert, tuned by gt_autotune and
 * gt_set_tuning (the GEMM tile only: its dense level is c and its splits
 * always use the ring-fed gather), read by gt_read_rows and scored by
 * gt_dense_scores at level c; gt_exhaustive_tree, gt_pair_bounds and
 * gt_query_static return GT_EINVAL for it. */

/* Streaming insertion (Sec. 4, "Streaming Setting"): append n_new rows f
 * (n_new x d) as items N .. N+n_new-1 (in the order given), then recompute
 * every ancestor pool that covers them, in place, with the same FP32
 * summation order as gt_build (a tree grown by inserts equals the tree built
 * over the whole database in one call, bit for bit).  The paper appends one
 * cumulative sum per item; the tree updates ceil(log2 N) ancestors.  Grows
 * the storage when N exceeds the capacity.  stream: cudaStream_t or NULL. */
gt_status gt_insert(gt_tree *t, const float *f, int64_t n_new, void *stream);

/* Range query by binary splitting (Sec. 2, Algorithm 1, traversed level by
 * level): for each of the B queries (B x d) return {i : q.f_i >= rho[q]}.
 * The traversal prunes a pool only when a rigorous upper bound on its exact
 * score (covering FP32 pool rounding, row quantisation and accumulation
 * error) is below rho; at the items, a BF16/FP8 score whose bound straddles
 * rho is re-scored in FP32 from the FP32 row, and one that still straddles
 * is settled in FP64.  The result is therefore exact in every
 * row format.  rho: B thresholds, 0 < rho <= 1. */
gt_status gt_query(gt_tree *t, const float *Q, int64_t B, const float *rho,
                   const gt_query_opts *opts, gt_csr *out);

/* gt_query with caller-owned outputs: the same sets written as CSR into
 * offsets (B + 1 int64) and ids (ids_cap int32), query q's ids at
 * ids[offsets[q] .. offsets[q+1]), ascending.  Q, rho, offsets and ids may
 * each be host or device memory; page-locked host buffers that the caller
 * reuses across calls avoid the per-call host allocation and the slow copy
 * into pageable memory of gt_query's host results.  *n_results receives the
 * number of neighbours; if it exceeds ids_cap the call returns GT_EOVERFLOW
 * and writes neither offsets nor ids (call again with a larger buffer).
 * opts as for gt_query (results_on_device is ignored). */
gt_status gt_query_into(gt_tree *t, const float *Q, int64_t B, const float *rho,
                        const gt_query_opts *opts, int64_t *offsets, int32_t *ids, int64_t ids_cap,
                        int64_t *n_results);

/* Exhaustive search over a database the caller holds (the paper's Exh
 * comparator, Sec. 4 and Table 1: every query is compared with every item).
 * For each of the B queries (B x d) it returns {i : q.f_i >= rho[q]} over the
 * N rows of F (N x d, FP32, entries >= 0), as CSR lists of row numbers of F,
 * ascending - the same exact sets gt_query returns for a tree built over F.
 *  - Method: the rows of F are rounded once into a BF16 copy (and padded into
 *    an FP32 copy for the recheck); a tensor-core GEMM scores every (query,
 *    item) pair in FP32; a pair whose rigorous upper bound is below rho is
 *    dropped, one whose lower bound reaches rho is kept, and the few in
 *    between are settled in FP64 from the FP32 rows.  No tree is built.
 *  - F, Q and rho may each be host or device memory; the caller keeps them.
 *  - The library keeps, per device, the storage of the two row copies and of
 *    the search's lists between calls (about 6 d N bytes plus the result
 *    lists), reused by the next call; calls from several threads are
 *    serialised.
 *  - opts as for gt_query; dtype and cutover are ignored (the GEMM reads BF16
 *    rows, the scan has no levels).
 *  - Errors: GT_EINVAL for N outside [1, 2^31), d outside [1, 2048], a null
 *    pointer or no tensor-core path; GT_EDOMAIN for a negative or non-finite
 *    entry of F or Q; GT_ENOMEM when the row copies do not fit. */
gt_status gt_exhaustive(const float *F, int64_t N, int32_t d, const float *Q, int64_t B,
                        const float *rho, const gt_query_opts *opts, gt_csr *out);

/* gt_exhaustive over the items of a built tree (its level-0 rows; the ids
 * are the tree's, as for gt_query).  Not available for a prefix-layout
 * tree, which keeps no BF16 item rows. */
gt_status gt_exhaustive_tree(gt_tree *t, const float *Q, int64_t B, const float *rho,
                             const gt_query_opts *opts, gt_csr *out);

/* Result of gt_autotune: the choices and the device milliseconds of a query
 * batch measured for each candidate (0 where not tried). */
typedef struct gt_autotune_result {
  int32_t cutover;        /* chosen dense cutover level */
  int32_t inflight;       /* chosen tests in flight per warp, plus 8 when the
                             query is read through L1 rather than held in
                             registers, or 16: rows fed to the tests through
                             a ring of shared-memory slots by bulk
                             asynchronous copies, or 32: the same gather in
                             one persistent launch whose warps drain the
                             dense GEMM's list as a shared work queue, each
                             carrying the entries it claims down to the
                             items (subtraction path, cutover 2..5; 0: the
                             format's default) */
  int32_t tile_n;         /* chosen GEMM tile: 128 (128 queries x 128 pools
                             on one SM), 256 (128 x 256), 512 (256 x 256 on
                             one SM) or 1024 (256 x 256 on a pair of SMs,
                             tcgen05 cta_group::2) */
  float best_ms;
  float ms_cutover[9];    /* stage 1: cutover c = 1..8 on the direct path,
                             default in-flight, tile 256 */
  float ms_cutover_sub[9];/* stage 1: the same on the subtraction path (c >= 2) */
  float ms_inflight[8];   /* stage 2: codes 1, 2, 4, 9, 10, 12, 16, 32 at the best cutover */
  float ms_tile[4];       /* stage 3: tiles 128, 256, 512, 1024 at the best of both */
  int32_t subtract;       /* 1 if the subtraction path was chosen (stage 1) */
} gt_autotune_result;

/* Tune the free choices of the query path for this tree and row format on a
 * sample batch (Q, rho as for gt_query), by coordinate descent: the level
 * whose pools the dense GEMM scores (the paper's early rounds prune little,
 * Sec. 4; the best level depends on N, d and the data) together with whether
 * the subtraction path (one gathered child per pool) pays, then how many
 * tests each warp keeps in flight, then the GEMM's tile shape.  Each candidate
 * runs three times, each run after the L2 cache is overwritten (a 256 MiB
 * device scratch, allocated for the call), and the best of the last two
 * counts.  The choices are
 * stored in the tree and used by gt_query with cutover = -1 (the tile width
 * and in-flight count by every later call). */
gt_status gt_autotune(gt_tree *t, const float *Q, int64_t B, const float *rho, int32_t dtype,
                      void *stream, gt_autotune_result *out);

/* Set by hand the choices gt_autotune stores for row format dtype: the
 * cutover level (used by gt_query with cutover = -1), the tests in flight
 * code and the GEMM tile (codes as in gt_autotune_result).  0 resets a choice
 * to its default; a negative value leaves it unchanged. */
gt_status gt_set_tuning(gt_tree *t, int32_t dtype, int32_t cutover, int32_t inflight,
                        int32_t tile);

/* Copy `count` rows of tree level `level` in format `dtype` to host memory
 * `out` (row r at out + r * d entries; GT_FP8 rows are d bytes, and
 * `scales_out`, if non-null, receives the per-row FP32 scales).  For checking
 * the tree's invariants.  A GT_LAYOUT_PREFIX tree keeps level 0 (the items)
 * in GT_F32 and level c (the blocks' totals) in GT_BF16; level -1 selects its
 * prefix rows (row i = the sum of items (i >> c) << c .. i, accumulated in
 * FP64 in item order and rounded to FP32, then to BF16 for the BF16 rows). */
gt_status gt_read_rows(const gt_tree *t, int32_t level, int32_t dtype, int64_t first,
                       int64_t count, void *out, float *scales_out);

/* Diagnostic: the raw dense scores q^t y of every query (B x d) against every
 * pool y of tree level `level` (Sec. 2: a pool's score is the query's dot
 * product with the pool sum), as the tensor-core GEMM of gt_query's cutover
 * computes them: BF16 inputs, FP32 accumulation, no threshold applied.
 * scores (host or device): B x rows(level) floats, row q for query q.
 * stream: cudaStream_t or NULL. */
gt_status gt_dense_scores(gt_tree *t, const float *Q, int64_t B, int32_t level, float *scores,
                          void *stream);

/* Diagnostic: the traversal's test of given (query, pool) pairs (Sec. 2: a
 * pool is pruned when its score is below rho, which is exact because no
 * member scores higher).  For pair i = (pairs[2i], pairs[2i+1]) = (query q,
 * row j of tree level `level`), computed by the same device code as the level
 * kernels of gt_query in row format `dtype` (lane-parallel FP32 accumulation,
 * FP8 scale applied):
 *   out[3i]     the low-precision score of query q against row j;
 *   out[3i + 1] U, the upper bound on q.y_j (y_j the exact pool: the sum, or
 *               for a max-pool tree the element-wise maximum, of its members'
 *               FP32 rows) that the traversal compares with rho to prune;
 *   out[3i + 2] L, the lower bound on q.y_j (the items' acceptance test; at a
 *               pool level, the right child's bound the subtraction path
 *               takes from the parent's).
 * Q: B x d FP32 (entries >= 0); pairs: n x 2 int32; out: n x 3 FP32; each a
 * host or a device pointer.  A pair naming a query >= B or a row outside the
 * level gets NaNs.  GT_EINVAL on a bad level, format or size; GT_EDOMAIN on
 * a negative or non-finite query entry.  stream: cudaStream_t or NULL. */
gt_status gt_pair_bounds(gt_tree *t, int32_t level, int32_t dtype, const float *Q, int64_t B,
                         const int32_t *pairs, int64_t n, float *out, void *stream);

/* Allocation-free range query (the paper has no counterpart: this is a
 * deployment variant of gt_query).  For callers that must not allocate
 * device memory while serving - cudaMalloc can synchronise the whole device
 * and stall other streams, and some processes hand all device memory to
 * another allocator up front.  It runs gt_query's traversal from the root
 * (no dense cutover) in row format `dtype`, with every scratch buffer inside
 * one fixed 32 MiB array of device memory that the library holds on each GPU
 * it is loaded on until the process exits.
 *  - Q (B x d FP32), rho (B), offsets (B + 1 int64) and ids (ids_cap int32)
 *    must be device pointers; 1 <= B <= 256.  Results are written as CSR:
 *    query q's ids at ids[offsets[q] .. offsets[q+1]), ascending.
 *  - *n_results receives the number of neighbours; if it exceeds ids_cap
 *    the call returns GT_EOVERFLOW without writing ids (call again with a
 *    larger buffer).
 *  - Fixed limits of the array: 256 queries per call; rows of at most 2048
 *    entries; 262,144 neighbours per call in all; per micro-batch 65,536 leaf
 *    pairs awaiting the FP64 recheck and about 1.8M (query, pool) pairs in
 *    each of two frontier lists.  A micro-batch whose frontier or recheck
 *    list overflows is re-run with half the queries.  GT_EOVERFLOW is
 *    returned (*n_results then 0) when the call's neighbours exceed 262,144
 *    (split the queries over more calls) or when one query's frontier alone
 *    does not fit.
 *  - The tree's device (the one current at gt_build) must be current
 *    (GT_EINVAL otherwise).  The first call on a device looks up the array's
 *    device address and keeps it; make that first call before any stream
 *    capture, and make no call on a device after cudaDeviceReset of it.
 *  - All calls share the array and see the previous call's leftovers (each
 *    call clears what it needs): calls that overlap on the GPU - other
 *    streams, other threads - race and must not be made.
 *  - stream: cudaStream_t or NULL (the tree's stream). */
gt_status gt_query_static(gt_tree *t, const float *Q, int64_t B, const float *rho, int32_t dtype,
                          int64_t *offsets, int32_t *ids, int64_t ids_cap, int64_t *n_results,
                          void *stream);

/* ---- Serving: continuous batching over one tree ------------------------
 * A request loop for range queries (Sec. 2) arriving over time, with
 * streaming inserts (Sec. 4) interleaved.  Every gt_server_step applies
 * queued inserts, admits a new group from the arrival queue (bounded by free
 * query slots and the frontier memory budget) whose dense cutover GEMM runs
 * in that step, moves the groups in flight below the cutover as the schedule
 * says (gt_server_schedule), and completes the groups that reach a decision.
 * A request that arrives while others are on the device joins at the next
 * step.  Each group answers for the tree as it was when the group was
 * admitted: {i < N_admit : q.f_i >= rho}, the same set it gets alone. */
typedef struct gt_server gt_server;

typedef struct gt_server_opts {
  void *stream;          /* cudaStream_t (NULL: the tree's stream) */
  int32_t dtype;         /* row format gathered below the cutover (gt_dtype) */
  int32_t cutover;       /* dense GEMM level (<= 0: the tree's tuned level, else 3) */
  int64_t max_group;     /* queries admitted per step at most (0: 4096) */
  int64_t scratch_bytes; /* device memory for the level lists (0: 4 GiB) */
  int64_t queue_capacity;/* queued queries held before the pinned queue grows
                            (0: max(4 x max_group, 16384)) */
  int32_t schedule;      /* how a group moves below the cutover, one of
                            gt_server_schedule (0: GT_SCHEDULE_AUTO) */
  int32_t reserved;
} gt_server_opts;

/* Schedules of the server.
 *   GT_SCHEDULE_LEVELS     one level per step: every step launches, for each
 *                          group in flight, the kernel of the level it is at,
 *                          so a group finishes c + 1 steps after admission and
 *                          up to c + 1 groups share each step.
 *   GT_SCHEDULE_DRAIN      each step drains the group admitted the step before
 *                          in one persistent launch (every level below the
 *                          cutover and its items, the warps working through
 *                          the GEMM's list as a shared queue) while it admits
 *                          the next group: two groups share each step and a
 *                          group finishes one step after admission.
 *   GT_SCHEDULE_IMMEDIATE  each step admits a group and answers it in the
 *                          same step (its GEMM, the same persistent launch,
 *                          the recheck and its neighbour lists): a request is
 *                          answered at the end of the first step that starts
 *                          after it arrives, and no group stays in flight
 *                          between steps.  A group whose lists overflow is
 *                          answered again, smaller, by a later step.  A group
 *                          of at most 64 queries has its GEMM one or two
 *                          levels above the server's cutover (at most level
 *                          5), where the GEMM reads fewer pool rows.
 *   GT_SCHEDULE_AUTO       GT_SCHEDULE_IMMEDIATE where it applies, else
 *                          GT_SCHEDULE_LEVELS.
 * DRAIN and IMMEDIATE need the subtraction path (sum pools, cutover 2 to 5,
 * tree layout); GT_EINVAL otherwise. */
typedef enum gt_server_schedule {
  GT_SCHEDULE_AUTO = 0,
  GT_SCHEDULE_LEVELS = 1,
  GT_SCHEDULE_DRAIN = 2,
  GT_SCHEDULE_IMMEDIATE = 3
} gt_server_schedule;

typedef struct gt_server_stats {
  int64_t submitted, admitted, completed, pending, inserted;
  int64_t steps, launches, retries, rechecks, refines;
  int64_t gathered_tests, dense_tests;
  int64_t cutover, max_group;
  int64_t schedule;      /* the gt_server_schedule in use (LEVELS, DRAIN or IMMEDIATE) */
  double busy_seconds;   /* host wall time spent inside gt_server_step */
} gt_server_stats;

/* Create a server over tree t (which must keep BF16 rows; a GT_LAYOUT_PREFIX
 * tree is served at its prefix_level; a GT_POOL_MAXMIN tree takes queries and
 * inserts of d entries, like gt_query, and is served one level per step).
 * The server owns its device buffers; the tree must outlive it and is
 * updated in place by queued inserts. */
gt_status gt_server_create(gt_tree *t, const gt_server_opts *opts, gt_server **out);
/* Queue n queries (host Q n x d, rho n, caller tags n); copied on return. */
gt_status gt_server_submit(gt_server *s, const float *Q, const float *rho, const int64_t *tags,
                           int64_t n);
/* Queue n rows (host, n x d) for insertion at the start of the next step.
 * The rows are checked here (GT_EDOMAIN for a negative or non-finite entry,
 * or a non-finite one for a GT_POOL_MAXMIN tree; nothing of the call is
 * queued then), so that the step applies them without waiting on the device. */
gt_status gt_server_insert(gt_server *s, const float *f, int64_t n);
/* One engine iteration (synchronous).  *in_flight: queries on the device. */
gt_status gt_server_step(gt_server *s, int64_t *in_flight);
/* Pop up to max_queries completed queries: tags[k], their ids at
 * ids[offsets[k] .. offsets[k+1]) ascending (offsets has max_queries + 1
 * entries, ids ids_cap), and, if n_snapshot is non-null, the tree size the
 * query was answered against.  *n_done receives the number popped. */
gt_status gt_server_poll(gt_server *s, int64_t max_queries, int64_t *n_done, int64_t *tags,
                         int64_t *offsets, int32_t *ids, int64_t ids_cap, int64_t *n_snapshot);
gt_status gt_server_get_stats(const gt_server *s, gt_server_stats *out);
void gt_server_free(gt_server *s);

/* Run the kernels of later calls on tree t (queries, the server's steps,
 * inserts) on grids sized for at most n SMs (n <= 0: all of the device's), so
 * that calls on several trees and streams can share the GPU side by side:
 * the persistent kernels (one block per SM) then leave the other SMs to the
 * other calls' kernels.  n >= 2.  The paper has no counterpart. */
gt_status gt_set_sm_limit(gt_tree *t, int32_t n);

/* Failure detection (the bounded device waits): every wait of the gather
 * kernels on their bulk copies gives up after 1 s, raises a status word that
 * the call reads, and the call returns GT_ETIMEOUT with no results instead of
 * leaving a kernel waiting.  To test that path without a fault, on != 0 makes
 * the ring-fed gather kernels of later calls on tree t start no copy, so
 * their first wait runs out at once with nothing in flight; 0 restores normal
 * operation.  The tree's rows are not touched.  The paper has no counterpart
 * (its implementation runs on a CPU). */
gt_status gt_set_wait_expiry(gt_tree *t, int32_t on);

/* What a tree is: its sizes, row formats and how its pools are formed. */
typedef struct gt_tree_info {
  int64_t n_items;       /* N */
  int64_t capacity;      /* items held before an insert must grow the storage */
  int32_t d;             /* entries per input row */
  int32_t row_width;     /* entries per stored row (2d for GT_POOL_MAXMIN) */
  int32_t levels;        /* L + 1 */
  int32_t pooling;       /* gt_pooling */
  int32_t layout;        /* gt_layout */
  int32_t prefix_level;  /* GT_LAYOUT_PREFIX: c (else 0) */
  uint32_t formats;      /* bitmask of (1 << gt_dtype) row formats kept */
  int32_t device;        /* CUDA device of the tree's memory */
} gt_tree_info;
gt_status gt_info(const gt_tree *t, gt_tree_info *out);

/* Checkpoint (the paper builds its index offline, Sec. 2; a built or grown
 * tree can be kept and reopened): gt_save writes to the file at `path` what
 * gt_load needs to rebuild the same tree - the stored item rows (FP32, in
 * tree order), the tree permutation, the build options (pooling, layout,
 * prefix level, formats, capacity) and the tuning choices.  gt_load rebuilds
 * it on the current device: rows, pools of every level and the ids returned
 * are bit for bit those of the saved tree (the build is deterministic).
 * Errors: GT_EINVAL for a bad argument, a file that cannot be opened, read or
 * written (gt_last_error gives the reason) or that is not a tree checkpoint;
 * GT_ENOMEM / GT_ECUDA as for gt_build.  stream: cudaStream_t or NULL. */
gt_status gt_save(const gt_tree *t, const char *path);
gt_status gt_load(const char *path, void *stream, gt_tree **out);

int64_t gt_size(const gt_tree *t);        /* current N */
int32_t gt_dim(const gt_tree *t);         /* d */
int32_t gt_levels(const gt_tree *t);      /* L + 1 = ceil(log2 N) + 1 */
void gt_free(gt_tree *t);                 /* release the tree (NULL is ignored) */
void gt_csr_free(gt_csr *c);              /* release a result (zeroes *c) */
const char *gt_last_error(void);          /* message of this thread's last error */

#ifdef __cplusplus
}
#endif

#endif /* GT_H */
