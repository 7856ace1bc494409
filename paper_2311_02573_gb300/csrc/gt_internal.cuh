// Internal declarations of the GPU library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <tuple>
#include <vector>

#include "../../include/gt.h"

namespace gt {

// A named NVTX range for the lifetime of the object (host-side tracing of the
// entry points and of each micro-batch; free when no tool is attached).
struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};

constexpr int kMaxLevels = 40;
// counter slots after the levels: [40] results, [41] rechecks, [42] refines,
// [43] segments left for the block sort of the CSR assembly
constexpr int kCsrListSlot = kMaxLevels + 3;
// CSR assembly (launch_csr_into) of at most this many queries runs in one
// block, which writes only the offsets and ids it is given (host-mapped
// buffers included)
constexpr int kCsrSmallMax = 64;
constexpr int kWarp = 32;

// Device-side status words (one array per tree, cleared per call).
enum Flag : int {
  kFlagDomain = 0,     // a negative / non-finite input entry
  kFlagOverflow = 1,   // a frontier or result list ran past its capacity
  kFlagTimeout = 2,    // a bounded wait gave up
  kFlagRho = 3,        // a threshold outside (0, 1]
  kFlagStray = 4,      // a result names a query outside the range being assembled
  kFlagCount = 8
};

// (query, pool) pair of the frontier: q is the query's index in the call's
// batch (a micro-batch holds queries [q0, q0 + b)), j the pool within its level.
struct __align__(8) Pair {
  uint32_t q, j;
};

// (query, parent pool, upper and lower bounds on the parent's exact score):
// the subtraction path tests one child of the parent and bounds the other as
// parent minus the tested child (Sec. 2: the left half's score is sim - rsim).
// The fourth word holds the lower bound as FP32 bits (0, which accepts
// nothing, where none is known); the prefix layout's entries hold the prefix
// score at the pool's end there instead.
struct __align__(16) SibPair {
  uint32_t q, p;
  float U;
  uint32_t pad;
};

// Error bounds (all quantities non-negative).  For a stored row yhat of a
// level-h pool y (exact sum of FP32 items) and a query q used exactly in FP32:
//   |ytilde_j - y_j| <= e_h y_j            (FP32 pool sums, e_h = (1+2^-24)^h - 1)
//   |yhat_j - ytilde_j| <= u ytilde_j + t   (row format: u, t per format / row)
//   |shat - sum q_j yhat_j| <= g sum q_j yhat_j   (FP32 accumulation, g = gamma_d)
// hence the exact pool score s obeys
//   s <= (shat / (1 - g) + t |q|_1) / ((1 - u)(1 - e_h))      (prune iff < rho)
//   s >= (shat / (1 + g) - t |q|_1) / ((1 + u)(1 + e_h))       (accept iff >= rho;
//                                      also the lower bound of a pool score)
// The kernels evaluate these in FP32 with constants inflated (or deflated) by
// 2^-20 relative, which covers the FP32 rounding of the few bound operations.
struct Bound {
  float cu;   // upper:  U = shat * cu + t * qn1 * ct_up
  float ct_up;
  float cl;   // lower:  Lo = (shat * cl - t * qn1 * ct_lo) * (1 - 2^-22)  (1 + e_h folded in)
  float ct_lo;
};

Bound make_bound(int fmt, int h, int d);

// Per-format constants.
__host__ __device__ constexpr int entry_bytes(int fmt) {
  return fmt == GT_F32 ? 4 : (fmt == GT_BF16 ? 2 : 1);
}

struct Workspace {
  // frontier ping-pong buffers
  Pair *front[2] = {nullptr, nullptr};
  int64_t front_cap = 0;  // pairs per buffer (allocated)
  int64_t front_lim = 0;  // pairs per buffer this call may use (<= front_cap)
  Pair *res = nullptr;    // accepted (q, position) pairs of the call
  int64_t res_cap = 0;
  Pair *rchk = nullptr;   // leaf pairs for the FP64 recheck
  int64_t rchk_cap = 0;
  Pair *defer = nullptr;  // FP8 leaf pairs whose bound straddles rho, re-scored
  int64_t defer_cap = 0;  // from BF16 rows by a ring-fed pass after the FP8 one
  uint32_t *counters = nullptr;  // device: [0..kMaxLevels) frontier counts,
                                 // [kMaxLevels] results, [+1] rechecks
  float *qf32 = nullptr;         // queries, padded FP32 rows
  __nv_bfloat16 *qbf16 = nullptr;  // queries, padded BF16 rows (GEMM operand)
  float *qn1 = nullptr;          // per-query upper bound on |q|_1
  float *rho = nullptr;          // per-query thresholds
  int64_t q_cap = 0;
  int64_t *bcnt = nullptr;       // per-query counts / cursors of the bucketing pass
  int64_t *boff = nullptr;       // per-query offsets of the bucketing pass
  float *stage = nullptr;        // host->device staging of inputs
  int64_t stage_bytes = 0;
  uint32_t *hcounters = nullptr; // pinned host mirror of counters + flags
  void *drain = nullptr;         // k_drain: the warps' private lists
  int64_t drain_cap = 0;         // (entries of 16 bytes)
};

// A captured CUDA graph of one micro-batch of the query path, keyed by
// everything its launches depend on (shape, choices, buffer addresses).
struct GraphKey {
  int cut, fmt, timing, tuned_g, tuned_bn, pad;
  int64_t q0, b, N, front_lim, res_cap, rchk_cap;
  const void *p[24];
};

struct GraphEntry {
  GraphKey key;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> events;  // timing events the graph records
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> marks;
  int64_t launches = 0, level_launches = 0;
};

inline void destroy_graph(GraphEntry &e) {
  if (e.exec) cudaGraphExecDestroy(e.exec);
  for (cudaEvent_t ev : e.events) cudaEventDestroy(ev);
  e.exec = nullptr;
  e.events.clear();
}

struct GraphCache {
  std::vector<GraphEntry> v;
  // entries evicted during a call: their timing events may still be read by
  // that call's timer, so they are destroyed when the call ends
  std::vector<GraphEntry> retired;
  void release_retired() {
    for (auto &e : retired) destroy_graph(e);
    retired.clear();
  }
  ~GraphCache() {
    for (auto &e : v) destroy_graph(e);
    release_retired();
  }
};

}  // namespace gt

struct gt_tree {
  int64_t N = 0;     // items
  int64_t cap = 0;   // items storable without reallocation
  int32_t d = 0;     // entries per stored row (2 d_in for split signed rows)
  int32_t d_in = 0;  // entries per row of the caller's inputs
  bool split_sign = false;  // GT_POOL_MAXMIN: rows and queries stored as
                            // [max(x, 0), max(-x, 0)], max pools over them,
                            // items decided by a signed FP64 dot product
  int32_t L = 0;     // top level: ceil(log2 N)
  int32_t Lcap = 0;  // top level storable: ceil(log2 cap)
  int64_t stride = 0;            // entries per stored row (d rounded up to 64)
  int64_t lvl_off[gt::kMaxLevels + 1] = {0};  // first row of level h
  int64_t total_rows = 0;
  uint32_t formats = 0;          // bitmask of (1 << gt_dtype)
  float *rows32 = nullptr;
  __nv_bfloat16 *rows16 = nullptr;
  uint8_t *rows8 = nullptr;
  float *scale8 = nullptr;       // FP8 row scales (powers of two)
  int32_t *perm = nullptr;       // device: tree position -> input row id
  int *flags = nullptr;          // device status words
  float max_norm_dev = 0.f;      // max | ||f||_2 - 1 | seen at build / insert
  cudaStream_t stream = nullptr;
  int sm_count = 0;              // SMs the tree's kernels size their grids for
  int sm_total = 0;              // SMs of the device (gt_set_sm_limit restores it)
  int device = 0;                // CUDA device the tree's memory lives on
  int tuned_cut[3] = {0, 0, 0};  // cutover level chosen by gt_autotune, per row format
  int tuned_g[3] = {0, 0, 0};    // tests in flight per warp chosen by gt_autotune
  int tuned_bn = 0;              // dense GEMM pool-tile width (0: 256)
  int pooling = GT_POOL_SUM;     // gt_pooling of the rows above level 0
  int layout = GT_LAYOUT_TREE;   // gt_layout.  GT_LAYOUT_PREFIX: rows32 holds the
                                 // items, rows16 the level-pc pools, pref16 /
                                 // pref32 the block prefix rows; lvl_off is 0
  int pc = 0;                    // prefix layout: blocks of 2^pc items
  __nv_bfloat16 *pref16 = nullptr;
  float *pref32 = nullptr;
  int tuned_sub[3] = {0, 0, 0};  // gt_autotune's choice: 1 subtraction path, -1 direct, 0 untuned
  int ring_batch = 32;           // k_ring's pairs per warp batch for the current launches
  int expire_waits = 0;          // gt_set_wait_expiry: ring kernels' first wait gives up
  bool graphs_ok = true;         // false after a failed capture: launch directly
  gt::GraphCache *graphs = nullptr;  // captured micro-batches (a pointer: views copy it)
  cudaStream_t aux_stream = nullptr; // capturable stream for legacy-stream callers
  cudaEvent_t aux_in = nullptr, aux_out = nullptr;
  gt::Workspace ws;
};

namespace gt {

// rows per level and layout for `cap` items
int top_level(int64_t n);  // ceil(log2 n), 0 for n <= 1
inline int64_t level_rows(int64_t n, int h) { return (n + ((int64_t)1 << h) - 1) >> h; }

// error plumbing (gt_api.cu)
gt_status set_error(gt_status st, const std::string &msg);
gt_status cuda_error(cudaError_t e, const char *what);
#define GT_CUDA(call)                                          \
  do {                                                         \
    cudaError_t _e = (call);                                   \
    if (_e != cudaSuccess) return gt::cuda_error(_e, #call);   \
  } while (0)

bool is_device_ptr(const void *p);

// tree kernels (gt_tree.cu)
gt_status tree_alloc(gt_tree *t, int64_t cap);
gt_status tree_build_level0(gt_tree *t, const float *F_dev, int64_t first, int64_t n,
                            const int32_t *perm_dev_or_null, cudaStream_t s,
                            bool stored_rows = false);
gt_status tree_build_levels(gt_tree *t, int64_t first_item, int64_t n_items, cudaStream_t s);
float tree_norm_dev(gt_tree *t);
// prefix layout (gt_tree.cu): storage for `cap` items, and the prefix rows and
// block totals of the blocks covering items [first, first + n)
gt_status prefix_alloc(gt_tree *t, int64_t cap);
gt_status prefix_build(gt_tree *t, int64_t first, int64_t n, cudaStream_t s);
// gt_insert's work without its checks and waits (gt_api.cu): for rows the
// caller has validated on the host; enqueued on s
gt_status insert_checked_async(gt_tree *t, const float *F_dev, int64_t n_new, cudaStream_t s);

// query-side kernels (gt_traverse.cu)
gt_status ws_reserve_queries(gt_tree *t, int64_t B);
gt_status ws_stage(gt_tree *t, int64_t bytes);
gt_status ws_reserve_frontier(gt_tree *t, int64_t pairs, int64_t results, int64_t rechecks);
void launch_prep_queries(gt_tree *t, const float *Q_dev, const float *rho_dev, int64_t B,
                         cudaStream_t s);
void launch_root(gt_tree *t, int64_t q0, int64_t b, Pair *out, uint32_t *count, cudaStream_t s);
// Subtraction at the items: entries (q, c, U) of level-1 pools c in; the
// right item 2c+1 is decided (results, rechecks), the left item 2c is written
// to `left` as a leaf pair when its bound U - L_right reaches rho.
void launch_items_sub(gt_tree *t, int fmt, const SibPair *in, const uint32_t *in_count,
                      uint32_t *left_count, cudaStream_t s);
bool items_sub_available(gt_tree *t, int fmt);
// Counter slot of the leaf pairs that the subtraction at the items passes on
// (a slot above every level a tree can have: N < 2^31 gives at most 32).
constexpr int kLeftItemsSlot = kMaxLevels - 1;
// Counter slot of the deferred FP8 leaf pairs (Workspace::defer).
constexpr int kDeferSlot = kMaxLevels - 2;
// Whether the FP8 leaf kernels of tree t defer their straddling pairs to a
// ring-fed BF16 pass (one more launch after each FP8 leaf launch).
bool defer_active(const gt_tree *t, int fmt);
// Level whose accumulated FP32 rounding the bounds of a level-h pool carry:
// h for sum pools, 0 for max pools (an element-wise maximum is exact).
// Rounding depth e_h of a level's stored pools: h FP32 additions for a tree
// pool, none for max pools; a prefix-layout row (and block total) is an FP64
// sum rounded once to FP32, covered by depth 2.
inline int bound_level(const gt_tree *t, int h) {
  if (t->layout == GT_LAYOUT_PREFIX) return 2;
  return t->pooling == GT_POOL_MAX ? 0 : h;
}
// Pairs a k_ring warp takes at a time for a group of b queries: 32, or 16
// and 8 for small groups, whose short lists then spread over more warps (at
// least the ring's depth, 8, so a refill reaches one batch ahead at most).
inline int ring_batch_for(int64_t b) { return b >= 1024 ? 32 : (b >= 256 ? 16 : 8); }
// Tests-in-flight code bit selecting the ring-fed gather kernel (k_ring).
constexpr int kInflightRing = 16;
// Tests-in-flight code selecting, on the subtraction path, one persistent
// launch (k_drain) for every level below the cutover instead of one launch
// per level (the ring-fed gather otherwise).
constexpr int kInflightDrain = 32;
// Counter slot of k_drain's work-queue head.
constexpr int kDrainHeadSlot = kMaxLevels + 4;
// Whether k_drain serves tree t in format fmt below cutover level cut (the
// subtraction path of a sum-pooled tree, 2 <= cut <= 5, rows that fit the ring).
bool drain_available(const gt_tree *t, int fmt, int cut);
// Device memory for k_drain's per-warp lists (outside any stream capture).
gt_status ws_reserve_drain(gt_tree *t);
// All levels below cutover `cut` and the items in one launch: `root` holds the
// GEMM's level-(cut-1) entries (grouped by query), `root_count` their count.
// The entries tested at each level h < cut - 1 are added to level_count[h]
// and the left items tested to *left_count (null: the workspace's level
// counters and its left-item slot).  `cleared`: the caller has zeroed the
// queue head (kDrainHeadSlot) and the deferred-pair count (kDeferSlot) of the
// workspace's counters already, in stream order before this launch.
void launch_drain(gt_tree *t, int fmt, int cut, const SibPair *root, const uint32_t *root_count,
                  cudaStream_t s, uint32_t *level_count = nullptr, uint32_t *left_count = nullptr,
                  bool cleared = false);
// Kernel attributes of the level kernels, set once before any stream capture.
void prepare_level_kernels();
void launch_level(gt_tree *t, int fmt, int h, int64_t q0, const Pair *in, const uint32_t *in_count,
                  Pair *out, uint32_t *out_count, cudaStream_t s);
// subtraction path at level h >= 1: `in` holds SibPairs (children at level h of
// parents at level h+1); out holds SibPairs for level h-1, or plain item pairs
// when h == 1
void launch_level_sub(gt_tree *t, int fmt, int h, const SibPair *in, const uint32_t *in_count,
                      void *out, uint32_t *out_count, cudaStream_t s, bool entries_out = false);
// Scale factors of the dense GEMM's bound at level h (gt_gemm.cu):
// acc * cl <= exact score <= acc * cu.
void gemm_bound(int h, double *cu, double *cl);
// prefix layout: split the level-h pools of `in` (SibPairs {q, pool, prefix
// score at the pool's start, at its end}) at their midpoints, one gathered
// prefix row each; the kept children go to `out` as SibPairs (h >= 2), or the
// items are decided into the result and recheck lists (h == 1).  false when
// the ring-fed gather's slots do not fit rows of this format and width.
bool launch_prefix(gt_tree *t, int fmt, int h, const SibPair *in, const uint32_t *in_count,
                   SibPair *out, uint32_t *out_count, cudaStream_t s);
void launch_recheck(gt_tree *t, int64_t q0, cudaStream_t s);
// The level kernels' test of n given (query, pool) pairs at level h: score,
// upper and lower bound per pair into out (gt_pair_bounds).
void launch_pair_bounds(gt_tree *t, int fmt, int h, const int32_t *pairs, int64_t n, int64_t n_queries,
                        float *out, cudaStream_t s);
// CSR assembly (see gt_traverse.cu) of the results of queries [q_lo, q_lo +
// B): cnt (zero on entry) and off are indexed by query, so off[q_lo ..
// q_lo + B] receives the offsets; n_dev, when given, is the device-side
// result count (clamped to n).  With `recheck` the FP64 recheck of the
// tree view's recheck list runs first (for at most kCsrSmallMax queries in
// the same launch as the CSR), appending to `res` with the count at n_dev.
void launch_csr_into(gt_tree *t, const Pair *res, uint32_t n, const uint32_t *n_dev, int64_t q_lo,
                     int64_t B, int64_t *cnt, int64_t *off, int32_t *ids, uint32_t *list_n,
                     cudaStream_t s, bool recheck = false);

// dense tensor-core GEMM with a threshold epilogue (gt_gemm.cu)
// mode 0: cutover - survivors' children at level h-1 go to `out`/`out_count`
// mode 1: items (exhaustive) - accepted pairs to results, straddling to rechecks
// mode 3: cutover for the subtraction path - one SibPair per surviving pool
// Group a frontier list by query (a counting sort; order within a query is
// arbitrary): `in` (count *n_dev, at most cap) into `out`.  sib: entries are
// SibPairs.  The micro-batch holds queries [q0, q0 + b).
void launch_bucket(gt_tree *t, bool sib, const void *in, void *out, const uint32_t *n_dev,
                   uint32_t cap, int64_t q0, int64_t b, cudaStream_t s);
gt_status launch_dense(gt_tree *t, int h, int mode, int64_t q0, int64_t b, Pair *out,
                       uint32_t *out_count, cudaStream_t s);
// mode 2: raw scores of queries [q0, q0+b) against every pool of level h into
// scores (device, row-major, leading dimension ld)
gt_status launch_dense_impl(gt_tree *t, int h, int mode, int64_t q0, int64_t b, Pair *out,
                            uint32_t *out_count, float *scores, int64_t ld, cudaStream_t s);
bool dense_available();

}  // namespace gt
