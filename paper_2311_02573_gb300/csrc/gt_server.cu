// Continuous-batching query server over one tree.
//
// A query's traversal below the dense cutover level c takes exactly c+1
// kernel rounds (Sec. 4's rounds): the GEMM that scores level c and emits
// level c-1, then one round per level down to the items.  The server runs
// those rounds for several groups of queries at once.  Each step:
//   1. applies queued inserts (Sec. 4, streaming setting) to the tree;
//   2. advances every group in flight by one level: the group at level h
//      is tested and its survivors' children become level h-1 (on the
//      subtraction path, the right child is tested and the left one bounded,
//      down to the items, as in gt_query);
//   3. the group at the item level is decided (bound, FP32 refine, FP64
//      recheck) and its neighbour lists are assembled and copied out;
//   4. admits a new group from the arrival queue, as many queries as the
//      free query slots and the frontier memory budget allow, runs its dense
//      GEMM and groups the survivors by query.
// Groups therefore overlap on the device: a request that arrives while others
// are in flight joins at the next step.  (That is the one-level-per-step
// schedule; the drain schedule takes a group through every level below the
// cutover in the step after its admission, and the immediate schedule in the
// step that admits it: gt_server_schedule.)  Every level's list holds exactly
// one group.  Each group records the tree size at admission and traverses
// that snapshot (later inserts only raise pool sums, so the bounds stay
// valid), so a query's answer is the same alone and in the mix.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstring>
#include <deque>
#include <vector>

#include <string>

#include "gt_internal.cuh"

namespace gt {
namespace {

constexpr int kMaxCut = 12;

struct Group {
  bool active = false;
  int level = 0;        // level its pairs are at (to be tested this step)
  int64_t s0 = 0, b = 0;  // query slots [s0, s0 + b)
  int64_t n_snap = 0;   // tree size when admitted
  std::vector<int64_t> tags;
};

}  // namespace
}  // namespace gt

struct gt_server {
  gt_tree *t = nullptr;
  cudaStream_t s = nullptr;
  int fmt = GT_BF16;
  int cut = 3;
  int64_t max_group = 4096;   // queries admitted per step at most (shrinks on overflow)
  int64_t group_stride = 0;   // query slots per ring position (the initial max_group)
  int64_t slots = 0;          // (cut + 1) x group_stride query slots
  int64_t list_cap = 0;    // pairs per level list
  int64_t queue_cap = 0;   // initial arrival-queue capacity (queries)
  // query bank (device)
  float *qf32 = nullptr, *qn1 = nullptr, *rho = nullptr;
  __nv_bfloat16 *qbf16 = nullptr;
  float *stage = nullptr;  // device staging of one group's raw queries + rho
  // arrival queue: a ring of pinned host rows (admission copies straight from it)
  float *ring_q = nullptr;   // [ring_cap x d]
  float *ring_rho = nullptr; // [ring_cap]
  std::vector<int64_t> ring_tag;
  int64_t ring_cap = 0, ring_head = 0, ring_size = 0;
  // insert staging (pinned host and device), reused every step
  float *ins_h = nullptr, *ins_d = nullptr;
  int64_t ins_cap = 0, ins_n = 0;
  // subtraction path (entries of 16 bytes in the level lists) and the
  // subtraction at the items
  bool sub = false, items_sub = false;
  // prefix layout: list h holds entries of level-(h+1) pools (16 bytes, as
  // on the subtraction path), each split at its midpoint by one prefix row
  bool pre = false;
  // one persistent launch (k_drain) takes a group from the GEMM's list to its
  // decided items: a group is admitted (GEMM) in one step and finished in the
  // next, so each step drains the group admitted the step before while it
  // admits the next one
  bool drain = false;
  // GT_SCHEDULE_IMMEDIATE: each step admits a group and answers it at once
  // (GEMM, the same persistent launch, recheck, CSR), so no group is left in
  // flight between steps
  bool immediate = false;
  void *drain_buf = nullptr;
  int64_t drain_cap = 0;
  // per level two lists (parity), results, rechecks, counters, flags
  gt::Pair *lists[gt::kMaxCut][2] = {};
  gt::Pair *gemm_out = nullptr;  // the new group's GEMM survivors before grouping by query
  int64_t *bcnt = nullptr, *boff = nullptr;  // grouping by query: counts, offsets
  gt::Pair *res = nullptr, *rchk = nullptr;
  int64_t res_cap = 0, rchk_cap = 0;
  uint32_t *counters = nullptr;  // [2h + p] list counts; [40] results, [41] rechecks, [42] refines
  int *flags = nullptr;
  uint32_t *hcounters = nullptr;  // pinned
  // CSR over all slots
  int64_t *cnt = nullptr, *off = nullptr;
  int32_t *ids = nullptr;
  int64_t ids_cap = 0;
  int64_t *hoff = nullptr;
  int32_t *hids = nullptr;
  int64_t hids_cap = 0;
  int64_t ids_guess = 4096;  // ids copied out with the step's counters
  // host state
  int64_t step_no = 0;
  std::vector<gt::Group> groups;  // ring of cut + 1 groups
  // completed queries, flat: tag, snapshot and ids[off[k], off[k+1])
  std::vector<int64_t> done_tag, done_snap, done_off{0};
  std::vector<int32_t> done_ids;
  size_t done_head = 0;
  double est_pairs_per_query = 0.0;  // peak level-(c-1) pairs per admitted query
  gt_server_stats st;
};

namespace gt {
namespace {

// A view of the tree whose workspace points at the server's buffers.
// Start of a step: the next-parity list counts of levels 0 .. cut-1, the
// result, recheck and refine counts, the left-item count, k_drain's queue
// head, the deferred FP8 pairs' count, the flags (words 64 ..) and k_drain's
// test counts (words kDrainCounts ..) start at zero; the current parity's
// counts are kept.
constexpr int kDrainCounts = 96;  // k_drain: [96 + h] tests at level h, [96 + 8] left items
__global__ void k_step_reset(uint32_t *counters, int np, int cut) {
  const int i = threadIdx.x;
  if (i < cut) counters[2 * i + np] = 0u;
  if (i < 3) counters[kMaxLevels + i] = 0u;
  if (i == 0) counters[kLeftItemsSlot] = 0u;
  if (i == 1) counters[kDrainHeadSlot] = 0u;  // k_drain's queue head and
  if (i == 2) counters[kDeferSlot] = 0u;      // deferred FP8 pairs
  if (i < kFlagCount) counters[64 + i] = 0u;
  if (i < 9) counters[kDrainCounts + i] = 0u;
}

gt_tree view_of(gt_server *S, int64_t n_snap, int64_t slot0) {
  gt_tree v = *S->t;
  v.N = n_snap;
  v.L = top_level(n_snap);
  v.ws = Workspace();
  Workspace &w = v.ws;
  w.qf32 = S->qf32 + slot0 * v.stride;
  w.qbf16 = S->qbf16 + slot0 * v.stride;
  w.qn1 = S->qn1 + slot0;
  w.rho = S->rho + slot0;
  w.q_cap = S->slots - slot0;
  w.front_cap = S->list_cap;
  w.front_lim = S->list_cap;
  w.res = S->res;
  w.res_cap = S->res_cap;
  w.rchk = S->rchk;
  w.rchk_cap = S->rchk_cap;
  w.counters = S->counters;
  w.bcnt = S->bcnt;
  w.boff = S->boff;
  w.drain = S->drain_buf;
  w.drain_cap = S->drain_cap;
  v.flags = S->flags;
  return v;
}

// Entries a level list holds: pairs, or subtraction entries (two pairs wide).
int64_t list_entries(const gt_server *S) { return S->sub ? S->list_cap / 2 : S->list_cap; }

gt_status server_alloc(gt_server *S) {
  const int64_t st = S->t->stride;
  GT_CUDA(cudaMalloc(&S->qf32, (size_t)S->slots * st * sizeof(float)));
  GT_CUDA(cudaMalloc(&S->qbf16, (size_t)S->slots * st * sizeof(__nv_bfloat16)));
  GT_CUDA(cudaMalloc(&S->qn1, (size_t)S->slots * sizeof(float)));
  GT_CUDA(cudaMalloc(&S->rho, (size_t)S->slots * sizeof(float)));
  // staging and queues hold the caller's rows (d_in entries: a GT_POOL_MAXMIN
  // tree stores them split, 2 d_in wide)
  GT_CUDA(cudaMalloc(&S->stage, (size_t)S->max_group * (S->t->d_in + 1) * sizeof(float)));
  S->ring_cap = S->queue_cap > 0 ? S->queue_cap : std::max<int64_t>(4 * S->max_group, 16384);
  GT_CUDA(cudaMallocHost(&S->ring_q, (size_t)S->ring_cap * S->t->d_in * sizeof(float)));
  GT_CUDA(cudaMallocHost(&S->ring_rho, (size_t)S->ring_cap * sizeof(float)));
  S->ring_tag.resize((size_t)S->ring_cap);
  S->ins_cap = 4096;
  GT_CUDA(cudaMallocHost(&S->ins_h, (size_t)S->ins_cap * S->t->d_in * sizeof(float)));
  GT_CUDA(cudaMalloc(&S->ins_d, (size_t)S->ins_cap * S->t->d_in * sizeof(float)));
  for (int h = 0; h < S->cut; ++h)
    for (int p = 0; p < 2; ++p) GT_CUDA(cudaMalloc(&S->lists[h][p], (size_t)S->list_cap * sizeof(Pair)));
  GT_CUDA(cudaMalloc(&S->gemm_out, (size_t)S->list_cap * sizeof(Pair)));
  GT_CUDA(cudaMalloc(&S->bcnt, (size_t)(S->slots + 1) * sizeof(int64_t)));
  GT_CUDA(cudaMalloc(&S->boff, (size_t)(S->slots + 1) * sizeof(int64_t)));
  GT_CUDA(cudaMalloc(&S->res, (size_t)S->res_cap * sizeof(Pair)));
  if (S->drain) {
    // k_drain's per-warp lists, sized like the batch path's (a tree view
    // reserves them, then the server keeps the buffer)
    gt_tree tmp = *S->t;
    tmp.ws = Workspace();
    tmp.graphs = nullptr;
    gt_status st = ws_reserve_drain(&tmp);
    if (st != GT_OK) return st;
    S->drain_buf = tmp.ws.drain;
    S->drain_cap = tmp.ws.drain_cap;
  }
  GT_CUDA(cudaMalloc(&S->rchk, (size_t)S->rchk_cap * sizeof(Pair)));
  // list counts, result counts and (from word 64) the status flags in one
  // allocation: a step clears them with one launch and reads them back with
  // one copy
  GT_CUDA(cudaMalloc(&S->counters, 128 * sizeof(uint32_t)));
  GT_CUDA(cudaMemset(S->counters, 0, 128 * sizeof(uint32_t)));
  S->flags = reinterpret_cast<int *>(S->counters + 64);
  GT_CUDA(cudaMallocHost(&S->hcounters, 128 * sizeof(uint32_t)));
  GT_CUDA(cudaMalloc(&S->cnt, (size_t)(S->slots + 1) * sizeof(int64_t)));
  GT_CUDA(cudaMalloc(&S->off, (size_t)(S->slots + 1) * sizeof(int64_t)));
  S->ids_cap = S->res_cap;
  GT_CUDA(cudaMalloc(&S->ids, (size_t)S->ids_cap * sizeof(int32_t)));
  GT_CUDA(cudaMallocHost(&S->hoff, (size_t)(S->slots + 1) * sizeof(int64_t)));
  S->hids_cap = S->res_cap;
  GT_CUDA(cudaMallocHost(&S->hids, (size_t)S->hids_cap * sizeof(int32_t)));
  return GT_OK;
}

void server_release(gt_server *S) {
  cudaFree(S->qf32); cudaFree(S->qbf16); cudaFree(S->qn1); cudaFree(S->rho);
  cudaFree(S->stage);
  if (S->ring_q) cudaFreeHost(S->ring_q);
  if (S->ring_rho) cudaFreeHost(S->ring_rho);
  if (S->ins_h) cudaFreeHost(S->ins_h);
  cudaFree(S->ins_d);
  for (int h = 0; h < kMaxCut; ++h)
    for (int p = 0; p < 2; ++p) cudaFree(S->lists[h][p]);
  cudaFree(S->gemm_out); cudaFree(S->bcnt); cudaFree(S->boff);
  cudaFree(S->drain_buf);
  cudaFree(S->res); cudaFree(S->rchk); cudaFree(S->counters);
  if (S->hcounters) cudaFreeHost(S->hcounters);
  cudaFree(S->cnt); cudaFree(S->off); cudaFree(S->ids);
  if (S->hoff) cudaFreeHost(S->hoff);
  if (S->hids) cudaFreeHost(S->hids);
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Queued inserts, in one batch, before any kernel of the step (the rows were
// checked by gt_server_insert; nothing here waits for the device).  The step
// synchronizes before it returns, so the pinned staging rows are not reused
// while their copy is in flight.
gt_status apply_inserts(gt_server *S) {
  if (S->ins_n == 0) return GT_OK;
  GT_CUDA(cudaMemcpyAsync(S->ins_d, S->ins_h, (size_t)S->ins_n * S->t->d_in * sizeof(float),
                          cudaMemcpyHostToDevice, S->s));
  gt_status st = insert_checked_async(S->t, S->ins_d, S->ins_n, S->s);
  if (st != GT_OK) return st;
  S->st.inserted += S->ins_n;
  S->ins_n = 0;
  return GT_OK;
}

// Queries to admit this step: the queue's head, at most max_group, and what
// the frontier budget holds (a group's level-(c-1) entries at most double per
// level below: a list's entries / 2^(c-1), with a 25% margin).
int64_t admit_count(const gt_server *S, int64_t list_room) {
  int64_t b = std::min<int64_t>(S->ring_size, S->max_group);
  if (b > 0 && S->est_pairs_per_query > 0) {
    const int64_t fit = (int64_t)((double)list_room / (1.25 * S->est_pairs_per_query));
    b = std::max<int64_t>(1, std::min(b, fit));
  }
  return b;
}

// The oldest b queued queries (one or two contiguous pieces of the pinned
// ring) into the staging buffer, then into query slots [s0, s0 + b).
gt_status stage_queries(gt_server *S, int64_t b, int64_t s0) {
  cudaStream_t s = S->s;
  const int d = S->t->d_in;
  const int64_t k0 = S->ring_head, n1 = std::min(b, S->ring_cap - k0), n2 = b - n1;
  GT_CUDA(cudaMemcpyAsync(S->stage, S->ring_q + k0 * d, (size_t)n1 * d * sizeof(float),
                          cudaMemcpyHostToDevice, s));
  GT_CUDA(cudaMemcpyAsync(S->stage + (size_t)b * d, S->ring_rho + k0, (size_t)n1 * sizeof(float),
                          cudaMemcpyHostToDevice, s));
  if (n2 > 0) {
    GT_CUDA(cudaMemcpyAsync(S->stage + (size_t)n1 * d, S->ring_q, (size_t)n2 * d * sizeof(float),
                            cudaMemcpyHostToDevice, s));
    GT_CUDA(cudaMemcpyAsync(S->stage + (size_t)b * d + n1, S->ring_rho, (size_t)n2 * sizeof(float),
                            cudaMemcpyHostToDevice, s));
  }
  gt_tree vq = view_of(S, S->t->N, s0);
  launch_prep_queries(&vq, S->stage, S->stage + (size_t)b * d, b, s);
  return GT_OK;
}

// The flags every step checks after its synchronize.
gt_status step_flags(gt_server *S, const uint32_t *hc) {
  if (hc[64 + kFlagTimeout]) return set_error(GT_ETIMEOUT, "a bounded device wait expired");
  if (hc[64 + kFlagDomain])
    return set_error(GT_EDOMAIN, S->t->split_sign ? "a query has a non-finite entry"
                                                  : "a query has a negative or non-finite entry");
  return GT_OK;
}

// Groups of at most this many queries skip the grouping by query before
// k_drain (GT_SCHEDULE_IMMEDIATE).
constexpr int64_t kUngroupedMax = 64;

// GT_SCHEDULE_IMMEDIATE: one step admits a group from the queue's head and
// answers it: the dense GEMM at the cutover, its survivors grouped by query,
// one persistent launch for every level below and the items (k_drain), the
// FP64 recheck and the CSR, then one synchronize.  A request waits for the
// next step to start and is answered when that step ends.  A group whose
// GEMM list or result list overflowed is answered again, smaller, in a later
// step (its queries stay at the queue's head); nothing else carries over
// between steps.
gt_status step_immediate(gt_server *S, int64_t *in_flight) {
  gt_tree *t = S->t;
  cudaStream_t s = S->s;
  const double t0 = now_s();
  const bool inserting = S->ins_n > 0;
  gt_status st = apply_inserts(S);
  if (st != GT_OK) return st;
  const int p = (int)(S->step_no & 1), np = 1 - p;
  const int64_t room = list_entries(S);
  const int64_t b = admit_count(S, room);
  // The dense level: the server's for large groups; for small ones (not
  // grouped by query) one or two levels higher, up to k_drain's limit.  The
  // GEMM's floor is a read of every pool row at its level, which halves per
  // level up, while the levels gathered below it add work in proportion to
  // the group (measured at N = 1M, d = 1000: groups of about 10 queries are
  // answered 13% sooner with the GEMM at level 5 than at level 3, groups of
  // about 200 fastest at level 3).
  int cut = S->cut;
  if (b <= kUngroupedMax) {
    const int up = std::min<int>(std::min(S->cut + (b <= 32 ? 2 : 1), 5), t->L);
    for (int c = up; c > S->cut; --c)
      if (drain_available(t, S->fmt, c)) {
        cut = c;
        break;
      }
  }
  int64_t launches = 0;
  if (b > 0) {
    k_step_reset<<<1, 64, 0, s>>>(S->counters, np, cut);
    const int64_t s0 = 0;  // one group at a time: the first group's slots
    st = stage_queries(S, b, s0);
    if (st != GT_OK) return st;
    gt_tree v = view_of(S, t->N, 0);
    v.ring_batch = ring_batch_for(b);
    uint32_t *gemm_count = S->counters + 2 * (cut - 1) + np;
    st = launch_dense(&v, cut, 3, s0, b, S->gemm_out, gemm_count, s);
    if (st != GT_OK) return st;
    // a small group's GEMM list goes to k_drain as it is (its warps then
    // take one or a few entries each, one query apiece); a large one is first
    // grouped by query, so that a warp's entries share their query
    const SibPair *queue = reinterpret_cast<const SibPair *>(S->gemm_out);
    if (b > kUngroupedMax) {
      launch_bucket(&v, true, S->gemm_out, S->lists[cut - 1][np], gemm_count, (uint32_t)room, s0, b, s);
      queue = reinterpret_cast<const SibPair *>(S->lists[cut - 1][np]);
      launches += 4;
    }
    launch_drain(&v, S->fmt, cut, queue, gemm_count, s, S->counters + kDrainCounts,
                 S->counters + kDrainCounts + 8, /*cleared=*/true);
    // a small group's recheck and CSR run in one block, which writes the
    // offsets and ids straight into the page-locked host buffers (mapped into
    // the device's address space), so they need no copy; a large group's
    // CSR is copied out (its ids in part, by a guess, the rest after the
    // synchronize when the guess was short)
    const bool small = b <= kCsrSmallMax;
    int64_t ids_pre = S->hids_cap;
    if (small) {
      launch_csr_into(&v, S->res, (uint32_t)S->res_cap, S->counters + kMaxLevels, s0, b, S->cnt, S->hoff,
                      S->hids, S->counters + kCsrListSlot, s, /*recheck=*/true);
    } else {
      launch_recheck(&v, 0, s);
      GT_CUDA(cudaMemsetAsync(S->cnt + s0, 0, (size_t)(b + 1) * sizeof(int64_t), s));
      launch_csr_into(&v, S->res, (uint32_t)S->res_cap, S->counters + kMaxLevels, s0, b, S->cnt, S->off,
                      S->ids, S->counters + kCsrListSlot, s);
      GT_CUDA(cudaMemcpyAsync(S->hoff, S->off + s0, (size_t)(b + 1) * sizeof(int64_t),
                              cudaMemcpyDeviceToHost, s));
      ids_pre = std::min<int64_t>(S->ids_guess, S->hids_cap);
      GT_CUDA(cudaMemcpyAsync(S->hids, S->ids, (size_t)ids_pre * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    }
    GT_CUDA(cudaGetLastError());
    GT_CUDA(cudaMemcpyAsync(S->hcounters, S->counters, 128 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    GT_CUDA(cudaStreamSynchronize(s));
    // reset, prep, GEMM, drain, then the recheck and the CSR's (one block
    // for both for a small group)
    launches += 4 + (small ? 1 : 7);
    const uint32_t *hc = S->hcounters;
    st = step_flags(S, hc);
    if (st != GT_OK) return st;
    if (hc[64 + kFlagStray])
      return set_error(GT_ECUDA, "internal error: a list entry names a query or row outside its "
                                 "buffers; step " + std::to_string(S->step_no));
    const uint32_t gemm_pairs = hc[2 * (cut - 1) + np];
    const double per_q = (double)gemm_pairs / (double)b;
    if (hc[64 + kFlagOverflow] || gemm_pairs > (uint32_t)room) {
      // the group did not fit (its GEMM list, or its results or rechecks):
      // its answers are dropped and its queries stay queued for a smaller
      // group
      if (b == 1)
        return set_error(GT_EOVERFLOW, "one query's frontier or neighbours exceed the server's budget");
      S->max_group = std::max<int64_t>(1, b / 2);
      if (cut == S->cut) S->est_pairs_per_query = std::max(S->est_pairs_per_query, per_q);
      ++S->st.retries;
    } else {
      const int64_t first = S->hoff[0], n_ids = S->hoff[b] - first;
      if (first + n_ids > ids_pre) {
        GT_CUDA(cudaMemcpyAsync(S->hids + ids_pre, S->ids + ids_pre,
                                (size_t)(first + n_ids - ids_pre) * sizeof(int32_t),
                                cudaMemcpyDeviceToHost, s));
        GT_CUDA(cudaStreamSynchronize(s));
      }
      S->ids_guess = std::max<int64_t>(4096, 2 * (first + n_ids));
      const size_t base_ids = S->done_ids.size();
      S->done_ids.insert(S->done_ids.end(), S->hids + first, S->hids + first + n_ids);
      for (int64_t i = 0; i < b; ++i) {
        S->done_tag.push_back(S->ring_tag[(size_t)((S->ring_head + i) % S->ring_cap)]);
        S->done_snap.push_back(t->N);
        S->done_off.push_back((int64_t)base_ids + (S->hoff[i + 1] - first));
      }
      S->ring_head = (S->ring_head + b) % S->ring_cap;
      S->ring_size -= b;
      // (the admission estimate is kept in the server's own level's terms)
      if (cut == S->cut) S->est_pairs_per_query = std::max(S->est_pairs_per_query * 0.9, per_q);
      S->st.admitted += b;
      S->st.completed += b;
      S->st.rechecks += hc[kMaxLevels + 1];
      S->st.refines += hc[kMaxLevels + 2];
      S->st.dense_tests += b * level_rows(t->N, cut);
      S->st.gathered_tests += gemm_pairs;
      for (int h = 0; h + 1 < cut; ++h) S->st.gathered_tests += hc[kDrainCounts + h];
      S->st.gathered_tests += hc[kDrainCounts + 8];
    }
  }
  if (b == 0 && inserting) GT_CUDA(cudaStreamSynchronize(s));  // the inserts' copy and kernels
  S->step_no += 1;
  S->st.steps += 1;
  S->st.launches += launches;
  S->st.busy_seconds += now_s() - t0;
  if (in_flight) *in_flight = 0;
  return GT_OK;
}

}  // namespace
}  // namespace gt

using namespace gt;

extern "C" {

gt_status gt_server_create(gt_tree *t, const gt_server_opts *opts, gt_server **out) {
  if (!t || !out) return set_error(GT_EINVAL, "null argument");
  *out = nullptr;
  const bool pre = t->layout == GT_LAYOUT_PREFIX;
  gt_server_opts o;
  std::memset(&o, 0, sizeof(o));
  o.dtype = GT_BF16;
  o.cutover = -1;
  if (opts) o = *opts;
  if (o.dtype < GT_F32 || o.dtype > GT_FP8 || !(t->formats & (1u << o.dtype)))
    return set_error(GT_EINVAL, "tree does not keep this row format");
  if (!dense_available() || !(t->formats & (1u << GT_BF16)))
    return set_error(GT_EINVAL, "the server needs the dense GEMM path and BF16 rows");
  if (pre && o.cutover >= 1 && o.cutover != t->pc)
    return set_error(GT_EINVAL, "a prefix-layout tree's dense level is its prefix_level");
  gt_server *S = new gt_server();
  S->t = t;
  S->s = o.stream ? (cudaStream_t)o.stream : t->stream;
  S->fmt = o.dtype;
  int cut = o.cutover >= 1 ? o.cutover : (t->tuned_cut[o.dtype] > 0 ? t->tuned_cut[o.dtype] : 3);
  cut = std::max(1, std::min(cut, std::min(t->L, kMaxCut)));
  if (pre) cut = t->pc;  // the level whose pools (the blocks' totals) are stored
  S->cut = cut;
  S->pre = pre;
  // the subtraction path as gt_query takes it: sum pools, a cutover above
  // level 1, unless gt_autotune found it slower for this format (the prefix
  // layout's lists hold entries like the subtraction path's)
  S->sub = pre || (cut >= 2 && t->pooling == GT_POOL_SUM && t->tuned_sub[o.dtype] != -1);
  S->items_sub = !pre && S->sub && items_sub_available(t, o.dtype);
  // one persistent launch for the levels below the cutover, where it applies
  // (unless the caller asked for one level per step)
  if (o.schedule < GT_SCHEDULE_AUTO || o.schedule > GT_SCHEDULE_IMMEDIATE) {
    delete S;
    return set_error(GT_EINVAL, "unknown schedule");
  }
  S->drain = o.schedule != GT_SCHEDULE_LEVELS && !pre && S->items_sub &&
             drain_available(t, o.dtype, cut);
  if ((o.schedule == GT_SCHEDULE_DRAIN || o.schedule == GT_SCHEDULE_IMMEDIATE) && !S->drain) {
    delete S;
    return set_error(GT_EINVAL, "the drain and immediate schedules need the subtraction path of "
                                "a sum-pooled tree with the cutover at level 2 to 5");
  }
  S->immediate = S->drain && o.schedule != GT_SCHEDULE_DRAIN;
  S->max_group = o.max_group > 0 ? o.max_group : 4096;
  S->group_stride = S->max_group;
  S->queue_cap = o.queue_capacity;
  S->slots = (int64_t)(cut + 1) * S->group_stride;
  const int64_t budget = o.scratch_bytes > 0 ? o.scratch_bytes : ((int64_t)4 << 30);
  // 2 lists per level, plus results and rechecks (each a quarter of a list)
  S->list_cap = std::max<int64_t>(1 << 16, budget / ((2 * cut + 1) * (int64_t)sizeof(Pair)));
  S->list_cap = std::min<int64_t>(S->list_cap, (int64_t)1 << 31);
  S->res_cap = std::max<int64_t>(1 << 16, S->list_cap / 4);
  S->rchk_cap = S->res_cap;
  S->groups.resize(cut + 1);
  std::memset(&S->st, 0, sizeof(S->st));
  gt_status st = server_alloc(S);
  if (st != GT_OK) {
    server_release(S);
    delete S;
    return st;
  }
  S->est_pairs_per_query = 0.0;
  *out = S;
  return GT_OK;
}

gt_status gt_server_submit(gt_server *S, const float *Q, const float *rho, const int64_t *tags,
                           int64_t n) {
  if (!S || (n > 0 && (!Q || !rho || !tags))) return set_error(GT_EINVAL, "null argument");
  const int d = S->t->d_in;
  for (int64_t i = 0; i < n; ++i) {
    if (!(rho[i] > 0.f) || !(rho[i] <= 1.f)) return set_error(GT_EINVAL, "rho must satisfy 0 < rho <= 1");
  }
  if (S->ring_size + n > S->ring_cap) {
    // grow the ring (rare): a new pinned ring holding the queue in order
    int64_t cap = S->ring_cap;
    while (cap < S->ring_size + n) cap *= 2;
    float *q = nullptr, *r = nullptr;
    GT_CUDA(cudaMallocHost(&q, (size_t)cap * d * sizeof(float)));
    if (cudaMallocHost(&r, (size_t)cap * sizeof(float)) != cudaSuccess) {
      cudaFreeHost(q);
      return set_error(GT_ENOMEM, "arrival queue growth failed");
    }
    std::vector<int64_t> tg((size_t)cap);
    for (int64_t i = 0; i < S->ring_size; ++i) {
      const int64_t k = (S->ring_head + i) % S->ring_cap;
      std::memcpy(q + i * d, S->ring_q + k * d, (size_t)d * sizeof(float));
      r[i] = S->ring_rho[k];
      tg[(size_t)i] = S->ring_tag[(size_t)k];
    }
    cudaFreeHost(S->ring_q);
    cudaFreeHost(S->ring_rho);
    S->ring_q = q;
    S->ring_rho = r;
    S->ring_tag.swap(tg);
    S->ring_cap = cap;
    S->ring_head = 0;
  }
  for (int64_t i = 0; i < n; ++i) {
    const int64_t k = (S->ring_head + S->ring_size + i) % S->ring_cap;
    std::memcpy(S->ring_q + k * d, Q + i * d, (size_t)d * sizeof(float));
    S->ring_rho[k] = rho[i];
    S->ring_tag[(size_t)k] = tags[i];
  }
  S->ring_size += n;
  S->st.submitted += n;
  return GT_OK;
}

gt_status gt_server_insert(gt_server *S, const float *f, int64_t n) {
  if (!S || (n > 0 && !f)) return set_error(GT_EINVAL, "null argument");
  const int d = S->t->d_in;
  // checked here, on the host, so that a step applies queued rows without
  // waiting for the device to check them (the rule gt_insert applies)
  const bool signed_rows = S->t->split_sign;
  for (int64_t i = 0; i < n * (int64_t)d; ++i) {
    const float x = f[i];
    if (!std::isfinite(x) || (!signed_rows && x < 0.f))
      return set_error(GT_EDOMAIN, signed_rows ? "inserted row has a non-finite entry"
                                               : "inserted row has a negative or non-finite entry");
  }
  if (S->ins_n + n > S->ins_cap) {
    int64_t cap = S->ins_cap;
    while (cap < S->ins_n + n) cap *= 2;
    float *h = nullptr, *dv = nullptr;
    GT_CUDA(cudaMallocHost(&h, (size_t)cap * d * sizeof(float)));
    if (cudaMalloc(&dv, (size_t)cap * d * sizeof(float)) != cudaSuccess) {
      cudaFreeHost(h);
      return set_error(GT_ENOMEM, "insert staging growth failed");
    }
    std::memcpy(h, S->ins_h, (size_t)S->ins_n * d * sizeof(float));
    cudaFreeHost(S->ins_h);
    cudaFree(S->ins_d);
    S->ins_h = h;
    S->ins_d = dv;
    S->ins_cap = cap;
  }
  std::memcpy(S->ins_h + S->ins_n * d, f, (size_t)n * d * sizeof(float));
  S->ins_n += n;
  return GT_OK;
}

gt_status gt_server_step(gt_server *S, int64_t *in_flight) {
  if (!S) return set_error(GT_EINVAL, "null server");
  TraceRange trace("gt_server_step");
  if (S->immediate) return step_immediate(S, in_flight);
  gt_tree *t = S->t;
  cudaStream_t s = S->s;
  const double t0 = now_s();
  // 1. queued inserts, in one batch, before any kernel of this step
  gt_status st_ins = apply_inserts(S);
  if (st_ins != GT_OK) return st_ins;
  const int p = (int)(S->step_no & 1), np = 1 - p;
  const int cut = S->cut;
  // next-parity list counts, results, rechecks and flags start at zero
  k_step_reset<<<1, 64, 0, s>>>(S->counters, np, cut);
  int64_t launches = 0;
  // 2.-3. advance every group in flight by one level
  Group *finishing = nullptr;
  for (auto &g : S->groups) {
    if (!g.active) continue;
    gt_tree v = view_of(S, g.n_snap, 0);
    v.ring_batch = ring_batch_for(g.b);
    const int h = g.level;
    if (S->drain) {
      // the group admitted last step: every level below the cutover and its
      // items in one launch, so it finishes in this step
      launch_drain(&v, S->fmt, cut, reinterpret_cast<const SibPair *>(S->lists[h][p]),
                   S->counters + 2 * h + p, s, S->counters + kDrainCounts,
                   S->counters + kDrainCounts + 8);
    } else if (S->pre) {
      // the level-(h+1) pools of list h split at their midpoints: the kept
      // level-h children go to list h-1, or at h = 0 the items are decided
      if (!launch_prefix(&v, S->fmt, h + 1, reinterpret_cast<const SibPair *>(S->lists[h][p]),
                         S->counters + 2 * h + p,
                         h > 0 ? reinterpret_cast<SibPair *>(S->lists[h - 1][np]) : nullptr,
                         h > 0 ? S->counters + 2 * (h - 1) + np : nullptr, s))
        return set_error(GT_EINVAL, "FP32 prefix rows this wide do not fit the gather's "
                                    "shared-memory slots (d <= 1152 fits)");
    } else if (S->sub && h >= 1) {
      launch_level_sub(&v, S->fmt, h, reinterpret_cast<const SibPair *>(S->lists[h][p]),
                       S->counters + 2 * h + p, S->lists[h - 1][np], S->counters + 2 * (h - 1) + np, s,
                       S->items_sub);
    } else if (S->items_sub) {
      // right items decided, left items by their bounds or from their rows
      launch_items_sub(&v, S->fmt, reinterpret_cast<const SibPair *>(S->lists[0][p]), S->counters + p,
                       S->counters + kLeftItemsSlot, s);
    } else {
      launch_level(&v, S->fmt, h, 0, S->lists[h][p], S->counters + 2 * h + p,
                   h > 0 ? S->lists[h - 1][np] : nullptr, h > 0 ? S->counters + 2 * (h - 1) + np : nullptr,
                   s);
    }
    ++launches;
    if (h == 0 || S->drain) {
      finishing = &g;
      launch_recheck(&v, 0, s);
      ++launches;
    }
  }
  // the finishing group's neighbour lists, assembled behind its leaf level
  // with the result count read on the device; its offsets and a guess of its
  // ids come back with the step's counters (only this group has results, so
  // its ids start at 0)
  int64_t ids_pre = 0;
  if (finishing) {
    gt_tree v = view_of(S, finishing->n_snap, 0);
    v.ring_batch = ring_batch_for(finishing->b);
    // the CSR over the finishing group's slots only (every result is one of its queries)
    const int64_t s0 = finishing->s0, nb = finishing->b;
    GT_CUDA(cudaMemsetAsync(S->cnt + s0, 0, (size_t)(nb + 1) * sizeof(int64_t), s));
    launch_csr_into(&v, S->res, (uint32_t)S->res_cap, S->counters + kMaxLevels, s0, nb, S->cnt,
                    S->off, S->ids, S->counters + kCsrListSlot, s);
    launches += 6;
    GT_CUDA(cudaMemcpyAsync(S->hoff, S->off + finishing->s0, (size_t)(finishing->b + 1) * sizeof(int64_t),
                            cudaMemcpyDeviceToHost, s));
    ids_pre = std::min<int64_t>(S->ids_guess, S->hids_cap);
    GT_CUDA(cudaMemcpyAsync(S->hids, S->ids, (size_t)ids_pre * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  }
  // 4. admit a new group: free ring position, slots, memory budget
  // (with cut + 1 ring positions and at most cut groups in flight, one is free)
  Group *fresh = nullptr;
  int64_t b = 0;
  for (auto &g : S->groups)
    if (!g.active) {
      fresh = &g;
      break;
    }
  // (the drain schedule's lists below the cutover are the warps' own)
  if (fresh) b = admit_count(S, S->drain ? list_entries(S) : list_entries(S) >> (S->cut - 1));
  int64_t fresh_s0 = 0;
  if (b > 0) {
    const int ring = (int)(fresh - S->groups.data());
    fresh_s0 = (int64_t)ring * S->group_stride;
    // queries into their slots; the GEMM then names them by slot number
    gt_status st_q = stage_queries(S, b, fresh_s0);
    if (st_q != GT_OK) return st_q;
    gt_tree v = view_of(S, t->N, 0);
    gt_status st = launch_dense(&v, cut, S->sub ? 3 : 0, fresh_s0, b, S->gemm_out,
                                S->counters + 2 * (cut - 1) + np, s);
    if (st != GT_OK) return st;
    // the GEMM's survivors grouped by query into the level-(c-1) list
    launch_bucket(&v, S->sub, S->gemm_out, S->lists[cut - 1][np], S->counters + 2 * (cut - 1) + np,
                  (uint32_t)list_entries(S), fresh_s0, b, s);
    launches += 6;  // prep, GEMM, bucketing (four)
  }
  GT_CUDA(cudaGetLastError());
  GT_CUDA(cudaMemcpyAsync(S->hcounters, S->counters, 128 * sizeof(uint32_t),
                          cudaMemcpyDeviceToHost, s));
  GT_CUDA(cudaStreamSynchronize(s));
  const uint32_t *hc = S->hcounters;
  gt_status st_f = step_flags(S, hc);
  if (st_f != GT_OK) return st_f;
  if (hc[64 + kFlagStray]) {
    std::string lv;
    for (auto &g : S->groups)
      if (g.active) lv += " [s0 " + std::to_string(g.s0) + " b " + std::to_string(g.b) + " level " +
                          std::to_string(g.level) + "]";
    return set_error(GT_ECUDA, "internal error: a result (query slot " +
                                   std::to_string((int)hc[64 + kFlagStray + 1]) + ", row " +
                                   std::to_string((int)hc[64 + kFlagStray + 2]) +
                                   ") outside the finishing group's queries; step " +
                                   std::to_string(S->step_no) + ", groups" + lv);
  }
  // level lists are sized so that only the new group's GEMM output can
  // overflow; results and rechecks are checked too
  // The new group may put at most list_cap / 2^(c-1) pairs at level c-1:
  // each level below at most doubles, so no older group's list can overflow.
  const uint32_t fresh_pairs = hc[2 * (cut - 1) + np];
  // (with k_drain only the GEMM's list is in device lists: the levels below
  // live in the warps' own lists)
  const uint32_t fresh_lim = (uint32_t)(S->drain ? list_entries(S) : list_entries(S) >> (cut - 1));
  bool fresh_overflow = b > 0 && fresh_pairs > fresh_lim;
  if (hc[64 + kFlagOverflow]) {
    bool older = hc[kMaxLevels] > (uint32_t)S->res_cap || hc[kMaxLevels + 1] > (uint32_t)S->rchk_cap;
    for (int h = 0; h + 1 < cut; ++h) older |= hc[2 * h + np] > (uint32_t)list_entries(S);
    if (older) return set_error(GT_EOVERFLOW, "a query group outgrew the server's frontier budget");
    fresh_overflow = b > 0;
  }
  // the finishing group's neighbour lists
  if (finishing) {
    const int64_t nb = finishing->b;
    const int64_t first = S->hoff[0], n_ids = S->hoff[nb] - first;
    if (first + n_ids > ids_pre) {
      GT_CUDA(cudaMemcpyAsync(S->hids + ids_pre, S->ids + ids_pre,
                              (size_t)(first + n_ids - ids_pre) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      GT_CUDA(cudaStreamSynchronize(s));
    }
    S->ids_guess = std::max<int64_t>(4096, 2 * (first + n_ids));
    const size_t base_ids = S->done_ids.size();
    S->done_ids.insert(S->done_ids.end(), S->hids + first, S->hids + first + n_ids);
    for (int64_t i = 0; i < nb; ++i) {
      S->done_tag.push_back(finishing->tags[(size_t)i]);
      S->done_snap.push_back(finishing->n_snap);
      S->done_off.push_back((int64_t)base_ids + (S->hoff[i + 1] - first));
    }
    S->st.completed += nb;
    S->st.rechecks += hc[kMaxLevels + 1];
    S->st.refines += hc[kMaxLevels + 2];
    finishing->active = false;
    finishing->tags.clear();
  }
  // advance the levels of the groups still in flight
  for (auto &g : S->groups)
    if (g.active) {
      S->st.gathered_tests += hc[2 * g.level + p];
      g.level -= 1;
    }
  // the finishing group's item tests (its level-0 list, and the left items)
  if (finishing && S->drain) {
    // its GEMM list and every level k_drain tested
    S->st.gathered_tests += hc[2 * (cut - 1) + p];
    for (int h = 0; h + 1 < cut; ++h) S->st.gathered_tests += hc[kDrainCounts + h];
    S->st.gathered_tests += hc[kDrainCounts + 8];
  } else if (finishing) {
    S->st.gathered_tests += hc[p] + (S->items_sub ? hc[kLeftItemsSlot] : 0);
  }
  if (b > 0) {
    if (fresh_overflow) {
      // the new group's survivors did not fit: leave it queued, admit fewer
      if (b == 1)
        return set_error(GT_EOVERFLOW, "one query's frontier exceeds the server's budget");
      S->max_group = std::max<int64_t>(1, b / 2);
      S->est_pairs_per_query = std::max(S->est_pairs_per_query, (double)fresh_pairs / (double)b);
      ++S->st.retries;
    } else {
      fresh->active = true;
      fresh->level = cut - 1;
      fresh->s0 = fresh_s0;
      fresh->b = b;
      fresh->n_snap = t->N;
      fresh->tags.resize((size_t)b);
      for (int64_t i = 0; i < b; ++i)
        fresh->tags[(size_t)i] = S->ring_tag[(size_t)((S->ring_head + i) % S->ring_cap)];
      S->ring_head = (S->ring_head + b) % S->ring_cap;
      S->ring_size -= b;
      const double per_q = (double)hc[2 * (cut - 1) + np] / (double)b;
      S->est_pairs_per_query = std::max(S->est_pairs_per_query * 0.9, per_q);
      S->st.dense_tests += b * level_rows(t->N, cut);
      S->st.admitted += b;
    }
  }
  S->step_no += 1;
  S->st.steps += 1;
  S->st.launches += launches;
  S->st.busy_seconds += now_s() - t0;
  int64_t fl = 0;
  for (auto &g : S->groups)
    if (g.active) fl += g.b;
  if (in_flight) *in_flight = fl;
  return GT_OK;
}

gt_status gt_server_poll(gt_server *S, int64_t max_queries, int64_t *n_done, int64_t *tags,
                         int64_t *offsets, int32_t *ids, int64_t ids_cap, int64_t *n_snapshot) {
  if (!S || !n_done || (max_queries > 0 && (!tags || !offsets))) return set_error(GT_EINVAL, "null argument");
  *n_done = 0;
  if (offsets) offsets[0] = 0;
  const size_t avail = S->done_tag.size() - S->done_head;
  size_t k = 0;
  const int64_t id0 = S->done_off[S->done_head];
  while (k < (size_t)max_queries && k < avail) {
    const size_t j = S->done_head + k;
    const int64_t end = S->done_off[j + 1] - id0;
    if (end > ids_cap) {
      if (k == 0) return set_error(GT_EOVERFLOW, "ids_cap is smaller than the next query's list");
      break;
    }
    tags[k] = S->done_tag[j];
    if (n_snapshot) n_snapshot[k] = S->done_snap[j];
    offsets[k + 1] = end;
    ++k;
  }
  if (k) std::memcpy(ids, S->done_ids.data() + id0, (size_t)offsets[k] * sizeof(int32_t));
  S->done_head += k;
  *n_done = (int64_t)k;
  // drop what every caller has taken
  if (S->done_head == S->done_tag.size()) {
    S->done_tag.clear();
    S->done_snap.clear();
    S->done_ids.clear();
    S->done_off.assign(1, 0);
    S->done_head = 0;
  }
  return GT_OK;
}

gt_status gt_server_get_stats(const gt_server *S, gt_server_stats *out) {
  if (!S || !out) return set_error(GT_EINVAL, "null argument");
  *out = S->st;
  out->pending = S->ring_size;
  out->cutover = S->cut;
  out->max_group = S->max_group;
  out->schedule = S->immediate ? GT_SCHEDULE_IMMEDIATE
                 : S->drain    ? GT_SCHEDULE_DRAIN
                               : GT_SCHEDULE_LEVELS;
  return GT_OK;
}

void gt_server_free(gt_server *S) {
  if (!S) return;
  cudaStreamSynchronize(S->s);
  server_release(S);
  delete S;
}

}  // extern "C"
