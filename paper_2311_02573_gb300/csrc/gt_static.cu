// gt_query_static: a range query that allocates no memory.
//
// Some callers cannot allocate device memory at query time: a serving thread
// with a hard latency budget (cudaMalloc can synchronise the device and stall
// every stream), a process whose device memory is owned by another
// allocator or already committed in full, or code that must not change the
// device's memory footprint after start-up.  This entry point runs the same
// traversal kernels as gt_query, but every scratch buffer they need (query
// copies, frontier lists, result and recheck lists, counters) lives in one
// fixed array in device global memory that the library declares at file
// scope, and the caller passes the output buffers.
//
// The array, g_static_scratch, is kStaticBytes (32 MiB) and exists on every
// GPU on which the library is loaded, from load until the process exits.  In
// host code its name is only a host-side stand-in, so the first call on each
// device looks up its device address with cudaGetSymbolAddress (that device
// current) and keeps it; that first call should come before any stream
// capture.  The kept address belongs to the device's current context: after
// cudaDeviceReset the process must not call gt_query_static on that device
// again.  All calls share the array and it keeps the last call's contents:
// each call clears the counters it relies on, and calls that overlap on the
// GPU (on different streams, or from different threads) race on it and must
// not be issued.
//
// Fixed limits of the array: 256 queries per call, rows of at most 2048
// entries, 262,144 neighbours per call in all (the result list is shared by
// the call's micro-batches), 65,536 leaf pairs of one micro-batch waiting for
// the FP64 recheck, and about 1.8M (query, pool) pairs in each of the two
// frontier lists of one micro-batch.  A micro-batch whose frontier or recheck
// list overflows is re-run with half the queries; a call whose results
// exceed the result list, or one query whose frontier alone does not fit,
// returns GT_EOVERFLOW.
#include <mutex>

#include "gt_internal.cuh"

namespace gt {
namespace {

constexpr int64_t kStaticBytes = (int64_t)32 << 20;
constexpr int64_t kStaticMaxQueries = 256;
constexpr int64_t kStaticMaxStride = 2048;

// layout of the array (byte offsets, all 256-byte aligned)
constexpr int64_t kOffCounters = 0;                               // 64 x u32
constexpr int64_t kOffFlags = 256;                                // 64 x int
constexpr int64_t kOffQn1 = 512;                                  // max queries x f32
constexpr int64_t kOffRho = kOffQn1 + kStaticMaxQueries * 4;      // max queries x f32
constexpr int64_t kOffCursor = kOffRho + kStaticMaxQueries * 4;   // (max queries + 1) x i64
constexpr int64_t kOffQ = 8192;                                   // max queries x stride x f32
constexpr int64_t kOffRes = kOffQ + kStaticMaxQueries * kStaticMaxStride * 4;
constexpr int64_t kResPairs = (int64_t)1 << 18;
constexpr int64_t kOffRchk = kOffRes + kResPairs * (int64_t)sizeof(Pair);
constexpr int64_t kRchkPairs = (int64_t)1 << 16;
constexpr int64_t kOffFront = kOffRchk + kRchkPairs * (int64_t)sizeof(Pair);
constexpr int64_t kFrontPairs = (kStaticBytes - kOffFront) / (2 * (int64_t)sizeof(Pair));
static_assert(kOffCursor + (kStaticMaxQueries + 1) * 8 <= kOffQ, "layout");
static_assert(kFrontPairs > 0, "layout");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

std::mutex g_setup_mutex;
void *g_scratch_addr[64] = {nullptr};

// Device address of g_static_scratch on the current device (looked up once).
gt_status scratch_address(void **out) {
  int dev = 0;
  GT_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(GT_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_static_scratch)");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return GT_OK;
}

}  // namespace
}  // namespace gt

using namespace gt;

extern "C" gt_status gt_query_static(gt_tree *t, const float *Q, int64_t B, const float *rho,
                                     int32_t dtype, int64_t *offsets, int32_t *ids,
                                     int64_t ids_cap, int64_t *n_results, void *stream) {
  if (n_results) *n_results = 0;
  if (!t || !Q || !rho || !offsets || !n_results || (ids_cap > 0 && !ids))
    return set_error(GT_EINVAL, "null argument");
  if (t->layout == GT_LAYOUT_PREFIX) return set_error(GT_EINVAL, "not available for a prefix-layout tree");
  if (B < 1 || B > kStaticMaxQueries)
    return set_error(GT_EINVAL, "gt_query_static takes 1 to 256 queries per call");
  if (ids_cap < 0) return set_error(GT_EINVAL, "negative ids capacity");
  if (t->stride > kStaticMaxStride) return set_error(GT_EINVAL, "dimension above 2048");
  if (dtype < GT_F32 || dtype > GT_FP8 || !(t->formats & (1u << dtype)))
    return set_error(GT_EINVAL, "tree does not keep this row format");
  if (!is_device_ptr(Q) || !is_device_ptr(rho) || !is_device_ptr(offsets) ||
      (ids_cap > 0 && !is_device_ptr(ids)))
    return set_error(GT_EINVAL, "gt_query_static needs device pointers for Q, rho and outputs");
  int dev = 0;
  GT_CUDA(cudaGetDevice(&dev));
  if (dev != t->device)
    return set_error(GT_EINVAL, "gt_query_static must be called with the tree's device current");
  cudaStream_t s = stream ? (cudaStream_t)stream : t->stream;
  void *base = nullptr;
  gt_status st = scratch_address(&base);
  if (st != GT_OK) return st;
  char *sc = reinterpret_cast<char *>(base);

  // a view of the tree whose workspace is the static array
  gt_tree v = *t;
  v.ring_batch = ring_batch_for(B);
  v.ws = Workspace();
  Workspace &w = v.ws;
  w.counters = reinterpret_cast<uint32_t *>(sc + kOffCounters);
  v.flags = reinterpret_cast<int *>(sc + kOffFlags);
  w.qn1 = reinterpret_cast<float *>(sc + kOffQn1);
  w.rho = reinterpret_cast<float *>(sc + kOffRho);
  w.qf32 = reinterpret_cast<float *>(sc + kOffQ);
  w.qbf16 = nullptr;
  w.q_cap = kStaticMaxQueries;
  w.res = reinterpret_cast<Pair *>(sc + kOffRes);
  w.res_cap = kResPairs;
  w.rchk = reinterpret_cast<Pair *>(sc + kOffRchk);
  w.rchk_cap = kRchkPairs;
  w.front[0] = reinterpret_cast<Pair *>(sc + kOffFront);
  w.front[1] = w.front[0] + kFrontPairs;
  w.front_cap = kFrontPairs;
  w.front_lim = kFrontPairs;
  int64_t *cursor = reinterpret_cast<int64_t *>(sc + kOffCursor);

  // the array keeps the previous call's contents: clear what starts at zero
  GT_CUDA(cudaMemsetAsync(sc, 0, 512, s));  // counters and flags
  launch_prep_queries(&v, Q, rho, B, s);
  uint32_t hc[64 + 16];
  GT_CUDA(cudaMemcpyAsync(hc + 64, v.flags, 16 * sizeof(int), cudaMemcpyDeviceToHost, s));
  GT_CUDA(cudaStreamSynchronize(s));
  if (hc[64 + kFlagDomain]) return set_error(GT_EDOMAIN, "Q has a negative or non-finite entry");
  if (hc[64 + kFlagRho]) return set_error(GT_EINVAL, "rho must satisfy 0 < rho <= 1");

  uint32_t R = 0;
  int64_t bm = B, q0 = 0;
  while (q0 < B) {
    const int64_t b = std::min(bm, B - q0);
    GT_CUDA(cudaMemsetAsync(w.counters, 0, kMaxLevels * sizeof(uint32_t), s));
    GT_CUDA(cudaMemsetAsync(w.counters + kMaxLevels + 1, 0, sizeof(uint32_t), s));
    GT_CUDA(cudaMemsetAsync(v.flags + kFlagOverflow, 0, sizeof(int), s));
    launch_root(&v, q0, b, w.front[v.L & 1], w.counters + v.L, s);
    for (int h = v.L; h >= 0; --h)
      launch_level(&v, dtype, h, q0, w.front[h & 1], w.counters + h,
                   h > 0 ? w.front[(h - 1) & 1] : nullptr, h > 0 ? w.counters + h - 1 : nullptr, s);
    launch_recheck(&v, q0, s);
    GT_CUDA(cudaGetLastError());
    GT_CUDA(cudaMemcpyAsync(hc, w.counters, 64 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    GT_CUDA(cudaMemcpyAsync(hc + 64, v.flags, 16 * sizeof(int), cudaMemcpyDeviceToHost, s));
    GT_CUDA(cudaStreamSynchronize(s));
    if (hc[64 + kFlagTimeout]) return set_error(GT_ETIMEOUT, "a bounded device wait expired");
    if (hc[64 + kFlagStray])
      return set_error(GT_ECUDA, "internal error: a list entry names a query or row outside its buffers");
    if (hc[64 + kFlagOverflow]) {
      // the result list holds every micro-batch's neighbours: fewer queries
      // per micro-batch cannot make the call's results fit
      if ((int64_t)hc[kMaxLevels] > kResPairs)
        return set_error(GT_EOVERFLOW, "the call's neighbours exceed the static result list "
                                       "(262,144 per call): split the queries over more calls");
      // a frontier or the recheck list: roll the result list back and retry
      // with fewer queries
      GT_CUDA(cudaMemcpyAsync(w.counters + kMaxLevels, &R, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
      GT_CUDA(cudaStreamSynchronize(s));
      if (b == 1)
        return set_error(GT_EOVERFLOW, "one query's frontier (or its leaf pairs awaiting the FP64 "
                                       "recheck) exceeds the static scratch's lists");
      bm = b / 2;
      continue;
    }
    R = hc[kMaxLevels];
    q0 += b;
  }
  *n_results = R;
  if ((int64_t)R > ids_cap)
    return set_error(GT_EOVERFLOW, "ids_cap is smaller than the number of neighbours "
                                   "(*n_results holds the count needed)");
  GT_CUDA(cudaMemsetAsync(cursor, 0, (size_t)(B + 1) * sizeof(int64_t), s));
  launch_csr_into(&v, w.res, R, nullptr, 0, B, cursor, offsets, ids, w.counters + kCsrListSlot, s);
  GT_CUDA(cudaGetLastError());
  // the CSR passes flag (and leave out) a result naming a query outside the call
  GT_CUDA(cudaMemcpyAsync(hc + 64, v.flags, 16 * sizeof(int), cudaMemcpyDeviceToHost, s));
  GT_CUDA(cudaStreamSynchronize(s));
  if (hc[64 + kFlagStray])
    return set_error(GT_ECUDA, "internal error: a result names a query outside the call");
  return GT_OK;
}
