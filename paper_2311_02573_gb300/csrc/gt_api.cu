// The C ABI of include/gt.h: argument checks, staging of host inputs,
// micro-batching of the query traversal, and error reporting.
#include <algorithm>
#include <cerrno>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "gt_internal.cuh"

namespace gt {

namespace {
thread_local std::string g_err;
}

gt_status set_error(gt_status st, const std::string &msg) {
  g_err = msg;
  return st;
}

gt_status cuda_error(cudaError_t e, const char *what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? GT_ENOMEM : GT_ECUDA;
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

namespace {

// The device address of page-locked (cudaHostAlloc'd or registered) host
// memory, which kernels can read in place; null for any other pointer.
const void *pinned_device_view(const void *p) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return attr.type == cudaMemoryTypeHost ? attr.devicePointer : nullptr;
}

// Bring `bytes` of a host or device input onto the device; `tmp` receives an
// allocation the caller must free when the input was on the host.
gt_status to_device(const void *p, size_t bytes, cudaStream_t s, const void **dev, void **tmp) {
  *tmp = nullptr;
  if (is_device_ptr(p)) {
    *dev = p;
    return GT_OK;
  }
  void *d = nullptr;
  GT_CUDA(cudaMalloc(&d, std::max<size_t>(bytes, 16)));
  cudaError_t e = cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    cudaFree(d);
    return cuda_error(e, "cudaMemcpyAsync(input)");
  }
  *dev = d;
  *tmp = d;
  return GT_OK;
}

void free_tree_storage(gt_tree *t) {
  cudaFree(t->rows32);
  cudaFree(t->rows16);
  cudaFree(t->rows8);
  cudaFree(t->scale8);
  cudaFree(t->perm);
  cudaFree(t->pref16);
  cudaFree(t->pref32);
  t->rows32 = nullptr;
  t->rows16 = nullptr;
  t->rows8 = nullptr;
  t->scale8 = nullptr;
  t->perm = nullptr;
  t->pref16 = nullptr;
  t->pref32 = nullptr;
}

void free_workspace(gt_tree *t) {
  Workspace &w = t->ws;
  cudaFree(w.front[0]);
  cudaFree(w.front[1]);
  cudaFree(w.res);
  cudaFree(w.rchk);
  cudaFree(w.defer);
  cudaFree(w.counters);
  cudaFree(w.qf32);
  cudaFree(w.qbf16);
  cudaFree(w.qn1);
  cudaFree(w.rho);
  cudaFree(w.stage);
  cudaFree(w.bcnt);
  cudaFree(w.boff);
  cudaFree(w.drain);
  if (w.hcounters) cudaFreeHost(w.hcounters);
  w = Workspace();
}

gt_status read_flags(gt_tree *t, cudaStream_t s, int *h) {
  GT_CUDA(cudaMemcpyAsync(h, t->flags, kFlagCount * sizeof(int), cudaMemcpyDeviceToHost, s));
  GT_CUDA(cudaStreamSynchronize(s));
  return GT_OK;
}

// CUDA-event timing of the kernels a call launches, by kind (opts->timing).
// While a CUDA graph is being captured the events are recorded as external
// events, so each replay of the graph records them again.
struct KernelTimer {
  bool on = false;
  bool capturing = false;
  cudaStream_t s = nullptr;
  std::vector<cudaEvent_t> *pool = nullptr;
  size_t used = 0;
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> marks;  // (kind, start, end)
  int open_kind = 0;
  cudaEvent_t open_start = nullptr;
  cudaEvent_t next() {
    if (used == pool->size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool->push_back(e);
    }
    return (*pool)[used++];
  }
  void record(cudaEvent_t e) {
    if (capturing)
      cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else
      cudaEventRecord(e, s);
  }
  void begin(int kind) {
    if (!on) return;
    open_kind = kind;
    open_start = next();
    record(open_start);
  }
  void end() {
    if (!on) return;
    cudaEvent_t e = next();
    record(e);
    marks.emplace_back(open_kind, open_start, e);
  }
  void collect(float *ms) {
    if (!on) return;
    cudaStreamSynchronize(s);
    for (auto &m : marks) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, std::get<1>(m), std::get<2>(m)) == cudaSuccess)
        ms[std::get<0>(m)] += t;
    }
    cudaGetLastError();
  }
};

std::vector<cudaEvent_t> &event_pool(gt_tree *t) {
  static thread_local std::vector<cudaEvent_t> pool;
  (void)t;
  return pool;
}

int64_t default_budget() {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return (int64_t)1 << 30;
  }
  return std::min<int64_t>((int64_t)fr / 4, (int64_t)16 << 30);
}

// Copy the first `rows_keep` rows of every level from the old layout to a
// freshly allocated one with capacity `cap`.
gt_status grow(gt_tree *t, int64_t cap) {
  gt_tree old = *t;
  t->rows32 = nullptr; t->rows16 = nullptr; t->rows8 = nullptr; t->scale8 = nullptr;
  t->perm = nullptr; t->pref16 = nullptr; t->pref32 = nullptr;
  const bool pre = t->layout == GT_LAYOUT_PREFIX;
  gt_status st = pre ? prefix_alloc(t, cap) : tree_alloc(t, cap);
  if (st != GT_OK) {
    free_tree_storage(t);
    *t = old;
    old.ws = Workspace();
    return st;
  }
  if (pre) {
    // the items move; their prefix rows and block totals are recomputed
    GT_CUDA(cudaMemcpyAsync(t->rows32, old.rows32, (size_t)old.N * t->stride * 4,
                            cudaMemcpyDeviceToDevice, t->stream));
    GT_CUDA(cudaMemcpyAsync(t->perm, old.perm, (size_t)old.N * 4, cudaMemcpyDeviceToDevice, t->stream));
    st = prefix_build(t, 0, old.N, t->stream);
    if (st != GT_OK) return st;
    GT_CUDA(cudaStreamSynchronize(t->stream));
    free_tree_storage(&old);
    return GT_OK;
  }
  for (int h = 0; h <= old.L; ++h) {
    const int64_t rows = level_rows(old.N, h);
    const size_t so = (size_t)old.lvl_off[h] * t->stride, sn = (size_t)t->lvl_off[h] * t->stride;
    const size_t n = (size_t)rows * t->stride;
    GT_CUDA(cudaMemcpyAsync(t->rows32 + sn, old.rows32 + so, n * 4, cudaMemcpyDeviceToDevice, t->stream));
    if (t->rows16)
      GT_CUDA(cudaMemcpyAsync(t->rows16 + sn, old.rows16 + so, n * 2, cudaMemcpyDeviceToDevice, t->stream));
    if (t->rows8) {
      GT_CUDA(cudaMemcpyAsync(t->rows8 + sn, old.rows8 + so, n, cudaMemcpyDeviceToDevice, t->stream));
      GT_CUDA(cudaMemcpyAsync(t->scale8 + t->lvl_off[h], old.scale8 + old.lvl_off[h], rows * 4,
                              cudaMemcpyDeviceToDevice, t->stream));
    }
  }
  GT_CUDA(cudaMemcpyAsync(t->perm, old.perm, (size_t)old.N * 4, cudaMemcpyDeviceToDevice, t->stream));
  GT_CUDA(cudaStreamSynchronize(t->stream));
  free_tree_storage(&old);
  return GT_OK;
}

// gt_exhaustive's scan contexts, one per device: a tree of level 0 alone
// (FP32 and BF16 rows of the items in input order) that each call rewrites
// from the caller's rows.  Its row storage, workspace and captured graphs are
// kept between calls; a call with another width d starts a fresh context.
constexpr int kMaxDevices = 64;
std::mutex g_scan_mutex;
gt_tree *g_scan[kMaxDevices] = {nullptr};

gt_status scan_context(int dev, int64_t N, int32_t d, gt_tree **out) {
  gt_tree *&x = g_scan[dev];
  if (x && x->d != d) {
    gt_free(x);
    x = nullptr;
  }
  if (!x) {
    x = new gt_tree();
    x->d = d;
    x->d_in = d;
    x->stride = ((int64_t)d + 63) / 64 * 64;
    x->formats = (1u << GT_F32) | (1u << GT_BF16);
    x->device = dev;
    cudaDeviceGetAttribute(&x->sm_count, cudaDevAttrMultiProcessorCount, dev);
    x->sm_total = x->sm_count;
    cudaError_t e = cudaMalloc(&x->flags, 64 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(x->flags, 0, 64 * sizeof(int));
    if (e != cudaSuccess || x->sm_count <= 0) {
      gt_free(x);
      x = nullptr;
      return e != cudaSuccess ? cuda_error(e, "scan context") : set_error(GT_ECUDA, "no CUDA device");
    }
  }
  if (N > x->cap) {
    free_tree_storage(x);
    x->cap = 0;
    const size_t n = (size_t)N * (size_t)x->stride;
    GT_CUDA(cudaMalloc(&x->rows32, n * sizeof(float)));
    GT_CUDA(cudaMalloc(&x->rows16, n * 2));
    GT_CUDA(cudaMalloc(&x->perm, (size_t)N * sizeof(int32_t)));
    x->cap = N;
  }
  // one level: the items (every row is rewritten in full, padding included)
  x->N = N;
  x->L = 0;
  x->Lcap = 0;
  x->lvl_off[0] = 0;
  x->lvl_off[1] = x->cap;
  x->total_rows = x->cap;
  *out = x;
  return GT_OK;
}

}  // namespace
}  // namespace gt

using namespace gt;

namespace gt {
// Append n_new device rows that the caller has already checked (finite, and
// non-negative unless the tree stores split signed rows): the items' rows,
// then every pool above them, enqueued on s with no wait for the device
// (storage grows first, synchronously, when the capacity is reached).
gt_status insert_checked_async(gt_tree *t, const float *F_dev, int64_t n_new, cudaStream_t s) {
  if (n_new <= 0) return GT_OK;
  const int64_t N1 = t->N + n_new;
  if (N1 >= ((int64_t)1 << 31)) return set_error(GT_EINVAL, "tree would exceed 2^31 items");
  if (N1 > t->cap) {
    gt_status st = grow(t, std::max<int64_t>(N1, 2 * t->cap));
    if (st != GT_OK) return st;
  }
  gt_status st = tree_build_level0(t, F_dev, t->N, n_new, nullptr, s);
  if (st != GT_OK) return st;
  const int64_t first = t->N;
  t->N = N1;
  t->L = top_level(N1);
  return t->layout == GT_LAYOUT_PREFIX ? prefix_build(t, first, n_new, s)
                                       : tree_build_levels(t, first, n_new, s);
}
}  // namespace gt

extern "C" {

const char *gt_last_error(void) { return g_err.c_str(); }

gt_status gt_build(const float *F, int64_t N, int32_t d, const gt_build_opts *opts, gt_tree **out) {
  TraceRange trace("gt_build");
  if (!out) return set_error(GT_EINVAL, "null output handle");
  *out = nullptr;
  if (!F) return set_error(GT_EINVAL, "null F");
  if (N < 1 || N >= ((int64_t)1 << 31)) return set_error(GT_EINVAL, "N must be in [1, 2^31)");
  if (d < 1 || d > 2048) return set_error(GT_EINVAL, "d must be in [1, 2048]");
  gt_build_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  const int64_t cap = std::max<int64_t>(N, o.capacity);
  if (cap >= ((int64_t)1 << 31)) return set_error(GT_EINVAL, "capacity must be < 2^31");
  if (o.pooling != GT_POOL_SUM && o.pooling != GT_POOL_MAX && o.pooling != GT_POOL_MAXMIN)
    return set_error(GT_EINVAL, "unknown pooling");
  const bool split = o.pooling == GT_POOL_MAXMIN;
  if (split && d > 1024) return set_error(GT_EINVAL, "GT_POOL_MAXMIN needs d <= 1024 (rows are 2d wide)");
  if (o.layout != GT_LAYOUT_TREE && o.layout != GT_LAYOUT_PREFIX)
    return set_error(GT_EINVAL, "unknown layout");
  const bool pre = o.layout == GT_LAYOUT_PREFIX;
  const int pc = o.prefix_level ? o.prefix_level : 3;
  if (pre) {
    if (o.pooling != GT_POOL_SUM)
      return set_error(GT_EINVAL, "the prefix layout holds sums: it needs GT_POOL_SUM");
    if (pc < 1 || pc > 12) return set_error(GT_EINVAL, "prefix_level must be in [1, 12]");
    if (o.formats & (1u << GT_FP8)) return set_error(GT_EINVAL, "the prefix layout keeps no FP8 rows");
    if (!dense_available()) return set_error(GT_EINVAL, "the prefix layout needs the dense GEMM path");
  }
  prepare_level_kernels();
  gt_tree *t = new gt_tree();
  t->N = N;
  // signed rows are stored split, [max(f, 0), max(-f, 0)]: 2d entries
  t->d_in = d;
  t->d = split ? 2 * d : d;
  t->split_sign = split;
  t->L = top_level(N);
  t->stride = ((int64_t)t->d + 63) / 64 * 64;
  if (pre) {
    // the formats of the prefix rows: BF16 always, FP32 on request
    t->formats = (1u << GT_BF16) | (o.formats & (1u << GT_F32));
    t->layout = GT_LAYOUT_PREFIX;
    t->pc = pc;
  } else {
    t->formats = (1u << GT_F32) | (o.formats ? o.formats : ((1u << GT_BF16) | (1u << GT_FP8)));
  }
  // split signed rows are pooled by element-wise maximum
  t->pooling = split ? GT_POOL_MAX : o.pooling;
  t->stream = (cudaStream_t)o.stream;
  int dev = 0;
  cudaGetDevice(&dev);
  t->device = dev;
  cudaDeviceGetAttribute(&t->sm_count, cudaDevAttrMultiProcessorCount, dev);
  t->sm_total = t->sm_count;
  if (t->sm_count <= 0) {
    delete t;
    return set_error(GT_ECUDA, "no CUDA device");
  }
  cudaStream_t s = t->stream;
  gt_status st = pre ? prefix_alloc(t, cap) : tree_alloc(t, cap);
  const void *Fd = nullptr;
  void *Ftmp = nullptr;
  int32_t *perm_dev = nullptr;
  int hflags[kFlagCount] = {0};
  if (st == GT_OK) st = to_device(F, (size_t)N * d * sizeof(float), s, &Fd, &Ftmp);
  if (st == GT_OK && o.perm) {
    std::vector<int32_t> p32((size_t)N);
    std::vector<char> seen((size_t)N, 0);
    for (int64_t i = 0; i < N; ++i) {
      const int64_t v = o.perm[i];
      if (v < 0 || v >= N || seen[(size_t)v]) {
        st = set_error(GT_EINVAL, "perm is not a permutation of 0..N-1");
        break;
      }
      seen[(size_t)v] = 1;
      p32[(size_t)i] = (int32_t)v;
    }
    if (st == GT_OK) {
      cudaError_t e = cudaMalloc(&perm_dev, (size_t)N * 4);
      if (e == cudaSuccess) e = cudaMemcpyAsync(perm_dev, p32.data(), (size_t)N * 4, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) st = cuda_error(e, "perm upload");
    }
  }
  if (st == GT_OK) st = tree_build_level0(t, (const float *)Fd, 0, N, perm_dev, s);
  if (st == GT_OK) st = read_flags(t, s, hflags);
  if (st == GT_OK && hflags[kFlagDomain])
    st = set_error(GT_EDOMAIN, split ? "F has a non-finite entry" : "F has a negative or non-finite entry");
  if (st == GT_OK) st = pre ? prefix_build(t, 0, N, s) : tree_build_levels(t, 0, N, s);
  if (st == GT_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_error(e, "build");
  }
  cudaFree(Ftmp);
  cudaFree(perm_dev);
  if (st != GT_OK) {
    gt_free(t);
    return st;
  }
  t->max_norm_dev = tree_norm_dev(t);
  *out = t;
  return GT_OK;
}

gt_status gt_insert(gt_tree *t, const float *f, int64_t n_new, void *stream) {
  TraceRange trace("gt_insert");
  if (!t) return set_error(GT_EINVAL, "null tree");
  if (n_new == 0) return GT_OK;
  if (!f || n_new < 0) return set_error(GT_EINVAL, "bad insert arguments");
  const int64_t N1 = t->N + n_new;
  if (N1 >= ((int64_t)1 << 31)) return set_error(GT_EINVAL, "tree would exceed 2^31 items");
  cudaStream_t s = stream ? (cudaStream_t)stream : t->stream;
  if (N1 > t->cap) {
    gt_status st = grow(t, std::max<int64_t>(N1, 2 * t->cap));
    if (st != GT_OK) return st;
  }
  // host rows go through the workspace's staging buffer (no allocation per call)
  const void *fd = f;
  gt_status st = GT_OK;
  if (!is_device_ptr(f)) {
    const int64_t bytes = n_new * t->d_in * (int64_t)sizeof(float);
    st = ws_stage(t, bytes);
    if (st != GT_OK) return st;
    GT_CUDA(cudaMemcpyAsync(t->ws.stage, f, (size_t)bytes, cudaMemcpyHostToDevice, s));
    fd = t->ws.stage;
  }
  cudaMemsetAsync(t->flags, 0, sizeof(int), s);
  st = tree_build_level0(t, (const float *)fd, t->N, n_new, nullptr, s);
  int hflags[kFlagCount] = {0};
  if (st == GT_OK) st = read_flags(t, s, hflags);
  if (st != GT_OK) return st;
  if (hflags[kFlagDomain])
    return set_error(GT_EDOMAIN, t->split_sign ? "inserted row has a non-finite entry"
                                               : "inserted row has a negative or non-finite entry");
  const int64_t first = t->N;
  t->N = N1;
  t->L = top_level(N1);
  st = t->layout == GT_LAYOUT_PREFIX ? prefix_build(t, first, n_new, s)
                                     : tree_build_levels(t, first, n_new, s);
  if (st != GT_OK) return st;
  GT_CUDA(cudaStreamSynchronize(s));
  return GT_OK;
}

static GraphEntry *find_graph(gt_tree *t, const GraphKey &k) {
  if (!t->graphs) return nullptr;
  for (auto &e : t->graphs->v)
    if (std::memcmp(&e.key, &k, sizeof(k)) == 0) return &e;
  return nullptr;
}

static GraphEntry *store_graph(gt_tree *t, GraphEntry &&e) {
  if (!t->graphs) t->graphs = new GraphCache();
  auto &v = t->graphs->v;
  if (v.size() >= 64) {  // keep the 64 most recent shapes (micro-batches)
    t->graphs->retired.push_back(std::move(v.front()));
    v.erase(v.begin());
  }
  v.push_back(std::move(e));
  return &v.back();
}

static gt_status run_search_on(gt_tree *t, const float *Q, int64_t B, const float *rho,
                               const gt_query_opts *opts, gt_csr *out, bool exhaustive,
                               cudaStream_t s);

// Work of a query call runs on the caller's stream, or - when that is the
// legacy default stream, which cannot be captured into a CUDA graph - on a
// non-blocking stream of the tree, ordered after the caller's stream by an
// event; the caller's stream then waits for the call's work.
static gt_status run_search(gt_tree *t, const float *Q, int64_t B, const float *rho,
                            const gt_query_opts *opts, gt_csr *out, bool exhaustive) {
  cudaStream_t user = (opts && opts->stream) ? (cudaStream_t)opts->stream : t->stream;
  if (user != nullptr && user != cudaStreamLegacy)
    return run_search_on(t, Q, B, rho, opts, out, exhaustive, user);
  if (!t->aux_stream) {
    GT_CUDA(cudaStreamCreateWithFlags(&t->aux_stream, cudaStreamNonBlocking));
    GT_CUDA(cudaEventCreateWithFlags(&t->aux_in, cudaEventDisableTiming));
    GT_CUDA(cudaEventCreateWithFlags(&t->aux_out, cudaEventDisableTiming));
  }
  GT_CUDA(cudaEventRecord(t->aux_in, user));
  GT_CUDA(cudaStreamWaitEvent(t->aux_stream, t->aux_in, 0));
  gt_status st = run_search_on(t, Q, B, rho, opts, out, exhaustive, t->aux_stream);
  cudaEventRecord(t->aux_out, t->aux_stream);
  cudaStreamWaitEvent(user, t->aux_out, 0);
  return st;
}

static gt_status run_search_on(gt_tree *t, const float *Q, int64_t B, const float *rho,
                               const gt_query_opts *opts, gt_csr *out, bool exhaustive,
                               cudaStream_t s) {
  TraceRange trace("gt_query");
  if (!t || !out) return set_error(GT_EINVAL, "null tree or output");
  std::memset(out, 0, sizeof(*out));
  if (B < 0) return set_error(GT_EINVAL, "negative query count");
  if (B > 0 && (!Q || !rho)) return set_error(GT_EINVAL, "null queries or thresholds");
  if (B >= ((int64_t)1 << 31)) return set_error(GT_EINVAL, "too many queries");
  gt_query_opts o;
  std::memset(&o, 0, sizeof(o));
  o.cutover = -1;
  if (opts) o = *opts;
  const int fmt = o.dtype;
  if (fmt < GT_F32 || fmt > GT_FP8) return set_error(GT_EINVAL, "unknown dtype");
  if (!(t->formats & (1u << fmt))) return set_error(GT_EINVAL, "tree does not keep this row format");
  gt_query_stats stats;
  std::memset(&stats, 0, sizeof(stats));
  stats.levels = t->L + 1;
  stats.cutover = -1;
  if (B == 0) {
    out->n_queries = 0;
    out->on_device = o.results_on_device;
    if (o.results_on_device) {
      GT_CUDA(cudaMalloc(&out->offsets, sizeof(int64_t)));
      GT_CUDA(cudaMemset(out->offsets, 0, sizeof(int64_t)));
      GT_CUDA(cudaMalloc(&out->ids, sizeof(int32_t)));
    } else {
      out->offsets = (int64_t *)std::calloc(1, sizeof(int64_t));
      out->ids = (int32_t *)std::calloc(1, sizeof(int32_t));
    }
    if (o.stats) *o.stats = stats;
    return GT_OK;
  }
  gt_status st = ws_reserve_queries(t, B);
  if (st != GT_OK) return st;
  // host inputs: page-locked ones are read in place by the preparation
  // kernel (over the CPU-GPU link, as part of the step: no separate copy);
  // pageable ones go through the workspace's staging buffer (no per-call
  // allocation)
  const void *Qd = Q, *rd = rho;
  bool q_host = !is_device_ptr(Q), r_host = !is_device_ptr(rho);
  if (q_host) {
    if (const void *p = pinned_device_view(Q)) {
      Qd = p;
      q_host = false;
    }
  }
  if (r_host) {
    if (const void *p = pinned_device_view(rho)) {
      rd = p;
      r_host = false;
    }
  }
  const int64_t qbytes = B * t->d_in * (int64_t)sizeof(float);
  const int64_t qpad = (qbytes + 255) / 256 * 256;
  if (q_host || r_host) {
    st = ws_stage(t, qpad + B * (int64_t)sizeof(float));
    if (st != GT_OK) return st;
    if (q_host) {
      GT_CUDA(cudaMemcpyAsync(t->ws.stage, Q, (size_t)qbytes, cudaMemcpyHostToDevice, s));
      Qd = t->ws.stage;
    }
    if (r_host) {
      char *dst = reinterpret_cast<char *>(t->ws.stage) + qpad;
      GT_CUDA(cudaMemcpyAsync(dst, rho, (size_t)B * sizeof(float), cudaMemcpyHostToDevice, s));
      rd = dst;
    }
  }
  // graphs evicted during this call are destroyed when it returns (after the
  // timer has read their events)
  struct RetiredGraphs {
    gt_tree *t;
    ~RetiredGraphs() {
      if (t->graphs) t->graphs->release_retired();
    }
  } retired_guard{t};
  KernelTimer tm;
  tm.on = o.timing != 0;
  tm.s = s;
  tm.pool = &event_pool(t);
  cudaMemsetAsync(t->flags, 0, kFlagCount * sizeof(int), s);
  tm.begin(5);
  launch_prep_queries(t, (const float *)Qd, (const float *)rd, B, s);
  tm.end();
  stats.launches += 1;
  // the input checks of the prep kernel are read at the first micro-batch's
  // sync (a bad input only makes the traversal prune or keep too much; no
  // list is written past its capacity)

  // level the traversal starts at, and whether a dense GEMM produces it
  int cut = -2;
  const bool pre = t->layout == GT_LAYOUT_PREFIX;
  if (pre) {
    // the dense GEMM scores the blocks' totals; the prefix splits do the rest
    if (exhaustive) return set_error(GT_EINVAL, "a prefix-layout tree keeps no BF16 item rows");
    if (o.cutover != -1 && o.cutover != t->pc)
      return set_error(GT_EINVAL, "a prefix-layout tree's dense level is its prefix_level");
    cut = t->pc;
  } else if (exhaustive) {
    if (t->split_sign)
      return set_error(GT_EINVAL, "a GT_POOL_MAXMIN tree decides items by a signed recheck: "
                                  "no exhaustive scan of its split rows");
    cut = 0;
  } else if (o.cutover >= 0) {
    if (o.cutover > t->L) return set_error(GT_EINVAL, "cutover above the root level");
    if (o.cutover == 0 && t->split_sign)
      return set_error(GT_EINVAL, "a GT_POOL_MAXMIN tree needs a cutover level >= 1");
    cut = o.cutover;
  } else if (o.cutover == -1) {
    // automatic: the level an earlier gt_autotune chose for this format, else
    // pools of 8 items (level 3), where the dense GEMM has absorbed the
    // levels in which few pools are pruned (Sec. 4 finds most rejections in
    // the last rounds)
    cut = -2;
    if (dense_available() && (t->formats & (1u << GT_BF16)) && t->L >= 6) {
      cut = t->tuned_cut[fmt] > 0 ? t->tuned_cut[fmt] : 3;
      cut = std::min(cut, t->L);
    }
  } else if (o.cutover != -2) {
    return set_error(GT_EINVAL, "bad cutover");
  }
  if (cut >= 0 && !dense_available()) return set_error(GT_EINVAL, "dense GEMM path not available");
  if (cut >= 0 && !(t->formats & (1u << GT_BF16)))
    return set_error(GT_EINVAL, "dense GEMM needs the tree's BF16 rows");
  stats.cutover = cut >= 0 ? cut : -1;
  prepare_level_kernels();
  // the subtraction path needs a dense cutover above level 1
  // (max pools: a parent is not the sum of its children, so no subtraction)
  // (the prefix layout's lists hold entries like the subtraction path's)
  const bool sub = pre || (cut >= 2 && t->pooling == GT_POOL_SUM &&
                           (o.subtract == 1 || (o.subtract == 0 && t->tuned_sub[fmt] != -1)));
  // with the subtraction path, the items are split the same way (right item
  // tested, left item bounded) where the ring-fed kernel's slots fit
  const bool items_sub = pre || (sub && items_sub_available(t, fmt));
  // every level below the cutover in one persistent launch (k_drain) when
  // the tree's tuning chose it
  const bool drain = !pre && sub && items_sub && t->tuned_g[fmt] == kInflightDrain &&
                     drain_available(t, fmt, cut);
  if (drain) {
    st = ws_reserve_drain(t);
    if (st != GT_OK) return st;
  }

  const int64_t budget = o.scratch_bytes > 0 ? o.scratch_bytes : default_budget();
  int64_t front_cap = std::max<int64_t>(1 << 10, budget * 7 / 10 / (2 * (int64_t)sizeof(Pair)));
  front_cap = std::min<int64_t>(front_cap, (int64_t)1 << 31);
  int64_t rchk_cap = std::max<int64_t>(1 << 14, front_cap / 16);
  int64_t res_cap = std::max<int64_t>(t->ws.res_cap, std::min<int64_t>(front_cap, B * 256));
  // the exhaustive scan's GEMM epilogue decides every item: it writes only the
  // result and recheck lists, so its frontier buffers stay at the minimum
  st = ws_reserve_frontier(t, exhaustive ? (1 << 10) : front_cap, res_cap, rchk_cap);
  if (st != GT_OK) return st;
  Workspace &w = t->ws;
  front_cap = std::min<int64_t>(front_cap, w.front_cap);
  w.front_lim = front_cap;

  int64_t bm = o.max_batch > 0 ? o.max_batch
                               : (exhaustive ? B : std::max<int64_t>(1, front_cap / 65536));
  bm = std::min(bm, B);
  if (!exhaustive) bm = std::min<int64_t>(bm, front_cap);  // the root list holds one pair per query
  uint32_t R = 0;  // results so far
  GT_CUDA(cudaMemsetAsync(w.counters, 0, 64 * sizeof(uint32_t), s));
  // the CSR output, assembled on the device behind the last micro-batch (its
  // result count is read there), so the host waits once at the end
  struct CsrBufs {
    int64_t *off = nullptr, *cnt = nullptr;
    int32_t *ids = nullptr;
    int64_t cap = -1;
    cudaStream_t s = nullptr;
    void release() {
      if (off) cudaFreeAsync(off, s);
      if (cnt) cudaFreeAsync(cnt, s);
      if (ids) cudaFreeAsync(ids, s);
      off = nullptr; cnt = nullptr; ids = nullptr; cap = -1;
    }
    ~CsrBufs() { release(); }
  } csr;
  csr.s = s;
  const int top = cut >= 0 ? cut : t->L;
  int64_t q0 = 0;
  while (q0 < B) {
    const int64_t b = std::min(bm, B - q0);
    TraceRange trace_mb("micro-batch");
    // everything one micro-batch does on the device, in stream order
    int64_t n_launch = 0, n_level = 0;
    auto enqueue = [&](KernelTimer &tmr) -> gt_status {
      t->ring_batch = ring_batch_for(b);
      GT_CUDA(cudaMemsetAsync(w.counters, 0, kMaxLevels * sizeof(uint32_t), s));
      GT_CUDA(cudaMemsetAsync(w.counters + kMaxLevels + 1, 0, sizeof(uint32_t), s));
      GT_CUDA(cudaMemsetAsync(t->flags + kFlagOverflow, 0, sizeof(int), s));
      int first_level;
      n_launch = 0;
      n_level = 0;
      if (cut < 0) {
        launch_root(t, q0, b, w.front[t->L & 1], w.counters + t->L, s);
        n_launch += 1;
        first_level = t->L;
      } else if (cut == 0) {
        tmr.begin(2);
        gt_status e = launch_dense(t, 0, 1, q0, b, nullptr, nullptr, s);
        tmr.end();
        if (e != GT_OK) return e;
        n_launch += 1;  // GEMM
        first_level = -1;  // the GEMM epilogue decided every item
      } else {
        tmr.begin(2);
        gt_status e = launch_dense(t, cut, sub ? 3 : 0, q0, b, w.front[cut & 1],
                                   w.counters + (cut - 1), s);
        tmr.end();
        if (e != GT_OK) return e;
        // group the GEMM's survivors by query for the level kernels
        tmr.begin(6);
        launch_bucket(t, sub, w.front[cut & 1], w.front[(cut - 1) & 1], w.counters + (cut - 1),
                      (uint32_t)(sub ? w.front_lim / 2 : w.front_lim), q0, b, s);
        tmr.end();
        n_launch += 5;  // GEMM + count, scan, scatter, count fix
        first_level = cut - 1;
      }
      if (drain) {
        // the GEMM's grouped level-(c-1) list is the work queue
        tmr.begin(0);
        launch_drain(t, fmt, cut, reinterpret_cast<const SibPair *>(w.front[(cut - 1) & 1]),
                     w.counters + (cut - 1), s);
        tmr.end();
        n_launch += 1;
        n_level += 1;
        first_level = -1;
      }
      for (int h = first_level; h >= 0; --h) {
        Pair *in = w.front[h & 1];
        Pair *outp = h > 0 ? w.front[(h - 1) & 1] : nullptr;
        tmr.begin(h > 0 ? 0 : 1);
        if (pre) {
          // entries of level-(h+1) pools in; kept level-h pools out, or at
          // h = 0 the items decided
          if (!launch_prefix(t, fmt, h + 1, reinterpret_cast<const SibPair *>(in), w.counters + h,
                             reinterpret_cast<SibPair *>(outp), h > 0 ? w.counters + h - 1 : nullptr, s))
            return set_error(GT_EINVAL, "FP32 prefix rows this wide do not fit the gather's "
                                        "shared-memory slots (d <= 1152 fits)");
        } else if (sub && h >= 1) {
          launch_level_sub(t, fmt, h, reinterpret_cast<const SibPair *>(in), w.counters + h, outp,
                           w.counters + h - 1, s, items_sub);
        } else if (sub && items_sub) {
          // the items: right items decided, left items by their bounds or,
          // when those straddle rho, from their rows in the same launch
          launch_items_sub(t, fmt, reinterpret_cast<const SibPair *>(in), w.counters,
                           w.counters + kLeftItemsSlot, s);
        } else {
          launch_level(t, fmt, h, q0, in, w.counters + h, outp, h > 0 ? w.counters + h - 1 : nullptr, s);
        }
        tmr.end();
        n_launch += 1;
        if (h > 0) n_level += 1;
      }
      if (drain && defer_active(t, fmt)) n_launch += 1;
      if (first_level >= 0 && defer_active(t, fmt)) n_launch += 1;
      tmr.begin(3);
      launch_recheck(t, q0, s);
      tmr.end();
      n_launch += 1;
      GT_CUDA(cudaGetLastError());
      GT_CUDA(cudaMemcpyAsync(w.hcounters, w.counters, 64 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
      GT_CUDA(cudaMemcpyAsync(w.hcounters + 64, t->flags, kFlagCount * sizeof(int), cudaMemcpyDeviceToHost, s));
      return GT_OK;
    };
    // replay a CUDA graph of this exact micro-batch if one was captured,
    // else capture one (falling back to direct launches if capture fails)
    GraphKey key;
    std::memset(&key, 0, sizeof(key));
    key.cut = cut; key.fmt = fmt; key.timing = tm.on ? 1 : 0;
    key.pad = (sub ? 1 : 0) | (t->expire_waits ? 2 : 0) | (t->sm_count << 8);
    key.tuned_g = t->tuned_g[fmt]; key.tuned_bn = t->tuned_bn;
    key.q0 = q0; key.b = b; key.N = t->N; key.front_lim = w.front_lim;
    key.res_cap = w.res_cap; key.rchk_cap = w.rchk_cap;
    const void *ptrs[] = {w.front[0], w.front[1], w.res, w.rchk, w.counters, w.hcounters, w.qf32,
                          w.qbf16, w.qn1, w.rho, w.bcnt, w.boff, w.defer,
                          t->rows32, t->rows16, t->rows8, t->scale8, t->perm, t->flags, s,
                          t->pref16, t->pref32};
    static_assert(sizeof(ptrs) / sizeof(ptrs[0]) <= sizeof(key.p) / sizeof(key.p[0]), "key");
    for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); ++i) key.p[i] = ptrs[i];
    GraphEntry *ge = o.no_graph ? nullptr : find_graph(t, key);
    if (ge) {
      GT_CUDA(cudaGraphLaunch(ge->exec, s));
      if (tm.on) tm.marks.insert(tm.marks.end(), ge->marks.begin(), ge->marks.end());
      n_launch = ge->launches;
      n_level = ge->level_launches;
      ++stats.graph_replays;
    } else if (!o.no_graph && t->graphs_ok) {
      GraphEntry fresh;
      KernelTimer gtm;
      gtm.on = tm.on;
      gtm.capturing = true;
      gtm.s = s;
      gtm.pool = &fresh.events;
      cudaGraph_t g = nullptr;
      cudaError_t ce = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
      if (ce == cudaSuccess) {
        st = enqueue(gtm);
        ce = cudaStreamEndCapture(s, &g);
        if (ce == cudaSuccess && (st != GT_OK || !g)) ce = cudaErrorStreamCaptureInvalidated;
      }
      if (ce == cudaSuccess) ce = cudaGraphInstantiate(&fresh.exec, g, 0);
      const bool ok = ce == cudaSuccess;
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      if (!ok)
        std::fprintf(stderr, "gt: CUDA graph capture failed (%s%s%s); launching directly\n",
                     cudaGetErrorString(ce), st != GT_OK ? ": " : "",
                     st != GT_OK ? g_err.c_str() : "");
      if (ok) {
        fresh.key = key;
        fresh.marks = gtm.marks;
        fresh.launches = n_launch;
        fresh.level_launches = n_level;
        ge = store_graph(t, std::move(fresh));
        GT_CUDA(cudaGraphLaunch(ge->exec, s));
        if (tm.on) tm.marks.insert(tm.marks.end(), ge->marks.begin(), ge->marks.end());
        ++stats.graph_captures;
      } else {
        // no graph for this tree from now on; run the launches directly
        for (cudaEvent_t e : fresh.events) cudaEventDestroy(e);
        if (fresh.exec) cudaGraphExecDestroy(fresh.exec);
        t->graphs_ok = false;
        st = enqueue(tm);
        if (st != GT_OK) return st;
      }
    } else {
      st = enqueue(tm);
      if (st != GT_OK) return st;
    }
    stats.launches += n_launch;
    stats.level_launches += n_level;
    if (q0 + b == B) {
      // the last micro-batch: enqueue the CSR assembly behind it
      if (csr.cap != w.res_cap) {
        csr.release();
        GT_CUDA(cudaMallocAsync((void **)&csr.off, (size_t)(B + 1) * sizeof(int64_t), s));
        GT_CUDA(cudaMallocAsync((void **)&csr.cnt, (size_t)(B + 1) * sizeof(int64_t), s));
        GT_CUDA(cudaMallocAsync((void **)&csr.ids, (size_t)std::max<int64_t>(w.res_cap, 1) * sizeof(int32_t), s));
        csr.cap = w.res_cap;
      }
      tm.begin(4);
      GT_CUDA(cudaMemsetAsync(csr.cnt, 0, (size_t)(B + 1) * sizeof(int64_t), s));
      launch_csr_into(t, w.res, (uint32_t)w.res_cap, w.counters + kMaxLevels, 0, B, csr.cnt, csr.off,
                      csr.ids, w.counters + kCsrListSlot, s);
      tm.end();
      GT_CUDA(cudaGetLastError());
      stats.launches += 6;
    }
    GT_CUDA(cudaStreamSynchronize(s));
    const uint32_t *hc = w.hcounters;
    if (hc[64 + kFlagDomain]) return set_error(GT_EDOMAIN, "Q has a negative or non-finite entry (non-finite only for a GT_POOL_MAXMIN tree)");
    if (hc[64 + kFlagRho]) return set_error(GT_EINVAL, "rho must satisfy 0 < rho <= 1");
    if (w.hcounters[64 + kFlagTimeout]) return set_error(GT_ETIMEOUT, "a bounded device wait expired");
    if (w.hcounters[64 + kFlagStray])
      return set_error(GT_ECUDA, "internal error: a list entry names a query outside its micro-batch");
    const int overflow = (int)w.hcounters[64 + kFlagOverflow];
    if (overflow) {
      ++stats.retries;
      // which list ran out?
      bool front_full = false;
      for (int h = 0; h < kMaxLevels; ++h)
        front_full |= hc[h] > (uint32_t)((sub && (h >= 1 || items_sub) && h != kLeftItemsSlot)
                                             ? front_cap / 2 : front_cap);
      front_full |= w.defer && hc[kDeferSlot] > (uint32_t)w.defer_cap;
      const bool res_full = hc[kMaxLevels] > (uint32_t)w.res_cap;
      const bool rchk_full = hc[kMaxLevels + 1] > (uint32_t)w.rchk_cap;
      // a list that overflowed and was reset within the micro-batch (the
      // deferred FP8 pairs are cleared between the two leaf passes) shows
      // no count above its capacity: shrink the micro-batch then too
      if (!res_full && !rchk_full) front_full = true;
      GT_CUDA(cudaMemcpyAsync(w.counters + kMaxLevels, &R, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
      if (res_full) {
        int64_t need = std::max<int64_t>(2 * w.res_cap, (int64_t)hc[kMaxLevels] + 1024);
        if (need >= ((int64_t)1 << 32)) return set_error(GT_EOVERFLOW, "result count exceeds 2^32");
        st = ws_reserve_frontier(t, w.front_cap, need, w.rchk_cap);
        if (st != GT_OK) return st;
      }
      if (rchk_full) {
        st = ws_reserve_frontier(t, w.front_cap, w.res_cap, std::max<int64_t>(2 * w.rchk_cap, hc[kMaxLevels + 1]));
        if (st != GT_OK) return st;
      }
      if (front_full) {
        if (b == 1) return set_error(GT_EOVERFLOW, "one query's frontier exceeds the scratch budget");
        bm = std::max<int64_t>(1, b / 2);
      }
      continue;
    }
    // success: account and adapt the micro-batch to the widest level seen
    uint32_t peak = 0;
    for (int h = 0; h <= top; ++h) {
      stats.level_tests[h] += hc[h];
      stats.gathered_tests += hc[h];
      peak = std::max(peak, hc[h]);
    }
    if (items_sub) {  // the left items tested after their right siblings
      stats.level_tests[0] += hc[kLeftItemsSlot];
      stats.gathered_tests += hc[kLeftItemsSlot];
      peak = std::max(peak, hc[kLeftItemsSlot]);
    }
    stats.rechecks += hc[kMaxLevels + 1];
    stats.micro_batches += 1;
    if (cut >= 0) stats.dense_tests += b * level_rows(t->N, cut);
    R = hc[kMaxLevels];
    q0 += b;
    if (o.max_batch <= 0 && peak > 0) {
      const double per_q = (double)peak / (double)b;
      bm = std::max<int64_t>(1, (int64_t)((double)front_cap / (1.5 * per_q)));
      bm = std::min<int64_t>(bm, front_cap);
    }
  }
  const double eb = entry_bytes(fmt);
  for (int h = 0; h <= top; ++h)
    stats.gathered_bytes += (double)stats.level_tests[h] * (t->d * eb + (fmt == GT_FP8 ? 4.0 : 0.0));
  stats.tests = stats.gathered_tests + stats.dense_tests;
  stats.results = R;
  stats.refines = w.hcounters[kMaxLevels + 2];
  out->n_queries = B;
  if (o.results_on_device) {
    out->offsets = csr.off;
    out->ids = csr.ids;
    out->on_device = 1;
    csr.off = nullptr;
    csr.ids = nullptr;
    csr.release();
  } else {
    int64_t *hoff = (int64_t *)std::malloc((size_t)(B + 1) * sizeof(int64_t));
    int32_t *hids = (int32_t *)std::malloc((size_t)std::max<uint32_t>(R, 1) * sizeof(int32_t));
    if (!hoff || !hids) {
      std::free(hoff);
      std::free(hids);
      return set_error(GT_ENOMEM, "host allocation of the result failed");
    }
    GT_CUDA(cudaMemcpyAsync(hoff, csr.off, (size_t)(B + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (R) GT_CUDA(cudaMemcpyAsync(hids, csr.ids, (size_t)R * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    csr.release();
    GT_CUDA(cudaStreamSynchronize(s));
    out->offsets = hoff;
    out->ids = hids;
    out->on_device = 0;
  }
  tm.collect(stats.kernel_ms);
  if (o.stats) *o.stats = stats;
  return GT_OK;
}

gt_status gt_query(gt_tree *t, const float *Q, int64_t B, const float *rho, const gt_query_opts *opts,
                   gt_csr *out) {
  return run_search(t, Q, B, rho, opts, out, false);
}

gt_status gt_query_into(gt_tree *t, const float *Q, int64_t B, const float *rho,
                        const gt_query_opts *opts, int64_t *offsets, int32_t *ids, int64_t ids_cap,
                        int64_t *n_results) {
  if (n_results) *n_results = 0;
  if (!t || !offsets || !n_results || (ids_cap > 0 && !ids) || ids_cap < 0)
    return set_error(GT_EINVAL, "null or bad output argument");
  gt_query_opts o;
  std::memset(&o, 0, sizeof(o));
  o.cutover = -1;
  if (opts) o = *opts;
  gt_query_stats stats;
  gt_query_stats *user_stats = o.stats;
  o.stats = &stats;
  o.results_on_device = 1;
  gt_csr csr;
  gt_status st = run_search(t, Q, B, rho, &o, &csr, false);
  if (user_stats && st == GT_OK) *user_stats = stats;
  if (st != GT_OK) return st;
  const int64_t R = stats.results;
  *n_results = R;
  if (R > ids_cap) {
    gt_csr_free(&csr);
    return set_error(GT_EOVERFLOW, "ids_cap is smaller than the number of neighbours "
                                   "(*n_results holds the count needed)");
  }
  cudaStream_t s = o.stream ? (cudaStream_t)o.stream : t->stream;
  cudaError_t e = cudaMemcpyAsync(offsets, csr.offsets, (size_t)(B + 1) * sizeof(int64_t),
                                  cudaMemcpyDefault, s);
  if (e == cudaSuccess && R > 0)
    e = cudaMemcpyAsync(ids, csr.ids, (size_t)R * sizeof(int32_t), cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  gt_csr_free(&csr);
  if (e != cudaSuccess) return cuda_error(e, "copying the results out");
  return GT_OK;
}

gt_status gt_exhaustive_tree(gt_tree *t, const float *Q, int64_t B, const float *rho,
                             const gt_query_opts *opts, gt_csr *out) {
  if (out) std::memset(out, 0, sizeof(*out));
  if (!dense_available()) return set_error(GT_EINVAL, "dense GEMM path not available");
  gt_query_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  o.dtype = GT_BF16;
  return run_search(t, Q, B, rho, &o, out, true);
}

gt_status gt_exhaustive(const float *F, int64_t N, int32_t d, const float *Q, int64_t B,
                        const float *rho, const gt_query_opts *opts, gt_csr *out) {
  TraceRange trace("gt_exhaustive");
  if (!out) return set_error(GT_EINVAL, "null output");
  std::memset(out, 0, sizeof(*out));
  if (!F) return set_error(GT_EINVAL, "null F");
  if (N < 1 || N >= ((int64_t)1 << 31)) return set_error(GT_EINVAL, "N must be in [1, 2^31)");
  if (d < 1 || d > 2048) return set_error(GT_EINVAL, "d must be in [1, 2048]");
  if (!dense_available()) return set_error(GT_EINVAL, "dense GEMM path not available");
  int dev = 0;
  GT_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(GT_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scan_mutex);
  gt_tree *x = nullptr;
  gt_status st = scan_context(dev, N, d, &x);
  if (st != GT_OK) return st;
  // the caller's rows, quantised into the context (FP32 master rows for the
  // FP64 recheck, BF16 rows for the GEMM) on the caller's stream
  cudaStream_t s = (opts && opts->stream) ? (cudaStream_t)opts->stream : nullptr;
  const void *Fd = F;
  if (!is_device_ptr(F)) {
    if (const void *p = pinned_device_view(F)) {
      Fd = p;  // page-locked host rows are read in place
    } else {
      const int64_t bytes = N * (int64_t)d * (int64_t)sizeof(float);
      st = ws_stage(x, bytes);
      if (st != GT_OK) return st;
      GT_CUDA(cudaMemcpyAsync(x->ws.stage, F, (size_t)bytes, cudaMemcpyHostToDevice, s));
      Fd = x->ws.stage;
    }
  }
  GT_CUDA(cudaMemsetAsync(x->flags, 0, kFlagCount * sizeof(int), s));
  st = tree_build_level0(x, (const float *)Fd, 0, N, nullptr, s);
  int hflags[kFlagCount] = {0};
  if (st == GT_OK) st = read_flags(x, s, hflags);
  if (st != GT_OK) return st;
  if (hflags[kFlagDomain]) return set_error(GT_EDOMAIN, "F has a negative or non-finite entry");
  gt_query_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  o.dtype = GT_BF16;
  return run_search(x, Q, B, rho, &o, out, true);
}

gt_status gt_dense_scores(gt_tree *t, const float *Q, int64_t B, int32_t level, float *scores,
                          void *stream) {
  if (!t || !Q || !scores || B < 1) return set_error(GT_EINVAL, "bad dense-score arguments");
  if (t->layout == GT_LAYOUT_PREFIX ? level != t->pc : (level < 0 || level > t->L))
    return set_error(GT_EINVAL, "level out of range");
  if (!dense_available()) return set_error(GT_EINVAL, "dense GEMM path not available");
  if (!(t->formats & (1u << GT_BF16))) return set_error(GT_EINVAL, "tree keeps no BF16 rows");
  cudaStream_t s = stream ? (cudaStream_t)stream : t->stream;
  gt_status st = ws_reserve_queries(t, B);
  if (st != GT_OK) return st;
  const void *Qd = Q;
  const int64_t qbytes = B * t->d_in * (int64_t)sizeof(float);
  const int64_t qpad = (qbytes + 255) / 256 * 256;
  st = ws_stage(t, qpad + B * (int64_t)sizeof(float));
  if (st != GT_OK) return st;
  if (!is_device_ptr(Q)) {
    GT_CUDA(cudaMemcpyAsync(t->ws.stage, Q, (size_t)qbytes, cudaMemcpyHostToDevice, s));
    Qd = t->ws.stage;
  }
  // thresholds are not used here; the preparation kernel wants valid ones
  std::vector<float> ones((size_t)B, 1.0f);
  float *rd = reinterpret_cast<float *>(reinterpret_cast<char *>(t->ws.stage) + qpad);
  GT_CUDA(cudaMemcpyAsync(rd, ones.data(), (size_t)B * sizeof(float), cudaMemcpyHostToDevice, s));
  GT_CUDA(cudaMemsetAsync(t->flags, 0, kFlagCount * sizeof(int), s));
  launch_prep_queries(t, (const float *)Qd, rd, B, s);
  int hflags[kFlagCount] = {0};
  st = read_flags(t, s, hflags);
  if (st != GT_OK) return st;
  if (hflags[kFlagDomain]) return set_error(GT_EDOMAIN, "Q has a negative or non-finite entry (non-finite only for a GT_POOL_MAXMIN tree)");
  const int64_t rows = level_rows(t->N, level);
  float *sd = scores;
  const bool host_out = !is_device_ptr(scores);
  if (host_out) GT_CUDA(cudaMallocAsync((void **)&sd, (size_t)B * rows * sizeof(float), s));
  st = launch_dense_impl(t, level, 2, 0, B, nullptr, nullptr, sd, rows, s);
  if (st == GT_OK && host_out)
    st = cudaMemcpyAsync(scores, sd, (size_t)B * rows * sizeof(float), cudaMemcpyDeviceToHost, s) ==
                 cudaSuccess
             ? GT_OK
             : set_error(GT_ECUDA, "copy of the scores failed");
  if (host_out) cudaFreeAsync(sd, s);
  GT_CUDA(cudaStreamSynchronize(s));
  if (st != GT_OK) return st;
  st = read_flags(t, s, hflags);
  if (st == GT_OK && hflags[kFlagTimeout]) return set_error(GT_ETIMEOUT, "dense GEMM wait expired");
  return st;
}

gt_status gt_pair_bounds(gt_tree *t, int32_t level, int32_t dtype, const float *Q, int64_t B,
                         const int32_t *pairs, int64_t n, float *out, void *stream) {
  if (!t || !Q || B < 1 || n < 0 || (n > 0 && (!pairs || !out)))
    return set_error(GT_EINVAL, "bad pair-bound arguments");
  if (t->layout == GT_LAYOUT_PREFIX) return set_error(GT_EINVAL, "not available for a prefix-layout tree");
  if (B >= ((int64_t)1 << 31)) return set_error(GT_EINVAL, "too many queries");
  if (level < 0 || level > t->L) return set_error(GT_EINVAL, "level out of range");
  if (dtype < GT_F32 || dtype > GT_FP8 || !(t->formats & (1u << dtype)))
    return set_error(GT_EINVAL, "tree does not keep this row format");
  if (n == 0) return GT_OK;
  cudaStream_t s = stream ? (cudaStream_t)stream : t->stream;
  gt_status st = ws_reserve_queries(t, B);
  if (st != GT_OK) return st;
  // staging: queries, thresholds (unused; the preparation wants valid ones),
  // pairs and scores, each 256-byte aligned
  auto pad = [](int64_t b) { return (b + 255) / 256 * 256; };
  const int64_t qbytes = B * t->d_in * (int64_t)sizeof(float);
  const int64_t o_rho = pad(qbytes), o_pairs = o_rho + pad(B * 4), o_out = o_pairs + pad(n * 8);
  st = ws_stage(t, o_out + pad(n * 12));
  if (st != GT_OK) return st;
  char *stg = reinterpret_cast<char *>(t->ws.stage);
  const void *Qd = Q;
  if (!is_device_ptr(Q)) {
    GT_CUDA(cudaMemcpyAsync(stg, Q, (size_t)qbytes, cudaMemcpyHostToDevice, s));
    Qd = stg;
  }
  std::vector<float> ones((size_t)B, 1.0f);
  GT_CUDA(cudaMemcpyAsync(stg + o_rho, ones.data(), (size_t)B * 4, cudaMemcpyHostToDevice, s));
  const int32_t *pd = pairs;
  if (!is_device_ptr(pairs)) {
    GT_CUDA(cudaMemcpyAsync(stg + o_pairs, pairs, (size_t)n * 8, cudaMemcpyHostToDevice, s));
    pd = reinterpret_cast<const int32_t *>(stg + o_pairs);
  }
  const bool host_out = !is_device_ptr(out);
  float *od = host_out ? reinterpret_cast<float *>(stg + o_out) : out;
  GT_CUDA(cudaMemsetAsync(t->flags, 0, kFlagCount * sizeof(int), s));
  launch_prep_queries(t, (const float *)Qd, reinterpret_cast<const float *>(stg + o_rho), B, s);
  launch_pair_bounds(t, dtype, level, pd, n, B, od, s);
  GT_CUDA(cudaGetLastError());
  if (host_out) GT_CUDA(cudaMemcpyAsync(out, od, (size_t)n * 12, cudaMemcpyDeviceToHost, s));
  int hflags[kFlagCount] = {0};
  st = read_flags(t, s, hflags);
  if (st != GT_OK) return st;
  if (hflags[kFlagDomain]) return set_error(GT_EDOMAIN, "Q has a negative or non-finite entry (non-finite only for a GT_POOL_MAXMIN tree)");
  return GT_OK;
}

gt_status gt_autotune(gt_tree *t, const float *Q, int64_t B, const float *rho, int32_t dtype,
                      void *stream, gt_autotune_result *out) {
  TraceRange trace("gt_autotune");
  if (!t || !Q || !rho || B < 1) return set_error(GT_EINVAL, "bad autotune arguments");
  const bool pre = t->layout == GT_LAYOUT_PREFIX;
  if (dtype < GT_F32 || dtype > GT_FP8 || !(t->formats & (1u << dtype)))
    return set_error(GT_EINVAL, "tree does not keep this row format");
  if (!dense_available() || !(t->formats & (1u << GT_BF16)) || (!pre && t->L < 2))
    return set_error(GT_EINVAL, "nothing to tune: no dense path for this tree");
  cudaStream_t s = stream ? (cudaStream_t)stream : t->stream;
  gt_autotune_result r;
  std::memset(&r, 0, sizeof(r));
  cudaEvent_t e0, e1;
  GT_CUDA(cudaEventCreate(&e0));
  GT_CUDA(cudaEventCreate(&e1));
  // device time of one batch at (cutover c, tests in flight g, tile width bn);
  // three runs, the best of the last two counts.  Each run starts with the L2
  // cache overwritten (a 256 MiB write, outside the timed events), as a step
  // after other work would: with the cache warm from the previous run, a
  // cutover whose pool rows about fit in L2 would look faster than it is.
  void *l2_flush = nullptr;
  const size_t flush_bytes = (size_t)256 << 20;
  if (cudaMalloc(&l2_flush, flush_bytes) != cudaSuccess) {
    cudaGetLastError();
    l2_flush = nullptr;
  }
  int cur_sub = -1;
  auto run = [&](int c, int g, int bn, float *ms_out) -> gt_status {
    t->tuned_g[dtype] = g;
    t->tuned_bn = bn;
    gt_query_opts o;
    std::memset(&o, 0, sizeof(o));
    o.stream = s;
    o.dtype = dtype;
    o.cutover = c;
    o.subtract = cur_sub;
    o.results_on_device = 1;
    float best_ms = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      gt_csr csr;
      if (l2_flush) cudaMemsetAsync(l2_flush, rep + 1, flush_bytes, s);
      cudaEventRecord(e0, s);
      gt_status st = run_search(t, Q, B, rho, &o, &csr, false);
      cudaEventRecord(e1, s);
      if (st != GT_OK) return st;
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      gt_csr_free(&csr);
      if (rep > 0) best_ms = std::min(best_ms, ms);
    }
    *ms_out = best_ms;
    return GT_OK;
  };
  const int cmax = std::min(t->L, 8);
  // in-flight codes: 1, 2, 4 tests per warp with the query in registers;
  // 9, 10, 12 the same with the query read through L1; 16 the ring-fed gather;
  // 32 the ring-fed gather in one persistent launch for every level below the
  // cutover (k_drain, subtraction path)
  const int gs[8] = {1, 2, 4, 9, 10, 12, 16, 32};
  // GEMM tiles: 128 queries x 128 pools, 128 x 256, 256 x 256 on one SM, 256 x
  // 256 on a pair of SMs (codes 128, 256, 512, 1024)
  const int bns[4] = {128, 256, 512, 1024};
  int best_c = 3, best_g = 0, best_bn = 256, best_sub = 0;
  float best = 1e30f;
  gt_status st = GT_OK;
  if (pre) {
    // the prefix layout fixes its dense level (prefix_level) and always splits
    // with the ring-fed gather: only the GEMM tile is free
    for (int bi = 0; bi < 4 && st == GT_OK; ++bi) {
      st = run(t->pc, 0, bns[bi], &r.ms_tile[bi]);
      if (st == GT_OK && r.ms_tile[bi] < best) {
        best = r.ms_tile[bi];
        best_bn = bns[bi];
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(l2_flush);
    if (st != GT_OK) {
      t->tuned_bn = 0;
      return st;
    }
    if (t->pc <= 8) r.ms_cutover[t->pc] = r.ms_tile[1];
    t->tuned_bn = best_bn;
    r.cutover = t->pc;
    r.inflight = kInflightRing;
    r.tile_n = best_bn;
    r.best_ms = best;
    r.subtract = 0;
    if (out) *out = r;
    return GT_OK;
  }
  // coordinate descent: cutover level with the direct and the subtraction
  // path, then tests in flight, then tile shape
  for (int c = 1; c <= cmax && st == GT_OK; ++c) {
    cur_sub = -1;
    st = run(c, 0, 256, &r.ms_cutover[c]);
    if (st == GT_OK && r.ms_cutover[c] < best) {
      best = r.ms_cutover[c];
      best_c = c;
      best_sub = 0;
    }
    if (st == GT_OK && c >= 2 && t->pooling == GT_POOL_SUM) {
      cur_sub = 1;
      st = run(c, 0, 256, &r.ms_cutover_sub[c]);
      if (st == GT_OK && r.ms_cutover_sub[c] < best) {
        best = r.ms_cutover_sub[c];
        best_c = c;
        best_sub = 1;
      }
    }
  }
  cur_sub = best_sub ? 1 : -1;
  for (int gi = 0; gi < 8 && st == GT_OK; ++gi) {
    st = run(best_c, gs[gi], 256, &r.ms_inflight[gi]);
    if (st == GT_OK && r.ms_inflight[gi] < best) {
      best = r.ms_inflight[gi];
      best_g = gs[gi];
    }
  }
  for (int bi = 0; bi < 4 && st == GT_OK; ++bi) {
    st = run(best_c, best_g, bns[bi], &r.ms_tile[bi]);
    if (st == GT_OK && r.ms_tile[bi] < best) {
      best = r.ms_tile[bi];
      best_bn = bns[bi];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(l2_flush);
  if (st != GT_OK) {
    t->tuned_g[dtype] = 0;
    t->tuned_bn = 0;
    return st;
  }
  t->tuned_sub[dtype] = best_sub ? 1 : -1;
  r.subtract = best_sub;
  t->tuned_cut[dtype] = best_c;
  t->tuned_g[dtype] = best_g;
  t->tuned_bn = best_bn;
  r.cutover = best_c;
  r.inflight = best_g;
  r.tile_n = best_bn;
  r.best_ms = best;
  if (out) *out = r;
  return GT_OK;
}

gt_status gt_set_tuning(gt_tree *t, int32_t dtype, int32_t cutover, int32_t inflight,
                        int32_t tile) {
  if (!t || dtype < GT_F32 || dtype > GT_FP8) return set_error(GT_EINVAL, "bad tuning arguments");
  if (t->layout == GT_LAYOUT_PREFIX && ((cutover > 0 && cutover != t->pc) || inflight > 0))
    return set_error(GT_EINVAL, "a prefix-layout tree's dense level is its prefix_level and its "
                                "splits always use the ring-fed gather: only the tile is tuned");
  if (cutover > t->L) return set_error(GT_EINVAL, "cutover above the root level");
  if (inflight > 0 && inflight != kInflightRing && inflight != kInflightDrain &&
      !((inflight & ~8) == 1 || (inflight & ~8) == 2 || (inflight & ~8) == 4))
    return set_error(GT_EINVAL, "tests in flight must be 1, 2 or 4 (plus 8 for the L1 query), "
                                "16 for the ring-fed gather, or 32 for one persistent launch "
                                "of every level");
  if (tile > 0 && tile != 128 && tile != 256 && tile != 512 && tile != 1024)
    return set_error(GT_EINVAL, "tile must be 128, 256, 512 or 1024");
  if (cutover >= 0) t->tuned_cut[dtype] = cutover;
  if (inflight >= 0) t->tuned_g[dtype] = inflight;
  if (tile >= 0) t->tuned_bn = tile;
  return GT_OK;
}

gt_status gt_read_rows(const gt_tree *t, int32_t level, int32_t dtype, int64_t first, int64_t count,
                       void *out, float *scales_out) {
  if (!t || !out) return set_error(GT_EINVAL, "null argument");
  if (t->layout == GT_LAYOUT_PREFIX) {
    // level 0: FP32 items; level c: BF16 block totals; -1: prefix rows
    const void *base = nullptr;
    if (level == 0 && dtype == GT_F32) base = t->rows32;
    else if (level == t->pc && dtype == GT_BF16) base = t->rows16;
    else if (level == -1 && dtype == GT_BF16) base = t->pref16;
    else if (level == -1 && dtype == GT_F32) base = t->pref32;
    if (!base) return set_error(GT_EINVAL, "level or format not kept by this prefix-layout tree");
    const int64_t rows = level == t->pc ? level_rows(t->N, level) : t->N;
    if (first < 0 || count < 0 || first + count > rows) return set_error(GT_EINVAL, "rows out of range");
    const int eb = entry_bytes(dtype);
    GT_CUDA(cudaMemcpy2D(out, (size_t)t->d * eb,
                         reinterpret_cast<const uint8_t *>(base) + (size_t)first * t->stride * eb,
                         (size_t)t->stride * eb, (size_t)t->d * eb, (size_t)count, cudaMemcpyDeviceToHost));
    return GT_OK;
  }
  if (level < 0 || level > t->L) return set_error(GT_EINVAL, "level out of range");
  if (first < 0 || count < 0 || first + count > level_rows(t->N, level))
    return set_error(GT_EINVAL, "rows out of range");
  if (dtype < GT_F32 || dtype > GT_FP8 || !(t->formats & (1u << dtype)))
    return set_error(GT_EINVAL, "format not kept");
  const int eb = entry_bytes(dtype);
  const uint8_t *base = dtype == GT_F32 ? (const uint8_t *)t->rows32
                        : dtype == GT_BF16 ? (const uint8_t *)t->rows16 : t->rows8;
  const size_t row0 = (size_t)(t->lvl_off[level] + first);
  GT_CUDA(cudaMemcpy2D(out, (size_t)t->d * eb, base + row0 * t->stride * eb, (size_t)t->stride * eb,
                       (size_t)t->d * eb, (size_t)count, cudaMemcpyDeviceToHost));
  if (scales_out && dtype == GT_FP8)
    GT_CUDA(cudaMemcpy(scales_out, t->scale8 + row0, (size_t)count * 4, cudaMemcpyDeviceToHost));
  return GT_OK;
}

gt_status gt_set_sm_limit(gt_tree *t, int32_t n) {
  if (!t) return set_error(GT_EINVAL, "null tree");
  if (n > 0 && n < 2) return set_error(GT_EINVAL, "an SM limit must be at least 2");
  t->sm_count = n > 0 ? std::min(n, t->sm_total) : t->sm_total;
  return GT_OK;
}

gt_status gt_set_wait_expiry(gt_tree *t, int32_t on) {
  if (!t) return set_error(GT_EINVAL, "null tree");
  t->expire_waits = on ? 1 : 0;
  return GT_OK;
}

gt_status gt_info(const gt_tree *t, gt_tree_info *out) {
  if (!t || !out) return set_error(GT_EINVAL, "null argument");
  std::memset(out, 0, sizeof(*out));
  out->n_items = t->N;
  out->capacity = t->cap;
  out->d = t->d_in;
  out->row_width = t->d;
  out->levels = t->L + 1;
  out->pooling = t->split_sign ? GT_POOL_MAXMIN : t->pooling;
  out->layout = t->layout;
  out->prefix_level = t->layout == GT_LAYOUT_PREFIX ? t->pc : 0;
  out->formats = t->formats;
  out->device = t->device;
  return GT_OK;
}

// Checkpoint file: this header, the tree permutation (N int32), then the
// stored item rows (N x row width FP32, tree order), all little-endian.
namespace {
struct CkptHeader {
  char magic[8];
  int64_t n, cap;
  int32_t d, d_in, pooling, layout, pc, split_sign;
  uint32_t formats;
  int32_t tuned_cut[3], tuned_g[3], tuned_bn, tuned_sub[3];
  int32_t reserved[5];
};
constexpr char kCkptMagic[8] = {'G', 'T', 'T', 'R', 'E', 'E', '1', 0};
constexpr int64_t kCkptChunkRows = 16384;

struct File {
  FILE *f = nullptr;
  ~File() {
    if (f) std::fclose(f);
  }
};
}  // namespace

gt_status gt_save(const gt_tree *t, const char *path) {
  if (!t || !path) return set_error(GT_EINVAL, "null argument");
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kCkptMagic, sizeof(h.magic));
  h.n = t->N;
  h.cap = t->cap;
  h.d = t->d;
  h.d_in = t->d_in;
  h.pooling = t->pooling;
  h.layout = t->layout;
  h.pc = t->pc;
  h.split_sign = t->split_sign ? 1 : 0;
  h.formats = t->formats;
  for (int i = 0; i < 3; ++i) {
    h.tuned_cut[i] = t->tuned_cut[i];
    h.tuned_g[i] = t->tuned_g[i];
    h.tuned_sub[i] = t->tuned_sub[i];
  }
  h.tuned_bn = t->tuned_bn;
  std::vector<int32_t> perm((size_t)t->N);
  GT_CUDA(cudaMemcpy(perm.data(), t->perm, (size_t)t->N * sizeof(int32_t), cudaMemcpyDeviceToHost));
  File f;
  f.f = std::fopen(path, "wb");
  if (!f.f) return set_error(GT_EINVAL, std::string("cannot open ") + path + ": " + std::strerror(errno));
  bool ok = std::fwrite(&h, sizeof(h), 1, f.f) == 1 &&
            std::fwrite(perm.data(), sizeof(int32_t), perm.size(), f.f) == perm.size();
  std::vector<float> rows;
  for (int64_t r0 = 0; ok && r0 < t->N; r0 += kCkptChunkRows) {
    const int64_t n = std::min<int64_t>(kCkptChunkRows, t->N - r0);
    rows.resize((size_t)n * t->d);
    GT_CUDA(cudaMemcpy2D(rows.data(), (size_t)t->d * sizeof(float), t->rows32 + (size_t)r0 * t->stride,
                         (size_t)t->stride * sizeof(float), (size_t)t->d * sizeof(float), (size_t)n,
                         cudaMemcpyDeviceToHost));
    ok = std::fwrite(rows.data(), sizeof(float), rows.size(), f.f) == rows.size();
  }
  if (!ok || std::fflush(f.f) != 0)
    return set_error(GT_EINVAL, std::string("cannot write ") + path + ": " + std::strerror(errno));
  return GT_OK;
}

gt_status gt_load(const char *path, void *stream, gt_tree **out) {
  if (!path || !out) return set_error(GT_EINVAL, "null argument");
  *out = nullptr;
  TraceRange trace("gt_load");
  File f;
  f.f = std::fopen(path, "rb");
  if (!f.f) return set_error(GT_EINVAL, std::string("cannot open ") + path + ": " + std::strerror(errno));
  CkptHeader h;
  if (std::fread(&h, sizeof(h), 1, f.f) != 1 || std::memcmp(h.magic, kCkptMagic, sizeof(h.magic)) != 0)
    return set_error(GT_EINVAL, std::string(path) + " is not a tree checkpoint");
  const bool pre = h.layout == GT_LAYOUT_PREFIX;
  if (h.n < 1 || h.cap < h.n || h.cap >= ((int64_t)1 << 31) || h.d < 1 || h.d > 2048 ||
      h.d_in < 1 || h.d != (h.split_sign ? 2 * h.d_in : h.d_in) ||
      (h.layout != GT_LAYOUT_TREE && !pre) || (h.pooling != GT_POOL_SUM && h.pooling != GT_POOL_MAX) ||
      (pre && (h.pc < 1 || h.pc > 12)))
    return set_error(GT_EINVAL, std::string(path) + ": inconsistent checkpoint header");
  std::vector<int32_t> perm((size_t)h.n);
  if (std::fread(perm.data(), sizeof(int32_t), perm.size(), f.f) != perm.size())
    return set_error(GT_EINVAL, std::string(path) + ": truncated checkpoint");
  prepare_level_kernels();
  gt_tree *t = new gt_tree();
  t->N = h.n;
  t->d = h.d;
  t->d_in = h.d_in;
  t->split_sign = h.split_sign != 0;
  t->L = top_level(h.n);
  t->stride = ((int64_t)t->d + 63) / 64 * 64;
  t->formats = h.formats;
  t->pooling = h.pooling;
  t->layout = h.layout;
  t->pc = pre ? h.pc : 0;
  for (int i = 0; i < 3; ++i) {
    t->tuned_cut[i] = h.tuned_cut[i];
    t->tuned_g[i] = h.tuned_g[i];
    t->tuned_sub[i] = h.tuned_sub[i];
  }
  t->tuned_bn = h.tuned_bn;
  t->stream = (cudaStream_t)stream;
  int dev = 0;
  cudaGetDevice(&dev);
  t->device = dev;
  cudaDeviceGetAttribute(&t->sm_count, cudaDevAttrMultiProcessorCount, dev);
  t->sm_total = t->sm_count;
  cudaStream_t s = t->stream;
  gt_status st = pre ? prefix_alloc(t, h.cap) : tree_alloc(t, h.cap);
  float *stage = nullptr;
  if (st == GT_OK) {
    cudaError_t e = cudaMalloc(&stage, (size_t)kCkptChunkRows * t->d * sizeof(float));
    if (e != cudaSuccess) st = cuda_error(e, "checkpoint staging");
  }
  std::vector<float> rows;
  for (int64_t r0 = 0; st == GT_OK && r0 < t->N; r0 += kCkptChunkRows) {
    const int64_t n = std::min<int64_t>(kCkptChunkRows, t->N - r0);
    rows.resize((size_t)n * t->d);
    if (std::fread(rows.data(), sizeof(float), rows.size(), f.f) != rows.size()) {
      st = set_error(GT_EINVAL, std::string(path) + ": truncated checkpoint");
      break;
    }
    cudaError_t e = cudaMemcpyAsync(stage, rows.data(), rows.size() * sizeof(float),
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      st = cuda_error(e, "checkpoint rows");
      break;
    }
    st = tree_build_level0(t, stage, r0, n, nullptr, s, true);
    if (st == GT_OK) {
      e = cudaStreamSynchronize(s);  // the host buffer is refilled next
      if (e != cudaSuccess) st = cuda_error(e, "checkpoint rows");
    }
  }
  int hflags[kFlagCount] = {0};
  if (st == GT_OK) st = read_flags(t, s, hflags);
  if (st == GT_OK && hflags[kFlagDomain])
    st = set_error(GT_EINVAL, std::string(path) + ": a stored row has a negative or non-finite entry");
  // the ids: the saved tree permutation (the level-0 pass wrote positions)
  if (st == GT_OK) {
    cudaError_t e = cudaMemcpyAsync(t->perm, perm.data(), perm.size() * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) st = cuda_error(e, "checkpoint permutation");
  }
  if (st == GT_OK) st = pre ? prefix_build(t, 0, t->N, s) : tree_build_levels(t, 0, t->N, s);
  if (st == GT_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_error(e, "checkpoint build");
  }
  cudaFree(stage);
  if (st != GT_OK) {
    gt_free(t);
    return st;
  }
  t->max_norm_dev = tree_norm_dev(t);
  *out = t;
  return GT_OK;
}

int64_t gt_size(const gt_tree *t) { return t ? t->N : 0; }
int32_t gt_dim(const gt_tree *t) { return t ? t->d_in : 0; }
int32_t gt_levels(const gt_tree *t) { return t ? t->L + 1 : 0; }

void gt_free(gt_tree *t) {
  if (!t) return;
  delete t->graphs;
  t->graphs = nullptr;
  if (t->aux_stream) {
    cudaStreamSynchronize(t->aux_stream);
    cudaStreamDestroy(t->aux_stream);
    cudaEventDestroy(t->aux_in);
    cudaEventDestroy(t->aux_out);
  }
  free_tree_storage(t);
  free_workspace(t);
  cudaFree(t->flags);
  delete t;
}

void gt_csr_free(gt_csr *c) {
  if (!c) return;
  if (c->on_device) {
    // allocated stream-ordered; the legacy stream orders the release after
    // the work of blocking streams
    cudaFreeAsync(c->offsets, 0);
    cudaFreeAsync(c->ids, 0);
  } else {
    std::free(c->offsets);
    std::free(c->ids);
  }
  std::memset(c, 0, sizeof(*c));
}

}  // extern "C"
