// Tree build and streaming insert: the pooled vectors of Sec. 2 (Eq. 1 gives
// the same pools as differences of cumulative sums; here each pool is a row).
//
// Level 0 row p is input row perm[p]; level h row j is fl32(level h-1 row 2j
// + level h-1 row 2j+1) (or the copy of row 2j when 2j+1 is past the end).
// Every row is written in FP32 and, when kept, in BF16 (round to nearest)
// and FP8 e4m3 with a power-of-two scale s = 2^e chosen so that max/s <= 448
// (so x/s and code*s are exact in FP32).  One warp per row, float4 traffic.
#include <algorithm>
#include <cstring>

#include "gt_internal.cuh"

namespace gt {

int top_level(int64_t n) {
  int L = 0;
  while (((int64_t)1 << L) < n) ++L;
  return L;
}

namespace {

struct RowsOut {
  float *r32;
  __nv_bfloat16 *r16;
  uint8_t *r8;
  float *s8;
  int64_t stride;  // entries per row, multiple of 64
  int max_pool;    // 1: a pool is the element-wise maximum of its children
};

// Row value layout in a warp: lane l holds float4 number (l + 32 k), k < KV4.
template <int KV4>
__device__ __forceinline__ void write_row(const RowsOut &o, int64_t row, const float4 (&v)[KV4],
                                          int nv4) {
  const int lane = threadIdx.x & 31;
  float4 *d32 = reinterpret_cast<float4 *>(o.r32 + row * o.stride);
  float mx = 0.f;
#pragma unroll
  for (int k = 0; k < KV4; ++k) {
    int i = lane + 32 * k;
    if (i < nv4) {
      d32[i] = v[k];
      mx = fmaxf(mx, fmaxf(fmaxf(v[k].x, v[k].y), fmaxf(v[k].z, v[k].w)));
    }
  }
  if (o.r16) {
    uint2 *d16 = reinterpret_cast<uint2 *>(o.r16 + row * o.stride);
#pragma unroll
    for (int k = 0; k < KV4; ++k) {
      int i = lane + 32 * k;
      if (i < nv4) {
        __nv_bfloat162 a = __floats2bfloat162_rn(v[k].x, v[k].y);
        __nv_bfloat162 b = __floats2bfloat162_rn(v[k].z, v[k].w);
        uint2 w;
        w.x = *reinterpret_cast<uint32_t *>(&a);
        w.y = *reinterpret_cast<uint32_t *>(&b);
        d16[i] = w;
      }
    }
  }
  if (o.r8) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    // scale 2^e with max / 2^e <= 448 = 0.875 * 2^9
    int E = 0;
    float m = frexpf(mx, &E);  // mx = m 2^E, m in [0.5, 1) (m = 0 for mx = 0)
    int e = (mx == 0.f) ? 0 : (m <= 0.875f ? E - 9 : E - 8);
    float inv = ldexpf(1.f, -e);
    uint32_t *d8 = reinterpret_cast<uint32_t *>(o.r8 + row * o.stride);
#pragma unroll
    for (int k = 0; k < KV4; ++k) {
      int i = lane + 32 * k;
      if (i < nv4) {
        __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(
            make_float2(v[k].x * inv, v[k].y * inv), __NV_SATFINITE, __NV_E4M3);
        __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(
            make_float2(v[k].z * inv, v[k].w * inv), __NV_SATFINITE, __NV_E4M3);
        d8[i] = (uint32_t)lo | ((uint32_t)hi << 16);
      }
    }
    if (lane == 0) o.s8[row] = ldexpf(1.f, e);
  }
}

// Entry j of a stored row built from input row `in` (d entries): the input
// entry itself, or with `split` (signed rows) entry j of [max(f, 0), max(-f, 0)]
// (2d entries); zero past the row.  `bad` records a non-finite input entry
// or, without split, a negative one.
__device__ __forceinline__ float row_entry(const float *in, int d, bool split, int j, bool &bad) {
  if (!split) {
    const float x = j < d ? __ldg(in + j) : 0.f;
    bad |= !(x >= 0.f) || !isfinite(x);
    return x;
  }
  if (j >= 2 * d) return 0.f;
  const float x = __ldg(in + (j < d ? j : j - d));
  bad |= !isfinite(x);
  return j < d ? (x > 0.f ? x : 0.f) : (x < 0.f ? -x : 0.f);
}

// Level 0: gather input rows (d contiguous floats each, any alignment), check
// the domain, pad to the row stride with zeros (signed rows: split first).
template <int KV4>
__global__ void __launch_bounds__(256) k_level0(const float *__restrict__ F, int64_t first,
                                                int64_t n, int d, int split,
                                                const int32_t *__restrict__ perm,
                                                int32_t *__restrict__ perm_out, RowsOut o,
                                                int *flags, unsigned *norm_dev_bits) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int nv4 = (int)(o.stride / 4);
  for (int64_t r = warp; r < n; r += nwarps) {
    const int64_t p = first + r;
    // with a permutation, F is the whole database; without, F holds the rows
    // for positions first..first+n-1 (a build or an insert batch)
    const int64_t src = perm ? (int64_t)perm[p] : r;
    const int64_t id = perm ? (int64_t)perm[p] : p;
    const float *in = F + src * (int64_t)d;
    float4 v[KV4];
    float ss = 0.f;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < KV4; ++k) {
      int i = lane + 32 * k;
      float x[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        int j = 4 * i + c;
        x[c] = i < nv4 ? row_entry(in, d, split != 0, j, bad) : 0.f;
        ss = fmaf(x[c], x[c], ss);
      }
      v[k] = make_float4(x[0], x[1], x[2], x[3]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicExch(&flags[kFlagDomain], 1);
    if (lane == 0) {
      float dev = fabsf(sqrtf(ss) - 1.f);
      atomicMax(norm_dev_bits, __float_as_uint(dev));
      perm_out[p] = (int32_t)id;
    }
    write_row<KV4>(o, p, v, nv4);
  }
}

// Level h >= 1, rows [j0, j1): fl32(child 2j + child 2j+1), or with max
// pooling max(child 2j, child 2j+1) element by element (exact).
template <int KV4>
__device__ __forceinline__ void sum_row(const RowsOut &o, int64_t child_base, int64_t child_rows,
                                        int64_t parent_base, int64_t j) {
  const int lane = threadIdx.x & 31;
  const int nv4 = (int)(o.stride / 4);
  const float4 *a = reinterpret_cast<const float4 *>(o.r32 + (child_base + 2 * j) * o.stride);
  const bool has_b = 2 * j + 1 < child_rows;
  const float4 *b = reinterpret_cast<const float4 *>(o.r32 + (child_base + 2 * j + 1) * o.stride);
  float4 v[KV4];
#pragma unroll
  for (int k = 0; k < KV4; ++k) {
    int i = lane + 32 * k;
    if (i < nv4) {
      float4 x = a[i];
      if (has_b) {
        float4 y = b[i];
        if (o.max_pool) {
          x.x = fmaxf(x.x, y.x); x.y = fmaxf(x.y, y.y); x.z = fmaxf(x.z, y.z); x.w = fmaxf(x.w, y.w);
        } else {
          x.x += y.x; x.y += y.y; x.z += y.z; x.w += y.w;
        }
      }
      v[k] = x;
    } else {
      v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  write_row<KV4>(o, parent_base + j, v, nv4);
}

template <int KV4>
__global__ void __launch_bounds__(256) k_level_sum(RowsOut o, int64_t child_base,
                                                   int64_t child_rows, int64_t parent_base,
                                                   int64_t j0, int64_t j1) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = j0 + warp; j < j1; j += nwarps) sum_row<KV4>(o, child_base, child_rows, parent_base, j);
}

// Several small levels in one block: level h rows [lo_h, hi_h) for h = h0..h1.
struct LevelRange {
  int64_t base[kMaxLevels + 1];
  int64_t rows[kMaxLevels + 1];  // rows present at each level (for the child test)
  int64_t lo[kMaxLevels + 1], hi[kMaxLevels + 1];
};

template <int KV4>
__global__ void __launch_bounds__(512) k_levels_small(RowsOut o, LevelRange lr, int h0, int h1) {
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int h = h0; h <= h1; ++h) {
    for (int64_t j = lr.lo[h] + warp; j < lr.hi[h]; j += nw)
      sum_row<KV4>(o, lr.base[h - 1], lr.rows[h - 1], lr.base[h], j);
    __syncthreads();  // level h is complete before level h+1 reads it
  }
}

// A short append (at most kChainRows rows to recompute at each of levels
// h0..h1): one block keeps each level's new FP32 rows in shared memory for the
// level above, and loads at the start, all at once, the rows it reads from
// memory: level h0-1's rows of the range and, for every level, the one
// existing row that can be a child of a new row (the left sibling of the
// range's first row, when that row is a right child).  A level is then a sum
// in shared memory and the rows' writes: the same sums, in the same order,
// as k_levels_small, without a dependent read from memory per level.
constexpr int kChainRows = 4;

template <int KV4>
__global__ void __launch_bounds__(256) k_levels_chain(RowsOut o, LevelRange lr, int h0, int h1) {
  extern __shared__ float4 chain_sm[];
  const int nv4 = (int)(o.stride / 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  float4 *prev = chain_sm;                       // 2 kChainRows rows
  float4 *cur = prev + 2 * kChainRows * nv4;     // kChainRows rows
  float4 *sib = cur + kChainRows * nv4;          // one row per level h0..h1
  const int n_first = (int)(lr.hi[h0 - 1] - lr.lo[h0 - 1]);
  const int n_lv = h1 - h0 + 1;
  for (int task = warp; task < n_first + n_lv; task += nw) {
    int64_t row;
    float4 *dst;
    if (task < n_first) {
      row = lr.base[h0 - 1] + lr.lo[h0 - 1] + task;
      dst = prev + (int64_t)task * nv4;
    } else {
      const int h = h0 + (task - n_first);
      const int64_t lo1 = lr.lo[h - 1];
      if ((lo1 & 1) == 0) continue;  // the first new row at h-1 is a left child
      row = lr.base[h - 1] + lo1 - 1;
      dst = sib + (int64_t)(h - h0) * nv4;
    }
    const float4 *src = reinterpret_cast<const float4 *>(o.r32 + row * o.stride);
    for (int i = lane; i < nv4; i += 32) dst[i] = src[i];
  }
  __syncthreads();
  for (int h = h0; h <= h1; ++h) {
    const int64_t lo1 = lr.lo[h - 1], rows1 = lr.rows[h - 1];
    const int n_cur = (int)(lr.hi[h] - lr.lo[h]);
    if (warp < n_cur) {
      const int64_t j = lr.lo[h] + warp;
      // child 2j always exists (j < rows at h); it is a new row of level h-1,
      // or (below the range) the loaded sibling; child 2j+1 may be missing
      const float4 *a = 2 * j >= lo1 ? prev + (2 * j - lo1) * nv4 : sib + (int64_t)(h - h0) * nv4;
      const bool has_b = 2 * j + 1 < rows1;
      const float4 *b = prev + (2 * j + 1 - lo1) * nv4;
      float4 v[KV4];
#pragma unroll
      for (int k = 0; k < KV4; ++k) {
        const int i = lane + 32 * k;
        if (i < nv4) {
          float4 x = a[i];
          if (has_b) {
            const float4 y = b[i];
            if (o.max_pool) {
              x.x = fmaxf(x.x, y.x); x.y = fmaxf(x.y, y.y); x.z = fmaxf(x.z, y.z); x.w = fmaxf(x.w, y.w);
            } else {
              x.x += y.x; x.y += y.y; x.z += y.z; x.w += y.w;
            }
          }
          v[k] = x;
          cur[(int64_t)warp * nv4 + i] = x;
        } else {
          v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      write_row<KV4>(o, lr.base[h] + j, v, nv4);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n_cur * nv4; t += blockDim.x) prev[t] = cur[t];
    __syncthreads();
  }
}

RowsOut rows_out(gt_tree *t) {
  RowsOut o;
  const bool pre = t->layout == GT_LAYOUT_PREFIX;  // rows16 holds pools there, not items
  o.r32 = t->rows32;
  o.r16 = pre ? nullptr : t->rows16;
  o.r8 = pre ? nullptr : t->rows8;
  o.s8 = t->scale8;
  o.stride = t->stride;
  o.max_pool = t->pooling == GT_POOL_MAX ? 1 : 0;
  return o;
}

int kv4_for(int64_t stride) {
  int need = (int)((stride / 4 + 31) / 32);
  int k = 1;
  while (k < need) k <<= 1;
  return k;
}

#define GT_DISPATCH_KV4(kv, ...)              \
  switch (kv) {                               \
    case 1: { constexpr int KV = 1; __VA_ARGS__; } break;   \
    case 2: { constexpr int KV = 2; __VA_ARGS__; } break;   \
    case 4: { constexpr int KV = 4; __VA_ARGS__; } break;   \
    case 8: { constexpr int KV = 8; __VA_ARGS__; } break;   \
    default: { constexpr int KV = 16; __VA_ARGS__; } break; \
  }

// Prefix layout: blocks [b0, b1) of 2^c items.  One warp per (block, 64
// columns): lane l keeps FP64 running sums of columns 2l and 2l+1 over the
// block's items in order, and writes after each item its prefix row (FP32
// round to nearest, BF16 by round to nearest of that FP32 value) and after
// the block's last item the block total as the level-c pool row (BF16).
__global__ void __launch_bounds__(256) k_prefix_rows(const float *items, int64_t stride, int64_t N,
                                                     int c, int64_t b0, int64_t b1,
                                                     __nv_bfloat16 *pref16, float *pref32,
                                                     __nv_bfloat16 *pool16) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t chunks = stride / 64;
  const int64_t work = (b1 - b0) * chunks;
  for (int64_t wi = warp; wi < work; wi += nwarps) {
    const int64_t blk = b0 + wi / chunks;
    const int64_t col = (wi % chunks) * 64 + 2 * lane;
    const int64_t first = blk << c;
    const int64_t last = min(first + ((int64_t)1 << c), N);
    double s0 = 0.0, s1 = 0.0;
    float2 v = make_float2(0.f, 0.f);
    for (int64_t i = first; i < last; ++i) {
      const float2 x = *reinterpret_cast<const float2 *>(items + i * stride + col);
      s0 += (double)x.x;
      s1 += (double)x.y;
      v = make_float2((float)s0, (float)s1);
      if (pref32) *reinterpret_cast<float2 *>(pref32 + i * stride + col) = v;
      *reinterpret_cast<__nv_bfloat162 *>(pref16 + i * stride + col) = __floats2bfloat162_rn(v.x, v.y);
    }
    *reinterpret_cast<__nv_bfloat162 *>(pool16 + blk * stride + col) = __floats2bfloat162_rn(v.x, v.y);
  }
}

}  // namespace

gt_status prefix_alloc(gt_tree *t, int64_t cap) {
  t->cap = cap;
  t->Lcap = top_level(cap);
  if (t->Lcap > kMaxLevels - 1) return set_error(GT_EINVAL, "capacity too large");
  for (int h = 0; h <= kMaxLevels; ++h) t->lvl_off[h] = 0;  // one level per array
  t->total_rows = cap;
  const size_t n = (size_t)cap * (size_t)t->stride;
  const size_t np = (size_t)level_rows(cap, t->pc) * (size_t)t->stride;
  GT_CUDA(cudaMalloc(&t->rows32, n * sizeof(float)));
  GT_CUDA(cudaMemsetAsync(t->rows32, 0, n * sizeof(float), t->stream));
  GT_CUDA(cudaMalloc(&t->pref16, n * 2));
  GT_CUDA(cudaMemsetAsync(t->pref16, 0, n * 2, t->stream));
  if (t->formats & (1u << GT_F32)) {
    GT_CUDA(cudaMalloc(&t->pref32, n * sizeof(float)));
    GT_CUDA(cudaMemsetAsync(t->pref32, 0, n * sizeof(float), t->stream));
  }
  GT_CUDA(cudaMalloc(&t->rows16, np * 2));
  GT_CUDA(cudaMemsetAsync(t->rows16, 0, np * 2, t->stream));
  GT_CUDA(cudaMalloc(&t->perm, (size_t)cap * sizeof(int32_t)));
  if (!t->flags) {
    GT_CUDA(cudaMalloc(&t->flags, 64 * sizeof(int)));
    GT_CUDA(cudaMemsetAsync(t->flags, 0, 64 * sizeof(int), t->stream));
  }
  return GT_OK;
}

gt_status prefix_build(gt_tree *t, int64_t first, int64_t n, cudaStream_t s) {
  if (n <= 0) return GT_OK;
  const int64_t b0 = first >> t->pc, b1 = ((first + n - 1) >> t->pc) + 1;
  const int64_t work = (b1 - b0) * (t->stride / 64);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((work + 7) / 8, (int64_t)t->sm_count * 16));
  k_prefix_rows<<<blocks, 256, 0, s>>>(t->rows32, t->stride, t->N, t->pc, b0, b1, t->pref16,
                                       t->pref32, t->rows16);
  GT_CUDA(cudaGetLastError());
  return GT_OK;
}

gt_status tree_alloc(gt_tree *t, int64_t cap) {
  t->cap = cap;
  t->Lcap = top_level(cap);
  if (t->Lcap > kMaxLevels - 1) return set_error(GT_EINVAL, "capacity too large");
  int64_t off = 0;
  for (int h = 0; h <= t->Lcap; ++h) {
    t->lvl_off[h] = off;
    off += level_rows(cap, h);
  }
  t->lvl_off[t->Lcap + 1] = off;
  t->total_rows = off;
  const size_t n = (size_t)off * (size_t)t->stride;
  GT_CUDA(cudaMalloc(&t->rows32, n * sizeof(float)));
  GT_CUDA(cudaMemsetAsync(t->rows32, 0, n * sizeof(float), t->stream));
  if (t->formats & (1u << GT_BF16)) {
    GT_CUDA(cudaMalloc(&t->rows16, n * 2));
    GT_CUDA(cudaMemsetAsync(t->rows16, 0, n * 2, t->stream));
  }
  if (t->formats & (1u << GT_FP8)) {
    GT_CUDA(cudaMalloc(&t->rows8, n));
    GT_CUDA(cudaMemsetAsync(t->rows8, 0, n, t->stream));
    GT_CUDA(cudaMalloc(&t->scale8, (size_t)off * sizeof(float)));
    GT_CUDA(cudaMemsetAsync(t->scale8, 0, (size_t)off * sizeof(float), t->stream));
  }
  GT_CUDA(cudaMalloc(&t->perm, (size_t)cap * sizeof(int32_t)));
  if (!t->flags) {
    GT_CUDA(cudaMalloc(&t->flags, 64 * sizeof(int)));
    GT_CUDA(cudaMemsetAsync(t->flags, 0, 64 * sizeof(int), t->stream));
  }
  return GT_OK;
}

gt_status tree_build_level0(gt_tree *t, const float *F_dev, int64_t first, int64_t n,
                            const int32_t *perm_dev, cudaStream_t s, bool stored_rows) {
  if (n <= 0) return GT_OK;
  RowsOut o = rows_out(t);
  // level-0 rows start at row 0; rows already in the stored form (a
  // checkpoint's) are t->d wide and are not split again
  const int kv = kv4_for(t->stride);
  unsigned *nb = reinterpret_cast<unsigned *>(t->flags + 32);
  int blocks = (int)std::min<int64_t>((n + 7) / 8, (int64_t)t->sm_count * 8);
  const int d_in = stored_rows ? t->d : t->d_in;
  const int split = (t->split_sign && !stored_rows) ? 1 : 0;
  GT_DISPATCH_KV4(kv, k_level0<KV><<<blocks, 256, 0, s>>>(F_dev, first, n, d_in, split, perm_dev,
                                                          t->perm, o, t->flags, nb));
  GT_CUDA(cudaGetLastError());
  return GT_OK;
}

// Recompute every pool of levels 1..L that covers items [first, first + n).
gt_status tree_build_levels(gt_tree *t, int64_t first, int64_t n, cudaStream_t s) {
  if (n <= 0 || t->L == 0) return GT_OK;
  RowsOut o = rows_out(t);
  const int kv = kv4_for(t->stride);
  LevelRange lr;
  for (int h = 0; h <= t->L; ++h) {
    lr.base[h] = t->lvl_off[h];
    lr.rows[h] = level_rows(t->N, h);
    lr.lo[h] = first >> h;
    lr.hi[h] = ((first + n - 1) >> h) + 1;
  }
  int h = 1;
  // big levels: one launch each
  for (; h <= t->L; ++h) {
    int64_t rows = lr.hi[h] - lr.lo[h];
    if (rows < 2048) break;
    int blocks = (int)std::min<int64_t>((rows + 7) / 8, (int64_t)t->sm_count * 8);
    GT_DISPATCH_KV4(kv, k_level_sum<KV><<<blocks, 256, 0, s>>>(o, lr.base[h - 1], lr.rows[h - 1],
                                                               lr.base[h], lr.lo[h], lr.hi[h]));
    GT_CUDA(cudaGetLastError());
  }
  // the remaining small levels: one block walks them in order (a short
  // append, with its rows and siblings in shared memory, when they fit)
  if (h <= t->L) {
    const int64_t row_bytes = t->stride * (int64_t)sizeof(float);
    const int64_t smem = (3 * kChainRows + (t->L - h + 1)) * row_bytes;
    static int smem_max = 0;
    if (!smem_max) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    }
    const bool chain = lr.hi[h] - lr.lo[h] <= kChainRows && lr.hi[h - 1] - lr.lo[h - 1] <= 2 * kChainRows &&
                       smem <= smem_max;
    if (chain) {
      GT_DISPATCH_KV4(kv, {
        static bool attr = false;
        if (!attr) {
          GT_CUDA(cudaFuncSetAttribute(k_levels_chain<KV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem_max));
          attr = true;
        }
        k_levels_chain<KV><<<1, 256, (size_t)smem, s>>>(o, lr, h, t->L);
      });
    } else {
      GT_DISPATCH_KV4(kv, k_levels_small<KV><<<1, 512, 0, s>>>(o, lr, h, t->L));
    }
    GT_CUDA(cudaGetLastError());
  }
  return GT_OK;
}

float tree_norm_dev(gt_tree *t) {
  unsigned bits = 0;
  cudaMemcpy(&bits, t->flags + 32, sizeof(unsigned), cudaMemcpyDeviceToHost);
  float f;
  std::memcpy(&f, &bits, sizeof(f));
  return f;
}

}  // namespace gt
