// Query traversal: Algorithm 1's binary splitting taken level by level (the
// "rounds" of Sec. 4), for a whole batch of queries at once.
//
// The frontier at level h is a list of (query, pool) pairs to test.  One warp
// tests one pair at a time: each lane loads 16-byte vectors of the pool row
// (streaming, no L1 allocation), multiplies them with the query entries it
// keeps in registers, and the warp sums the lanes.  A warp walks 32
// consecutive pairs, remembers which survived in a bit mask, and then writes
// the survivors' children (2j, 2j+1 at level h-1) with one atomic add and a
// warp prefix sum, so children of one query stay adjacent and the next level
// reloads the query rarely.  At level 0 the survivors are items: accepted
// outright when the lower bound clears rho, else queued for the FP64 recheck.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "gt_internal.cuh"

namespace gt {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ uint4 ld_stream(const void *p) {
  uint4 r;
  asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
      : "l"(p));
  return r;
}

template <int FMT>
struct RowFmt;
template <>
struct RowFmt<GT_F32> { static constexpr int EPV = 4; };
template <>
struct RowFmt<GT_BF16> { static constexpr int EPV = 8; };
template <>
struct RowFmt<GT_FP8> { static constexpr int EPV = 16; };

template <int FMT>
__device__ __forceinline__ float vdot(const uint4 w, const float *q, float acc);

template <>
__device__ __forceinline__ float vdot<GT_F32>(const uint4 w, const float *q, float acc) {
  acc = fmaf(__uint_as_float(w.x), q[0], acc);
  acc = fmaf(__uint_as_float(w.y), q[1], acc);
  acc = fmaf(__uint_as_float(w.z), q[2], acc);
  acc = fmaf(__uint_as_float(w.w), q[3], acc);
  return acc;
}

__device__ __forceinline__ float bf16x2_dot(uint32_t x, const float *q, float acc) {
  acc = fmaf(__uint_as_float(x << 16), q[0], acc);
  acc = fmaf(__uint_as_float(x & 0xffff0000u), q[1], acc);
  return acc;
}

template <>
__device__ __forceinline__ float vdot<GT_BF16>(const uint4 w, const float *q, float acc) {
  acc = bf16x2_dot(w.x, q + 0, acc);
  acc = bf16x2_dot(w.y, q + 2, acc);
  acc = bf16x2_dot(w.z, q + 4, acc);
  acc = bf16x2_dot(w.w, q + 6, acc);
  return acc;
}

__device__ __forceinline__ float fp8x4_dot(uint32_t x, const float *q, float acc) {
  __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(x & 0xffffu), __NV_E4M3);
  __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(x >> 16), __NV_E4M3);
  float2 a = __half22float2(*reinterpret_cast<__half2 *>(&lo));
  float2 b = __half22float2(*reinterpret_cast<__half2 *>(&hi));
  acc = fmaf(a.x, q[0], acc);
  acc = fmaf(a.y, q[1], acc);
  acc = fmaf(b.x, q[2], acc);
  acc = fmaf(b.y, q[3], acc);
  return acc;
}

template <>
__device__ __forceinline__ float vdot<GT_FP8>(const uint4 w, const float *q, float acc) {
  acc = fp8x4_dot(w.x, q + 0, acc);
  acc = fp8x4_dot(w.y, q + 4, acc);
  acc = fp8x4_dot(w.z, q + 8, acc);
  acc = fp8x4_dot(w.w, q + 12, acc);
  return acc;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
  return v;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    uint32_t t = __shfl_up_sync(FULL, v, off);
    if (lane >= off) v += t;
  }
  return v;
}

// Append `n` (0..2) pairs per lane to list `out` with one atomic per warp.
// A list that runs past its capacity raises the overflow flag; the pairs
// below the capacity are still written, so it has no hole below it (the next
// pass reads min(count, cap) pairs; the call then retries with fewer queries).
__device__ __forceinline__ void warp_append(Pair *out, uint32_t *count, uint32_t cap, int *flags,
                                            uint32_t n, Pair a, Pair b) {
  const uint32_t incl = warp_incl_scan(n);
  const uint32_t tot = __shfl_sync(FULL, incl, 31);
  if (tot == 0) return;
  uint32_t base = 0;
  if ((threadIdx.x & 31) == 0) base = atomicAdd(count, tot);
  base = __shfl_sync(FULL, base, 0);
  if (n == 0) return;
  const uint32_t pos = base + incl - n;
  if ((uint64_t)pos + n > cap) {
    atomicExch(&flags[kFlagOverflow], 1);
    if (pos < cap) out[pos] = a;   // n == 2 with only the first below the capacity
    return;
  }
  out[pos] = a;
  if (n == 2) out[pos + 1] = b;
}

struct LevelArgs {
  const uint8_t *rows;   // row 0 of this level in the gathered format
  const float *scales;   // FP8 scales of this level (else null)
  int64_t row_bytes;
  int nvec;              // 16-byte vectors covering d entries
  uint32_t n_child;      // rows at level h-1
  const float *qf32;
  int64_t qstride;
  const float *qn1;
  const float *rho;
  const Pair *in;
  const uint32_t *in_count;
  uint32_t in_cap;
  Pair *out;
  uint32_t *out_count;
  uint32_t out_cap;
  Pair *res;
  uint32_t *res_count;
  uint32_t res_cap;
  Pair *rchk;
  uint32_t *rchk_count;
  uint32_t rchk_cap;
  int *flags;
  Bound bd;
  const float *rows32;   // level-0 FP32 rows (leaf refine)
  Bound bd32;            // FP32 bound at level 0
  const __nv_bfloat16 *rows16;  // level-0 BF16 rows (first refine of FP8 leaves; may be null)
  Bound bd16;            // BF16 bound at level 0
  uint32_t *refine_count;
  int inflight;          // tests in flight per warp (0: the format's default)
  uint32_t n_rows;       // rows at this level (subtraction path: the right child may be missing)
  uint32_t batch;        // k_ring: pairs a warp takes at a time (8, 16 or 32)
  uint32_t q_lim;        // query rows of the workspace: an entry's query is below it
  Pair *defer;           // FP8 leaves: straddling pairs go here for the BF16 pass
  uint32_t *defer_count; //   (null: re-scored from the BF16 row in the same warp)
  uint32_t defer_cap;
  // prefix layout (k_ring modes 5, 6): the entries' pools are at level pre_h
  // inside blocks of 2^pre_c of the n_items items; a score at a block's end
  // is the dense GEMM's, bounded by g_cl * s <= exact <= g_cu * s
  uint32_t pre_h, pre_c, n_items;
  float g_cu, g_cl;
  // split signed rows (GT_POOL_MAXMIN): a leaf's score bounds q.f from above
  // only, so every leaf that the bound keeps goes to the signed FP64 recheck
  int no_accept;
  // failure-detection test (gt_set_wait_limit): the ring kernels start no
  // copy, and their first bounded wait gives up at once
  int expire;
};

// A list entry naming a query or a row outside its buffers can only come from
// a corrupted list: the kernel replaces its indices by valid ones, so that it
// reads nothing outside its buffers, and raises kFlagStray when it exits; the
// call then fails with an error and none of its results are used.
__device__ __forceinline__ bool entry_ok(const LevelArgs &a, uint32_t q, uint32_t row) {
  return q < a.q_lim && row < a.n_rows;
}

__device__ __forceinline__ void raise_stray(const LevelArgs &a, bool stray) {
  if (__any_sync(FULL, stray) && (threadIdx.x & 31) == 0) atomicExch(&a.flags[kFlagStray], 1);
}

// Query entries 4e..4e+3 of 16-byte row vector v (EPV entries): from the
// registers the warp loaded (QL1 = false), or read through L1 from the
// padded FP32 query row (QL1 = true: fewer registers, more warps per SM).
template <int EPV, bool QL1>
__device__ __forceinline__ float4 qchunk(const float *qreg, const float4 *qrow, int k, int v, int e) {
  if (QL1) return __ldg(qrow + v * (EPV / 4) + e);
  return make_float4(qreg[k * EPV + 4 * e + 0], qreg[k * EPV + 4 * e + 1],
                     qreg[k * EPV + 4 * e + 2], qreg[k * EPV + 4 * e + 3]);
}

template <int FMT, int KV, bool QL1>
__device__ __forceinline__ float row_dot(const uint4 (&w)[KV], const float *qreg,
                                         const float4 *qrow, int nvec) {
  constexpr int EPV = RowFmt<FMT>::EPV;
  const int lane = threadIdx.x & 31;
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < KV; ++k) {
    if (QL1) {
      const int v = lane + 32 * k;
      if (v < nvec) {
        float qv[EPV];
#pragma unroll
        for (int e = 0; e < EPV / 4; ++e) {
          const float4 x = qchunk<EPV, true>(qreg, qrow, k, v, e);
          qv[4 * e] = x.x; qv[4 * e + 1] = x.y; qv[4 * e + 2] = x.z; qv[4 * e + 3] = x.w;
        }
        acc = vdot<FMT>(w[k], qv, acc);
      }
    } else {
      acc = vdot<FMT>(w[k], &qreg[k * EPV], acc);
    }
  }
  return acc;
}

// Bounds of one tested pair from its (all-reduced) accumulator: U at or
// above and Lo at or below the exact score of the row's pool (the prune and
// the accept tests; the constants are make_bound's, the FP8 scale and the
// e4m3 subnormal term applied here).
template <int FMT>
__device__ __forceinline__ void test_bounds_scaled(const LevelArgs &a, float acc, float sc, float qn1,
                                                   float &U, float &Lo) {
  float tq = 0.f;
  if (FMT == GT_FP8) {
    acc *= sc;                      // exact: sc is a power of two
    tq = sc * 0x1p-10f * qn1;       // half the e4m3 subnormal spacing, times |q|_1
  }
  U = fmaf(acc, a.bd.cu, tq * a.bd.ct_up);
  Lo = (acc * a.bd.cl - tq * a.bd.ct_lo) * (1.f - 0x1p-22f);
}

// The same with row j's FP8 scale read here.
template <int FMT>
__device__ __forceinline__ void test_bounds(const LevelArgs &a, float acc, uint32_t j, float qn1,
                                            float &U, float &Lo) {
  test_bounds_scaled<FMT>(a, acc, FMT == GT_FP8 ? a.scales[j] : 1.f, qn1, U, Lo);
}

// FP32 re-score of item row j with the query entries the warp holds (the
// same entries of the FP32 master row): 0 when the FP32 bound prunes it, 1
// when it accepts it, 2 when the score is still within the bound of rho.
template <int FMT, int KV, bool QL1>
__device__ __forceinline__ int refine32(const LevelArgs &a, uint32_t j, float rho, const float *qreg,
                                        const float4 *qrow) {
  constexpr int EPV = RowFmt<FMT>::EPV;
  const int lane = threadIdx.x & 31;
  const float4 *r32 = reinterpret_cast<const float4 *>(a.rows32 + (size_t)j * a.qstride);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < KV; ++k) {
    const int v = lane + 32 * k;
    if (v < a.nvec) {
#pragma unroll
      for (int e = 0; e < EPV / 4; ++e) {
        const float4 x = r32[v * (EPV / 4) + e];
        const float4 y = qchunk<EPV, QL1>(qreg, qrow, k, v, e);
        s = fmaf(x.x, y.x, s);
        s = fmaf(x.y, y.y, s);
        s = fmaf(x.z, y.z, s);
        s = fmaf(x.w, y.w, s);
      }
    }
  }
  s = warp_sum(s);
  if (s * a.bd32.cu < rho) return 0;
  return s * a.bd32.cl * (1.f - 0x1p-22f) >= rho ? 1 : 2;
}

// Re-score leaf item j whose low-precision bound straddles rho, warp-wide,
// with the query entries the warp holds: from its BF16 row first for an FP8
// tree keeping BF16 rows (half the bytes of the FP32 row; its bound is 16
// times tighter than FP8's), then from the FP32 master row.  0 pruned, 1
// accepted, 2 still within the FP32 bound of rho (FP64 recheck).
template <int FMT, int KV, bool QL1>
__device__ __forceinline__ int leaf_rescore(const LevelArgs &a, uint32_t j, float rho,
                                            const float *qreg, const float4 *qrow,
                                            uint32_t &n_refine) {
  constexpr int EPV = RowFmt<FMT>::EPV;
  const int lane = threadIdx.x & 31;
  if (FMT == GT_FP8 && !QL1 && a.rows16) {
    // this lane's FP8 vector v holds entries 16v .. 16v+15, two BF16 vectors
    // of the item's BF16 row (the row is padded to the stride, so the second
    // of the last pair stays in it)
    const uint4 *r16 = reinterpret_cast<const uint4 *>(a.rows16 + (size_t)j * a.qstride);
    float s16 = 0.f;
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      const int v = lane + 32 * k;
      if (v < a.nvec) {
        s16 = vdot<GT_BF16>(r16[2 * v], &qreg[k * EPV], s16);
        s16 = vdot<GT_BF16>(r16[2 * v + 1], &qreg[k * EPV + 8], s16);
      }
    }
    s16 = warp_sum(s16);
    ++n_refine;
    if (s16 * a.bd16.cu < rho) return 0;
    if (s16 * a.bd16.cl * (1.f - 0x1p-22f) >= rho) return 1;
  }
  // FP32 refine: the same entries of the FP32 master row
  ++n_refine;
  return refine32<FMT, KV, QL1>(a, j, rho, qreg, qrow);
}

// Decide one tested pair from its (all-reduced) accumulator.  Sets bit `bit`
// of m_pass (kept / accepted) or m_rchk (FP64 recheck).  At the leaves a
// score whose low-precision bound straddles rho is first re-scored in FP32
// from the FP32 item row with the query entries already in registers; only
// a score still within the FP32 bound of rho goes to the FP64 recheck.
template <int FMT, int KV, bool LEAF, bool QL1>
__device__ __forceinline__ void decide(const LevelArgs &a, float acc, uint32_t j, float qn1,
                                       float rho, const float *qreg, const float4 *qrow, int bit,
                                       uint32_t &m_pass, uint32_t &m_rchk, uint32_t &m_defer,
                                       uint32_t &n_refine) {
  constexpr int EPV = RowFmt<FMT>::EPV;
  float U, Lo;
  test_bounds<FMT>(a, acc, j, qn1, U, Lo);
  if (U < rho) return;
  if (!LEAF) {
    m_pass |= 1u << bit;
    return;
  }
  if (a.no_accept) {
    m_rchk |= 1u << bit;
    return;
  }
  if (Lo >= rho) {
    m_pass |= 1u << bit;
    return;
  }
  if (FMT == GT_F32) {
    m_rchk |= 1u << bit;
    return;
  }
  if (FMT == GT_FP8 && !QL1 && a.rows16 && a.defer) {
    // re-scored from the BF16 row by the pass after this kernel (its rows
    // prefetched like any other gather, not waited for here)
    m_defer |= 1u << bit;
    ++n_refine;
    return;
  }
  const int r = leaf_rescore<FMT, KV, QL1>(a, j, rho, qreg, qrow, n_refine);
  if (r == 1)
    m_pass |= 1u << bit;
  else if (r == 2)
    m_rchk |= 1u << bit;
}

// One warp per (query, pool) test.  A warp takes 32 consecutive pairs; runs
// of up to G consecutive pairs of the same query are tested together (their
// row loads issued back to back, their sums reduced interleaved), which keeps
// G rows in flight per warp.
template <int FMT, int KV, bool LEAF, int G, bool QL1>
__global__ void __launch_bounds__(256) k_level(const LevelArgs a) {
  constexpr int EPV = RowFmt<FMT>::EPV;
  const int lane = threadIdx.x & 31;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  const uint32_t n = min(*a.in_count, a.in_cap);
  float qreg[QL1 ? 1 : KV * EPV];
  const float4 *qrow = nullptr;
  uint32_t cur_q = 0xffffffffu;
  float qn1 = 0.f, rho = 0.f;
  uint32_t n_refine = 0;
  bool stray = false;
  for (uint32_t base = gw * 32; base < n; base += nw * 32) {
    const uint32_t idx = base + lane;
    Pair pr;
    if (idx < n) {
      pr = a.in[idx];
      if (!entry_ok(a, pr.q, pr.j)) {
        stray = true;
        pr.q = 0;
        pr.j = 0;
      }
    } else {
      pr.q = 0xffffffffu;
      pr.j = 0;
    }
    const int cnt = (int)min(32u, n - base);
    uint32_t m_pass = 0, m_rchk = 0, m_defer = 0;
    int i = 0;
    while (i < cnt) {
      const uint32_t q = __shfl_sync(FULL, pr.q, i);
      // length of the run of pairs i, i+1, ... that share query q (<= G)
      const uint32_t same = __ballot_sync(FULL, pr.q == q && lane < cnt);
      const uint32_t tail = ~(same >> i);
      const int run = tail ? __ffs(tail) - 1 : 32 - i;
      const int g = min(run, G);
      if (q != cur_q) {
        cur_q = q;
        qrow = reinterpret_cast<const float4 *>(a.qf32 + (size_t)q * a.qstride);
        if (!QL1) {
#pragma unroll
          for (int k = 0; k < KV; ++k) {
            const int v = lane + 32 * k;
#pragma unroll
            for (int e = 0; e < EPV / 4; ++e) {
              float4 x = v < a.nvec ? qrow[v * (EPV / 4) + e] : make_float4(0.f, 0.f, 0.f, 0.f);
              qreg[k * EPV + 4 * e + 0] = x.x;
              qreg[k * EPV + 4 * e + 1] = x.y;
              qreg[k * EPV + 4 * e + 2] = x.z;
              qreg[k * EPV + 4 * e + 3] = x.w;
            }
          }
        }
        qn1 = a.qn1[q];
        rho = a.rho[q];
      }
      if (g == G) {
        uint32_t j[G];
        uint4 w[G][KV];
#pragma unroll
        for (int u = 0; u < G; ++u) {
          j[u] = __shfl_sync(FULL, pr.j, i + u);
          const uint8_t *row = a.rows + (size_t)j[u] * a.row_bytes;
#pragma unroll
          for (int k = 0; k < KV; ++k) {
            const int v = lane + 32 * k;
            w[u][k] = v < a.nvec ? ld_stream(row + 16 * v) : make_uint4(0u, 0u, 0u, 0u);
          }
        }
        float acc[G];
#pragma unroll
        for (int u = 0; u < G; ++u) acc[u] = row_dot<FMT, KV, QL1>(w[u], qreg, qrow, a.nvec);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
          for (int u = 0; u < G; ++u) acc[u] += __shfl_xor_sync(FULL, acc[u], off);
        }
#pragma unroll
        for (int u = 0; u < G; ++u)
          decide<FMT, KV, LEAF, QL1>(a, acc[u], j[u], qn1, rho, qreg, qrow, i + u, m_pass, m_rchk,
                                     m_defer, n_refine);
        i += G;
      } else {
        const uint32_t j = __shfl_sync(FULL, pr.j, i);
        const uint8_t *row = a.rows + (size_t)j * a.row_bytes;
        uint4 w[KV];
#pragma unroll
        for (int k = 0; k < KV; ++k) {
          const int v = lane + 32 * k;
          w[k] = v < a.nvec ? ld_stream(row + 16 * v) : make_uint4(0u, 0u, 0u, 0u);
        }
        float acc = row_dot<FMT, KV, QL1>(w, qreg, qrow, a.nvec);
        acc = warp_sum(acc);
        decide<FMT, KV, LEAF, QL1>(a, acc, j, qn1, rho, qreg, qrow, i, m_pass, m_rchk, m_defer, n_refine);
        i += 1;
      }
    }
    const bool mine = (m_pass >> lane) & 1u;
    if (!LEAF) {
      const uint32_t c0 = 2u * pr.j;
      const uint32_t nch = mine ? (1u + (c0 + 1u < a.n_child ? 1u : 0u)) : 0u;
      Pair x, y;
      x.q = pr.q; x.j = c0;
      y.q = pr.q; y.j = c0 + 1u;
      warp_append(a.out, a.out_count, a.out_cap, a.flags, nch, x, y);
    } else {
      warp_append(a.res, a.res_count, a.res_cap, a.flags, mine ? 1u : 0u, pr, pr);
      const bool rc = (m_rchk >> lane) & 1u;
      warp_append(a.rchk, a.rchk_count, a.rchk_cap, a.flags, rc ? 1u : 0u, pr, pr);
      if (FMT == GT_FP8 && __any_sync(FULL, m_defer != 0u))
        warp_append(a.defer, a.defer_count, a.defer_cap, a.flags, (m_defer >> lane) & 1u, pr, pr);
    }
  }
  raise_stray(a, stray);
  if (LEAF && n_refine && lane == 0) atomicAdd(a.refine_count, n_refine);
}

// Subtraction path, one entry's test: from the right child's accumulator,
// its upper bound Ur and the left child's bound Ul = Up - L_right (rounded up).
template <int FMT>
__device__ __forceinline__ void sub_test(const LevelArgs &a, float acc, uint32_t r, float qn1,
                                         float Up, float &Ul, float &Ur, float &Lr) {
  test_bounds<FMT>(a, acc, r, qn1, Ur, Lr);
  // The last row of a level is the one pool an insert can extend after its
  // parent's bound was taken (a server group keeps the tree of its admission
  // while later steps append items): its current row would bound the grown
  // pool, not the one under the parent, so it is not subtracted.
  if (r + 1u >= a.n_rows) Lr = 0.f;
  Ul = __fsub_ru(Up, fmaxf(Lr, 0.f));
}

// Subtraction path, the children's lower bounds.  The tested (right) child
// keeps its own row's lower bound Lr, except when that row is the level's last
// (the one pool an insert can extend while a served group still holds the
// entry: the current row may then hold members the entry's pool lacks).  The
// other child's exact score is the parent's minus the tested child's, so
// Ll = L_parent - U_right (rounded down) bounds it from below; with no right
// child the left child is the parent's whole pool.  0 is a valid lower bound
// of every (non-negative) score and accepts nothing.
__device__ __forceinline__ void sub_lower(float Lp, bool has_r, bool r_last, float Ur, float Lr_row,
                                          float &Ll, float &Lr) {
  Ll = has_r ? fmaxf(__fsub_rd(Lp, Ur), 0.f) : Lp;
  Lr = (has_r && !r_last) ? fmaxf(Lr_row, 0.f) : 0.f;
}

// Subtraction path, a warp's output: lane i holds entry e of its batch;
// bit i of m_left / m_right says whether that entry's children survive, with
// bounds my_ul / my_ur (upper) and my_ll / my_lr (lower).  Survivors become
// entries for the next level, or at the leaves the item pairs of the
// surviving level-1 pools.
template <bool TO_LEAF>
__device__ __forceinline__ void sub_emit(const LevelArgs &a, void *out_v, const SibPair &e,
                                         uint32_t m_left, uint32_t m_right, float my_ul,
                                         float my_ur, float my_ll, float my_lr) {
  const int lane = threadIdx.x & 31;
  const bool kl = (m_left >> lane) & 1u, kr = (m_right >> lane) & 1u;
  const uint32_t c_l = 2u * e.p, c_r = 2u * e.p + 1u;
  if (TO_LEAF) {
    // the items of each surviving level-1 pool c: 2c and 2c+1 (if present)
    const uint32_t nl = kl ? 1u + (2u * c_l + 1u < a.n_child ? 1u : 0u) : 0u;
    const uint32_t nr = kr ? 1u + (2u * c_r + 1u < a.n_child ? 1u : 0u) : 0u;
    const uint32_t tot = nl + nr;
    const uint32_t incl = warp_incl_scan(tot);
    const uint32_t all = __shfl_sync(FULL, incl, 31);
    if (all) {
      uint32_t b0 = 0;
      if (lane == 0) b0 = atomicAdd(a.out_count, all);
      b0 = __shfl_sync(FULL, b0, 0);
      uint32_t pos = b0 + incl - tot;
      Pair *out = reinterpret_cast<Pair *>(out_v);
      if (tot) {
        // past the capacity: the overflow flag, and only the pairs below it
        // written (no hole below the capacity)
        if ((uint64_t)pos + tot > a.out_cap) atomicExch(&a.flags[kFlagOverflow], 1);
        const uint32_t cap = a.out_cap;
        Pair x;
        x.q = e.q;
        if (kl) {
          x.j = 2u * c_l;
          if (pos < cap) out[pos] = x;
          ++pos;
          if (2u * c_l + 1u < a.n_child) { x.j = 2u * c_l + 1u; if (pos < cap) out[pos] = x; ++pos; }
        }
        if (kr) {
          x.j = 2u * c_r;
          if (pos < cap) out[pos] = x;
          ++pos;
          if (2u * c_r + 1u < a.n_child) { x.j = 2u * c_r + 1u; if (pos < cap) out[pos] = x; ++pos; }
        }
      }
    }
  } else {
    const uint32_t tot = (kl ? 1u : 0u) + (kr ? 1u : 0u);
    const uint32_t incl = warp_incl_scan(tot);
    const uint32_t all = __shfl_sync(FULL, incl, 31);
    if (all) {
      uint32_t b0 = 0;
      if (lane == 0) b0 = atomicAdd(a.out_count, all);
      b0 = __shfl_sync(FULL, b0, 0);
      uint32_t pos = b0 + incl - tot;
      SibPair *out = reinterpret_cast<SibPair *>(out_v);
      if (tot) {
        if ((uint64_t)pos + tot > a.out_cap) atomicExch(&a.flags[kFlagOverflow], 1);
        SibPair x;
        x.q = e.q;
        if (kl) {
          x.p = c_l; x.U = my_ul; x.pad = __float_as_uint(my_ll);
          if (pos < a.out_cap) out[pos] = x;
          ++pos;
        }
        if (kr) {
          x.p = c_r; x.U = my_ur; x.pad = __float_as_uint(my_lr);
          if (pos < a.out_cap) out[pos] = x;
        }
      }
    }
  }
}

// Prefix layout, a warp's output: lane i holds entry e = {q, pool p, prefix
// score at p's start (U field), at p's end (pad bits)} and in my_mid the
// prefix score at p's midpoint; bit i of m_left / m_right says whether child
// 2p / 2p+1 is kept.  Each kept child is written with its own two endpoint
// scores.
__device__ __forceinline__ void pre_emit(const LevelArgs &a, void *out_v, const SibPair &e,
                                         uint32_t m_left, uint32_t m_right, float my_mid) {
  const int lane = threadIdx.x & 31;
  const bool kl = (m_left >> lane) & 1u, kr = (m_right >> lane) & 1u;
  const uint32_t tot = (kl ? 1u : 0u) + (kr ? 1u : 0u);
  const uint32_t incl = warp_incl_scan(tot);
  const uint32_t all = __shfl_sync(FULL, incl, 31);
  if (!all) return;
  uint32_t b0 = 0;
  if (lane == 0) b0 = atomicAdd(a.out_count, all);
  b0 = __shfl_sync(FULL, b0, 0);
  uint32_t pos = b0 + incl - tot;
  SibPair *out = reinterpret_cast<SibPair *>(out_v);
  if (!tot) return;
  if ((uint64_t)pos + tot > a.out_cap) atomicExch(&a.flags[kFlagOverflow], 1);
  SibPair x;
  x.q = e.q;
  if (kl) {
    x.p = 2u * e.p; x.U = e.U; x.pad = __float_as_uint(my_mid);
    if (pos < a.out_cap) out[pos] = x;
    ++pos;
  }
  if (kr) {
    x.p = 2u * e.p + 1u; x.U = my_mid; x.pad = e.pad;
    if (pos < a.out_cap) out[pos] = x;
  }
}

// Subtraction path, level h >= 1.  Entry (q, p, U_p): the children of parent
// p (level h+1) are pools 2p and 2p+1 at level h.  The right child is tested;
// the left child's exact score is the parent's minus the right's, so
//   s_left <= U_p - L_right      (rounded up)
// bounds it without gathering its row (Algorithm 1 tests the right half and
// takes the left half as sim - rsim).  A missing right child means the left
// child has the parent's members: U_left = U_p.  Survivors are passed on as
// entries for level h-1, or, at h = 1, as the item pairs of the leaf level.
template <int FMT, int KV, bool TO_LEAF>
__global__ void __launch_bounds__(256) k_level_sub(const LevelArgs a, const SibPair *in,
                                                   void *out_v) {
  constexpr int EPV = RowFmt<FMT>::EPV;
  const int lane = threadIdx.x & 31;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  const uint32_t n = min(*a.in_count, a.in_cap);
  float qreg[KV * EPV];
  uint32_t cur_q = 0xffffffffu;
  float qn1 = 0.f, rho = 0.f;
  bool stray = false;
  for (uint32_t base = gw * 32; base < n; base += nw * 32) {
    const uint32_t idx = base + lane;
    SibPair e;
    if (idx < n) {
      e = in[idx];
      if (!entry_ok(a, e.q, 2u * e.p)) {  // the left child is always a row
        stray = true;
        e.q = 0; e.p = 0;
      }
    } else {
      e.q = 0xffffffffu; e.p = 0; e.U = 0.f; e.pad = 0;
    }
    const int cnt = (int)min(32u, n - base);
    float my_ul = 0.f, my_ur = 0.f;   // bounds of this lane's entry's children
    float my_ll = 0.f, my_lr = 0.f;
    uint32_t m_left = 0, m_right = 0;
    for (int i = 0; i < cnt; ++i) {
      const uint32_t q = __shfl_sync(FULL, e.q, i);
      const uint32_t p = __shfl_sync(FULL, e.p, i);
      const float Up = __shfl_sync(FULL, e.U, i);
      const float Lp = __uint_as_float(__shfl_sync(FULL, e.pad, i));
      if (q != cur_q) {
        cur_q = q;
        const float4 *qrow = reinterpret_cast<const float4 *>(a.qf32 + (size_t)q * a.qstride);
#pragma unroll
        for (int k = 0; k < KV; ++k) {
          const int v = lane + 32 * k;
#pragma unroll
          for (int c = 0; c < EPV / 4; ++c) {
            float4 x = v < a.nvec ? qrow[v * (EPV / 4) + c] : make_float4(0.f, 0.f, 0.f, 0.f);
            qreg[k * EPV + 4 * c + 0] = x.x;
            qreg[k * EPV + 4 * c + 1] = x.y;
            qreg[k * EPV + 4 * c + 2] = x.z;
            qreg[k * EPV + 4 * c + 3] = x.w;
          }
        }
        qn1 = a.qn1[q];
        rho = a.rho[q];
      }
      const uint32_t r = 2u * p + 1u;
      float Ul = Up, Ur = 0.f, Lr = 0.f;
      const bool has_r = r < a.n_rows;
      if (has_r) {
        const uint8_t *row = a.rows + (size_t)r * a.row_bytes;
        uint4 w[KV];
#pragma unroll
        for (int k = 0; k < KV; ++k) {
          const int v = lane + 32 * k;
          w[k] = v < a.nvec ? ld_stream(row + 16 * v) : make_uint4(0u, 0u, 0u, 0u);
        }
        float acc = row_dot<FMT, KV, false>(w, qreg, nullptr, a.nvec);
        acc = warp_sum(acc);
        sub_test<FMT>(a, acc, r, qn1, Up, Ul, Ur, Lr);
      }
      if (Ul >= rho) m_left |= 1u << i;
      if (has_r && Ur >= rho) m_right |= 1u << i;
      if (lane == i) {
        my_ul = Ul;
        my_ur = Ur;
        sub_lower(Lp, has_r, r + 1u >= a.n_rows, Ur, Lr, my_ll, my_lr);
      }
    }
    sub_emit<TO_LEAF>(a, out_v, e, m_left, m_right, my_ul, my_ur, my_ll, my_lr);
  }
  raise_stray(a, stray);
}

// ---- Ring-fed gather --------------------------------------------------------
// The level kernels above keep one row (or G rows) in registers per warp, so
// the rows an SM has in flight are bounded by its resident warps and their
// registers.  k_ring keeps them in shared memory instead: every warp owns a
// ring of `depth` row slots and, while it tests pair t, the row of its pair
// t + depth is already on its way into a slot by a bulk asynchronous copy
// (cp.async.bulk, completing on the slot's mbarrier).  Like k_level, a warp
// takes 32 consecutive pairs at a time, so on a query-grouped list it reloads
// its query rarely and its output stays grouped.  Each warp alone fills and
// drains its slots, so no warp waits on another (a warp that stalls, say on a
// query reload, delays only itself) and a slot's barrier is never waited on
// more than one phase ahead.  Every wait is bounded (1 s); on expiry the
// kernel raises the timeout flag, lets the copies it issued land and returns.
constexpr int kRingWarps = 24;               // warps per block, one block per SM
constexpr int kRingMaxDepth = 8;             // slots per warp at most
constexpr uint64_t kRingWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t ring_now() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void ring_bar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void ring_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void ring_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool ring_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// wait for the phase of parity `parity` of `bar`; false after limit_ns
__device__ __forceinline__ bool ring_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  if (ring_test(bar, parity)) return true;
  const uint64_t t0 = ring_now();
  while (!ring_test(bar, parity)) {
    if (ring_now() - t0 > limit_ns) return false;
  }
  return true;
}

__device__ __forceinline__ void ring_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// MODE 0: frontier level (pairs in, children out); 1: leaves (pairs in,
// results and rechecks out); 2: subtraction level (entries in and out); 3:
// subtraction into the leaves (entries in, item pairs out); 4: subtraction
// at the items (entries of level-1 pools in: the right item is decided like
// a leaf, results and rechecks out; the left item is accepted on its lower
// bound, the pool's minus the right item's upper bound, or else, while its
// upper bound reaches rho, gathered and decided like a leaf in the same
// launch); 5: prefix split (entries {q, pool, prefix score at
// the pool's start, at its end} in, the kept children out as entries); 6:
// prefix split of level-1 pools (both items decided: results and rechecks
// out).  In modes 5 and 6 the gathered row is the prefix row that ends at the
// pool's midpoint, and each child scores as a difference of prefix scores.
template <int FMT, int KV, int MODE>
__global__ void __launch_bounds__(32 * kRingWarps, 1)
    k_ring(const LevelArgs a, const void *in_v, void *out_v, uint32_t depth, uint32_t slot_bytes) {
  constexpr int EPV = RowFmt<FMT>::EPV;
  constexpr bool PRE = MODE >= 5;
  constexpr bool SUB = MODE >= 2 && !PRE;
  constexpr bool LEAF = MODE == 1 || MODE == 4 || MODE == 6;
  constexpr uint32_t kNoRow = 0xffffffffu;
  extern __shared__ __align__(128) uint8_t ring_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t sbase = (smem_addr(ring_raw) + 127u) & ~127u;
  const uint8_t *gbase = ring_raw + (sbase - smem_addr(ring_raw));
  // this warp's slots and their barriers
  const uint32_t slot0 = sbase + (uint32_t)warp * depth * slot_bytes;
  const uint8_t *gslot0 = gbase + (size_t)warp * depth * slot_bytes;
  const uint32_t full0 = sbase + kRingWarps * depth * slot_bytes + (uint32_t)warp * depth * 8u;
  const uint32_t n = min(*a.in_count, a.in_cap);
  const uint32_t bw = a.batch;  // 8, 16 or 32 (>= depth: a refill reaches the next batch at most)
  const uint32_t copy_bytes = (uint32_t)a.nvec * 16u;
  if (lane == 0) {
    for (uint32_t k = 0; k < depth; ++k) ring_bar_init(full0 + 8u * k, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const Pair *inp = reinterpret_cast<const Pair *>(in_v);
  const SibPair *ins = reinterpret_cast<const SibPair *>(in_v);
  const uint32_t gw = blockIdx.x * kRingWarps + (uint32_t)warp;
  const uint32_t nw = gridDim.x * kRingWarps;
  // the warp's batches: pairs [bw b, bw b + bw) for b = gw, gw + nw, ...
  // (bw = a.batch: 32, or 16 or 8 for small lists, which then spread over
  // more warps);
  // lane i holds pair i of a batch, as an entry (q, pool, U); the row to
  // gather is the pool (pairs) or its right child (entries)
  bool stray = false;
  auto load_batch = [&](uint32_t b, SibPair &e, uint32_t &row) {
    const uint32_t idx = bw * b + (uint32_t)lane;
    row = kNoRow;
    if ((uint64_t)bw * b >= n || (uint32_t)lane >= bw || idx >= n) {
      e.q = 0xffffffffu; e.p = 0; e.U = 0.f; e.pad = 0;
      return;
    }
    if (PRE) {
      e = ins[idx];
      if (!entry_ok(a, e.q, e.p)) {
        stray = true;
        e.q = 0; e.p = 0;
      }
      // the prefix row ending at the midpoint; none when the pool has no
      // right half (the left half is then the whole pool)
      const uint32_t mid = (e.p << a.pre_h) + (1u << (a.pre_h - 1u));
      if (mid < a.n_items) row = mid - 1u;
    } else if (SUB) {
      e = ins[idx];
      if (!entry_ok(a, e.q, 2u * e.p)) {  // the left child is always a row
        stray = true;
        e.q = 0; e.p = 0;
      }
      // MODE 4 reads the bounds again after the batch (fewer registers held
      // across the loop)
      if (MODE == 4) { e.U = 0.f; e.pad = 0; }
      const uint32_t r = 2u * e.p + 1u;
      if (r < a.n_rows) row = r;
    } else {
      const Pair x = inp[idx];
      e.q = x.q; e.p = x.j; e.U = 0.f; e.pad = 0;
      if (!entry_ok(a, e.q, e.p)) {
        stray = true;
        e.q = 0; e.p = 0;
      }
      row = e.p;
    }
  };
  // lane 0 starts the copy of `row` into slot k (or completes the slot's
  // phase without one when the entry has no row to gather)
  auto issue = [&](uint32_t k, uint32_t row) {
    if (lane != 0) return;
    if (row != kNoRow) {
      ring_expect(full0 + 8u * k, copy_bytes);
      ring_copy(slot0 + k * slot_bytes, a.rows + (size_t)row * a.row_bytes, copy_bytes, full0 + 8u * k);
    } else {
      ring_arrive(full0 + 8u * k);
    }
  };
  auto batch_len = [&](uint32_t b) -> uint32_t {
    return (uint64_t)bw * b < n ? min(bw, n - bw * b) : 0u;
  };

  float qreg[KV * EPV];
  uint32_t cur_q = 0xffffffffu;
  float qn1 = 0.f, rho = 0.f;
  uint32_t n_refine = 0;
  bool ok = true;
  // query q's entries into registers (this lane's share), with its bounds
  auto load_query = [&](uint32_t q) {
    cur_q = q;
    const float4 *qrow = reinterpret_cast<const float4 *>(a.qf32 + (size_t)q * a.qstride);
#pragma unroll
    for (int kk = 0; kk < KV; ++kk) {
      const int v = lane + 32 * kk;
#pragma unroll
      for (int x = 0; x < EPV / 4; ++x) {
        const float4 y = v < a.nvec ? qrow[v * (EPV / 4) + x] : make_float4(0.f, 0.f, 0.f, 0.f);
        qreg[kk * EPV + 4 * x + 0] = y.x;
        qreg[kk * EPV + 4 * x + 1] = y.y;
        qreg[kk * EPV + 4 * x + 2] = y.z;
        qreg[kk * EPV + 4 * x + 3] = y.w;
      }
    }
    qn1 = a.qn1[q];
    rho = a.rho[q];
  };
  SibPair e_cur, e_nxt;
  uint32_t r_cur, r_nxt;
  uint32_t b = gw;
  load_batch(b, e_cur, r_cur);
  load_batch(b + nw, e_nxt, r_nxt);
  uint32_t len_cur = batch_len(b), len_nxt = batch_len(b + nw);
  // prime the ring: the first `depth` pairs of the warp's stream (a warp's
  // stream holds fewer than 2^32 pairs: the list's length is a uint32).
  // With a.expire (a failure-detection test) no copy is started, so the
  // first wait below runs out with nothing in flight.
  uint32_t t_issued = 0;  // pairs of the stream whose copy was started
  for (uint32_t k = 0; k < (a.expire ? 0u : depth); ++k) {
    uint32_t row;
    bool have;
    if (k < len_cur) {
      row = __shfl_sync(FULL, r_cur, k);
      have = true;
    } else if (k - len_cur < len_nxt && len_cur == bw) {
      row = __shfl_sync(FULL, r_nxt, k - len_cur);
      have = true;
    } else {
      have = false;
      row = kNoRow;
    }
    if (!have) break;
    issue(k, row);
    ++t_issued;
  }
  uint32_t t = 0;  // stream position of the pair being tested
  // its slot t % depth and that slot's phase parity (t / depth) & 1, advanced
  // by one per pair (no division in the loop)
  uint32_t k = 0, ph = 0;
  while (len_cur > 0 && ok) {
    uint32_t m_a = 0, m_b = 0;   // pass / recheck, or left / right survives
    uint32_t m_c = 0;            // MODE 4: the left item is tested next
    uint32_t m_d = 0;            // FP8 leaves: re-scored by the BF16 pass
    uint32_t m_e = 0;            // MODE 4: the left item accepted on its lower bound
    uint32_t m_la = 0, m_lr = 0, m_ld = 0;  // MODE 4: the left item tested from its row:
                                            // accepted, FP64 recheck, BF16 re-score
    float my_ul = 0.f, my_ur = 0.f, my_ll = 0.f, my_lr = 0.f;
    // At the pool levels (modes 0, 2, 3, 5) the per-pair loop only gathers
    // and scores: wait for the row, dot product, refill the slot, warp sum.
    // The score of pair i is kept by lane i, and after the batch every lane
    // decides its own pair (the bounds, the subtraction, the prune test).  At
    // the items (modes 1, 4) each pair is decided in the loop, with the
    // query that is loaded for it: a straddling score is re-scored there and
    // then, while the ring's next copies are in flight.
    constexpr bool PER_LANE = MODE != 1 && MODE != 4;
    float my_acc = 0.f;
    // this lane's pair's query terms (and FP8 row scale), loaded ahead of the
    // loop so that their latency hides behind it
    const bool mine = (uint32_t)lane < len_cur;
    const float qn1_l = (PER_LANE && !PRE && mine) ? a.qn1[e_cur.q] : 0.f;
    const float rho_l = (PER_LANE && mine) ? a.rho[e_cur.q] : INFINITY;
    const float sc_l =
        (FMT == GT_FP8 && PER_LANE && !PRE && mine && r_cur != kNoRow) ? a.scales[r_cur] : 1.f;
    // refill slot kk with the row of stream position tt + depth (tt is the
    // position of this batch's pair ii)
    auto refill = [&](uint32_t kk, uint32_t tt, uint32_t ii) {
      const uint32_t tn = tt + depth;
      const uint32_t in_batch = ii + depth;  // position relative to this batch
      uint32_t row = kNoRow;
      bool have = false;
      if (in_batch < len_cur) {
        row = __shfl_sync(FULL, r_cur, in_batch);
        have = true;
      } else if (len_cur == bw && in_batch - bw < len_nxt) {
        row = __shfl_sync(FULL, r_nxt, in_batch - bw);
        have = true;
      }
      if (have && tn == t_issued) {
        issue(kk, row);
        ++t_issued;
      }
    };
    // BF16 rows at the pool levels: two pairs per pass, both slots waited,
    // one proxy fence and one warp barrier, both refills, and the two warp
    // sums folded into one butterfly (after the first exchange lanes 0-15
    // carry pair i's sum and lanes 16-31 pair i+1's; each half then ends with
    // exactly warp_sum's value).  A pass's second slot is the one after k
    // (slot 0 of the next phase when k is the last; the depth may be odd).
    // (2% faster for BF16 rows of up to 1024 entries; slower for FP8 and FP32
    // rows, and more registers than wider rows have, so those keep one pair
    // per pass.)
    constexpr bool TWO = PER_LANE && FMT == GT_BF16 && KV <= 4;
    if constexpr (TWO) {
      for (uint32_t i = 0; i < len_cur; i += 2, t += 2) {
        const bool two = i + 1u < len_cur;
        const uint32_t q0 = __shfl_sync(FULL, e_cur.q, i);
        const uint32_t row0 = __shfl_sync(FULL, r_cur, i);
        const uint32_t q1 = __shfl_sync(FULL, e_cur.q, two ? i + 1u : i);
        const uint32_t row1 = __shfl_sync(FULL, r_cur, two ? i + 1u : i);
        const bool wrap = k + 1u == depth;
        const uint32_t k2 = wrap ? 0u : k + 1u, ph2 = wrap ? (ph ^ 1u) : ph;
        if (q0 != cur_q) load_query(q0);
        bool good = ring_wait(full0 + 8u * k, ph, a.expire ? 0ull : kRingWaitNs);
        if (two && good) good = ring_wait(full0 + 8u * k2, ph2, kRingWaitNs);
        if (!__all_sync(FULL, good)) {
          ok = false;
          break;
        }
        uint4 w[KV];
        {
          const uint4 *rowp = reinterpret_cast<const uint4 *>(gslot0 + (size_t)k * slot_bytes);
          const bool has = row0 != kNoRow;
#pragma unroll
          for (int kk = 0; kk < KV; ++kk) {
            const int v = lane + 32 * kk;
            w[kk] = (has && v < a.nvec) ? rowp[v] : make_uint4(0u, 0u, 0u, 0u);
          }
        }
        const float acc0 = row_dot<FMT, KV, false>(w, qreg, nullptr, a.nvec);
        float acc1 = 0.f;
        if (two) {
          if (q1 != cur_q) load_query(q1);  // the pass straddles a query boundary
          const uint4 *rowp = reinterpret_cast<const uint4 *>(gslot0 + (size_t)k2 * slot_bytes);
          const bool has = row1 != kNoRow;
#pragma unroll
          for (int kk = 0; kk < KV; ++kk) {
            const int v = lane + 32 * kk;
            w[kk] = (has && v < a.nvec) ? rowp[v] : make_uint4(0u, 0u, 0u, 0u);
          }
          acc1 = row_dot<FMT, KV, false>(w, qreg, nullptr, a.nvec);
        }
        // the slots' next contents arrive through the async proxy: order this
        // warp's reads of them before the copies that refill them
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        refill(k, t, i);
        k = k2;
        ph = ph2;
        if (two) {
          refill(k, t + 1u, i + 1u);
          if (++k == depth) {
            k = 0;
            ph ^= 1u;
          }
        }
        const bool hi = (lane & 16) != 0;
        float keep = hi ? acc1 : acc0;
        keep += __shfl_xor_sync(FULL, hi ? acc0 : acc1, 16);
#pragma unroll
        for (int off = 8; off > 0; off >>= 1) keep += __shfl_xor_sync(FULL, keep, off);
        const float s0 = __shfl_sync(FULL, keep, 0), s1 = __shfl_sync(FULL, keep, 16);
        if ((uint32_t)lane == i) my_acc = s0;
        if (two && (uint32_t)lane == i + 1u) my_acc = s1;
      }
    } else {
      for (uint32_t i = 0; i < len_cur; ++i, ++t) {
        const uint32_t q = __shfl_sync(FULL, e_cur.q, i);
        const uint32_t rowi = __shfl_sync(FULL, r_cur, i);
        const bool has = rowi != kNoRow;
        if (q != cur_q) load_query(q);
        const bool good = ring_wait(full0 + 8u * k, ph, a.expire ? 0ull : kRingWaitNs);
        if (!__all_sync(FULL, good)) {
          ok = false;
          break;
        }
        uint4 w[KV];
        const uint4 *rowp = reinterpret_cast<const uint4 *>(gslot0 + (size_t)k * slot_bytes);
#pragma unroll
        for (int kk = 0; kk < KV; ++kk) {
          const int v = lane + 32 * kk;
          w[kk] = (has && v < a.nvec) ? rowp[v] : make_uint4(0u, 0u, 0u, 0u);
        }
        float acc = row_dot<FMT, KV, false>(w, qreg, nullptr, a.nvec);
        // the slot's next contents arrive through the async proxy: order this
        // warp's reads of it before the copy that refills it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        refill(k, t, i);
        if (++k == depth) {
          k = 0;
          ph ^= 1u;
        }
        acc = warp_sum(acc);
        if (MODE == 1) {
          decide<FMT, KV, true, false>(a, acc, rowi, qn1, rho, qreg, nullptr, (int)i, m_a, m_b,
                                       m_d, n_refine);
        } else if (MODE == 4) {
          // MODE 4: the right item decided here; its score kept by lane i,
          // which bounds the left item after the batch
          if (has)
            decide<FMT, KV, true, false>(a, acc, rowi, qn1, rho, qreg, nullptr, (int)i, m_a, m_b,
                                         m_d, n_refine);
          if ((uint32_t)lane == i) my_acc = acc;
        } else if ((uint32_t)lane == i) {
          my_acc = acc;
        }
      }
    }
    if (!ok) break;
    if (!PRE && PER_LANE) {
      // this lane's pair: the gathered row's score and bounds
      const bool has = mine && r_cur != kNoRow;
      float U = 0.f, Lo = 0.f;
      if (has) test_bounds_scaled<FMT>(a, my_acc, sc_l, qn1_l, U, Lo);
      // subtraction: the left child's exact score is the parent's minus the
      // right child's, so Ul = U_parent - L_right (rounded up) bounds it.  The
      // last row of a level is the one pool an insert can extend after its
      // parent's bound was taken (a server group keeps the tree of its
      // admission while later steps append items): its current row would
      // bound the grown pool, not the one under the parent, so it is not
      // subtracted.
      float Ul = e_cur.U;
      if (SUB && has) Ul = __fsub_ru(e_cur.U, r_cur + 1u >= a.n_rows ? 0.f : fmaxf(Lo, 0.f));
      if (MODE == 0) {
        m_a = __ballot_sync(FULL, has && U >= rho_l);
      } else if (MODE == 2 || MODE == 3) {
        m_a = __ballot_sync(FULL, mine && Ul >= rho_l);
        m_b = __ballot_sync(FULL, has && U >= rho_l);
        my_ul = Ul;
        my_ur = U;
        if (MODE == 2) {
          const bool r_last = r_cur + 1u >= a.n_rows;
          sub_lower(__uint_as_float(e_cur.pad), has, r_last, U, r_last ? 0.f : Lo, my_ll, my_lr);
        }
      }
    }
    if (MODE == 4) {
      // this lane's level-1 pool: the left item's exact score is the pool's
      // minus the right item's, so it is accepted without its row when
      // L_pool - U_right (rounded down) reaches rho, and otherwise tested from
      // its row while U_pool - L_right (rounded up) does.  No right item: the
      // left item is the whole pool.
      // (its query's terms are read here: kept out of the loop's registers)
      const bool has = mine && r_cur != kNoRow;
      float Up = 0.f, Lp = 0.f, rho_4 = INFINITY;
      if (mine) {
        const SibPair ee = ins[bw * b + (uint32_t)lane];
        Up = ee.U;
        Lp = __uint_as_float(ee.pad);
        rho_4 = a.rho[e_cur.q];
      }
      float U = 0.f, Lo = 0.f;
      if (has) test_bounds<FMT>(a, my_acc, r_cur, a.qn1[e_cur.q], U, Lo);
      const float Ul = has ? __fsub_ru(Up, r_cur + 1u >= a.n_rows ? 0.f : fmaxf(Lo, 0.f)) : Up;
      const float Ll = has ? __fsub_rd(Lp, U) : Lp;
      const bool al = mine && !a.no_accept && Ll >= rho_4;
      m_e = __ballot_sync(FULL, al);
      m_c = __ballot_sync(FULL, mine && !al && Ul >= rho_4);
      // the left items whose bounds straddle rho (a few per batch) are
      // gathered and decided here, warp-wide, one at a time, like any leaf:
      // no list and no launch of their own
      uint32_t need = m_c;
      while (need) {
        const int j = __ffs(need) - 1;
        need &= need - 1u;
        const uint32_t qj = __shfl_sync(FULL, e_cur.q, j);
        const uint32_t item = 2u * __shfl_sync(FULL, e_cur.p, j);
        if (qj != cur_q) load_query(qj);
        const uint8_t *row = a.rows + (size_t)item * a.row_bytes;
        uint4 w[KV];
#pragma unroll
        for (int kk = 0; kk < KV; ++kk) {
          const int v = lane + 32 * kk;
          w[kk] = v < a.nvec ? ld_stream(row + 16 * v) : make_uint4(0u, 0u, 0u, 0u);
        }
        const float acc = warp_sum(row_dot<FMT, KV, false>(w, qreg, nullptr, a.nvec));
        decide<FMT, KV, true, false>(a, acc, item, qn1, rho, qreg, nullptr, j, m_la, m_lr, m_ld,
                                     n_refine);
      }
      // (counted with the tests, as left items)
      if (m_c && lane == 0) atomicAdd(a.out_count, (uint32_t)__popc(m_c));
    }
    if (PRE) {
      my_ul = my_acc;
      // Each lane decides its own entry: the pool [lo, hi) and its prefix
      // scores S(lo), S(hi) (0 at a block's start; the GEMM's block total at
      // its end; else gathered prefix scores) and S(mid) from this batch's
      // test.  Each bound holds the exact S (the row format's and the FP32
      // accumulation's error terms), so a difference of bounds, rounded
      // outward, holds a child's exact score.
      const bool hasr = r_cur != kNoRow;
      const uint32_t bmask = (1u << a.pre_c) - 1u;
      const uint32_t lo = e_cur.p << a.pre_h;
      const uint32_t hi = min(lo + (1u << a.pre_h), a.n_items);
      const float s_lo = e_cur.U, s_hi = __uint_as_float(e_cur.pad);
      float lu = 0.f, ld = 0.f, hu, hd, mu = 0.f, md = 0.f;
      if (lo & bmask) test_bounds<FMT>(a, s_lo, 0u, 0.f, lu, ld);
      if ((hi & bmask) == 0u || hi == a.n_items) {
        hu = __fmul_ru(s_hi, a.g_cu);
        hd = __fmul_rd(s_hi, a.g_cl);
      } else {
        test_bounds<FMT>(a, s_hi, 0u, 0.f, hu, hd);
      }
      if (hasr) test_bounds<FMT>(a, my_ul, 0u, 0.f, mu, md);
      if (MODE == 5) {
        // no right half: the left half is the kept pool itself
        m_a = __ballot_sync(FULL, mine && (!hasr || __fsub_ru(mu, ld) >= rho_l));
        m_b = __ballot_sync(FULL, mine && hasr && __fsub_ru(hu, md) >= rho_l);
        if (!hasr) my_ul = s_hi;
      } else {
        // items lo and lo + 1 (when present): 1 accepted on the lower bound,
        // 3 while only the upper bound reaches rho (re-scored below from the
        // item's FP32 row: a bound relative to the item's own score), then 2
        // (FP64 recheck) if still doubtful, 0 pruned
        int rl = 0, rr = 0;
        if (mine) {
          const float Ul = __fsub_ru(hasr ? mu : hu, ld), Ll = __fsub_rd(hasr ? md : hd, lu);
          rl = Ll >= rho_l ? 1 : (Ul >= rho_l ? 3 : 0);
          if (hasr) {
            const float Ur = __fsub_ru(hu, md), Lr = __fsub_rd(hd, mu);
            rr = Lr >= rho_l ? 1 : (Ur >= rho_l ? 3 : 0);
          }
        }
        // the re-scores, warp-wide, one item at a time, with its query loaded
#pragma unroll 1
        for (uint32_t side = 0; side < 2; ++side) {
          uint32_t need = __ballot_sync(FULL, (side ? rr : rl) == 3);
          while (need) {
            const int j = __ffs(need) - 1;
            need &= need - 1u;
            const uint32_t qj = __shfl_sync(FULL, e_cur.q, j);
            if (qj != cur_q) load_query(qj);
            const uint32_t pos = (__shfl_sync(FULL, e_cur.p, j) << a.pre_h) + side;
            ++n_refine;
            const int r = refine32<FMT, KV, false>(a, pos, rho, qreg, nullptr);
            if (lane == j) (side ? rr : rl) = r;
          }
        }
        m_a = __ballot_sync(FULL, rl == 1);
        m_b = __ballot_sync(FULL, rl == 2);
        m_c = __ballot_sync(FULL, rr == 1);
        m_d = __ballot_sync(FULL, rr == 2);
      }
    }
    Pair pr;
    pr.q = e_cur.q;
    pr.j = e_cur.p;
    if (MODE == 0) {
      const bool mine = (m_a >> lane) & 1u;
      const uint32_t c0 = 2u * pr.j;
      const uint32_t nch = mine ? (1u + (c0 + 1u < a.n_child ? 1u : 0u)) : 0u;
      Pair x, y;
      x.q = pr.q; x.j = c0;
      y.q = pr.q; y.j = c0 + 1u;
      warp_append(a.out, a.out_count, a.out_cap, a.flags, nch, x, y);
    } else if (MODE == 1) {
      warp_append(a.res, a.res_count, a.res_cap, a.flags, (m_a >> lane) & 1u, pr, pr);
      warp_append(a.rchk, a.rchk_count, a.rchk_cap, a.flags, (m_b >> lane) & 1u, pr, pr);
      if (FMT == GT_FP8 && m_d)
        warp_append(a.defer, a.defer_count, a.defer_cap, a.flags, (m_d >> lane) & 1u, pr, pr);
    } else if (MODE == 4) {
      Pair right, left;
      right.q = pr.q; right.j = 2u * pr.j + 1u;
      left.q = pr.q; left.j = 2u * pr.j;
      const bool ar = (m_a >> lane) & 1u, al = ((m_e | m_la) >> lane) & 1u;
      warp_append(a.res, a.res_count, a.res_cap, a.flags, (ar ? 1u : 0u) + (al ? 1u : 0u),
                  ar ? right : left, left);
      const bool cr = (m_b >> lane) & 1u, cl = (m_lr >> lane) & 1u;
      warp_append(a.rchk, a.rchk_count, a.rchk_cap, a.flags, (cr ? 1u : 0u) + (cl ? 1u : 0u),
                  cr ? right : left, left);
      if (FMT == GT_FP8 && (m_d | m_ld)) {
        const bool dr = (m_d >> lane) & 1u, dl = (m_ld >> lane) & 1u;
        warp_append(a.defer, a.defer_count, a.defer_cap, a.flags, (dr ? 1u : 0u) + (dl ? 1u : 0u),
                    dr ? right : left, left);
      }
    } else if (MODE == 5) {
      pre_emit(a, out_v, e_cur, m_a, m_b, my_ul);
    } else if (MODE == 6) {
      Pair l, r;
      l.q = e_cur.q; l.j = e_cur.p << 1;
      r.q = e_cur.q; r.j = (e_cur.p << 1) + 1u;
      const bool al = (m_a >> lane) & 1u, ar = (m_c >> lane) & 1u;
      warp_append(a.res, a.res_count, a.res_cap, a.flags, (al ? 1u : 0u) + (ar ? 1u : 0u), al ? l : r, r);
      const bool cl = (m_b >> lane) & 1u, cr = (m_d >> lane) & 1u;
      warp_append(a.rchk, a.rchk_count, a.rchk_cap, a.flags, (cl ? 1u : 0u) + (cr ? 1u : 0u), cl ? l : r, r);
    } else {
      sub_emit<MODE == 3>(a, out_v, e_cur, m_a, m_b, my_ul, my_ur, my_ll, my_lr);
    }
    // next batch
    b += nw;
    e_cur = e_nxt;
    r_cur = r_nxt;
    len_cur = len_nxt;
    load_batch(b + nw, e_nxt, r_nxt);
    len_nxt = batch_len(b + nw);
    // a batch shorter than bw is the warp's last; copies past it were never started
  }
  if (!ok) {
    if (lane == 0) atomicExch(&a.flags[kFlagTimeout], 1);
  }
  // every copy this warp started has landed before it exits
  if (lane == 0) {
    const uint64_t t0 = ring_now();
    for (uint32_t tt = t_issued > depth ? t_issued - depth : 0; tt < t_issued; ++tt) {
      const uint32_t ks = tt % depth, pk = (tt / depth) & 1u;
      while (!ring_test(full0 + 8u * ks, pk) && ring_now() - t0 < kRingWaitNs) {
      }
    }
  }
  raise_stray(a, stray);
  if (LEAF && n_refine && lane == 0) atomicAdd(a.refine_count, n_refine);
}

// ---- One persistent launch for every level below the cutover ---------------
// k_drain: the warps of one persistent grid drain a shared work queue, the
// list of (query, pool, bound) entries the dense GEMM leaves at level c-1
// (grouped by query).  A warp claims 32 consecutive entries at a time and
// carries their subtrees down to the items itself, level by level, in
// private lists: the entries' right children are gathered (the ring of
// k_ring) and tested, the left ones bounded by subtraction (Algorithm 1's
// sim - rsim, as an upper bound), the survivors become the warp's next list
// (at most twice as long), and at the items the right item of each surviving
// level-1 pool is decided, then the left items that their bound keeps.  All
// levels of the batch run in this one launch; a warp never waits for another
// (the queue is complete before the launch), so the only waits are the
// ring's bounded ones.  Levels whose lists are short no longer pay a launch
// and a tail each.
constexpr int kDrainMaxCut = 5;        // lists of 32 << (c - 1) entries per warp

struct DrainLevel {
  int64_t row0;      // first row of the level (row index into the format's rows)
  uint32_t n_rows;   // rows at the level
  Bound bd;          // the level's bound constants (row format, FP32 pool sums)
};

// (the gathered rows and FP8 scales, from row 0 of level 0, are the
// LevelArgs' rows and scales)
struct DrainArgs {
  DrainLevel lvl[kDrainMaxCut];
  const SibPair *root;       // the queue: entries of level-c pools (children at c - 1)
  const uint32_t *root_count;
  uint32_t root_cap;
  uint32_t *head;            // next queue position to claim (zero at launch)
  uint32_t *level_count;     // [h]: entries tested at level h < c - 1
  uint32_t *left_count;      // left items tested
  SibPair *scratch;          // per warp: two lists of wcap entries, then wcap item pairs
  uint32_t wcap;
  int cut;
};

template <int FMT, int KV>
__global__ void __launch_bounds__(32 * kRingWarps, 1)
    k_drain(const LevelArgs a, const DrainArgs g, uint32_t depth, uint32_t slot_bytes) {
  constexpr int EPV = RowFmt<FMT>::EPV;
  constexpr uint32_t kNoRow = 0xffffffffu;
  extern __shared__ __align__(128) uint8_t ring_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t sbase = (smem_addr(ring_raw) + 127u) & ~127u;
  const uint8_t *gbase = ring_raw + (sbase - smem_addr(ring_raw));
  // after the slots and their barriers: the block's test counts per level,
  // then of left items (all shared memory is dynamic, so the kernel may
  // take the same opt-in size as k_ring)
  uint32_t *blk_count = reinterpret_cast<uint32_t *>(
      const_cast<uint8_t *>(gbase) + (size_t)kRingWarps * depth * (slot_bytes + 8u));
  if (threadIdx.x <= kDrainMaxCut) blk_count[threadIdx.x] = 0u;
  __syncthreads();
  const uint32_t slot0 = sbase + (uint32_t)warp * depth * slot_bytes;
  const uint8_t *gslot0 = gbase + (size_t)warp * depth * slot_bytes;
  const uint32_t full0 = sbase + kRingWarps * depth * slot_bytes + (uint32_t)warp * depth * 8u;
  const uint32_t copy_bytes = (uint32_t)a.nvec * 16u;
  if (lane == 0) {
    for (uint32_t k = 0; k < depth; ++k) ring_bar_init(full0 + 8u * k, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const uint32_t gw = blockIdx.x * kRingWarps + (uint32_t)warp;
  SibPair *listA = g.scratch + (size_t)gw * (2u * g.wcap + (g.wcap + 1u) / 2u);
  SibPair *listB = listA + g.wcap;
  Pair *left = reinterpret_cast<Pair *>(listB + g.wcap);
  const uint32_t n_root = min(*g.root_count, g.root_cap);

  float qreg[KV * EPV];
  uint32_t cur_q = 0xffffffffu;
  float qn1 = 0.f, rho = 0.f;
  uint32_t n_refine = 0;
  bool ok = true, stray = false;
  auto load_query = [&](uint32_t q) {
    cur_q = q;
    const float4 *qrow = reinterpret_cast<const float4 *>(a.qf32 + (size_t)q * a.qstride);
#pragma unroll
    for (int kk = 0; kk < KV; ++kk) {
      const int v = lane + 32 * kk;
#pragma unroll
      for (int x = 0; x < EPV / 4; ++x) {
        const float4 y = v < a.nvec ? qrow[v * (EPV / 4) + x] : make_float4(0.f, 0.f, 0.f, 0.f);
        qreg[kk * EPV + 4 * x + 0] = y.x;
        qreg[kk * EPV + 4 * x + 1] = y.y;
        qreg[kk * EPV + 4 * x + 2] = y.z;
        qreg[kk * EPV + 4 * x + 3] = y.w;
      }
    }
    qn1 = a.qn1[q];
    rho = a.rho[q];
  };
  // the ring: stream position t is the pair being tested (slot k, phase
  // parity ph); copies are started in stream order up to t + depth - 1
  uint32_t t = 0, k = 0, ph = 0, t_issued = 0, k_iss = 0;
  auto issue = [&](const uint8_t *rows_lvl, uint32_t row) {
    if (lane == 0) {
      const uint32_t bar = full0 + 8u * k_iss;
      if (row != kNoRow) {
        ring_expect(bar, copy_bytes);
        ring_copy(slot0 + k_iss * slot_bytes, rows_lvl + (size_t)row * a.row_bytes, copy_bytes, bar);
      } else {
        ring_arrive(bar);
      }
    }
    ++t_issued;
    if (++k_iss == depth) k_iss = 0;
  };

  // One list of n entries (src) at level h, in batches of 32.  kind 0: the
  // entries are pools of level h + 1 (h >= 1), their children at level h are
  // tested and the kept ones appended to dst as entries for level h - 1;
  // kind 1 (h = 0): the entries are level-1 pools, the right item is decided
  // and the left item appended to `left` when its bound keeps it; kind 2: the
  // item pairs of `left` are decided.
  auto run_list = [&](int kind, int h, const SibPair *src, const Pair *srcp, uint32_t n, SibPair *dst,
                      uint32_t &dst_n) {
    const DrainLevel L = g.lvl[h];
    const uint8_t *rows_lvl = a.rows + (size_t)L.row0 * a.row_bytes;
    const float *scales_lvl = FMT == GT_FP8 ? a.scales + L.row0 : nullptr;
    auto fetch = [&](uint32_t b0, SibPair &e, uint32_t &row) {
      const uint32_t idx = b0 + (uint32_t)lane;
      row = kNoRow;
      e.q = 0xffffffffu; e.p = 0; e.U = 0.f; e.pad = 0;
      if (b0 >= n || idx >= n) return;
      if (kind == 2) {
        const Pair x = srcp[idx];
        e.q = x.q; e.p = x.j;
        row = x.j;
      } else {
        e = src[idx];
        const uint32_t r = 2u * e.p + 1u;
        if (r < L.n_rows) row = r;
      }
    };
    SibPair e_cur, e_nxt;
    uint32_t r_cur, r_nxt;
    fetch(0, e_cur, r_cur);
    fetch(32, e_nxt, r_nxt);
    if (lane == 0) atomicAdd(&blk_count[kind == 2 ? kDrainMaxCut : h], n);
    for (uint32_t b0 = 0; b0 < n && ok; b0 += 32) {
      const uint32_t len = min(32u, n - b0);
      const uint32_t len_nxt = b0 + 32 < n ? min(32u, n - b0 - 32) : 0u;
      // row of stream position x >= t0 (this batch starts at t0, then the
      // next batch of the list)
      const uint32_t t0 = t;
      auto row_at = [&](uint32_t x, bool &have) -> uint32_t {
        const uint32_t rel = x - t0;
        have = true;
        if (rel < len) return __shfl_sync(FULL, r_cur, rel);
        if (len == 32 && rel - 32 < len_nxt) return __shfl_sync(FULL, r_nxt, rel - 32);
        have = false;
        return kNoRow;
      };
      // the first pairs of a list were not prefetched: start their copies
      // (none with a.expire: a failure-detection test)
      while (!a.expire && t_issued < t + depth) {
        bool have;
        const uint32_t row = row_at(t_issued, have);
        if (!have) break;
        issue(rows_lvl, row);
      }
      const bool mine = (uint32_t)lane < len;
      const float qn1_l = mine ? a.qn1[e_cur.q] : 0.f;
      const float rho_l = mine ? a.rho[e_cur.q] : INFINITY;
      const float sc_l = (FMT == GT_FP8 && mine && r_cur != kNoRow) ? scales_lvl[r_cur] : 1.f;
      float my_acc = 0.f;
      for (uint32_t i = 0; i < len; ++i, ++t) {
        const uint32_t q = __shfl_sync(FULL, e_cur.q, i);
        const bool has = __shfl_sync(FULL, r_cur, i) != kNoRow;
        if (q != cur_q) load_query(q);
        const bool good = ring_wait(full0 + 8u * k, ph, a.expire ? 0ull : kRingWaitNs);
        if (!__all_sync(FULL, good)) {
          ok = false;
          break;
        }
        uint4 w[KV];
        const uint4 *rowp = reinterpret_cast<const uint4 *>(gslot0 + (size_t)k * slot_bytes);
#pragma unroll
        for (int kk = 0; kk < KV; ++kk) {
          const int v = lane + 32 * kk;
          w[kk] = (has && v < a.nvec) ? rowp[v] : make_uint4(0u, 0u, 0u, 0u);
        }
        float acc = row_dot<FMT, KV, false>(w, qreg, nullptr, a.nvec);
        // the slot's next contents arrive through the async proxy: order this
        // warp's reads of it before the copy that refills it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (!a.expire && t_issued == t + depth) {
          bool have;
          const uint32_t row = row_at(t + depth, have);
          if (have) issue(rows_lvl, row);
        }
        if (++k == depth) {
          k = 0;
          ph ^= 1u;
        }
        acc = warp_sum(acc);
        if ((uint32_t)lane == i) my_acc = acc;
      }
      if (!ok) break;
      // every lane decides its own pair
      const bool has = mine && r_cur != kNoRow;
      float U = 0.f, Lo = 0.f;
      if (has) {
        float acc = my_acc, tq = 0.f;
        if (FMT == GT_FP8) {
          acc *= sc_l;
          tq = sc_l * 0x1p-10f * qn1_l;
        }
        U = fmaf(acc, L.bd.cu, tq * L.bd.ct_up);
        Lo = (acc * L.bd.cl - tq * L.bd.ct_lo) * (1.f - 0x1p-22f);
      }
      // subtraction (kinds 0, 1): the left child's bound; the last row of a
      // level is not subtracted (an insert may have extended it since the
      // parent's bound was taken)
      const bool r_last = r_cur + 1u >= L.n_rows;
      float Ul = e_cur.U;
      if (kind != 2 && has) Ul = __fsub_ru(e_cur.U, r_last ? 0.f : fmaxf(Lo, 0.f));
      // the children's lower bounds (the right one's own, the left one's by
      // subtraction)
      float Ll = 0.f, Lr = 0.f;
      if (kind != 2) sub_lower(__uint_as_float(e_cur.pad), has, r_last, U, r_last ? 0.f : Lo, Ll, Lr);
      if (kind == 0) {
        const bool kl = mine && Ul >= rho_l, kr = has && U >= rho_l;
        const uint32_t cntl = (kl ? 1u : 0u) + (kr ? 1u : 0u);
        const uint32_t incl = warp_incl_scan(cntl);
        uint32_t pos = dst_n + incl - cntl;
        SibPair x;
        x.q = e_cur.q;
        if (kl) { x.p = 2u * e_cur.p; x.U = Ul; x.pad = __float_as_uint(Ll); dst[pos++] = x; }
        if (kr) { x.p = 2u * e_cur.p + 1u; x.U = U; x.pad = __float_as_uint(Lr); dst[pos++] = x; }
        dst_n += __shfl_sync(FULL, incl, 31);
      } else {
        // the gathered item: 0 pruned, 1 accepted, 2 FP64 recheck, 3 re-score
        // here, 4 re-scored from its BF16 row by the pass after this kernel
        int c = 0;
        if (has && U >= rho_l) {
          if (Lo >= rho_l) c = 1;
          else if (FMT == GT_F32) c = 2;
          else if (FMT == GT_FP8 && a.rows16 && a.defer) c = 4;
          else c = 3;
        }
        // kind 1: the left item of a kept level-1 pool is accepted on its
        // lower bound, or else goes to `left` for a direct test while its
        // upper bound reaches rho
        const bool al = kind == 1 && mine && !a.no_accept && Ll >= rho_l;
        if (kind == 1) {
          const bool kl = mine && !al && Ul >= rho_l;
          const uint32_t incl = warp_incl_scan(kl ? 1u : 0u);
          if (kl) {
            Pair x;
            x.q = e_cur.q;
            x.j = 2u * e_cur.p;
            left[dst_n + incl - 1u] = x;
          }
          dst_n += __shfl_sync(FULL, incl, 31);
        }
        uint32_t need = __ballot_sync(FULL, c == 3);
        while (need) {
          const int j = __ffs(need) - 1;
          need &= need - 1u;
          const uint32_t qj = __shfl_sync(FULL, e_cur.q, j);
          if (qj != cur_q) load_query(qj);
          const int r = leaf_rescore<FMT, KV, false>(a, __shfl_sync(FULL, r_cur, j), rho, qreg,
                                                     nullptr, n_refine);
          if (lane == j) c = r;
        }
        Pair it, il;
        it.q = e_cur.q;
        it.j = r_cur;
        il.q = e_cur.q;
        il.j = 2u * e_cur.p;
        warp_append(a.res, a.res_count, a.res_cap, a.flags, (c == 1 ? 1u : 0u) + (al ? 1u : 0u),
                    c == 1 ? it : il, il);
        warp_append(a.rchk, a.rchk_count, a.rchk_cap, a.flags, c == 2 ? 1u : 0u, it, it);
        if (FMT == GT_FP8) {
          const uint32_t m_d = __ballot_sync(FULL, c == 4);
          if (m_d) {
            warp_append(a.defer, a.defer_count, a.defer_cap, a.flags, c == 4 ? 1u : 0u, it, it);
            n_refine += (uint32_t)__popc(m_d);
          }
        }
      }
      __syncwarp();   // the warp's list writes before its reads of them
      e_cur = e_nxt;
      r_cur = r_nxt;
      fetch(b0 + 64, e_nxt, r_nxt);
    }
  };

  // entries per claim: 32, or fewer when the queue is short (a small served
  // group), so that its subtrees spread over as many warps as the grid has
  // instead of queuing behind one another in a few warps
  const uint32_t n_warps = gridDim.x * kRingWarps;
  const uint32_t claim = max(1u, min(32u, (n_root + n_warps - 1u) / n_warps));
  while (ok) {
    // claim the next entries of the queue
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(g.head, claim);
    base = __shfl_sync(FULL, base, 0);
    if (base >= n_root) break;
    const uint32_t cnt = min(claim, n_root - base);
    // a queue entry naming a query or a row outside its buffers can only
    // come from a corrupted list: flagged, and its subtree left out
    bool bad = false;
    if ((uint32_t)lane < cnt) {
      const SibPair e = g.root[base + lane];
      bad = !(e.q < a.q_lim && 2u * e.p < g.lvl[g.cut - 1].n_rows);
    }
    if (__any_sync(FULL, bad)) {
      stray = true;
      continue;
    }
    uint32_t n = cnt;
    const SibPair *src = g.root + base;
    SibPair *dst = listA;
    for (int h = g.cut - 1; h >= 1 && ok; --h) {
      uint32_t dn = 0;
      run_list(0, h, src, nullptr, n, dst, dn);
      src = dst;
      dst = dst == listA ? listB : listA;
      n = dn;
    }
    uint32_t nl = 0;
    if (ok) run_list(1, 0, src, nullptr, n, nullptr, nl);
    uint32_t unused = 0;
    if (ok) run_list(2, 0, nullptr, left, nl, nullptr, unused);
  }
  if (!ok && lane == 0) atomicExch(&a.flags[kFlagTimeout], 1);
  // every copy this warp started has landed before it exits
  if (lane == 0) {
    const uint64_t t0 = ring_now();
    for (uint32_t tt = t_issued > depth ? t_issued - depth : 0; tt < t_issued; ++tt) {
      const uint32_t ks = tt % depth, pk = (tt / depth) & 1u;
      while (!ring_test(full0 + 8u * ks, pk) && ring_now() - t0 < kRingWaitNs) {
      }
    }
  }
  raise_stray(a, stray);
  if (n_refine && lane == 0) atomicAdd(a.refine_count, n_refine);
  __syncthreads();
  if (threadIdx.x < (unsigned)g.cut - 1u && blk_count[threadIdx.x])
    atomicAdd(&g.level_count[threadIdx.x], blk_count[threadIdx.x]);
  if (threadIdx.x == 0 && blk_count[kDrainMaxCut])
    atomicAdd(g.left_count, blk_count[kDrainMaxCut]);
}

// Diagnostic twin of the level kernels' test: one warp per given (query,
// pool) pair loads the pool's row and the query exactly as k_level and k_ring
// do, forms the same lane-parallel dot product and warp sum, and writes the
// score with the bounds test_bounds() gives the traversal.  A pair naming a
// query or a row out of range gets NaNs.
template <int FMT, int KV>
__global__ void __launch_bounds__(256) k_pair_bounds(const LevelArgs a, const int32_t *__restrict__ pairs,
                                                     int64_t n, uint32_t n_queries, float *__restrict__ out) {
  constexpr int EPV = RowFmt<FMT>::EPV;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = gw; i < n; i += nw) {
    const int32_t q = pairs[2 * i], j = pairs[2 * i + 1];
    if (q < 0 || (uint32_t)q >= n_queries || j < 0 || (uint32_t)j >= a.n_rows) {
      if (lane < 3) out[3 * i + lane] = __int_as_float(0x7fc00000);
      continue;
    }
    float qreg[KV * EPV];
    const float4 *qrow = reinterpret_cast<const float4 *>(a.qf32 + (size_t)q * a.qstride);
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      const int v = lane + 32 * k;
#pragma unroll
      for (int x = 0; x < EPV / 4; ++x) {
        const float4 y = v < a.nvec ? qrow[v * (EPV / 4) + x] : make_float4(0.f, 0.f, 0.f, 0.f);
        qreg[k * EPV + 4 * x + 0] = y.x;
        qreg[k * EPV + 4 * x + 1] = y.y;
        qreg[k * EPV + 4 * x + 2] = y.z;
        qreg[k * EPV + 4 * x + 3] = y.w;
      }
    }
    const uint8_t *row = a.rows + (size_t)j * a.row_bytes;
    uint4 w[KV];
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      const int v = lane + 32 * k;
      w[k] = v < a.nvec ? ld_stream(row + 16 * v) : make_uint4(0u, 0u, 0u, 0u);
    }
    float acc = row_dot<FMT, KV, false>(w, qreg, nullptr, a.nvec);
    acc = warp_sum(acc);
    float U, Lo;
    test_bounds<FMT>(a, acc, (uint32_t)j, a.qn1[q], U, Lo);
    if (lane == 0) {
      out[3 * i + 0] = FMT == GT_FP8 ? acc * a.scales[j] : acc;
      out[3 * i + 1] = U;
      out[3 * i + 2] = Lo;
    }
  }
}

// FP64 recheck of leaf pairs whose bound straddles rho: the exact decision
// q.f >= rho from the FP32 rows (products of FP32 values are exact in FP64).
// Few pairs reach it, so each warp takes one pair at a time (grid-strided)
// and the FP64 dot products of different pairs run in parallel.
//
// Split signed rows (d_half > 0): the stored item and query rows are
// [max(x, 0), max(-x, 0)], so x_j = row_j - row_{d_half + j} exactly, and the
// recheck forms the signed q.f from those differences (exact FP64 products).
struct RecheckArgs {
  const Pair *rchk;         // the doubtful (query, item) pairs and their count
  const uint32_t *count;
  uint32_t cap;
  const float *rows32;      // FP32 item rows (row stride `stride`)
  int64_t stride;
  int nv4;                  // 16-byte vectors of an item row
  int d_half;               // split signed rows: the caller's width, else 0
  const float *qf32;
  const float *rho;
  Pair *res;                // accepted pairs are appended here
  uint32_t *res_count;
  uint32_t res_cap;
  uint32_t q_lim, n_items;  // valid query slots and items (a corrupted entry is flagged)
  int *flags;
};

// The pairs warp gw of nw takes: gw, gw + nw, ...
__device__ __forceinline__ void recheck_pairs(const RecheckArgs &a, uint32_t gw, uint32_t nw,
                                              int lane) {
  const uint32_t n = min(*a.count, a.cap);
  for (uint32_t i = gw; i < n; i += nw) {
    const Pair pr = a.rchk[i];
    if (pr.q >= a.q_lim || pr.j >= a.n_items) {  // a corrupted list: flagged, left out
      if (lane == 0) atomicExch(&a.flags[kFlagStray], 1);
      continue;
    }
    double acc = 0.0;
    if (a.d_half > 0) {
      const float *f = a.rows32 + (size_t)pr.j * a.stride;
      const float *qq = a.qf32 + (size_t)pr.q * a.stride;
      for (int j = lane; j < a.d_half; j += 32) {
        const double x = (double)f[j] - (double)f[a.d_half + j];
        const double y = (double)qq[j] - (double)qq[a.d_half + j];
        acc = fma(x, y, acc);
      }
    } else {
      const float4 *f = reinterpret_cast<const float4 *>(a.rows32 + (size_t)pr.j * a.stride);
      const float4 *qq = reinterpret_cast<const float4 *>(a.qf32 + (size_t)pr.q * a.stride);
      for (int v = lane; v < a.nv4; v += 32) {
        const float4 x = f[v], y = qq[v];
        acc = fma((double)x.x, (double)y.x, acc);
        acc = fma((double)x.y, (double)y.y, acc);
        acc = fma((double)x.z, (double)y.z, acc);
        acc = fma((double)x.w, (double)y.w, acc);
      }
    }
    acc = warp_sum_d(acc);
    if (lane == 0 && acc >= (double)a.rho[pr.q]) {
      const uint32_t pos = atomicAdd(a.res_count, 1u);
      if (pos < a.res_cap)
        a.res[pos] = pr;
      else
        atomicExch(&a.flags[kFlagOverflow], 1);
    }
  }
}

__global__ void __launch_bounds__(256) k_recheck(const RecheckArgs a) {
  recheck_pairs(a, (blockIdx.x * blockDim.x + threadIdx.x) >> 5, (gridDim.x * blockDim.x) >> 5,
                (int)(threadIdx.x & 31));
}

// Queries: pad to the row stride (FP32 and BF16), |q|_1 upper bound, domain
// checks on entries and thresholds.  One warp per query.  With `split`
// (signed rows) a query of d entries is stored as [max(q, 0), max(-q, 0)],
// and only non-finite entries are refused.
__global__ void __launch_bounds__(256) k_prep_queries(const float *__restrict__ Q, int64_t B, int d,
                                                      int split, int64_t stride,
                                                      const float *__restrict__ rho_in,
                                                      float *qf32, __nv_bfloat16 *qbf16, float *qn1,
                                                      float *rho_out, int *flags) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  constexpr int U = 8;  // loads a lane has in flight before it uses them
  const int64_t n_in = split ? 2 * (int64_t)d : (int64_t)d;
  for (int64_t q = warp; q < B; q += nwarps) {
    const float *in = Q + q * (int64_t)d;
    float s = 0.f;
    bool bad = false;
    // a lane's entries j = lane, lane + 32, ... in that order (so the sum's
    // rounding does not depend on U), read U at a time: for a small batch the
    // kernel is one row per warp and waits on memory, not on arithmetic
    for (int64_t j0 = lane; j0 < stride; j0 += 32 * U) {
      float y[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t j = j0 + 32 * u;
        y[u] = j < n_in ? in[j < d ? j : j - d] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t j = j0 + 32 * u;
        if (j >= stride) break;
        float x;
        if (!split) {
          x = y[u];
          bad |= !(x >= 0.f) || !isfinite(x);
        } else if (j < n_in) {
          bad |= !isfinite(y[u]);
          x = j < d ? (y[u] > 0.f ? y[u] : 0.f) : (y[u] < 0.f ? -y[u] : 0.f);
        } else {
          x = 0.f;
        }
        s += x;
        qf32[q * stride + j] = x;
        if (qbf16) qbf16[q * stride + j] = __float2bfloat16_rn(x);
      }
    }
    s = warp_sum(s);
    if (__any_sync(FULL, bad) && lane == 0) atomicExch(&flags[kFlagDomain], 1);
    if (lane == 0) {
      // fl32 sum of n non-negative terms: exact |q|_1 <= s / (1 - gamma_n)
      const int n_terms = split ? 2 * d : d;
      qn1[q] = s * (1.f + 2.f * (float)(n_terms + 1) * 0x1p-24f);
      const float r = rho_in[q];
      if (!(r > 0.f) || !(r <= 1.f)) atomicExch(&flags[kFlagRho], 1);
      rho_out[q] = r;
    }
  }
}

__global__ void k_root(Pair *out, uint32_t *count, uint32_t q0, uint32_t b) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < b; i += gridDim.x * blockDim.x) {
    Pair p;
    p.q = q0 + i;
    p.j = 0;
    out[i] = p;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = b;
}

// ---- CSR assembly ---------------------------------------------------------
// Counting sort of a frontier list by query.  The GEMM epilogue appends the
// survivors of 32 queries at a time, so its list interleaves queries; grouped,
// a warp of the level kernels keeps one query in registers for a whole run of
// pairs, and the children it appends stay grouped for the next level.
// The epilogue writes one query's survivors of a 32-pool chunk together, so
// neighbouring entries mostly share a query: the lanes of a warp that hold
// the same query combine their atomics (__match_any_sync), and the loops step
// whole warps so that every lane takes part in each vote.
template <typename E>
__global__ void k_bucket_count(const E *in, const uint32_t *n_dev, uint32_t cap, uint32_t q0,
                               uint32_t b, int64_t *cnt, int *flags) {
  const uint32_t n = min(*n_dev, cap);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x + threadIdx.x - lane; base < n; base += stride) {
    const uint32_t i = base + lane;
    uint32_t k = 0xffffffffu;
    if (i < n) {
      k = in[i].q - q0;  // the micro-batch holds queries [q0, q0 + b)
      if (k >= b) {      // the list's count would then cover entries the scatter leaves out
        atomicExch(&flags[kFlagStray], 1);
        k = 0xffffffffu;
      }
    }
    const uint32_t peers = __match_any_sync(FULL, k);
    if (k != 0xffffffffu && lane == (uint32_t)(__ffs(peers) - 1))
      atomicAdd(reinterpret_cast<unsigned long long *>(&cnt[k]), (unsigned long long)__popc(peers));
  }
}

template <typename E>
__global__ void k_bucket_scatter(const E *in, const uint32_t *n_dev, uint32_t cap, uint32_t q0,
                                 uint32_t b, const int64_t *off, int64_t *cursor, E *out) {
  const uint32_t n = min(*n_dev, cap);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x + threadIdx.x - lane; base < n; base += stride) {
    const uint32_t i = base + lane;
    E e;
    uint32_t k = 0xffffffffu;
    if (i < n) {
      e = in[i];
      k = e.q - q0;
      if (k >= b) k = 0xffffffffu;
    }
    const uint32_t peers = __match_any_sync(FULL, k);
    const int leader = __ffs(peers) - 1;
    unsigned long long slot = 0;
    if (k != 0xffffffffu && (int)lane == leader)
      slot = atomicAdd(reinterpret_cast<unsigned long long *>(&cursor[k]),
                       (unsigned long long)__popc(peers));
    slot = __shfl_sync(FULL, slot, leader);
    if (k != 0xffffffffu) out[off[k] + (int64_t)slot + __popc(peers & ((1u << lane) - 1u))] = e;
  }
}

// After the scatter: a list that fit (count <= cap) gets the number of
// entries the scatter wrote, so an entry left out (flagged by the count pass)
// can never leave a stale tail inside the count.  An overflowed count is kept:
// it tells the host which list to shrink.
__global__ void k_bucket_fix_count(uint32_t *n_dev, uint32_t cap, const int64_t *off, uint32_t b) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && *n_dev <= cap) *n_dev = (uint32_t)off[b];
}

// Result count: the host's n, or min(*n_dev, n) when the count is still on
// the device (the CSR is then enqueued behind the traversal without a sync).
__device__ __forceinline__ uint32_t csr_n(uint32_t n, const uint32_t *n_dev) {
  return n_dev ? min(*n_dev, n) : n;
}

// The result list comes in runs of one query (a warp of the leaf kernels
// appends the results of one query's pairs together), so lanes holding the
// same query combine their atomics (__match_any_sync).  Loops step whole
// warps so that every lane takes part in each vote.
__global__ void k_csr_count(const Pair *res, uint32_t n_cap, const uint32_t *n_dev, uint32_t q_lo,
                            uint32_t q_hi, int64_t *cnt, int *flags) {
  const uint32_t n = csr_n(n_cap, n_dev);
  const uint32_t lane = threadIdx.x & 31u;
  for (uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; w0 < n;
       w0 += gridDim.x * blockDim.x) {
    const uint32_t i = w0 + lane;
    uint32_t q = i < n ? res[i].q : 0xffffffffu;
    if (i < n && (q < q_lo || q >= q_hi)) {  // not a query of this range: flagged, left out
      // the first one seen is kept in flags[kFlagStray + 1, + 2] (query, row)
      if (atomicExch(&flags[kFlagStray], 1) == 0) {
        flags[kFlagStray + 1] = (int)q;
        flags[kFlagStray + 2] = (int)res[i].j;
      }
      q = 0xffffffffu;
    }
    const uint32_t peers = __match_any_sync(FULL, q);
    if (q != 0xffffffffu && lane == (uint32_t)(__ffs(peers) - 1))
      atomicAdd(reinterpret_cast<unsigned long long *>(&cnt[q]), (unsigned long long)__popc(peers));
  }
}

// Exclusive scan of cnt[0..B) into off[0..B] (one block).
__global__ void __launch_bounds__(1024) k_scan(const int64_t *cnt, int64_t B, int64_t *off) {
  // one block: thread t sums a contiguous chunk, the chunk sums are scanned
  // by warp shuffles (two barriers), then each thread writes its chunk
  __shared__ int64_t wsum[32];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int64_t per = (B + 1023) / 1024;
  const int64_t lo = std::min<int64_t>(B, t * per), hi = std::min<int64_t>(B, lo + per);
  int64_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += cnt[i];
  int64_t v = s;  // inclusive scan of the chunk sums within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) wsum[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int64_t x = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    wsum[lane] = x;
  }
  __syncthreads();
  int64_t run = (wid ? wsum[wid - 1] : 0) + v - s;
  for (int64_t i = lo; i < hi; ++i) {
    off[i] = run;
    run += cnt[i];
  }
  if (t == 1023) off[B] = wsum[31];
}

__global__ void k_csr_fill(const Pair *res, uint32_t n_cap, const uint32_t *n_dev, uint32_t q_lo,
                           uint32_t q_hi, const int64_t *off, int64_t *cursor, const int32_t *perm,
                           int32_t *ids) {
  const uint32_t n = csr_n(n_cap, n_dev);
  const uint32_t lane = threadIdx.x & 31u;
  for (uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; w0 < n;
       w0 += gridDim.x * blockDim.x) {
    const uint32_t i = w0 + lane;
    Pair p;
    p.q = 0xffffffffu;
    p.j = 0;
    if (i < n) p = res[i];
    const bool mine = i < n && p.q >= q_lo && p.q < q_hi;  // k_csr_count flagged the others
    if (!mine) p.q = 0xffffffffu;
    const uint32_t peers = __match_any_sync(FULL, p.q);
    const int leader = __ffs(peers) - 1;
    unsigned long long slot = 0;
    if (mine && (int)lane == leader)
      slot = atomicAdd(reinterpret_cast<unsigned long long *>(&cursor[p.q]),
                       (unsigned long long)__popc(peers));
    slot = __shfl_sync(FULL, slot, leader);
    if (mine) ids[off[p.q] + (int64_t)slot + __popc(peers & ((1u << lane) - 1u))] = perm[p.j];
  }
}

// Ascending sort of each query's ids: a bitonic network whose merge steps all
// sort upward, so a segment of any length n sorts in place with the missing
// entries n..2^k-1 acting as +inf (never moved).  Segments up to 4096 ids sort
// in shared memory; longer ones in global memory (one block per segment).
constexpr int kSortSmem = 4096;

__device__ __forceinline__ void cas(int32_t *a, int i, int p) {
  int32_t x = a[i], y = a[p];
  if (y < x) {
    a[i] = y;
    a[p] = x;
  }
}

template <bool SMEM>
__device__ void bitonic(int32_t *a, int64_t n) {
  int64_t np2 = 1;
  while (np2 < n) np2 <<= 1;
  for (int64_t k = 2; k <= np2; k <<= 1) {
    for (int64_t i = threadIdx.x; i < np2 / 2; i += blockDim.x) {
      // flip step: pair lanes mirrored inside each block of size k
      const int64_t blk = i / (k / 2), off = i % (k / 2);
      const int64_t lo = blk * k + off, hi = blk * k + (k - 1 - off);
      if (hi < n) cas(a, (int)lo, (int)hi);
    }
    __syncthreads();
    for (int64_t j = k / 4; j >= 1; j >>= 1) {
      for (int64_t i = threadIdx.x; i < np2 / 2; i += blockDim.x) {
        const int64_t blk = i / j, off = i % j;
        const int64_t lo = blk * 2 * j + off, hi = lo + j;
        if (hi < n) cas(a, (int)lo, (int)hi);
      }
      __syncthreads();
    }
  }
}

// Ascending sort of one segment of n <= 32 KPL ids, ids[s .. s + n), by one
// warp: KPL ids per lane (id index i = 32 k + lane), a bitonic network whose
// partners i ^ stride sit in another lane (stride < 32, a shuffle) or another
// register of the same lane.
template <int KPL>
__device__ __forceinline__ void warp_sort_ids(int32_t *ids, int64_t s, int64_t n) {
  constexpr int CAP = 32 * KPL;
  const int lane = threadIdx.x & 31;
  int32_t v[KPL];
#pragma unroll
  for (int k = 0; k < KPL; ++k) {
    const int i = 32 * k + lane;
    v[k] = i < n ? ids[s + i] : 0x7fffffff;
  }
#pragma unroll
  for (int size = 2; size <= CAP; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
#pragma unroll
      for (int k = 0; k < KPL; ++k) {
        const int i = 32 * k + lane;
        const bool up = (i & size) == 0;
        if (stride >= 32) {
          const int kp = k ^ (stride >> 5);
          if (kp > k) {
            const int32_t a = v[k], b = v[kp];
            const int32_t lo_v = min(a, b), hi_v = max(a, b);
            v[k] = up ? lo_v : hi_v;
            v[kp] = up ? hi_v : lo_v;
          }
        } else {
          const int32_t p = __shfl_xor_sync(FULL, v[k], stride);
          const bool lower = (lane & stride) == 0;
          v[k] = (lower == up) ? min(v[k], p) : max(v[k], p);
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < KPL; ++k) {
    const int i = 32 * k + lane;
    if (i < n) ids[s + i] = v[k];
  }
}

// Segments of lo < n <= 32 KPL ids, one warp each.  Longer segments are
// appended to `list` (when given) for k_csr_sort.
template <int KPL>
__global__ void __launch_bounds__(256) k_csr_sort_warp(const int64_t *off, int32_t *ids, int64_t B,
                                                       int64_t lo, int64_t *list,
                                                       uint32_t *list_n) {
  constexpr int CAP = 32 * KPL;
  const int lane = threadIdx.x & 31;
  const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (q >= B) return;
  const int64_t s = off[q], n = off[q + 1] - s;
  if (n > CAP) {
    if (list && lane == 0) list[atomicAdd(list_n, 1u)] = q;
    return;
  }
  if (n <= lo || n <= 1) return;
  warp_sort_ids<KPL>(ids, s, n);
}

// The CSR of a few queries (B <= kCsrSmallMax) in one block: counts per query
// in shared memory, their scan, the fill (ids through the tree permutation)
// and the sort of each query's ids by one warp, or by the whole block for a
// segment longer than a warp sorts.  One launch instead of the six of the
// general passes: a served group's step is bound by such fixed costs.
//
// With `recheck` the block first runs the FP64 recheck of the doubtful pairs
// (a served group of a few queries has few of them), whose accepted pairs it
// appends to the result list before counting it: the recheck and the CSR of a
// small group in one launch.  The count is then read past the L1 cache, since
// the recheck's appends updated it in L2.
__global__ void __launch_bounds__(1024, 1) k_csr_small(const Pair *res, uint32_t n_cap,
                                                    const uint32_t *n_dev, uint32_t q_lo,
                                                    uint32_t B, int64_t *off_r,
                                                    const int32_t *perm, int32_t *ids, int *flags,
                                                    const RecheckArgs rc, int recheck) {
  __shared__ uint32_t cnt[kCsrSmallMax + 1], cur[kCsrSmallMax + 1];
  __shared__ int64_t start[kCsrSmallMax + 1];
  __shared__ uint32_t n_long, longq[kCsrSmallMax];
  __shared__ int32_t buf[kSortSmem];
  const uint32_t tid = threadIdx.x;
  if (recheck) recheck_pairs(rc, tid >> 5, blockDim.x >> 5, (int)(tid & 31u));
  if (tid <= B) {
    cnt[tid] = 0u;
    cur[tid] = 0u;
  }
  if (tid == 0) n_long = 0u;
  __syncthreads();
  const uint32_t n = n_dev ? min(__ldcg(n_dev), n_cap) : n_cap;
  for (uint32_t i = tid; i < n; i += blockDim.x) {
    const Pair p = res[i];
    if (p.q < q_lo || p.q - q_lo >= B) {  // not a query of this range: flagged, left out
      if (atomicExch(&flags[kFlagStray], 1) == 0) {
        flags[kFlagStray + 1] = (int)p.q;
        flags[kFlagStray + 2] = (int)p.j;
      }
      continue;
    }
    atomicAdd(&cnt[p.q - q_lo], 1u);
  }
  __syncthreads();
  if (tid == 0) {
    int64_t run = 0;
    for (uint32_t q = 0; q < B; ++q) {
      start[q] = run;
      run += cnt[q];
    }
    start[B] = run;
  }
  __syncthreads();
  if (tid <= B) off_r[tid] = start[tid];
  for (uint32_t i = tid; i < n; i += blockDim.x) {
    const Pair p = res[i];
    if (p.q < q_lo || p.q - q_lo >= B) continue;
    const uint32_t q = p.q - q_lo;
    ids[start[q] + atomicAdd(&cur[q], 1u)] = perm[p.j];
  }
  __syncthreads();  // the block's writes of ids before its warps read them back
  const uint32_t warp = tid >> 5, lane = tid & 31u;
  for (uint32_t q = warp; q < B; q += blockDim.x >> 5) {
    const int64_t m = cnt[q];
    if (m > 512) {
      if (lane == 0) longq[atomicAdd(&n_long, 1u)] = q;
    } else if (m > 1) {
      warp_sort_ids<16>(ids, start[q], m);
    }
  }
  __syncthreads();
  // the long segments, by the whole block: in shared memory up to kSortSmem
  // ids, in place in memory beyond
  for (uint32_t e = 0; e < n_long; ++e) {
    const uint32_t q = longq[e];
    const int64_t s = start[q], m = cnt[q];
    if (m <= kSortSmem) {
      for (int64_t i = tid; i < m; i += blockDim.x) buf[i] = ids[s + i];
      __syncthreads();
      bitonic<true>(buf, m);
      for (int64_t i = tid; i < m; i += blockDim.x) ids[s + i] = buf[i];
    } else {
      bitonic<false>(ids + s, m);
    }
    __syncthreads();
  }
}

// Segments longer than a warp sorts: one block per listed segment.
__global__ void __launch_bounds__(256) k_csr_sort(const int64_t *off, int32_t *ids,
                                                  const int64_t *list, const uint32_t *list_n) {
  __shared__ int32_t buf[kSortSmem];
  const uint32_t nl = *list_n;
  for (uint32_t e = blockIdx.x; e < nl; e += gridDim.x) {
    const int64_t q = list[e];
    const int64_t s = off[q], n = off[q + 1] - s;
    if (n <= kSortSmem) {
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) buf[i] = ids[s + i];
      __syncthreads();
      bitonic<true>(buf, n);
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) ids[s + i] = buf[i];
    } else {
      bitonic<false>(ids + s, n);
    }
    __syncthreads();
  }
}

template <int FMT>
int kv_for(int64_t d) {
  constexpr int EPV = RowFmt<FMT>::EPV;
  int nvec = (int)((d + EPV - 1) / EPV);
  return (nvec + 31) / 32 <= 1024 / (32 * EPV) ? 1024 / (32 * EPV) : 2048 / (32 * EPV);
}

// Grid of a grid-strided kernel: its resident blocks per SM (looked up once
// per kernel, in `per_sm`) times the SMs the launch may use.
int grid_for(const void *fn, int block, int sm_count, int &per_sm) {
  if (!per_sm) {
    int r = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, fn, block, 0);
    per_sm = std::max(1, r);
  }
  return per_sm * sm_count;
}

// G: tests a warp keeps in flight (bytes in flight per warp at d = 1000:
// G x 4 KB for FP32, G x 2 KB for BF16, G x 1 KB for FP8).  Default FP32 2,
// BF16 / FP8 4; gt_autotune may choose another per tree and format.
template <int FMT>
constexpr int default_inflight() { return FMT == GT_F32 ? 2 : 4; }

template <int FMT, int KV, bool LEAF, int G, bool QL1>
void launch_level_g(const LevelArgs &a, int sm_count, cudaStream_t s) {
  static int per_sm = 0;
  const int grid = grid_for((const void *)k_level<FMT, KV, LEAF, G, QL1>, 256, sm_count, per_sm);
  k_level<FMT, KV, LEAF, G, QL1><<<grid, 256, 0, s>>>(a);
}

// a.inflight: tests in flight per warp (1, 2, 4), plus 8 when the query is
// read through L1 instead of held in registers (0: the format's default)
template <int FMT, int KV, bool LEAF>
void launch_level_t(const LevelArgs &a, int sm_count, cudaStream_t s) {
  const int code = a.inflight > 0 ? a.inflight : default_inflight<FMT>();
  const int g = code & 7;
  if (code & 8) {
    if (g == 1) launch_level_g<FMT, KV, LEAF, 1, true>(a, sm_count, s);
    else if (g == 2) launch_level_g<FMT, KV, LEAF, 2, true>(a, sm_count, s);
    else launch_level_g<FMT, KV, LEAF, 4, true>(a, sm_count, s);
  } else {
    if (g == 1) launch_level_g<FMT, KV, LEAF, 1, false>(a, sm_count, s);
    else if (g == 2) launch_level_g<FMT, KV, LEAF, 2, false>(a, sm_count, s);
    else launch_level_g<FMT, KV, LEAF, 4, false>(a, sm_count, s);
  }
}

// Shared memory a k_ring block may use (the device's opt-in maximum).
int ring_smem_max() {
  static int m = 0;
  if (!m) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&m, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  return m;
}

template <int FMT, int KV, int MODE>
void ring_attr() {
  cudaFuncSetAttribute(k_ring<FMT, KV, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       ring_smem_max());
}

template <int FMT, int KV>
void ring_attr_modes() {
  ring_attr<FMT, KV, 0>();
  ring_attr<FMT, KV, 1>();
  ring_attr<FMT, KV, 2>();
  ring_attr<FMT, KV, 3>();
  ring_attr<FMT, KV, 4>();
}

template <int FMT, int KV>
void drain_attr() {
  cudaFuncSetAttribute(k_drain<FMT, KV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       ring_smem_max());
}

// Slots per warp of k_ring for rows of nvec 16-byte vectors: as many as fit
// in the block's shared memory, at most kRingMaxDepth; 0 (no ring) below 2.
uint32_t ring_depth(int nvec, uint32_t *slot_bytes) {
  *slot_bytes = ((uint32_t)nvec * 16u + 127u) & ~127u;
  const uint32_t d = (uint32_t)(ring_smem_max() - 256) / (kRingWarps * (*slot_bytes + 8u));
  return d >= 2 ? std::min<uint32_t>(d, kRingMaxDepth) : 0u;
}

template <int FMT, int KV>
bool launch_drain_t(const LevelArgs &a, const DrainArgs &g, int sm_count, cudaStream_t s) {
  uint32_t slot = 0;
  const uint32_t depth = ring_depth(a.nvec, &slot);
  if (!depth) return false;
  // the ring, its barriers, the alignment pad and the block's counters
  const size_t smem = (size_t)kRingWarps * depth * (slot + 8u) + 256u;
  k_drain<FMT, KV><<<sm_count, 32 * kRingWarps, smem, s>>>(a, g, depth, slot);
  return true;
}

template <int FMT, int KV, int MODE>
bool launch_ring(const LevelArgs &a, const void *in, void *out, int sm_count, cudaStream_t s) {
  uint32_t slot = 0;
  const uint32_t depth = ring_depth(a.nvec, &slot);
  if (!depth) return false;
  const size_t smem = (size_t)kRingWarps * depth * (slot + 8u) + 128u;
  k_ring<FMT, KV, MODE><<<sm_count, 32 * kRingWarps, smem, s>>>(a, in, out, depth, slot);
  return true;
}

template <int FMT, bool LEAF>
void launch_level_f(const LevelArgs &a, int64_t d, int sm_count, cudaStream_t s) {
  constexpr int EPV = RowFmt<FMT>::EPV;
  constexpr int KV1 = 1024 / (32 * EPV), KV2 = 2048 / (32 * EPV);
  const bool narrow = kv_for<FMT>(d) == KV1;
  if (a.inflight & kInflightRing) {
    const bool done = narrow ? launch_ring<FMT, KV1, LEAF ? 1 : 0>(a, a.in, a.out, sm_count, s)
                             : launch_ring<FMT, KV2, LEAF ? 1 : 0>(a, a.in, a.out, sm_count, s);
    if (done) return;
    LevelArgs b = a;
    b.inflight = 0;  // rows too wide for the ring: the format's default
    if (narrow) launch_level_t<FMT, KV1, LEAF>(b, sm_count, s);
    else launch_level_t<FMT, KV2, LEAF>(b, sm_count, s);
    return;
  }
  if (narrow)
    launch_level_t<FMT, KV1, LEAF>(a, sm_count, s);
  else
    launch_level_t<FMT, KV2, LEAF>(a, sm_count, s);
}

}  // namespace

Bound make_bound(int fmt, int h, int d) {
  const double u32 = std::ldexp(1.0, -24);
  const double g = d * u32 / (1.0 - d * u32);
  const double eh = std::expm1(h * std::log1p(u32));
  const double u = fmt == GT_F32 ? 0.0 : (fmt == GT_BF16 ? std::ldexp(1.0, -8) : std::ldexp(1.0, -4));
  const double up = 1.0 + std::ldexp(1.0, -20), dn = 1.0 - std::ldexp(1.0, -20);
  auto round_up = [](double x) {
    float f = (float)x;
    if ((double)f < x) f = std::nextafter(f, INFINITY);
    return f;
  };
  auto round_dn = [](double x) {
    float f = (float)x;
    if ((double)f > x) f = std::nextafter(f, 0.0f);
    return f;
  };
  Bound b;
  b.cu = round_up(up / ((1.0 - g) * (1.0 - u) * (1.0 - eh)));
  b.ct_up = round_up(up / ((1.0 - u) * (1.0 - eh)));
  b.cl = round_dn(dn / ((1.0 + g) * (1.0 + u) * (1.0 + eh)));
  b.ct_lo = round_up(up / ((1.0 + u) * (1.0 + eh)));
  return b;
}

gt_status ws_reserve_queries(gt_tree *t, int64_t B) {
  Workspace &w = t->ws;
  if (B <= w.q_cap) return GT_OK;
  cudaFree(w.qf32);
  cudaFree(w.qbf16);
  cudaFree(w.qn1);
  cudaFree(w.rho);
  cudaFree(w.bcnt);
  cudaFree(w.boff);
  w.qf32 = nullptr; w.qbf16 = nullptr; w.qn1 = nullptr; w.rho = nullptr; w.q_cap = 0;
  w.bcnt = nullptr; w.boff = nullptr;
  GT_CUDA(cudaMalloc(&w.qf32, (size_t)B * t->stride * sizeof(float)));
  GT_CUDA(cudaMalloc(&w.qbf16, (size_t)B * t->stride * sizeof(__nv_bfloat16)));
  GT_CUDA(cudaMalloc(&w.qn1, (size_t)B * sizeof(float)));
  GT_CUDA(cudaMalloc(&w.rho, (size_t)B * sizeof(float)));
  GT_CUDA(cudaMalloc(&w.bcnt, (size_t)(B + 1) * sizeof(int64_t)));
  GT_CUDA(cudaMalloc(&w.boff, (size_t)(B + 1) * sizeof(int64_t)));
  w.q_cap = B;
  return GT_OK;
}

gt_status ws_stage(gt_tree *t, int64_t bytes) {
  Workspace &w = t->ws;
  if (bytes <= w.stage_bytes) return GT_OK;
  cudaFree(w.stage);
  w.stage = nullptr;
  w.stage_bytes = 0;
  GT_CUDA(cudaMalloc(&w.stage, (size_t)bytes));
  w.stage_bytes = bytes;
  return GT_OK;
}

gt_status ws_reserve_frontier(gt_tree *t, int64_t pairs, int64_t results, int64_t rechecks) {
  Workspace &w = t->ws;
  if (!w.counters) {
    GT_CUDA(cudaMalloc(&w.counters, 64 * sizeof(uint32_t)));
    GT_CUDA(cudaMallocHost(&w.hcounters, 128 * sizeof(uint32_t)));
  }
  if (pairs > w.front_cap) {
    cudaFree(w.front[0]);
    cudaFree(w.front[1]);
    w.front[0] = w.front[1] = nullptr;
    w.front_cap = 0;
    GT_CUDA(cudaMalloc(&w.front[0], (size_t)pairs * sizeof(Pair)));
    GT_CUDA(cudaMalloc(&w.front[1], (size_t)pairs * sizeof(Pair)));
    w.front_cap = pairs;
  }
  if (results > w.res_cap) {
    Pair *n = nullptr;
    GT_CUDA(cudaMalloc(&n, (size_t)results * sizeof(Pair)));
    if (w.res) {
      // keep what earlier micro-batches of this call produced
      GT_CUDA(cudaMemcpy(n, w.res, (size_t)w.res_cap * sizeof(Pair), cudaMemcpyDeviceToDevice));
      cudaFree(w.res);
    }
    w.res = n;
    w.res_cap = results;
  }
  if (rechecks > w.rchk_cap) {
    cudaFree(w.rchk);
    w.rchk = nullptr;
    GT_CUDA(cudaMalloc(&w.rchk, (size_t)rechecks * sizeof(Pair)));
    w.rchk_cap = rechecks;
  }
  // FP8 leaves that straddle rho, for the BF16 pass (trees keeping both formats)
  const int64_t defer = std::max<int64_t>(1 << 16, w.front_cap / 4);
  if ((t->formats & (1u << GT_FP8)) && (t->formats & (1u << GT_BF16)) && defer > w.defer_cap) {
    cudaFree(w.defer);
    w.defer = nullptr;
    w.defer_cap = 0;
    GT_CUDA(cudaMalloc(&w.defer, (size_t)defer * sizeof(Pair)));
    w.defer_cap = defer;
  }
  return GT_OK;
}

void launch_prep_queries(gt_tree *t, const float *Q_dev, const float *rho_dev, int64_t B,
                         cudaStream_t s) {
  Workspace &w = t->ws;
  int blocks = (int)std::min<int64_t>((B + 7) / 8, (int64_t)t->sm_count * 8);
  if (blocks < 1) blocks = 1;
  k_prep_queries<<<blocks, 256, 0, s>>>(Q_dev, B, t->d_in, t->split_sign ? 1 : 0, t->stride,
                                        rho_dev, w.qf32, w.qbf16, w.qn1, w.rho, t->flags);
}

void launch_root(gt_tree *t, int64_t q0, int64_t b, Pair *out, uint32_t *count, cudaStream_t s) {
  int blocks = (int)std::min<int64_t>((b + 255) / 256, 1024);
  k_root<<<std::max(blocks, 1), 256, 0, s>>>(out, count, (uint32_t)q0, (uint32_t)b);
}

void prepare_level_kernels() {
  static bool done = false;
  if (done) return;
  done = true;
  ring_attr_modes<GT_F32, 8>();
  ring_attr_modes<GT_F32, 16>();
  ring_attr_modes<GT_BF16, 4>();
  ring_attr_modes<GT_BF16, 8>();
  ring_attr_modes<GT_FP8, 2>();
  ring_attr_modes<GT_FP8, 4>();
  ring_attr<GT_F32, 8, 5>();
  ring_attr<GT_F32, 8, 6>();
  ring_attr<GT_F32, 16, 5>();
  ring_attr<GT_F32, 16, 6>();
  ring_attr<GT_BF16, 4, 5>();
  ring_attr<GT_BF16, 4, 6>();
  ring_attr<GT_BF16, 8, 5>();
  ring_attr<GT_BF16, 8, 6>();
  drain_attr<GT_F32, 8>();
  drain_attr<GT_F32, 16>();
  drain_attr<GT_BF16, 4>();
  drain_attr<GT_BF16, 8>();
  drain_attr<GT_FP8, 2>();
  drain_attr<GT_FP8, 4>();
  cudaGetLastError();
}

bool drain_available(const gt_tree *t, int fmt, int cut) {
  uint32_t slot = 0;
  return cut >= 2 && cut <= kDrainMaxCut && t->layout == GT_LAYOUT_TREE &&
         t->pooling == GT_POOL_SUM && !t->split_sign &&
         ring_depth((int)((t->d * entry_bytes(fmt) + 15) / 16), &slot) > 0;
}

gt_status ws_reserve_drain(gt_tree *t) {
  Workspace &w = t->ws;
  // per warp: two lists of 32 << (c - 1) entries and the left items, for c
  // up to kDrainMaxCut
  const int64_t wcap = (int64_t)32 << (kDrainMaxCut - 1);
  const int64_t per_warp = 2 * wcap + (wcap + 1) / 2;
  const int64_t n = (int64_t)t->sm_count * kRingWarps * per_warp;
  if (w.drain && w.drain_cap >= n) return GT_OK;
  cudaFree(w.drain);
  w.drain = nullptr;
  w.drain_cap = 0;
  GT_CUDA(cudaMalloc(&w.drain, (size_t)n * sizeof(SibPair)));
  w.drain_cap = n;
  return GT_OK;
}

static void launch_deferred_bf16(gt_tree *t, cudaStream_t s);

void launch_drain(gt_tree *t, int fmt, int cut, const SibPair *root, const uint32_t *root_count,
                  cudaStream_t s, uint32_t *level_count, uint32_t *left_count, bool cleared) {
  Workspace &w = t->ws;
  LevelArgs a;
  std::memset(&a, 0, sizeof(a));
  a.expire = t->expire_waits;
  a.no_accept = t->split_sign ? 1 : 0;
  const int eb = entry_bytes(fmt);
  a.rows = fmt == GT_F32 ? reinterpret_cast<const uint8_t *>(t->rows32)
           : fmt == GT_BF16 ? reinterpret_cast<const uint8_t *>(t->rows16)
                            : t->rows8;
  a.scales = fmt == GT_FP8 ? t->scale8 : nullptr;
  a.row_bytes = t->stride * eb;
  a.nvec = (int)((t->d * eb + 15) / 16);
  a.qf32 = w.qf32;
  a.qstride = t->stride;
  a.qn1 = w.qn1;
  a.rho = w.rho;
  a.res = w.res;
  a.res_count = w.counters + kMaxLevels;
  a.res_cap = (uint32_t)std::min<int64_t>(w.res_cap, 0xffffffffLL);
  a.rchk = w.rchk;
  a.rchk_count = w.counters + kMaxLevels + 1;
  a.rchk_cap = (uint32_t)w.rchk_cap;
  a.flags = t->flags;
  a.q_lim = (uint32_t)w.q_cap;
  a.rows32 = t->rows32;
  a.bd32 = make_bound(GT_F32, 0, t->d);
  a.rows16 = t->rows16;
  a.bd16 = make_bound(GT_BF16, 0, t->d);
  a.refine_count = w.counters + kMaxLevels + 2;
  const bool defer = defer_active(t, fmt);
  if (defer) {
    if (!cleared) cudaMemsetAsync(w.counters + kDeferSlot, 0, sizeof(uint32_t), s);
    a.defer = w.defer;
    a.defer_count = w.counters + kDeferSlot;
    a.defer_cap = (uint32_t)w.defer_cap;
  }
  DrainArgs g;
  std::memset(&g, 0, sizeof(g));
  for (int h = 0; h < cut; ++h) {
    g.lvl[h].row0 = t->lvl_off[h];
    g.lvl[h].n_rows = (uint32_t)level_rows(t->N, h);
    g.lvl[h].bd = make_bound(fmt, bound_level(t, h), t->d);
  }
  g.root = root;
  g.root_count = root_count;
  g.root_cap = (uint32_t)(w.front_lim / 2);  // SibPairs are two Pairs wide
  g.head = w.counters + kDrainHeadSlot;
  g.level_count = level_count ? level_count : w.counters;
  g.left_count = left_count ? left_count : w.counters + kLeftItemsSlot;
  g.scratch = reinterpret_cast<SibPair *>(w.drain);
  g.wcap = 32u << (cut - 1);
  g.cut = cut;
  if (!cleared) cudaMemsetAsync(g.head, 0, sizeof(uint32_t), s);
  const bool wide = kv_for<GT_F32>(t->d) != 1024 / (32 * 4);
  if (fmt == GT_BF16)
    wide ? launch_drain_t<GT_BF16, 8>(a, g, t->sm_count, s) : launch_drain_t<GT_BF16, 4>(a, g, t->sm_count, s);
  else if (fmt == GT_FP8)
    wide ? launch_drain_t<GT_FP8, 4>(a, g, t->sm_count, s) : launch_drain_t<GT_FP8, 2>(a, g, t->sm_count, s);
  else
    wide ? launch_drain_t<GT_F32, 16>(a, g, t->sm_count, s) : launch_drain_t<GT_F32, 8>(a, g, t->sm_count, s);
  if (defer) launch_deferred_bf16(t, s);
}

bool launch_prefix(gt_tree *t, int fmt, int h, const SibPair *in, const uint32_t *in_count,
                   SibPair *out, uint32_t *out_count, cudaStream_t s) {
  Workspace &w = t->ws;
  LevelArgs a;
  std::memset(&a, 0, sizeof(a));
  a.expire = t->expire_waits;
  const int eb = entry_bytes(fmt);
  a.rows = fmt == GT_F32 ? reinterpret_cast<const uint8_t *>(t->pref32)
                         : reinterpret_cast<const uint8_t *>(t->pref16);
  a.row_bytes = t->stride * eb;
  a.nvec = (int)((t->d * eb + 15) / 16);
  a.n_rows = (uint32_t)level_rows(t->N, h);
  a.qf32 = w.qf32;
  a.qstride = t->stride;
  a.qn1 = w.qn1;
  a.rho = w.rho;
  a.in_count = in_count;
  a.in_cap = (uint32_t)(w.front_lim / 2);  // SibPairs are two Pairs wide
  a.out = reinterpret_cast<Pair *>(out);
  a.out_count = out_count;
  a.out_cap = (uint32_t)(w.front_lim / 2);
  a.res = w.res;
  a.res_count = w.counters + kMaxLevels;
  a.res_cap = (uint32_t)std::min<int64_t>(w.res_cap, 0xffffffffLL);
  a.rchk = w.rchk;
  a.rchk_count = w.counters + kMaxLevels + 1;
  a.rchk_cap = (uint32_t)w.rchk_cap;
  a.flags = t->flags;
  a.bd = make_bound(fmt, bound_level(t, h), t->d);
  a.batch = (uint32_t)t->ring_batch;
  a.q_lim = (uint32_t)w.q_cap;
  a.rows32 = t->rows32;  // the items (FP32 re-score of doubtful leaves)
  a.bd32 = make_bound(GT_F32, 0, t->d);
  a.refine_count = w.counters + kMaxLevels + 2;
  a.pre_h = (uint32_t)h;
  a.pre_c = (uint32_t)t->pc;
  a.n_items = (uint32_t)t->N;
  {
    double cu, cl;
    gemm_bound(bound_level(t, t->pc), &cu, &cl);
    float fu = (float)cu, fl = (float)cl;
    if ((double)fu < cu) fu = std::nextafter(fu, INFINITY);
    if ((double)fl > cl) fl = std::nextafter(fl, 0.0f);
    a.g_cu = fu;
    a.g_cl = fl;
  }
  const bool wide = kv_for<GT_F32>(t->d) != 1024 / (32 * 4);
  if (fmt == GT_BF16) {
    if (h > 1)
      return wide ? launch_ring<GT_BF16, 8, 5>(a, in, out, t->sm_count, s)
                  : launch_ring<GT_BF16, 4, 5>(a, in, out, t->sm_count, s);
    return wide ? launch_ring<GT_BF16, 8, 6>(a, in, out, t->sm_count, s)
                : launch_ring<GT_BF16, 4, 6>(a, in, out, t->sm_count, s);
  }
  if (h > 1)
    return wide ? launch_ring<GT_F32, 16, 5>(a, in, out, t->sm_count, s)
                : launch_ring<GT_F32, 8, 5>(a, in, out, t->sm_count, s);
  return wide ? launch_ring<GT_F32, 16, 6>(a, in, out, t->sm_count, s)
              : launch_ring<GT_F32, 8, 6>(a, in, out, t->sm_count, s);
}

bool defer_active(const gt_tree *t, int fmt) {
  // split signed rows accept no leaf on a bound: nothing is deferred
  return fmt == GT_FP8 && t->ws.defer && t->rows16 && !t->split_sign;
}

// The deferred FP8 leaf pairs, re-scored from the BF16 item rows by the
// ring-fed leaf kernel (their straddlers go on to the FP32 refine and the FP64
// recheck as usual).
static void launch_deferred_bf16(gt_tree *t, cudaStream_t s) {
  Workspace &w = t->ws;
  LevelArgs a;
  std::memset(&a, 0, sizeof(a));
  a.expire = t->expire_waits;
  a.rows = reinterpret_cast<const uint8_t *>(t->rows16);  // level 0 starts at row 0
  a.row_bytes = t->stride * 2;
  a.nvec = (int)((t->d * 2 + 15) / 16);
  a.n_rows = (uint32_t)t->N;
  a.qf32 = w.qf32;
  a.qstride = t->stride;
  a.qn1 = w.qn1;
  a.rho = w.rho;
  a.in = w.defer;
  a.in_count = w.counters + kDeferSlot;
  a.in_cap = (uint32_t)w.defer_cap;
  a.res = w.res;
  a.res_count = w.counters + kMaxLevels;
  a.res_cap = (uint32_t)std::min<int64_t>(w.res_cap, 0xffffffffLL);
  a.rchk = w.rchk;
  a.rchk_count = w.counters + kMaxLevels + 1;
  a.rchk_cap = (uint32_t)w.rchk_cap;
  a.flags = t->flags;
  a.bd = make_bound(GT_BF16, 0, t->d);
  a.batch = (uint32_t)t->ring_batch;
  a.q_lim = (uint32_t)w.q_cap;
  a.rows32 = t->rows32;
  a.bd32 = make_bound(GT_F32, 0, t->d);
  a.refine_count = w.counters + kMaxLevels + 2;
  a.inflight = kInflightRing;
  launch_level_f<GT_BF16, true>(a, t->d, t->sm_count, s);
}

void launch_level(gt_tree *t, int fmt, int h, int64_t /*q0*/, const Pair *in,
                  const uint32_t *in_count, Pair *out, uint32_t *out_count, cudaStream_t s) {
  Workspace &w = t->ws;
  LevelArgs a;
  std::memset(&a, 0, sizeof(a));
  a.expire = t->expire_waits;
  const int eb = entry_bytes(fmt);
  const uint8_t *base = fmt == GT_F32 ? reinterpret_cast<const uint8_t *>(t->rows32)
                        : fmt == GT_BF16 ? reinterpret_cast<const uint8_t *>(t->rows16)
                                         : t->rows8;
  a.rows = base + (size_t)t->lvl_off[h] * t->stride * eb;
  a.scales = fmt == GT_FP8 ? t->scale8 + t->lvl_off[h] : nullptr;
  a.row_bytes = t->stride * eb;
  a.nvec = (int)((t->d * eb + 15) / 16);
  a.n_child = h > 0 ? (uint32_t)level_rows(t->N, h - 1) : 0u;
  a.n_rows = (uint32_t)level_rows(t->N, h);
  a.qf32 = w.qf32;
  a.qstride = t->stride;
  a.qn1 = w.qn1;
  a.rho = w.rho;
  a.in = in;
  a.in_count = in_count;
  a.in_cap = (uint32_t)w.front_lim;
  a.out = out;
  a.out_count = out_count;
  a.out_cap = (uint32_t)w.front_lim;
  a.res = w.res;
  a.res_count = w.counters + kMaxLevels;
  a.res_cap = (uint32_t)std::min<int64_t>(w.res_cap, 0xffffffffLL);
  a.rchk = w.rchk;
  a.rchk_count = w.counters + kMaxLevels + 1;
  a.rchk_cap = (uint32_t)w.rchk_cap;
  a.flags = t->flags;
  a.bd = make_bound(fmt, bound_level(t, h), t->d);
  a.batch = (uint32_t)t->ring_batch;
  a.q_lim = (uint32_t)w.q_cap;
  a.rows32 = t->rows32;  // level 0 starts at row 0
  a.bd32 = make_bound(GT_F32, 0, t->d);
  a.rows16 = t->rows16;
  a.bd16 = make_bound(GT_BF16, 0, t->d);
  a.refine_count = w.counters + kMaxLevels + 2;
  a.inflight = t->tuned_g[fmt];
  const int64_t d = t->d;
  if (h > 0) {
    if (fmt == GT_F32) launch_level_f<GT_F32, false>(a, d, t->sm_count, s);
    else if (fmt == GT_BF16) launch_level_f<GT_BF16, false>(a, d, t->sm_count, s);
    else launch_level_f<GT_FP8, false>(a, d, t->sm_count, s);
  } else {
    a.no_accept = t->split_sign ? 1 : 0;
    const bool defer = defer_active(t, fmt);
    if (defer) {
      cudaMemsetAsync(w.counters + kDeferSlot, 0, sizeof(uint32_t), s);
      a.defer = w.defer;
      a.defer_count = w.counters + kDeferSlot;
      a.defer_cap = (uint32_t)w.defer_cap;
    }
    if (fmt == GT_F32) launch_level_f<GT_F32, true>(a, d, t->sm_count, s);
    else if (fmt == GT_BF16) launch_level_f<GT_BF16, true>(a, d, t->sm_count, s);
    else launch_level_f<GT_FP8, true>(a, d, t->sm_count, s);
    if (defer) launch_deferred_bf16(t, s);
  }
}

void launch_pair_bounds(gt_tree *t, int fmt, int h, const int32_t *pairs, int64_t n, int64_t n_queries,
                        float *out, cudaStream_t s) {
  Workspace &w = t->ws;
  LevelArgs a;
  std::memset(&a, 0, sizeof(a));
  a.expire = t->expire_waits;
  const int eb = entry_bytes(fmt);
  const uint8_t *base = fmt == GT_F32 ? reinterpret_cast<const uint8_t *>(t->rows32)
                        : fmt == GT_BF16 ? reinterpret_cast<const uint8_t *>(t->rows16)
                                         : t->rows8;
  a.rows = base + (size_t)t->lvl_off[h] * t->stride * eb;
  a.scales = fmt == GT_FP8 ? t->scale8 + t->lvl_off[h] : nullptr;
  a.row_bytes = t->stride * eb;
  a.nvec = (int)((t->d * eb + 15) / 16);
  a.n_rows = (uint32_t)level_rows(t->N, h);
  a.qf32 = w.qf32;
  a.qstride = t->stride;
  a.qn1 = w.qn1;
  a.bd = make_bound(fmt, bound_level(t, h), t->d);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, (int64_t)t->sm_count * 8));
  const uint32_t nq = (uint32_t)n_queries;
  auto go = [&](auto kern) { kern<<<blocks, 256, 0, s>>>(a, pairs, n, nq, out); };
  const bool narrow32 = kv_for<GT_F32>(t->d) == 1024 / (32 * 4);
  if (fmt == GT_F32) {
    if (narrow32) go(k_pair_bounds<GT_F32, 8>); else go(k_pair_bounds<GT_F32, 16>);
  } else if (fmt == GT_BF16) {
    if (narrow32) go(k_pair_bounds<GT_BF16, 4>); else go(k_pair_bounds<GT_BF16, 8>);
  } else {
    if (narrow32) go(k_pair_bounds<GT_FP8, 2>); else go(k_pair_bounds<GT_FP8, 4>);
  }
}

void launch_level_sub(gt_tree *t, int fmt, int h, const SibPair *in, const uint32_t *in_count,
                      void *out, uint32_t *out_count, cudaStream_t s, bool entries_out) {
  Workspace &w = t->ws;
  LevelArgs a;
  std::memset(&a, 0, sizeof(a));
  a.expire = t->expire_waits;
  const int eb = entry_bytes(fmt);
  const uint8_t *base = fmt == GT_F32 ? reinterpret_cast<const uint8_t *>(t->rows32)
                        : fmt == GT_BF16 ? reinterpret_cast<const uint8_t *>(t->rows16)
                                         : t->rows8;
  a.rows = base + (size_t)t->lvl_off[h] * t->stride * eb;
  a.scales = fmt == GT_FP8 ? t->scale8 + t->lvl_off[h] : nullptr;
  a.row_bytes = t->stride * eb;
  a.nvec = (int)((t->d * eb + 15) / 16);
  a.n_rows = (uint32_t)level_rows(t->N, h);
  a.n_child = (uint32_t)level_rows(t->N, h - 1);
  a.qf32 = w.qf32;
  a.qstride = t->stride;
  a.qn1 = w.qn1;
  a.rho = w.rho;
  a.in_count = in_count;
  a.in_cap = (uint32_t)(w.front_lim / 2);                       // SibPairs are two Pairs wide
  a.out_count = out_count;
  const bool to_leaf = h == 1 && !entries_out;
  a.out_cap = (uint32_t)(to_leaf ? w.front_lim : w.front_lim / 2);
  a.flags = t->flags;
  a.bd = make_bound(fmt, bound_level(t, h), t->d);
  a.batch = (uint32_t)t->ring_batch;
  a.q_lim = (uint32_t)w.q_cap;
  const bool wide = kv_for<GT_F32>(t->d) != 1024 / (32 * 4);
  // the subtraction levels take the ring-fed gather whenever its slots fit
  {
    bool done;
    if (fmt == GT_BF16)
      done = wide ? (to_leaf ? launch_ring<GT_BF16, 8, 3>(a, in, out, t->sm_count, s)
                             : launch_ring<GT_BF16, 8, 2>(a, in, out, t->sm_count, s))
                  : (to_leaf ? launch_ring<GT_BF16, 4, 3>(a, in, out, t->sm_count, s)
                             : launch_ring<GT_BF16, 4, 2>(a, in, out, t->sm_count, s));
    else if (fmt == GT_FP8)
      done = wide ? (to_leaf ? launch_ring<GT_FP8, 4, 3>(a, in, out, t->sm_count, s)
                             : launch_ring<GT_FP8, 4, 2>(a, in, out, t->sm_count, s))
                  : (to_leaf ? launch_ring<GT_FP8, 2, 3>(a, in, out, t->sm_count, s)
                             : launch_ring<GT_FP8, 2, 2>(a, in, out, t->sm_count, s));
    else
      done = wide ? (to_leaf ? launch_ring<GT_F32, 16, 3>(a, in, out, t->sm_count, s)
                             : launch_ring<GT_F32, 16, 2>(a, in, out, t->sm_count, s))
                  : (to_leaf ? launch_ring<GT_F32, 8, 3>(a, in, out, t->sm_count, s)
                             : launch_ring<GT_F32, 8, 2>(a, in, out, t->sm_count, s));
    if (done) return;
  }
  auto go = [&](auto kern) {
    static int per_sm = 0;
    const int grid = grid_for((const void *)kern, 256, t->sm_count, per_sm);
    kern<<<grid, 256, 0, s>>>(a, in, out);
  };
  if (fmt == GT_BF16) {
    if (wide) { if (to_leaf) go(k_level_sub<GT_BF16, 8, true>); else go(k_level_sub<GT_BF16, 8, false>); }
    else { if (to_leaf) go(k_level_sub<GT_BF16, 4, true>); else go(k_level_sub<GT_BF16, 4, false>); }
  } else if (fmt == GT_FP8) {
    if (wide) { if (to_leaf) go(k_level_sub<GT_FP8, 4, true>); else go(k_level_sub<GT_FP8, 4, false>); }
    else { if (to_leaf) go(k_level_sub<GT_FP8, 2, true>); else go(k_level_sub<GT_FP8, 2, false>); }
  } else {
    if (wide) { if (to_leaf) go(k_level_sub<GT_F32, 16, true>); else go(k_level_sub<GT_F32, 16, false>); }
    else { if (to_leaf) go(k_level_sub<GT_F32, 8, true>); else go(k_level_sub<GT_F32, 8, false>); }
  }
}

void launch_items_sub(gt_tree *t, int fmt, const SibPair *in, const uint32_t *in_count,
                      uint32_t *left_count, cudaStream_t s) {
  Workspace &w = t->ws;
  LevelArgs a;
  std::memset(&a, 0, sizeof(a));
  a.expire = t->expire_waits;
  const int eb = entry_bytes(fmt);
  const uint8_t *base = fmt == GT_F32 ? reinterpret_cast<const uint8_t *>(t->rows32)
                        : fmt == GT_BF16 ? reinterpret_cast<const uint8_t *>(t->rows16)
                                         : t->rows8;
  a.rows = base;  // level 0
  a.scales = fmt == GT_FP8 ? t->scale8 : nullptr;
  a.row_bytes = t->stride * eb;
  a.nvec = (int)((t->d * eb + 15) / 16);
  a.n_rows = (uint32_t)t->N;
  a.no_accept = t->split_sign ? 1 : 0;
  a.qf32 = w.qf32;
  a.qstride = t->stride;
  a.qn1 = w.qn1;
  a.rho = w.rho;
  a.in_count = in_count;
  a.in_cap = (uint32_t)(w.front_lim / 2);
  a.out = nullptr;              // the left items are decided in the launch;
  a.out_count = left_count;     // their count is kept with the tests
  a.out_cap = 0;
  a.res = w.res;
  a.res_count = w.counters + kMaxLevels;
  a.res_cap = (uint32_t)std::min<int64_t>(w.res_cap, 0xffffffffLL);
  a.rchk = w.rchk;
  a.rchk_count = w.counters + kMaxLevels + 1;
  a.rchk_cap = (uint32_t)w.rchk_cap;
  a.flags = t->flags;
  a.bd = make_bound(fmt, 0, t->d);
  a.batch = (uint32_t)t->ring_batch;
  a.q_lim = (uint32_t)w.q_cap;
  a.rows32 = t->rows32;
  a.bd32 = make_bound(GT_F32, 0, t->d);
  a.rows16 = t->rows16;
  a.bd16 = make_bound(GT_BF16, 0, t->d);
  a.refine_count = w.counters + kMaxLevels + 2;
  const bool wide = kv_for<GT_F32>(t->d) != 1024 / (32 * 4);
  const bool defer = defer_active(t, fmt);
  if (defer) {
    cudaMemsetAsync(w.counters + kDeferSlot, 0, sizeof(uint32_t), s);
    a.defer = w.defer;
    a.defer_count = w.counters + kDeferSlot;
    a.defer_cap = (uint32_t)w.defer_cap;
  }
  if (fmt == GT_BF16)
    wide ? launch_ring<GT_BF16, 8, 4>(a, in, nullptr, t->sm_count, s)
         : launch_ring<GT_BF16, 4, 4>(a, in, nullptr, t->sm_count, s);
  else if (fmt == GT_FP8)
    wide ? launch_ring<GT_FP8, 4, 4>(a, in, nullptr, t->sm_count, s)
         : launch_ring<GT_FP8, 2, 4>(a, in, nullptr, t->sm_count, s);
  else
    wide ? launch_ring<GT_F32, 16, 4>(a, in, nullptr, t->sm_count, s)
         : launch_ring<GT_F32, 8, 4>(a, in, nullptr, t->sm_count, s);
  if (defer) launch_deferred_bf16(t, s);
}

bool items_sub_available(gt_tree *t, int fmt) {
  uint32_t slot = 0;
  return ring_depth((int)((t->d * entry_bytes(fmt) + 15) / 16), &slot) > 0;
}

static RecheckArgs recheck_args(gt_tree *t) {
  Workspace &w = t->ws;
  RecheckArgs a;
  a.rchk = w.rchk;
  a.count = w.counters + kMaxLevels + 1;
  a.cap = (uint32_t)w.rchk_cap;
  a.rows32 = t->rows32;
  a.stride = t->stride;
  a.nv4 = (int)((t->d + 3) / 4);
  a.d_half = t->split_sign ? t->d_in : 0;
  a.qf32 = w.qf32;
  a.rho = w.rho;
  a.res = w.res;
  a.res_count = w.counters + kMaxLevels;
  a.res_cap = (uint32_t)w.res_cap;
  a.q_lim = (uint32_t)w.q_cap;
  a.n_items = (uint32_t)t->N;
  a.flags = t->flags;
  return a;
}

void launch_recheck(gt_tree *t, int64_t /*q0*/, cudaStream_t s) {
  static int per_sm = 0;
  const int grid = grid_for((const void *)k_recheck, 256, t->sm_count, per_sm);
  k_recheck<<<grid, 256, 0, s>>>(recheck_args(t));
}

// CSR assembly of the result pairs res[0..n) into offsets (B + 1) and ids.
// `cnt` (B + 1 int64, zeroed by the caller) is the per-query counter, then the
// fill cursor, then the list of segments too long for one warp; `list_n` is a
// device counter (cleared here).  With n_dev the count is read on the device
// (clamped to n), so the work can be enqueued before the count is known.
void launch_csr_into(gt_tree *t, const Pair *res, uint32_t n, const uint32_t *n_dev, int64_t q_lo,
                     int64_t B, int64_t *cnt, int64_t *off, int32_t *ids, uint32_t *list_n,
                     cudaStream_t s, bool recheck) {
  const bool any = n > 0;
  const int blocks = n_dev ? t->sm_count * 4
                           : (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, t->sm_count * 8));
  // the results' queries lie in [q_lo, q_lo + B): count and fill index the
  // arrays by query, the scan and the sorts see the range only
  int64_t *cnt_r = cnt + q_lo, *off_r = off + q_lo;
  const uint32_t q_hi = (uint32_t)(q_lo + B);
  if (B >= 1 && B <= kCsrSmallMax) {
    // one block for the CSR of a few queries (and, asked to, their recheck)
    k_csr_small<<<1, 1024, 0, s>>>(res, n, n_dev, (uint32_t)q_lo, (uint32_t)B, off_r, t->perm, ids,
                                   t->flags, recheck_args(t), recheck ? 1 : 0);
    return;
  }
  if (recheck) launch_recheck(t, 0, s);
  if (any) k_csr_count<<<blocks, 256, 0, s>>>(res, n, n_dev, (uint32_t)q_lo, q_hi, cnt, t->flags);
  k_scan<<<1, 1024, 0, s>>>(cnt_r, B, off_r);
  cudaMemsetAsync(cnt_r, 0, (size_t)(B + 1) * sizeof(int64_t), s);
  if (any && B) {
    cudaMemsetAsync(list_n, 0, sizeof(uint32_t), s);
    k_csr_fill<<<blocks, 256, 0, s>>>(res, n, n_dev, (uint32_t)q_lo, q_hi, off, cnt, t->perm, ids);
    const unsigned wblocks = (unsigned)((B * 32 + 255) / 256);
    k_csr_sort_warp<8><<<wblocks, 256, 0, s>>>(off_r, ids, B, 0, nullptr, nullptr);
    k_csr_sort_warp<16><<<wblocks, 256, 0, s>>>(off_r, ids, B, 256, cnt_r, list_n);
    k_csr_sort<<<t->sm_count * 2, 256, 0, s>>>(off_r, ids, cnt_r, list_n);
  }
}

void launch_bucket(gt_tree *t, bool sib, const void *in, void *out, const uint32_t *n_dev,
                   uint32_t cap, int64_t q0, int64_t b, cudaStream_t s) {
  Workspace &w = t->ws;
  // a full SM's worth of warps each: the passes are bound by load and
  // atomic latency, not by bandwidth
  const int blocks = t->sm_count * 8;
  const uint32_t uq0 = (uint32_t)q0, ub = (uint32_t)b;
  cudaMemsetAsync(w.bcnt, 0, (size_t)(b + 1) * sizeof(int64_t), s);
  if (sib)
    k_bucket_count<<<blocks, 256, 0, s>>>(reinterpret_cast<const SibPair *>(in), n_dev, cap, uq0, ub,
                                           w.bcnt, t->flags);
  else
    k_bucket_count<<<blocks, 256, 0, s>>>(reinterpret_cast<const Pair *>(in), n_dev, cap, uq0, ub,
                                           w.bcnt, t->flags);
  k_scan<<<1, 1024, 0, s>>>(w.bcnt, b, w.boff);
  cudaMemsetAsync(w.bcnt, 0, (size_t)(b + 1) * sizeof(int64_t), s);
  if (sib)
    k_bucket_scatter<<<blocks, 256, 0, s>>>(reinterpret_cast<const SibPair *>(in), n_dev, cap, uq0, ub,
                                             w.boff, w.bcnt, reinterpret_cast<SibPair *>(out));
  else
    k_bucket_scatter<<<blocks, 256, 0, s>>>(reinterpret_cast<const Pair *>(in), n_dev, cap, uq0, ub,
                                             w.boff, w.bcnt, reinterpret_cast<Pair *>(out));
  k_bucket_fix_count<<<1, 32, 0, s>>>(const_cast<uint32_t *>(n_dev), cap, w.boff, ub);
}

}  // namespace gt
