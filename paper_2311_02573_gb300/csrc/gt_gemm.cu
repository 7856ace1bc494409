// Dense scoring of every (query, pool) pair of one tree level on the 5th
// generation tensor cores: S = Q_bf16 . P_bf16^T with FP32 accumulation.
//
// This replaces the upper levels of the traversal (a pool pruned above level
// h would have been pruned at level h too, since all scores are >= 0) and is
// also the exhaustive scan of the paper's Exh comparator (level 0).
//
// Persistent, warp-specialised kernel, one CTA per SM:
//   warp 0      TMA producer: 128x64 query tile + 256x64 pool tile per stage
//               (128-byte swizzle), 4-stage ring guarded by mbarriers;
//   warp 1      allocates 512 TMEM columns (two 128x256 FP32 accumulators)
//               and issues tcgen05.mma (M=128 queries, N=256 pools, K=16);
//   warps 2..9  epilogue, two warps per TMEM lane quarter, each taking half
//               of the columns: tcgen05.ld 64 columns at a time, threshold
//               with a rigorous bound, a warp vote, and the rare survivors
//               appended with one atomic per warp.
// Each epilogue thread owns one query (one TMEM lane).
//
// Every mbarrier wait is bounded (%globaltimer, 1 s); on expiry the kernel
// raises the timeout flag, drains what it has in flight and returns.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "gt_internal.cuh"

namespace gt {

namespace {

constexpr int BM = 128;   // queries per MMA (TMEM lanes)
constexpr int BK = 64;    // K entries per stage: 128 bytes of BF16

// CTA tile: MSUB x 128 queries by BN pools.  MSUB = 1 keeps two accumulator
// buffers in TMEM so the epilogue of one tile overlaps the MMAs of the next;
// MSUB = 2 shares every pool stage between two 128-query MMAs (halving the
// shared-memory bytes an SM ingests per FLOP) with one accumulator buffer
// and eight epilogue warps.  The stage ring uses as many stages as fit in
// 192 KiB.
template <int MSUB_, int BN_>
struct Tile {
  static constexpr int MSUB = MSUB_;
  static constexpr int BN = BN_;
  static constexpr int BMC = BM * MSUB;                  // queries per CTA tile
  static constexpr int A_SUB = BM * BK * 2;              // 16 KiB per 128-query slab
  static constexpr int A_BYTES = MSUB * A_SUB;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int STAGES = (192 * 1024) / STAGE_BYTES;
  static constexpr int NBUF = MSUB == 1 ? 2 : 1;          // accumulator buffers
  static constexpr int TMEM_COLS = NBUF * MSUB * BN;      // 512 / 256 / 512
  // epilogue warps: four per 128-query accumulator (one per TMEM lane
  // quarter); with one accumulator, two per lane quarter, each taking half
  // of the tile's columns
  static constexpr int EPI_SPLIT = MSUB == 1 ? 2 : 1;
  static constexpr int EPI_WARPS = 4 * MSUB * EPI_SPLIT;
  static constexpr int THREADS = 64 + 32 * EPI_WARPS;     // producer, MMA, epilogue
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
};
constexpr uint64_t kWaitNs = 1000000000ull;

struct DenseArgs {
  int mode;            // 0: children of survivors; 1: leaf decisions; 2: raw scores
  uint32_t n_pools;    // rows of the level
  uint32_t q0, nq;     // queries [q0, q0 + nq)
  int k_blocks;
  uint32_t n_child;    // rows at level h-1 (mode 0)
  const float *rho;    // per query threshold; the epilogue keeps (or, for mode
                       // 0 and 3, takes as a candidate) a pool when acc >=
                       // rho * inv_cu rounded down, and accepts an item (mode 1)
                       // when acc >= rho * inv_cl rounded up
  float inv_cu, inv_cl;
  Pair *out;
  uint32_t *out_count;
  uint32_t out_cap;
  Pair *rchk;
  uint32_t *rchk_count;
  uint32_t rchk_cap;
  float *scores;       // mode 2: [nq x ld]
  int64_t ld;
  int *flags;
  float cu_up;         // mode 3: upper bound on a pool's exact score = acc * cu_up
  float cl_dn;         // mode 3: lower bound on a pool's exact score = acc * cl_dn
  int pad_lower;       // mode 3: the entry's fourth word holds that lower bound (tree
                       // layout) rather than the raw score (prefix layout)
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of barrier `bar`, at most kWaitNs; false on expiry
// or when another role already gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = now_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (now_ns() - t0 > kWaitNs) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

// UMMA shared-memory descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes in 8-row (1024-byte) atoms.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);       // start address
  d |= (uint64_t)1 << 16;                         // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;               // stride byte offset: one 8-row atom
  d |= (uint64_t)1 << 46;                         // descriptor version (tcgen05)
  d |= (uint64_t)2 << 61;                         // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: BF16 x BF16 -> FP32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4)                      // D format: F32
         | (1u << 7)                    // A format: BF16
         | (1u << 10)                   // B format: BF16
         | ((uint32_t)(N >> 3) << 17)   // N / 8
         | ((uint32_t)(M >> 4) << 24);  // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 64 consecutive 32-bit columns of the thread's TMEM lane, one wait
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&r)[64]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
        "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
        "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
        "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, v, off);
    if (lane >= off) v += t;
  }
  return v;
}

// Reserve `n` slots per lane of a list with one atomic per warp; returns the
// lane's first slot (0xffffffff when n is 0).  A list that runs past its
// capacity raises the overflow flag; the caller writes only the slots below
// the capacity, so a list that overflowed still has no hole below it (the
// next pass reads min(count, cap) entries).
__device__ __forceinline__ uint32_t warp_reserve(uint32_t *count, uint32_t cap, int *flags,
                                                 uint32_t n) {
  const uint32_t incl = warp_incl_scan(n);
  const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
  if (tot == 0) return 0xffffffffu;
  uint32_t base = 0;
  if ((threadIdx.x & 31) == 0) base = atomicAdd(count, tot);
  base = __shfl_sync(0xffffffffu, base, 0);
  if (n == 0) return 0xffffffffu;
  const uint32_t pos = base + incl - n;
  if ((uint64_t)pos + n > cap) atomicExch(&flags[kFlagOverflow], 1);
  return pos;
}

// Element hh * 32 + i of r for a run-time i in [0, 32): a select tree over
// compile-time indices, so r stays in registers.
__device__ __forceinline__ uint32_t pick32(const uint32_t (&r)[64], int hh, int i) {
  uint32_t x[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const uint32_t lo = hh ? r[32 + 2 * k] : r[2 * k];
    const uint32_t hi = hh ? r[33 + 2 * k] : r[2 * k + 1];
    x[k] = (i & 1) ? hi : lo;
  }
#pragma unroll
  for (int w = 8, b = 2; w >= 1; w >>= 1, b <<= 1) {
#pragma unroll
    for (int k = 0; k < w; ++k) x[k] = (i & b) ? x[2 * k + 1] : x[2 * k];
  }
  return x[0];
}

// Epilogue of one accumulator tile for the calling thread's query `row`
// (within the batch): BN columns starting at TMEM address `tcol` (the thread's
// lane and the buffer's first column), scoring pools col0 .. col0 + BN - 1.
// Survivors are rare, so each 32-column group costs one compare per column
// and a warp vote; the appends run only when some lane of the warp has one.
// The accumulator registers are indexed only with compile-time indices (no
// local-memory copy of them).
template <int BN>
__device__ __forceinline__ void epilogue_tile(const DenseArgs &a, uint32_t tcol, uint32_t row,
                                              uint32_t col0) {
  const bool qvalid = row < a.nq;
  const uint32_t q = a.q0 + row;
  const float r = qvalid ? a.rho[q] : 0.f;
  const float keep = qvalid ? __fmul_rd(r, a.inv_cu) : INFINITY;
  const float accept = (qvalid && a.mode == 1) ? __fmul_ru(r, a.inv_cl) : INFINITY;
#pragma unroll 1
  for (int c = 0; c < BN / 64; ++c) {
    uint32_t r[64];
    tmem_ld64(tcol + c * 64, r);
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const uint32_t m0 = col0 + c * 64 + hh * 32;
      if (a.mode == 2) {
        if (qvalid) {
#pragma unroll
          for (int i = 0; i < 32; ++i)
            if (m0 + i < a.n_pools)
              a.scores[(int64_t)row * a.ld + m0 + i] = __uint_as_float(r[hh * 32 + i]);
        }
        continue;
      }
      // columns past the level's last pool, and rows past the micro-batch
      // (their operand rows are other slots' data, which may hold anything,
      // even infinities that would pass an infinite threshold), are never kept
      const uint32_t lim = a.n_pools > m0 ? min(a.n_pools - m0, 32u) : 0u;
      const uint32_t in_mask = !qvalid ? 0u : (lim >= 32u ? 0xffffffffu : ((1u << lim) - 1u));
      uint32_t m_keep = 0;
#pragma unroll
      for (int i = 0; i < 32; ++i)
        m_keep |= (__uint_as_float(r[hh * 32 + i]) >= keep ? 1u : 0u) << i;
      m_keep &= in_mask;
      if (!__any_sync(0xffffffffu, m_keep != 0u)) continue;
      if (a.mode == 3) {
        // subtraction path: one entry per surviving pool, with its upper bound
        uint32_t pos = warp_reserve(a.out_count, a.out_cap, a.flags, __popc(m_keep));
        if (pos != 0xffffffffu) {
          SibPair *o = reinterpret_cast<SibPair *>(a.out);
          for (uint32_t mk = m_keep; mk; mk &= mk - 1, ++pos) {
            const int i = __ffs(mk) - 1;
            SibPair e;
            e.q = q;
            e.p = m0 + i;
            const float raw = __uint_as_float(pick32(r, hh, i));
            e.U = __fmul_ru(raw, a.cu_up);
            // tree layout: the pool's lower bound (none for the level's last
            // pool, the one pool an insert can extend while a served group
            // still holds this entry); prefix layout: the raw score, the
            // block total the splits below difference against
            e.pad = !a.pad_lower ? pick32(r, hh, i)
                                 : __float_as_uint(m0 + i + 1u < a.n_pools ? __fmul_rd(raw, a.cl_dn) : 0.f);
            if (pos < a.out_cap) o[pos] = e;
          }
        }
      } else if (a.mode == 0) {
        // children of every surviving pool: (q, 2m) and (q, 2m+1) if it exists
        uint32_t n = 0;
        for (uint32_t mk = m_keep; mk; mk &= mk - 1) {
          const uint32_t m = m0 + __ffs(mk) - 1;
          n += 1u + (2u * m + 1u < a.n_child ? 1u : 0u);
        }
        uint32_t pos = warp_reserve(a.out_count, a.out_cap, a.flags, n);
        if (pos != 0xffffffffu) {
          for (uint32_t mk = m_keep; mk; mk &= mk - 1) {
            const uint32_t m = m0 + __ffs(mk) - 1;
            Pair p0;
            p0.q = q;
            p0.j = 2u * m;
            if (pos < a.out_cap) a.out[pos] = p0;
            ++pos;
            if (2u * m + 1u < a.n_child) {
              Pair p1;
              p1.q = q;
              p1.j = 2u * m + 1u;
              if (pos < a.out_cap) a.out[pos] = p1;
              ++pos;
            }
          }
        }
      } else {
        // items: accepted outright, or straddling rho -> FP64 recheck
        uint32_t m_acc = 0;
#pragma unroll
        for (int i = 0; i < 32; ++i)
          m_acc |= (__uint_as_float(r[hh * 32 + i]) >= accept ? 1u : 0u) << i;
        m_acc &= m_keep;
        const uint32_t m_rc = m_keep & ~m_acc;
        uint32_t pos = warp_reserve(a.out_count, a.out_cap, a.flags, __popc(m_acc));
        if (pos != 0xffffffffu) {
          for (uint32_t mk = m_acc; mk; mk &= mk - 1, ++pos) {
            Pair p;
            p.q = q;
            p.j = m0 + __ffs(mk) - 1;
            if (pos < a.out_cap) a.out[pos] = p;
          }
        }
        pos = warp_reserve(a.rchk_count, a.rchk_cap, a.flags, __popc(m_rc));
        if (pos != 0xffffffffu) {
          for (uint32_t mk = m_rc; mk; mk &= mk - 1, ++pos) {
            Pair p;
            p.q = q;
            p.j = m0 + __ffs(mk) - 1;
            if (pos < a.rchk_cap) a.rchk[pos] = p;
          }
        }
      }
    }
  }
}

template <int MSUB, int BN>
__global__ void __launch_bounds__(Tile<MSUB, BN>::THREADS, 1)
    k_dense(const __grid_constant__ CUtensorMap tmap_q, const __grid_constant__ CUtensorMap tmap_p,
            const DenseArgs a) {
  using T = Tile<MSUB, BN>;
  constexpr int STAGES = T::STAGES;
  constexpr int A_BYTES = T::A_BYTES;
  constexpr int B_BYTES = T::B_BYTES;
  constexpr int STAGE_BYTES = T::STAGE_BYTES;
  constexpr int TMEM_COLS = T::TMEM_COLS;
  constexpr int NBUF = T::NBUF;
  constexpr int BMC = T::BMC;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  uint8_t *gbase = smem_raw + (base - smem_u32(smem_raw));
  const uint32_t sA = base;                          // STAGES x A_BYTES
  const uint32_t sB = base + STAGES * A_BYTES;       // STAGES x B_BYTES
  uint64_t *bars = reinterpret_cast<uint64_t *>(gbase + STAGES * STAGE_BYTES);
  const uint32_t full0 = smem_u32(bars);
  const uint32_t empty0 = full0 + 8 * STAGES;
  const uint32_t tfull0 = empty0 + 8 * STAGES;
  const uint32_t tempty0 = tfull0 + 16;
  const uint32_t done_bar = tempty0 + 16;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(gbase + STAGES * STAGE_BYTES + 8 * (2 * STAGES + 5));
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t n_qt = (a.nq + BMC - 1) / BMC;
  const uint32_t n_pt = (a.n_pools + BN - 1) / BN;
  const uint32_t n_tiles = n_qt * n_pt;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, T::EPI_WARPS * 32);
    }
    mbar_init(done_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap_q)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap_p)) : "memory");
      uint32_t it = 0;
      bool ok = true;
      for (uint32_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        const uint32_t pt = t / n_qt, qt = t % n_qt;
        for (int kb = 0; kb < a.k_blocks; ++kb, ++it) {
          const uint32_t s = it % STAGES, ph = (it / STAGES) & 1u;
          if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
#pragma unroll
          for (int m = 0; m < MSUB; ++m)
            tma_load_2d(sA + s * A_BYTES + m * T::A_SUB, &tmap_q, full0 + 8 * s, kb * BK,
                        (int)(a.q0 + qt * BMC + m * BM));
          tma_load_2d(sB + s * B_BYTES, &tmap_p, full0 + 8 * s, kb * BK, (int)(pt * BN));
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(&a.flags[kFlagTimeout], 1);
      }
      // drain: the last STAGES issued loads must have landed before exit
      const uint32_t first = it > (uint32_t)STAGES ? it - STAGES : 0u;
      for (uint32_t j = first; j < it; ++j) {
        const uint32_t s = j % STAGES, ph = (j / STAGES) & 1u;
        const uint64_t t0 = now_ns();
        while (!mbar_try_wait(full0 + 8 * s, ph) && now_ns() - t0 < kWaitNs) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(BM, BN);
      uint32_t it = 0, tile_i = 0;
      bool ok = true;
      for (uint32_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++tile_i) {
        const uint32_t b = tile_i % NBUF, bph = (tile_i / NBUF) & 1u;
        if (!mbar_wait(tempty0 + 8 * b, bph ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t d_tmem = tmem + b * MSUB * BN;
        for (int kb = 0; kb < a.k_blocks; ++kb, ++it) {
          const uint32_t s = it % STAGES, ph = (it / STAGES) & 1u;
          if (!mbar_wait(full0 + 8 * s, ph, abort_flag)) {
            ok = false;
            break;
          }
          fence_after();
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) {
            const uint64_t bd = sw128_desc(sB + s * B_BYTES + k * 32);
#pragma unroll
            for (int m = 0; m < MSUB; ++m) {
              const uint64_t ad = sw128_desc(sA + s * A_BYTES + m * T::A_SUB + k * 32);
              mma_bf16(d_tmem + m * BN, ad, bd, idesc, (kb | k) != 0 ? 1u : 0u);
            }
          }
          mma_commit(empty0 + 8 * s);  // frees the stage once these MMAs are done
        }
        if (!ok) break;
        mma_commit(tfull0 + 8 * b);    // accumulator b is complete
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(&a.flags[kFlagTimeout], 1);
      }
      // drain: every MMA issued by this thread has completed
      mma_commit(done_bar);
      const uint64_t t0 = now_ns();
      while (!mbar_try_wait(done_bar, 0) && now_ns() - t0 < kWaitNs) {
      }
    }
  } else {
    // ---------------- epilogue (warps 2 .. 2 + EPI_WARPS - 1) ----------------
    constexpr int SPLIT = T::EPI_SPLIT, BNW = BN / SPLIT;  // columns per warp
    const uint32_t quarter = (uint32_t)(warp & 3);  // TMEM lanes 32*quarter .. +31
    const uint32_t grp = (uint32_t)(warp - 2) / 4;
    const uint32_t msub = grp / SPLIT;              // which 128-query accumulator
    const uint32_t part = grp % SPLIT;              // which share of the columns
    uint32_t tile_i = 0;
    for (uint32_t t = blockIdx.x; t < n_tiles; t += gridDim.x, ++tile_i) {
      const uint32_t pt = t / n_qt, qt = t % n_qt;
      const uint32_t b = tile_i % NBUF, bph = (tile_i / NBUF) & 1u;
      if (!mbar_wait(tfull0 + 8 * b, bph, abort_flag)) {
        *abort_flag = 1;
        atomicExch(&a.flags[kFlagTimeout], 1);
        break;
      }
      fence_after();
      const uint32_t row = qt * BMC + msub * BM + quarter * 32 + lane;  // query within the batch
      epilogue_tile<BNW>(a, tmem + ((quarter * 32u) << 16) + (b * MSUB + msub) * BN + part * BNW, row,
                         pt * BN + part * BNW);
      fence_before();
      mbar_arrive(tempty0 + 8 * b);  // accumulator b may be overwritten
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// The same GEMM on a pair of SMs (a cluster of two CTAs, tcgen05 cta_group::2):
// one 256-query x 256-pool tile per pair.  CTA r of the pair loads query rows
// 128r .. 128r+127 and pool rows 128r .. 128r+127 of the tile (32 KiB per
// 64-entry K stage, six stages); the leader CTA (r = 0) issues
// tcgen05.mma.cta_group::2 with M = 256, N = 256, which reads both CTAs'
// operands and leaves rows 128r .. 128r+127 x all 256 columns in CTA r's TMEM.
// Per SM this moves 32 KiB through shared memory per 128x256x64 block of MMA
// work instead of 48 KiB, with two accumulator buffers per CTA kept, so the
// epilogue of one tile overlaps the MMAs of the next.
//
// Barriers: full[s] lives in the leader (both CTAs' loads complete on it; the
// leader's producer posts the expected bytes of both), empty[s] and tfull[b]
// in both CTAs (the leader's MMA commits multicast to the pair), tempty[b] in
// the leader (the four epilogue warps of each CTA arrive on it).
struct Pair2 {
  static constexpr int BMC = 256;                 // queries per pair tile
  static constexpr int BN = 256;                  // pools per pair tile
  static constexpr int A_BYTES = BM * BK * 2;     // 16 KiB: this CTA's 128 query rows
  static constexpr int B_BYTES = 128 * BK * 2;    // 16 KiB: this CTA's 128 pool rows
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int STAGES = (192 * 1024) / STAGE_BYTES;   // 6
  static constexpr int NBUF = 2;
  static constexpr int TMEM_COLS = NBUF * BN;      // 512
  static constexpr int EPI_WARPS = 8;               // two per TMEM lane quarter
  static constexpr int THREADS = 64 + 32 * EPI_WARPS;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
};

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// address of the same shared variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t map_to_rank(uint32_t saddr, uint32_t rank) {
  uint32_t out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(saddr), "r"(rank));
  return out;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

// TMA load into this CTA's shared memory, completing on an mbarrier that may
// be in the peer CTA (cluster address)
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap *map,
                                                 uint32_t bar_cluster, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void mma_bf16_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                              uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// arrive on barrier `bar` (same offset) in every CTA of `mask` once the
// MMAs issued so far have completed
__device__ __forceinline__ void mma_commit_pair(uint32_t bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(bar),
      "h"(mask)
      : "memory");
}

// Barrier 1 over the 8 epilogue warps (256 threads): true if any of them
// passed `fail`.
__device__ __forceinline__ bool epi_barrier_any(bool fail) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n"
      " barrier.cta.red.or.pred po, 1, 256, pi;\n selp.u32 %0, 1, 0, po;\n}\n"
      : "=r"(r)
      : "r"(fail ? 1u : 0u)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity,
                                                  volatile int *abort_flag) {
  if (mbar_try_wait_cluster(bar, parity)) return true;
  const uint64_t t0 = now_ns();
  while (!mbar_try_wait_cluster(bar, parity)) {
    if (*abort_flag) return false;
    if (now_ns() - t0 > kWaitNs) return false;
  }
  return true;
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(Pair2::THREADS, 1)
    k_dense_pair(const __grid_constant__ CUtensorMap tmap_q, const __grid_constant__ CUtensorMap tmap_p,
                 const DenseArgs a) {
  using T = Pair2;
  constexpr int STAGES = T::STAGES;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  uint8_t *gbase = smem_raw + (base - smem_u32(smem_raw));
  const uint32_t sA = base;                            // STAGES x A_BYTES
  const uint32_t sB = base + STAGES * T::A_BYTES;      // STAGES x B_BYTES
  uint64_t *bars = reinterpret_cast<uint64_t *>(gbase + STAGES * T::STAGE_BYTES);
  const uint32_t full0 = smem_u32(bars);
  const uint32_t empty0 = full0 + 8 * STAGES;
  const uint32_t tfull0 = empty0 + 8 * STAGES;
  const uint32_t tempty0 = tfull0 + 16;
  const uint32_t done_bar = tempty0 + 16;
  uint32_t *tmem_slot =
      reinterpret_cast<uint32_t *>(gbase + STAGES * T::STAGE_BYTES + 8 * (2 * STAGES + 5));
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const uint32_t cid = blockIdx.x >> 1, n_clusters = gridDim.x >> 1;
  const uint32_t n_qt = (a.nq + T::BMC - 1) / T::BMC;
  const uint32_t n_pt = (a.n_pools + T::BN - 1) / T::BN;
  const uint32_t n_tiles = n_qt * n_pt;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, 2);   // one arrival per CTA of the pair
    }
    mbar_init(done_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    // one warp of each CTA of the pair allocates, collectively
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(T::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  fence_before();
  cluster_sync_all();  // barriers initialised and TMEM allocated in both CTAs
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t full0_l = map_to_rank(full0, 0);     // the leader's full barriers
  const uint32_t tempty0_l = map_to_rank(tempty0, 0); // the leader's tmem-empty barriers

  if (warp == 0) {
    // ---------------- TMA producer (both CTAs) ----------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap_q)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap_p)) : "memory");
      uint32_t it = 0;
      bool ok = true;
      for (uint32_t t = cid; t < n_tiles && ok; t += n_clusters) {
        const uint32_t pt = t / n_qt, qt = t % n_qt;
        for (int kb = 0; kb < a.k_blocks; ++kb, ++it) {
          const uint32_t s = it % STAGES, ph = (it / STAGES) & 1u;
          if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          if (leader) mbar_expect_tx(full0 + 8 * s, 2 * T::STAGE_BYTES);
          tma_load_2d_pair(sA + s * T::A_BYTES, &tmap_q, full0_l + 8 * s, kb * BK,
                           (int)(a.q0 + qt * T::BMC + rank * BM));
          tma_load_2d_pair(sB + s * T::B_BYTES, &tmap_p, full0_l + 8 * s, kb * BK,
                           (int)(pt * T::BN + rank * 128));
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(&a.flags[kFlagTimeout], 1);
      }
      // drain: the last STAGES loads have been consumed by the MMAs (their
      // empty barriers completed) before this CTA may exit
      const uint32_t first = it > (uint32_t)STAGES ? it - STAGES : 0u;
      const uint64_t t0 = now_ns();
      for (uint32_t j = first; j < it; ++j) {
        const uint32_t s = j % STAGES, ph = (j / STAGES) & 1u;
        while (!mbar_try_wait(empty0 + 8 * s, ph) && now_ns() - t0 < kWaitNs) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (leader CTA only) ----------------
    if (leader && lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(2 * BM, T::BN);
      uint32_t it = 0, tile_i = 0;
      bool ok = true;
      for (uint32_t t = cid; t < n_tiles && ok; t += n_clusters, ++tile_i) {
        const uint32_t b = tile_i % T::NBUF, bph = (tile_i / T::NBUF) & 1u;
        if (!mbar_wait_cluster(tempty0 + 8 * b, bph ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t d_tmem = tmem + b * T::BN;
        for (int kb = 0; kb < a.k_blocks; ++kb, ++it) {
          const uint32_t s = it % STAGES, ph = (it / STAGES) & 1u;
          if (!mbar_wait(full0 + 8 * s, ph, abort_flag)) {
            ok = false;
            break;
          }
          fence_after();
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) {
            const uint64_t ad = sw128_desc(sA + s * T::A_BYTES + k * 32);
            const uint64_t bd = sw128_desc(sB + s * T::B_BYTES + k * 32);
            mma_bf16_pair(d_tmem, ad, bd, idesc, (kb | k) != 0 ? 1u : 0u);
          }
          mma_commit_pair(empty0 + 8 * s, 0x3);  // frees stage s in both CTAs
        }
        if (!ok) break;
        mma_commit_pair(tfull0 + 8 * b, 0x3);    // accumulator b complete in both CTAs
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(&a.flags[kFlagTimeout], 1);
      }
      // drain: every MMA issued by this thread has completed
      mma_commit_pair(done_bar, 0x1);
      const uint64_t t0 = now_ns();
      while (!mbar_try_wait(done_bar, 0) && now_ns() - t0 < kWaitNs) {
      }
    }
  } else {
    // ---------------- epilogue (warps 2 .. 9, both CTAs) ----------------
    constexpr int BNW = T::BN / 2;                  // columns per warp
    const uint32_t quarter = (uint32_t)(warp & 3);  // TMEM lanes 32*quarter .. +31
    const uint32_t part = (uint32_t)(warp - 2) / 4; // which half of the columns
    uint32_t tile_i = 0;
    for (uint32_t t = cid; t < n_tiles; t += n_clusters, ++tile_i) {
      const uint32_t pt = t / n_qt, qt = t % n_qt;
      const uint32_t b = tile_i % T::NBUF, bph = (tile_i / T::NBUF) & 1u;
      const bool ok = mbar_wait(tfull0 + 8 * b, bph, abort_flag);
      if (!ok) {
        *abort_flag = 1;
        atomicExch(&a.flags[kFlagTimeout], 1);
      } else {
        fence_after();
        const uint32_t row = qt * T::BMC + rank * BM + quarter * 32 + lane;  // query within the batch
        epilogue_tile<BNW>(a, tmem + ((quarter * 32u) << 16) + b * T::BN + part * BNW, row,
                           pt * T::BN + part * BNW);
      }
      fence_before();
      // the eight epilogue warps agree (named barrier 1) that the accumulator
      // is read, or that one of them gave up; then one thread releases it to
      // the leader's MMA: one cluster-scope arrival per CTA and tile
      if (epi_barrier_any(!ok)) break;
      if (warp == 2 && lane == 0) {
        if (leader)
          mbar_arrive(tempty0 + 8 * b);
        else
          mbar_arrive_cluster(tempty0_l + 8 * b);
      }
    }
  }
  fence_before();
  __syncthreads();
  cluster_sync_all();  // no CTA leaves while its pair may still touch its memory
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(T::TMEM_COLS)
                 : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  }
  return fn;
}

bool make_map(CUtensorMap *m, const void *base, uint64_t rows, uint64_t cols_elems,
              uint64_t row_bytes, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {cols_elems, rows};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor-core accumulation error model: relative error of the FP32 sum of
// non-negative BF16 products at most 2^-12 (far above any rounding or
// truncation the accumulator can make over K <= 2048; checked against FP64 on
// adversarial inputs by the tests).
constexpr double kGammaTC = 1.0 / 4096.0;

}  // namespace

int pair_clusters();

bool dense_available() {
  static int ok = -1;
  if (ok < 0) {
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    ok = (major == 10 && minor == 3 && encode_fn() != nullptr) ? 1 : 0;
    cudaGetLastError();
    if (ok == 1) pair_clusters();  // kernel attributes set before any stream capture
  }
  return ok == 1;
}

// Scale factors of the GEMM-path bound at level h: queries and rows both in
// BF16 (u = 2^-8 each), FP32 pool sums (e_h), tensor-core accumulation:
// acc * cl <= exact score <= acc * cu.
void gemm_bound(int h, double *cu, double *cl) {
  const double u = std::ldexp(1.0, -8);
  const double eh = std::expm1(h * std::log1p(std::ldexp(1.0, -24)));
  *cu = (1.0 + kGammaTC) / ((1.0 - u) * (1.0 - u) * (1.0 - eh)) * (1.0 + std::ldexp(1.0, -20));
  *cl = 1.0 / ((1.0 + kGammaTC) * (1.0 + u) * (1.0 + u) * (1.0 + eh)) * (1.0 - std::ldexp(1.0, -20));
}

// Clusters of two CTAs of k_dense_pair that can be resident at once (one CTA
// per SM); 0 if the pair kernel cannot run.  Sets the kernel's shared-memory
// attribute, so it is first called outside any stream capture.
int pair_clusters() {
  static int n = -1;
  if (n < 0) {
    n = 0;
    if (cudaFuncSetAttribute(k_dense_pair, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Pair2::SMEM_BYTES) == cudaSuccess) {
      cudaLaunchConfig_t cfg;
      std::memset(&cfg, 0, sizeof(cfg));
      int dev = 0, sms = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cfg.gridDim = dim3((unsigned)std::max(2, sms / 2 * 2));
      cfg.blockDim = dim3(Pair2::THREADS);
      cfg.dynamicSmemBytes = Pair2::SMEM_BYTES;
      int c = 0;
      if (cudaOccupancyMaxActiveClusters(&c, k_dense_pair, &cfg) == cudaSuccess) n = c;
    }
    cudaGetLastError();
  }
  return n;
}

gt_status launch_dense_impl(gt_tree *t, int h, int mode, int64_t q0, int64_t b, Pair *out,
                            uint32_t *out_count, float *scores, int64_t ld, cudaStream_t s) {
  Workspace &w = t->ws;
  if (!dense_available()) return set_error(GT_EINVAL, "dense GEMM path not available");
  if (!t->rows16) return set_error(GT_EINVAL, "dense GEMM needs BF16 rows");
  if (!w.rho || w.q_cap < b + q0)
    return set_error(GT_EINVAL, "dense GEMM queries were not reserved");
  double cu, cl;
  gemm_bound(bound_level(t, h), &cu, &cl);
  // The epilogue's per-query thresholds on the raw accumulator: a pool is kept
  // when acc * cu >= rho (cu bounds the exact score from above), an item
  // accepted when acc * cl >= rho; as acc >= rho * (1/cu) and acc >= rho *
  // (1/cl), with 1/cu rounded down and 1/cl rounded up here and the products
  // rounded the same ways in the kernel, so the comparisons stay rigorous.
  float inv_cu = (float)(1.0 / cu), inv_cl = (float)(1.0 / cl);
  if ((double)inv_cu > 1.0 / cu) inv_cu = std::nextafter(inv_cu, 0.0f);
  if ((double)inv_cl < 1.0 / cl) inv_cl = std::nextafter(inv_cl, INFINITY);
  const int64_t rows = level_rows(t->N, h);
  CUtensorMap mq, mp;
  if (!make_map(&mq, w.qbf16, (uint64_t)w.q_cap, (uint64_t)t->stride, (uint64_t)t->stride * 2, BM))
    return set_error(GT_ECUDA, "cuTensorMapEncodeTiled(queries) failed");
  const __nv_bfloat16 *pbase = t->rows16 + (size_t)t->lvl_off[h] * t->stride;
  // tile shape: tuned_bn 128 -> 128x128, 512 -> 256x256 on one SM, 1024 ->
  // 256x256 on a pair of SMs, else 128x256
  int shape = t->tuned_bn == 128 ? 1 : (t->tuned_bn == 512 ? 2 : (t->tuned_bn == 1024 ? 3 : 0));
  if (shape == 3 && pair_clusters() < 1) shape = 0;
  if (!make_map(&mp, pbase, (uint64_t)rows, (uint64_t)t->stride, (uint64_t)t->stride * 2,
                (shape == 1 || shape == 3) ? 128 : 256))
    return set_error(GT_ECUDA, "cuTensorMapEncodeTiled(pools) failed");
  DenseArgs a;
  a.mode = mode;
  a.n_pools = (uint32_t)rows;
  a.q0 = (uint32_t)q0;
  a.nq = (uint32_t)b;
  a.k_blocks = (int)(t->stride / BK);
  a.n_child = h > 0 ? (uint32_t)level_rows(t->N, h - 1) : 0u;
  a.rho = w.rho;
  a.inv_cu = inv_cu;
  a.inv_cl = inv_cl;
  if (mode == 1) {
    a.out = w.res;
    a.out_count = w.counters + kMaxLevels;
    a.out_cap = (uint32_t)std::min<int64_t>(w.res_cap, 0xffffffffLL);
    a.rchk = w.rchk;
    a.rchk_count = w.counters + kMaxLevels + 1;
    a.rchk_cap = (uint32_t)w.rchk_cap;
  } else {
    a.out = out;
    a.out_count = out_count;
    a.out_cap = (uint32_t)(mode == 3 ? w.front_lim / 2 : w.front_lim);
    a.rchk = nullptr;
    a.rchk_count = nullptr;
    a.rchk_cap = 0;
  }
  a.scores = scores;
  a.ld = ld;
  a.flags = t->flags;
  {
    float c = (float)cu;
    if ((double)c < cu) c = std::nextafter(c, INFINITY);
    a.cu_up = c;
    float l = (float)cl;
    if ((double)l > cl) l = std::nextafter(l, 0.0f);
    a.cl_dn = l;
  }
  // the lower bounds feed the accept test of left items reached by
  // subtraction (sum pools only; a signed tree accepts nothing from bounds)
  a.pad_lower = t->layout != GT_LAYOUT_PREFIX && t->pooling == GT_POOL_SUM && !t->split_sign;
  const int bmc = (shape == 2 || shape == 3) ? 256 : 128, bn = shape == 1 ? 128 : 256;
  const int64_t tiles = ((b + bmc - 1) / bmc) * ((rows + bn - 1) / bn);
  const int grid = shape == 3 ? 2 * (int)std::max<int64_t>(
                                      1, std::min<int64_t>({tiles, (int64_t)pair_clusters(),
                                                            (int64_t)t->sm_count / 2}))
                              : (int)std::max<int64_t>(1, std::min<int64_t>(tiles, t->sm_count));
  auto go = [&](auto kern, int threads, int smem) -> gt_status {
    static bool attr[4] = {false, false, false, false};
    if (!attr[shape]) {
      GT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      attr[shape] = true;
    }
    kern<<<grid, threads, smem, s>>>(mq, mp, a);
    return GT_OK;
  };
  gt_status st;
  if (shape == 3) st = go(k_dense_pair, Pair2::THREADS, Pair2::SMEM_BYTES);
  else if (shape == 1) st = go(k_dense<1, 128>, Tile<1, 128>::THREADS, Tile<1, 128>::SMEM_BYTES);
  else if (shape == 2) st = go(k_dense<2, 256>, Tile<2, 256>::THREADS, Tile<2, 256>::SMEM_BYTES);
  else st = go(k_dense<1, 256>, Tile<1, 256>::THREADS, Tile<1, 256>::SMEM_BYTES);
  if (st != GT_OK) return st;
  GT_CUDA(cudaGetLastError());
  return GT_OK;
}

gt_status launch_dense(gt_tree *t, int h, int mode, int64_t q0, int64_t b, Pair *out,
                       uint32_t *out_count, cudaStream_t s) {
  return launch_dense_impl(t, h, mode, q0, b, out, out_count, nullptr, 0, s);
}

}  // namespace gt
