// Batched dense kernels of the spaND factorization (FP64, sm_103a).
//
// All blocks live in "panel rows": cluster c owns an m_c x ncols_c
// column-major array (ld = m_c) holding its blocks A_cd for d in its
// neighbour list (and itself), ordered by cluster id.  Every kernel below is
// batched over a task array built by the host for one step of Algorithm 2
// (§3): one CTA per task, variable sizes, no atomics, so results do not
// depend on scheduling.
#include <cooperative_groups.h>

#include <cstdio>

#include "spand_real.h"

namespace spand {
namespace SPAND_NS {

namespace {

constexpr int kWarp = 32;

__device__ __forceinline__ real_t warp_sum(real_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Copies and scatters.
// ---------------------------------------------------------------------------
__global__ void k_copy(const CopyTask* __restrict__ tasks) {
  const CopyTask t = tasks[blockIdx.x];
  const int total = t.rows * t.cols;
  if (!t.trans) {
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int i = e % t.rows, j = e / t.rows;
      t.dst[i + (size_t)j * t.dst_ld] = t.src[i + (size_t)j * t.src_ld];
    }
  } else {
    // read src (cols x rows) along its columns, write dst transposed
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int j = e % t.cols, i = e / t.cols;
      t.dst[i + (size_t)j * t.dst_ld] = t.src[j + (size_t)i * t.src_ld];
    }
  }
}

__global__ void k_scatter(const double* __restrict__ val, const int64_t* __restrict__ dst,
                          real_t* __restrict__ base_lo, real_t* __restrict__ base_hi,
                          int64_t split, int64_t nnz) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = dst[e];
    if (d < 0) continue;
    if (d < split) base_lo[d] = (real_t)val[e];
    else base_hi[d - split] = (real_t)val[e];
  }
}

__global__ void k_set_identity(const PotrfTask* __restrict__ tasks) {
  const PotrfTask t = tasks[blockIdx.x];
  const int total = t.m * t.m;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int i = e % t.m, j = e / t.m;
    t.a[i + (size_t)j * t.ld] = (i == j) ? 1.0 : 0.0;
  }
}

// ---------------------------------------------------------------------------
// Batched Cholesky A = L L^T (lower), in place.  Right-looking, one column
// per step; the block is staged in shared memory when it fits.
// ---------------------------------------------------------------------------
__device__ void potrf_body(real_t* a, int m, int ld, int id, int* err, real_t* s_inv,
                           int* s_fail) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int j = 0; j < m; ++j) {
    if (tid == 0) {
      const real_t d = a[j + (size_t)j * ld];
      if (!(d > 0.0)) {
        *s_fail = 1;
        if (err) atomicCAS(err, 0, id + 1);
      } else {
        // one reciprocal square root instead of a square root and a division
        // (each a long sequence of warp-wide instructions on the FP64 pipe)
        const real_t inv = rsqrt(d);
        a[j + (size_t)j * ld] = d * inv;
        *s_inv = inv;
      }
    }
    __syncthreads();
    if (*s_fail) return;
    const real_t inv = *s_inv;
    for (int i = j + 1 + tid; i < m; i += nt) a[i + (size_t)j * ld] *= inv;
    __syncthreads();
    for (int c = j + 1 + warp; c < m; c += nw) {
      const real_t lc = a[c + (size_t)j * ld];
      real_t* col = a + (size_t)c * ld;
      const real_t* lj = a + (size_t)j * ld;
      for (int r = c + lane; r < m; r += kWarp) col[r] -= lj[r] * lc;
    }
    __syncthreads();
  }
}

__global__ void k_potrf(const PotrfTask* __restrict__ tasks, int smem_cap) {
  extern __shared__ real_t sm[];
  __shared__ real_t s_inv;
  __shared__ int s_fail;
  const PotrfTask t = tasks[blockIdx.x];
  if (threadIdx.x == 0) s_fail = 0;
  __syncthreads();
  const int m = t.m;
  if (m == 0) return;
  if (m * m <= smem_cap) {
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = e % m, j = e / m;
      sm[e] = (i >= j) ? t.a[i + (size_t)j * t.ld] : 0.0;
    }
    __syncthreads();
    potrf_body(sm, m, m, t.id, t.err, &s_inv, &s_fail);
    __syncthreads();
    if (s_fail) return;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = e % m, j = e / m;
      t.a[i + (size_t)j * t.ld] = sm[e];
    }
  } else {
    potrf_body(t.a, m, t.ld, t.id, t.err, &s_inv, &s_fail);
    __syncthreads();
    if (s_fail) return;
    // zero the strict upper triangle so the block is exactly L
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = e % m, j = e / m;
      if (i < j) t.a[i + (size_t)j * t.ld] = 0.0;
    }
  }
}

// ---------------------------------------------------------------------------
// Batched triangular solve with a lower factor, 32 right-hand sides per CTA.
// The right-hand sides are staged in shared memory (row-major, 32 wide) and
// solved by 32-row blocks.  The diagonal block is solved column by column by
// all warps: after x_j is final, every warp subtracts L_ij x_j from its rows i
// of the block (independent FMAs), and warp 0, which holds row j+1, finishes
// it with the reciprocal pivot (one division per block, across the lanes: on
// GB300's narrow FP64 pipe a division costs tens of warp-wide instructions).
// Then all warps update the rows below with the block's solution (4 partial
// sums per row, the row of L read by the lanes at once and shuffled).  Rows of an identity right-hand side above its unit entry
// stay zero and are skipped.
// ---------------------------------------------------------------------------
constexpr int kTrsmNC = 32;
constexpr int kTrsmThreads = 128;

__device__ void trsm_blocked(const real_t* __restrict__ L, size_t ldl, int m, real_t* xs,
                             int row0, int nc, real_t* rd) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int rb = row0; rb < m; rb += 32) {
    const int re = min(m, rb + 32);
    if (warp == 0 && rb + lane < re) rd[lane] = (real_t)1 / L[(size_t)(rb + lane) * (ldl + 1)];
    __syncthreads();
    if (warp == 0 && lane < nc) xs[rb * kTrsmNC + lane] *= rd[0];
    __syncthreads();
    for (int j = rb; j + 1 < re; ++j) {
      if (lane < nc) {
        const real_t xj = xs[j * kTrsmNC + lane];
        const real_t* Lj = L + (size_t)j * ldl;
        for (int i = j + 1 + warp; i < re; i += nw) {
          real_t xi = fma(-Lj[i], xj, xs[i * kTrsmNC + lane]);
          if (i == j + 1) xi *= rd[i - rb];
          xs[i * kTrsmNC + lane] = xi;
        }
      }
      __syncthreads();
    }
    // rows below the block: lane j loads L(i, rb + j) (the row's 32 entries in
    // flight at once, the next row's while this one is summed) and the lanes
    // take them by shuffle
    const int w = re - rb;
    auto lrow = [&](int i) {
      return (i < m && lane < w) ? L[i + (size_t)(rb + lane) * ldl] : (real_t)0.0;
    };
    real_t lnext = lrow(re + warp);
    for (int i = re + warp; i < m; i += nw) {
      const real_t lv = lnext;
      lnext = lrow(i + nw);
      // two partial sums: each extra one costs an FP64 add per row on the narrow pipe
      real_t s0 = 0.0, s1 = 0.0;
      int j = 0;
      for (; j + 3 < w; j += 4) {
        s0 = fma(__shfl_sync(0xffffffffu, lv, j), xs[(rb + j) * kTrsmNC + lane], s0);
        s1 = fma(__shfl_sync(0xffffffffu, lv, j + 1), xs[(rb + j + 1) * kTrsmNC + lane], s1);
        s0 = fma(__shfl_sync(0xffffffffu, lv, j + 2), xs[(rb + j + 2) * kTrsmNC + lane], s0);
        s1 = fma(__shfl_sync(0xffffffffu, lv, j + 3), xs[(rb + j + 3) * kTrsmNC + lane], s1);
      }
      for (; j < w; ++j) s0 = fma(__shfl_sync(0xffffffffu, lv, j), xs[(rb + j) * kTrsmNC + lane], s0);
      if (lane < nc) xs[i * kTrsmNC + lane] -= s0 + s1;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kTrsmThreads) k_trsm(const TrsmTask* __restrict__ tasks,
                                                       int smem_rows) {
  extern __shared__ real_t sm[];  // smem_rows x kTrsmNC
  __shared__ real_t s_rd[32];     // reciprocal pivots of a diagonal block
  const TrsmTask t = tasks[blockIdx.x];
  const int m = t.m, nc = t.ncols;
  if (m == 0 || nc == 0) return;
  const real_t* L = t.L;
  const size_t ldl = t.ldl;
  if (m <= smem_rows) {
    int row0 = 0;
    if (t.pad >= 0) {
      // X = L^{-1} [e_{c0} .. e_{c0+nc-1}]
      const int c0 = t.pad;
      row0 = c0 - (c0 % 32);
      for (int e = threadIdx.x; e < m * kTrsmNC; e += blockDim.x) {
        const int i = e / kTrsmNC, cc = e % kTrsmNC;
        sm[e] = (i == c0 + cc) ? 1.0 : 0.0;
      }
    } else if (!t.trans) {
      for (int e = threadIdx.x; e < m * nc; e += blockDim.x) {
        const int i = e % m, cc = e / m;
        sm[i * kTrsmNC + cc] = t.X[i + (size_t)cc * t.ldx];
      }
    } else {
      for (int e = threadIdx.x; e < m * nc; e += blockDim.x) {
        const int cc = e % nc, i = e / nc;
        sm[i * kTrsmNC + cc] = t.X[cc + (size_t)i * t.ldx];
      }
    }
    __syncthreads();
    trsm_blocked(L, ldl, m, sm, row0, nc, s_rd);
    if (!t.trans || t.pad >= 0) {
      for (int e = threadIdx.x; e < m * nc; e += blockDim.x) {
        const int i = e % m, cc = e / m;
        t.X[i + (size_t)cc * t.ldx] = sm[i * kTrsmNC + cc];
      }
    } else {
      for (int e = threadIdx.x; e < m * nc; e += blockDim.x) {
        const int cc = e % nc, i = e / nc;
        t.X[cc + (size_t)i * t.ldx] = sm[i * kTrsmNC + cc];
      }
    }
  } else if (threadIdx.x < nc && t.pad >= 0) {
    // very large factor: one right-hand side per thread, in place in global memory
    const int c = threadIdx.x;
    real_t* x = t.X + (size_t)c * t.ldx;
    const int cc = t.pad + c;
    for (int i = 0; i < cc; ++i) x[i] = 0.0;
    for (int i = cc; i < m; ++i) {
      real_t s = (i == cc) ? 1.0 : 0.0;
      const real_t* Li = L + i;
      for (int j = cc; j < i; ++j) s -= Li[j * ldl] * x[j];
      x[i] = s / Li[i * ldl];
    }
  } else if (threadIdx.x < nc) {
    const int c = threadIdx.x;
    real_t* x = t.trans ? t.X + c : t.X + (size_t)c * t.ldx;
    const size_t inc = t.trans ? (size_t)t.ldx : 1;
    for (int i = 0; i < m; ++i) {
      real_t s = x[i * inc];
      const real_t* Li = L + i;
      for (int j = 0; j < i; ++j) s -= Li[j * ldl] * x[j * inc];
      x[i * inc] = s / Li[i * ldl];
    }
  }
}

// ---------------------------------------------------------------------------
// Explicit Q^T = H_{nref-1} ... H_0 of an interface (for the apply), 32
// columns per CTA: lane c follows column c0+c from the unit vector through
// the reflectors; the 4 warps share the rows of every dot product and update
// (so that all four FP64 units of the SM work), 32-row chunks each, combining
// partial sums in shared memory.
// ---------------------------------------------------------------------------
constexpr int kFqThreads = 128;

__global__ void __launch_bounds__(kFqThreads) k_form_qt(const FormQtTask* __restrict__ tasks,
                                                        int smem_rows) {
  extern __shared__ real_t sm[];  // smem_rows x kTrsmNC, then 4 x kTrsmNC partial sums
  const FormQtTask t = tasks[blockIdx.x];
  const int m = t.m, nc = t.ncols;
  if (m == 0 || nc == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  real_t* part = sm + (size_t)smem_rows * kTrsmNC;
  if (m > smem_rows) {
    // very large block: one column per lane of warp 0, in global memory
    if (warp == 0 && lane < nc) {
      real_t* x = t.Qt + (size_t)lane * m;
      const int j = t.c0 + lane;
      for (int i = 0; i < m; ++i) x[i] = (i == j) ? 1.0 : 0.0;
      for (int s = 0; s < t.nref; ++s) {
        const real_t* v = t.V + (size_t)s * m;
        real_t d = 0.0;
        for (int i = s; i < m; ++i) d = fma(v[i], x[i], d);
        const real_t f = t.tau[s] * d;
        for (int i = s; i < m; ++i) x[i] = fma(-f, v[i], x[i]);
      }
    }
    return;
  }
  for (int e = threadIdx.x; e < m * kTrsmNC; e += blockDim.x) {
    const int i = e / kTrsmNC, c = e % kTrsmNC;
    sm[e] = (i == t.c0 + c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int s = 0; s < t.nref; ++s) {
    const real_t* v = t.V + (size_t)s * m;
    // warp w takes the 32-row chunks s + 32 (w + k nw): the lanes load the
    // chunk of v at once (coalesced) and take its entries by shuffle; four
    // partial sums per lane
    real_t d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
    for (int i0 = s + 32 * warp; i0 < m; i0 += 32 * nw) {
      const int w = min(32, m - i0);
      const real_t vv = lane < w ? v[i0 + lane] : (real_t)0.0;
      const real_t* q = sm + (size_t)i0 * kTrsmNC + lane;
      int j = 0;
      for (; j + 3 < w; j += 4) {
        d0 = fma(__shfl_sync(0xffffffffu, vv, j), q[j * kTrsmNC], d0);
        d1 = fma(__shfl_sync(0xffffffffu, vv, j + 1), q[(j + 1) * kTrsmNC], d1);
        d2 = fma(__shfl_sync(0xffffffffu, vv, j + 2), q[(j + 2) * kTrsmNC], d2);
        d3 = fma(__shfl_sync(0xffffffffu, vv, j + 3), q[(j + 3) * kTrsmNC], d3);
      }
      for (; j < w; ++j) d0 = fma(__shfl_sync(0xffffffffu, vv, j), q[j * kTrsmNC], d0);
    }
    part[warp * kTrsmNC + lane] = (d0 + d1) + (d2 + d3);
    __syncthreads();
    real_t dt = 0.0;
    for (int w = 0; w < nw; ++w) dt += part[w * kTrsmNC + lane];
    const real_t f = t.tau[s] * dt;
    for (int i0 = s + 32 * warp; i0 < m; i0 += 32 * nw) {
      const int w = min(32, m - i0);
      const real_t vv = lane < w ? v[i0 + lane] : (real_t)0.0;
      real_t* q = sm + (size_t)i0 * kTrsmNC + lane;
      for (int j = 0; j < w; ++j) q[j * kTrsmNC] = fma(-f, __shfl_sync(0xffffffffu, vv, j), q[j * kTrsmNC]);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < m * nc; e += blockDim.x) {
    const int i = e % m, cc = e / m;
    t.Qt[i + (size_t)cc * m] = sm[i * kTrsmNC + cc];
  }
}

// ---------------------------------------------------------------------------
// Schur-complement tiles: T -= sum_c A_c^T B_c (K-chunks staged in smem),
// written back to the target block and, transposed, to its mirror.
// ---------------------------------------------------------------------------
constexpr int kTile = 32;
constexpr int kKc = 32;

__global__ void __launch_bounds__(256) k_schur(const SchurTile* __restrict__ tiles,
                                               const SchurContrib* __restrict__ contribs) {
  __shared__ real_t As[kKc][kTile + 1];
  __shared__ real_t Bs[kKc][kTile + 1];
  const SchurTile t = tiles[blockIdx.x];
  const int tid = threadIdx.x;
  const int ti = tid & 31;        // output row
  const int tj = (tid >> 5) * 4;  // first of 4 output columns
  real_t acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int ci = t.cbegin; ci < t.cend; ++ci) {
    const SchurContrib c = contribs[ci];
    // kind 0: element (k, i) at k + i*ld (columns of W^T); kind 1: at k*ld + i
    const size_t sk_a = c.pad ? (size_t)c.lda : 1, si_a = c.pad ? 1 : (size_t)c.lda;
    const size_t sk_b = c.pad ? (size_t)c.ldb : 1, si_b = c.pad ? 1 : (size_t)c.ldb;
    const real_t* ca = c.a + (size_t)t.i0 * si_a;
    const real_t* cb = c.b + (size_t)t.j0 * si_b;
    for (int k0 = 0; k0 < c.K; k0 += kKc) {
      const int kk = min(kKc, c.K - k0);
      if (!c.pad) {
        for (int e = tid; e < kKc * kTile; e += 256) {
          const int k = e % kKc, i = e / kKc;
          As[k][i] = (k < kk && i < t.rows) ? ca[(k0 + k) * sk_a + i * si_a] : 0.0;
          Bs[k][i] = (k < kk && i < t.cols) ? cb[(k0 + k) * sk_b + i * si_b] : 0.0;
        }
      } else {
        for (int e = tid; e < kKc * kTile; e += 256) {
          const int i = e % kTile, k = e / kTile;
          As[k][i] = (k < kk && i < t.rows) ? ca[(k0 + k) * sk_a + i * si_a] : 0.0;
          Bs[k][i] = (k < kk && i < t.cols) ? cb[(k0 + k) * sk_b + i * si_b] : 0.0;
        }
      }
      __syncthreads();
      // only the chunk's kk rows, and only warps with a column in the tile (the
      // zero padding would add exact zeros at the full FP64 instruction cost)
      if (tj < t.cols) {
#pragma unroll 4
        for (int k = 0; k < kk; ++k) {
          const real_t a = As[k][ti];
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q] += a * Bs[k][tj + q];
        }
      }
      __syncthreads();
    }
  }
  if (ti < t.rows) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = tj + q;
      if (j < t.cols) {
        real_t* d = t.dst + ti + (size_t)j * t.ld;
        const real_t v = *d - acc[q];
        *d = v;
        if (t.mirror) t.mirror[j + (size_t)ti * t.ld_mirror] = v;
      }
    }
  }
}

#ifdef SPAND_SINGLE
// ---------------------------------------------------------------------------
// Schur tiles on the tensor cores (FP32 storage only): one 128 x 128 output
// tile per CTA, T -= sum_c A_c^T B_c accumulated by tcgen05.mma (kind::tf32)
// into tensor memory.  Each operand value x is split into a TF32 head and a
// TF32 tail (hi = rn(x), lo = rn(x - hi), both rounded to nearest), and every
// K-chunk issues hi*hi + hi*lo + lo*hi: the products of the heads and tails are
// exact in the FP32 accumulator, and the dropped lo*lo term and the tail's own
// rounding are below 2^-21 relative, close to FP32 arithmetic.
//
// Operands are staged by the CTA's threads (plain loads: the panel rows have
// arbitrary leading dimensions, which the 16-byte stride rule of TMA tensor
// copies does not allow) into shared memory in the K-major layout with the
// 128-byte swizzle: row r of a 128 x 32 chunk is 128 bytes at r * 128, its
// 16-byte piece q stored at piece q ^ (r & 7).  One thread issues the MMAs
// (K = 8 per instruction, 4 per chunk and product) and commits them to an
// mbarrier; the CTA waits on it (bounded) before restaging.  The accumulator
// is read back with tcgen05.ld, warp w holding rows 32w .. 32w + 31.
// ---------------------------------------------------------------------------
constexpr int kTcM = 128, kTcN = 128, kTcK = 32, kTcThreads = 128;
constexpr int kTcTileBytes = kTcM * kTcK * 4;             // one 128 x 32 FP32 chunk: 16 KB
constexpr int kTcSmem = 4 * kTcTileBytes + 1024;          // A hi/lo, B hi/lo, 1024-byte alignment
constexpr long long kTcWaitPolls = 1LL << 22;             // mbarrier polls before giving up

__device__ __forceinline__ uint32_t tc_smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of a K-major operand with the 128-byte
// swizzle: start address, leading byte offset (unused by this layout), stride
// byte offset 1024 (eight 128-byte rows), descriptor version 1, swizzle code 2.
__device__ __forceinline__ unsigned long long tc_desc(uint32_t saddr) {
  unsigned long long d = 0;
  d |= (unsigned long long)((saddr >> 4) & 0x3FFFu);
  d |= (unsigned long long)1 << 16;
  d |= (unsigned long long)(1024 >> 4) << 32;
  d |= (unsigned long long)1 << 46;
  d |= (unsigned long long)2 << 61;
  return d;
}

// Instruction descriptor: FP32 accumulator, TF32 A and B, both K-major, N, M.
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) |
                              ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, unsigned long long da, unsigned long long db,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(kTcIdesc), "r"(accumulate));
}

__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < kTcWaitPolls; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// element (r, k) of a swizzled 128 x 32 chunk
__device__ __forceinline__ int tc_sw(int r, int k) {
  return r * kTcK + ((((k >> 2) ^ (r & 7)) << 2) | (k & 3));
}

__global__ void __launch_bounds__(kTcThreads)
    k_schur_tc(const SchurTile* __restrict__ tiles, const SchurContrib* __restrict__ contribs,
               int* __restrict__ err) {
  extern __shared__ unsigned char tc_raw[];
  __shared__ __align__(8) unsigned long long s_bar;
  __shared__ uint32_t s_tmem;
  const SchurTile t = tiles[blockIdx.x];
  if (t.cend <= t.cbegin) return;  // no contribution (the same for the whole CTA)
  float* base = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~(uintptr_t)1023);
  float* Ah = base;
  float* Al = base + kTcM * kTcK;
  float* Bh = base + 2 * kTcM * kTcK;
  float* Bl = base + 3 * kTcM * kTcK;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t bar = tc_smem_addr(&s_bar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc_smem_addr(&s_tmem)),
                 "r"(kTcN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = s_tmem;
  uint32_t parity = 0;
  bool ok = true, first = true;
  for (int ci = t.cbegin; ci < t.cend && ok; ++ci) {
    const SchurContrib c = contribs[ci];  // K-major: element (k, i) at k + i * ld
    const float* ca = c.a + (size_t)t.i0 * c.lda;
    const float* cb = c.b + (size_t)t.j0 * c.ldb;
    for (int k0 = 0; k0 < c.K && ok; k0 += kTcK) {
      const int k = lane;
      const bool kin = k0 + k < c.K;
#pragma unroll 4
      for (int r = warp; r < kTcM; r += kTcThreads / 32) {
        const float a = (kin && r < t.rows) ? ca[(size_t)(k0 + k) + (size_t)r * c.lda] : 0.f;
        const float b = (kin && r < t.cols) ? cb[(size_t)(k0 + k) + (size_t)r * c.ldb] : 0.f;
        const float ah = tf32_rn(a), bh = tf32_rn(b);
        const int o = tc_sw(r, k);
        Ah[o] = ah;
        Al[o] = tf32_rn(a - ah);
        Bh[o] = bh;
        Bl[o] = tf32_rn(b - bh);
      }
      // the generic-proxy stores become visible to the tensor cores
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t sah = tc_smem_addr(Ah), sal = tc_smem_addr(Al);
        const uint32_t sbh = tc_smem_addr(Bh), sbl = tc_smem_addr(Bl);
#pragma unroll
        for (int kk = 0; kk < kTcK / 8; ++kk) {
          const uint32_t off = kk * 32;  // 8 TF32 values along K
          tc_mma(tmem, tc_desc(sah + off), tc_desc(sbh + off), (first && kk == 0) ? 0u : 1u);
          tc_mma(tmem, tc_desc(sah + off), tc_desc(sbl + off), 1u);
          tc_mma(tmem, tc_desc(sal + off), tc_desc(sbh + off), 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         bar)
                     : "memory");
      }
      first = false;
      ok = tc_wait(bar, parity);  // the MMAs have read the staged chunk
      parity ^= 1u;
      ok = __syncthreads_and(ok);
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    const int row = warp * 32 + lane;
#pragma unroll 1
    for (int cb0 = 0; cb0 < kTcN; cb0 += 32) {
      uint32_t v[32];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
          "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
          "%28, %29, %30, %31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
            "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
            "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
            "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < t.rows) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = cb0 + j;
          if (col < t.cols) {
            float* d = t.dst + row + (size_t)col * t.ld;
            const float val = *d - __uint_as_float(v[j]);
            *d = val;
            if (t.mirror) t.mirror[col + (size_t)row * t.ld_mirror] = val;
          }
        }
      }
    }
  } else {
    if (tid == 0) atomicExch(err, 1);
    // MMAs possibly still in flight: give them a bounded wait before freeing
    // the tensor memory they write
    tc_wait(bar, parity ^ 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcN));
}
#endif

// ---------------------------------------------------------------------------
// Batched early-stopping column-pivoted Householder QR (Algorithm 1), one CTA
// per interface, in place on the interface's panel row.  Columns are never
// swapped: the row ends up holding Q^T A_pw in the original column order
// (coarse rows 0..r-1, E below).  Pivot: largest squared trailing norm,
// recomputed at every step, ties to the lowest column; step t is taken while
// nu_t^2 >= eps^2 nu_0^2 (the superfine scheme continues to eps^4 nu_0^2).
// Afterwards the coarse rows are mirrored into the neighbours' rows, the
// diagonal block becomes I_r and t.cur[p] = r.
// ---------------------------------------------------------------------------
constexpr int kQrThreads = 256;
constexpr int kQrcMaxThreads = 512;  // the cluster RRQR runs 256 or 512 threads per CTA
// Register budgets of the FP64 on-chip RRQR kernels (compile-time knobs).
// Under __launch_bounds__(512) the compiler gives the cluster kernel 64
// registers and spills; a stated cap of 128 compiles to 112 without spills.
// Measured on the 128^3 diffusion workload (FP64, untuned shapes), cluster
// kernel per factorization: cap 128 401 ms, cap 72 (64 registers, no spills)
// 438 ms, the compiler's 64 with spills 416 ms; the multi-CTA kernel under
// its own 256-thread bound (128 registers) 92 ms, capped at 96 registers 96 ms.
// SPAND_QR_ACC2: two partial sums in the update's dot products (else four;
// 401 vs 409 ms).
#ifndef SPAND_QR_ACC2
#define SPAND_QR_ACC2 1
#endif
#ifndef SPAND_QRC_REGS
#define SPAND_QRC_REGS 128
#endif
#ifndef SPAND_GSM_REGS
#define SPAND_GSM_REGS 0
#endif
#if SPAND_QRC_REGS > 0
#define kQrcRegCap __maxnreg__(SPAND_QRC_REGS)
#else
#define kQrcRegCap __launch_bounds__(kQrcMaxThreads)
#endif
#if defined(SPAND_SINGLE) || SPAND_GSM_REGS <= 0
#define kQrGsmRegCap __launch_bounds__(kQrThreads)
#else
#define kQrGsmRegCap __maxnreg__(SPAND_GSM_REGS)
#endif

struct ArgMax {
  real_t v;
  int i;
};

__device__ __forceinline__ ArgMax better(ArgMax a, ArgMax b) {
  if (b.v > a.v || (b.v == a.v && b.i < a.i && b.i >= 0)) return b;
  return a;
}

__global__ void __launch_bounds__(kQrThreads)
    k_rrqr(const RRQRTask* __restrict__ tasks, const RRQRSeg* __restrict__ segs) {
  extern __shared__ real_t sm[];
  __shared__ ArgMax s_red[kQrThreads / kWarp];
  __shared__ double s_sec[kQrThreads / kWarp];
  const RRQRTask t = tasks[blockIdx.x];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kQrThreads / kWarp;
  const int m = t.m;
  const size_t ld = t.ld;
  real_t* norms = sm;                             // ncols_max
  real_t* v = norms + t.ncols_max;                // m
  int* cols = reinterpret_cast<int*>(v + m);      // ncols_max
  int* segoff = cols + t.ncols_max;               // nseg + 1
  const int nseg = t.seg_end - t.seg_begin;
  if (tid == 0) {
    int acc = 0;
    for (int s = 0; s < nseg; ++s) {
      segoff[s] = acc;
      acc += t.cur[segs[t.seg_begin + s].cl];
    }
    segoff[nseg] = acc;
  }
  __syncthreads();
  const int N = segoff[nseg];
  for (int s = 0; s < nseg; ++s) {
    const int base = segs[t.seg_begin + s].col, o = segoff[s], w = segoff[s + 1] - o;
    for (int c = tid; c < w; c += kQrThreads) cols[o + c] = base + c;
  }
  __syncthreads();
  // initial squared column norms
  for (int c = warp; c < N; c += nw) {
    const real_t* col = t.A + (size_t)cols[c] * ld;
    real_t s = 0.0;
    for (int i = lane; i < m; i += kWarp) s += col[i] * col[i];
    s = warp_sum(s);
    if (lane == 0) norms[c] = s;
  }
  __syncthreads();
  const double eps = t.eps;
  const int scheme = t.scheme;
  const double thr1 = eps * eps;
  const double thr2 = thr1 * thr1;
  const int maxsteps = min(m, N);
  int r = -1, nsteps = 0, flags = 0;
  double nu0sq = 0.0;
  for (int step = 0; step < maxsteps; ++step) {
    // argmax over non-pivoted columns (pivoted ones hold -1)
    ArgMax best{-1.0, -1};
    for (int c = tid; c < N; c += kQrThreads) best = better(best, ArgMax{norms[c], c});
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ArgMax other{__shfl_xor_sync(0xffffffffu, best.v, o), __shfl_xor_sync(0xffffffffu, best.i, o)};
      best = better(best, other);
    }
    if (lane == 0) s_red[warp] = best;
    __syncthreads();
    if (tid == 0) {
      ArgMax b = s_red[0];
      for (int w = 1; w < nw; ++w) b = better(b, s_red[w]);
      s_red[0] = b;
    }
    __syncthreads();
    best = s_red[0];
    __syncthreads();
    double nusq = (double)best.v;
    if (sizeof(real_t) < sizeof(double)) {
      // FP32 storage: nu_0 and near-threshold decisions use the FP64 norm
      const bool nearthr = step == 0 || fabs(nusq - thr1 * nu0sq) <= 1e-4 * thr1 * nu0sq ||
                           (scheme == SPAND_SECOND_ORDER_SUPERFINE &&
                            fabs(nusq - thr2 * nu0sq) <= 1e-4 * thr2 * nu0sq);
      if (nearthr && best.i >= 0) {
        if (warp == 0) {
          const real_t* pc0 = t.A + (size_t)cols[best.i] * ld;
          double s64 = 0.0;
          for (int i = step + lane; i < m; i += kWarp) {
            const double a = (double)pc0[i];
            s64 = fma(a, a, s64);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) s64 += __shfl_xor_sync(0xffffffffu, s64, o);
          if (lane == 0) s_sec[0] = s64;
        }
        __syncthreads();
        nusq = s_sec[0];
        __syncthreads();
      }
    }
    // second largest candidate norm, for the near-tie flag
    {
      real_t sec = -1.0;
      for (int c = tid; c < N; c += kQrThreads)
        if (c != best.i) sec = fmax(sec, norms[c]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sec = fmax(sec, __shfl_xor_sync(0xffffffffu, sec, o));
      if (lane == 0) s_sec[warp] = sec;
      __syncthreads();
      if (tid == 0) {
        double m2 = -1.0;
        for (int w = 0; w < nw; ++w) m2 = fmax(m2, s_sec[w]);
        if (m2 >= 0.0 && nusq > 0.0 && nusq - m2 <= 1e-12 * nusq) flags |= 1;
      }
      __syncthreads();
    }
    if (step == 0) {
      nu0sq = nusq;
      if (nu0sq == 0.0) {
        r = 0;
        break;
      }
    }
    if (tid == 0) {
      if (fabs(nusq - thr1 * nu0sq) <= 1e-10 * thr1 * nu0sq) flags |= 2;
      if (scheme == SPAND_SECOND_ORDER_SUPERFINE && fabs(nusq - thr2 * nu0sq) <= 1e-10 * thr2 * nu0sq)
        flags |= 2;
    }
    if (r < 0 && nusq < thr1 * nu0sq) {
      r = step;
      if (scheme != SPAND_SECOND_ORDER_SUPERFINE) break;
    }
    if (scheme == SPAND_SECOND_ORDER_SUPERFINE && nusq < thr2 * nu0sq) break;
    real_t* pc = t.A + (size_t)cols[best.i] * ld;
    const double alpha = pc[step];
    const double normx = sqrt(nusq);
    double beta, tau;
    if (normx == 0.0) {
      beta = alpha;
      tau = 0.0;
    } else {
      beta = alpha >= 0.0 ? -normx : normx;
      tau = (beta - alpha) / beta;
    }
    const double den = alpha - beta;
    for (int i = tid; i < m; i += kQrThreads) {
      real_t vi;
      if (i < step) vi = 0.0;
      else if (i == step) vi = 1.0;
      else vi = (normx == 0.0) ? 0.0 : (real_t)(pc[i] / den);
      v[i] = vi;
      t.V[i + (size_t)step * m] = vi;
    }
    if (tid == 0) {
      t.tau[step] = tau;
      norms[best.i] = -1.0;
    }
    __syncthreads();
    for (int i = step + tid; i < m; i += kQrThreads) pc[i] = (i == step) ? beta : 0.0;
    // apply H_step to the other non-pivoted columns; refresh their norms
    for (int c = warp; c < N; c += nw) {
      if (norms[c] < 0.0) continue;
      real_t* col = t.A + (size_t)cols[c] * ld;
      real_t d = 0.0;
      for (int i = step + lane; i < m; i += kWarp) d += v[i] * col[i];
      d = warp_sum(d);
      const real_t f = tau * d;
      real_t s = 0.0;
      for (int i = step + lane; i < m; i += kWarp) {
        const real_t a = col[i] - f * v[i];
        col[i] = a;
        if (i > step) s += a * a;
      }
      s = warp_sum(s);
      if (lane == 0) norms[c] = s;
    }
    __syncthreads();
    nsteps = step + 1;
  }
  if (r < 0) r = nsteps;
  if (tid == 0) {
    t.rank[t.id] = r;
    t.nref[t.id] = nsteps;
    t.flag[t.id] = flags;
  }
  __syncthreads();
  // coarse rows -> neighbours' rows (transposed), diagonal block -> I_r
  for (int s = 0; s < nseg; ++s) {
    const RRQRSeg g = segs[t.seg_begin + s];
    const int w = segoff[s + 1] - segoff[s];
    const int tot = w * r;
    for (int e = tid; e < tot; e += kQrThreads) {
      const int i = e % r, c = e / r;
      g.mirror[c + (size_t)i * g.mirror_ld] = t.A[i + (size_t)(g.col + c) * ld];
    }
  }
  for (int e = tid; e < r * r; e += kQrThreads) {
    const int i = e % r, j = e / r;
    t.diag[i + (size_t)j * ld] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  if (tid == 0) t.cur[t.id] = r;
}

// ---------------------------------------------------------------------------
// The same QR spread over several CTAs that synchronise through global
// memory (one cooperative launch, all CTAs resident): for interface blocks
// too large for the shared memory of a thread-block cluster.  CTA k of a
// task owns a contiguous slice of its columns; per step every CTA publishes
// its best and second-best candidate, one barrier, every CTA merges the
// candidates, reads the pivot column from global memory and forms v itself,
// the owner records v and tau, and every CTA updates its own columns.  The
// owner stores the R entries into the pivot column one barrier later, once
// every CTA has read it.  Each column is processed by one warp exactly as in
// k_rrqr, so the results equal k_rrqr's bit for bit.  Barrier waits are
// bounded: a wait that runs out raises the task's abort flag and the
// problem's error word, and every CTA of the task leaves.
// ---------------------------------------------------------------------------
struct GridSlot {  // one CTA's candidates of one step (6 ints)
  double best, second;
  int idx, pad;
};

// limit: polls of the counter before the wait gives up (the task's wait_limit,
// about a second by default).
__device__ __forceinline__ bool qr_grid_barrier(int* ctr, int* abort, int target, long long limit) {
  __shared__ int s_ok;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(ctr, 1);
    int ok = 1;
    long long it = 0;
    while (*(volatile int*)ctr < target) {
      if (*(volatile int*)abort) {
        ok = 0;
        break;
      }
      if (++it > limit) {
        atomicExch(abort, 1);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The merge of the G CTAs' candidates of a step (largest best, ties to the
// lowest column; second = the largest of the others): thread k < G loads CTA
// k's slot (all loads in flight at once), the warps reduce with shuffles and
// thread 0 merges the warps.  The norms are compared as the bit patterns of
// the doubles (integers order non-negative doubles as their values; -1, no
// candidate, sorts below), so the merge issues no FP64 instruction.  Called by
// every thread of the CTA; the result is returned to every thread.  red_*:
// shared scratch of kQrThreads / 32.
__device__ __forceinline__ void grid_merge(const GridSlot* sl, int G, long long* red_b,
                                           long long* red_s, int* red_i, double* out_best,
                                           double* out_sec, int* out_idx) {
  __shared__ long long s_b, s_s;
  __shared__ int s_i;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  long long b = -1, s2 = -1;
  int ix = -1;
  for (int k = tid; k < G; k += blockDim.x) {
    const long long kb = __double_as_longlong(__ldcg(&sl[k].best));
    const long long ks = __double_as_longlong(__ldcg(&sl[k].second));
    const int ki = __ldcg(&sl[k].idx);
    if (ki < 0) continue;
    if (kb > b || (kb == b && (ix < 0 || ki < ix))) {
      s2 = max(max(s2, ks), b);
      b = kb;
      ix = ki;
    } else {
      s2 = max(max(s2, ks), kb);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long ob = __shfl_xor_sync(0xffffffffu, b, o);
    const long long os = __shfl_xor_sync(0xffffffffu, s2, o);
    const int oi = __shfl_xor_sync(0xffffffffu, ix, o);
    if (oi >= 0 && (ob > b || (ob == b && (ix < 0 || oi < ix)))) {
      s2 = max(max(s2, os), b);
      b = ob;
      ix = oi;
    } else {
      s2 = max(max(s2, os), oi >= 0 ? ob : -1ll);
    }
  }
  if (lane == 0) {
    red_b[warp] = b;
    red_s[warp] = s2;
    red_i[warp] = ix;
  }
  __syncthreads();
  if (tid == 0) {
    long long bb = -1, ss = -1;
    int ii = -1;
    for (int w = 0; w < nw; ++w) {
      const long long ob = red_b[w], os = red_s[w];
      const int oi = red_i[w];
      if (oi >= 0 && (ob > bb || (ob == bb && (ii < 0 || oi < ii)))) {
        ss = max(max(ss, os), bb);
        bb = ob;
        ii = oi;
      } else {
        ss = max(max(ss, os), oi >= 0 ? ob : -1ll);
      }
    }
    s_b = bb;
    s_s = ss;
    s_i = ii;
  }
  __syncthreads();
  *out_best = s_b >= 0 ? __longlong_as_double(s_b) : -1.0;
  *out_sec = s_s >= 0 ? __longlong_as_double(s_s) : -1.0;
  *out_idx = s_i;
  __syncthreads();  // the scratch and the result may be reused at once
}

__global__ void __launch_bounds__(kQrThreads)
    k_rrqr_grid(const RRQRGridTask* __restrict__ tasks, int ntasks, const RRQRSeg* __restrict__ segs) {
  extern __shared__ real_t sm[];
  __shared__ double s_red[kQrThreads / kWarp], s_sec[kQrThreads / kWarp];
  __shared__ int s_idx[kQrThreads / kWarp];
  __shared__ double s_nu64;
  // the task of this CTA
  int lo = 0, hi = ntasks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tasks[mid].cta0 <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const RRQRGridTask gt = tasks[lo];
  const RRQRTask& t = gt.t;
  const int crank = (int)blockIdx.x - gt.cta0, G = gt.ncta;
  int* ctr = gt.ws;
  int* abort = gt.ws + 1;
  GridSlot* slots = reinterpret_cast<GridSlot*>(gt.ws + 4);  // [2][G]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kQrThreads / kWarp;
  const int m = t.m;
  const size_t ld = t.ld;
  const int nseg = t.seg_end - t.seg_begin;
  const int cpb_max = (t.ncols_max + G - 1) / G;
  real_t* v = sm;                                       // m
  real_t* norms = v + m;                                // cpb_max: FP64 d (downdated), -1 once pivoted
  real_t* errb = norms + cpb_max;                       // cpb_max: FP64 E (see k_rrqr_cluster)
  real_t* cand = errb + cpb_max;                        // cpb_max: exact norms of the candidates
  int* cols = reinterpret_cast<int*>(cand + cpb_max);   // cpb_max
  int* memb = cols + cpb_max;                           // cpb_max
  int* segoff = memb + cpb_max;                         // nseg + 1
  // FP64 storage downdates the trailing norms (the scheme and its bounds are
  // described at k_rrqr_cluster); FP32 storage recomputes them at every step
  constexpr bool kDown = sizeof(real_t) == sizeof(double);
  const double u64 = 1.1102230246251565e-16;
  const double gam = 1.01 * (m + 2) * u64, cst = (8.0 * m + 64.0) * u64;
  __shared__ double s_lbg[kQrThreads / kWarp];
  __shared__ int s_nm;
  if (tid == 0) {
    int acc = 0;
    for (int s = 0; s < nseg; ++s) {
      segoff[s] = acc;
      acc += t.cur[segs[t.seg_begin + s].cl];
    }
    segoff[nseg] = acc;
  }
  __syncthreads();
  const int N = segoff[nseg];
  const int cpb = (N + G - 1) / G;
  const int g0 = crank * cpb, nloc = max(0, min(N, g0 + cpb) - g0);
  for (int l = tid; l < nloc; l += kQrThreads) {
    const int g = g0 + l;
    int a = 0, b = nseg - 1;  // last segment with segoff <= g
    while (a < b) {
      const int mid = (a + b + 1) >> 1;
      if (segoff[mid] <= g) a = mid;
      else b = mid - 1;
    }
    cols[l] = segs[t.seg_begin + a].col + (g - segoff[a]);
  }
  __syncthreads();
  for (int l = warp; l < nloc; l += nw) {
    const real_t* col = t.A + (size_t)cols[l] * ld;
    real_t s = 0.0;
    for (int i = lane; i < m; i += kWarp) s += col[i] * col[i];
    s = warp_sum(s);
    if (lane == 0) {
      norms[l] = s;
      cand[l] = s;
      errb[l] = gam * s;
    }
  }
  __syncthreads();
  const double eps = t.eps;
  const int scheme = t.scheme;
  const double thr1 = eps * eps;
  const double thr2 = thr1 * thr1;
  const int maxsteps = min(m, N);
  int r = -1, nsteps = 0, flags = 0, nbar = 0;
  bool ok = true;
  double nu0sq = 0.0;
  int pend_l = -1, pend_step = 0;  // own pivot column still to receive its R entries
  double pend_beta = 0.0;
  for (int step = 0; step < maxsteps; ++step) {
    // local best (ties to the lowest column) and local second best
    double bv = -1.0, sv = -1.0;
    int bi = -1;
    for (int l = tid; l < nloc; l += kQrThreads) {
      const double x = (double)cand[l];
      if (x < 0.0) continue;
      if (x > bv || (x == bv && g0 + l < bi)) {
        sv = fmax(sv, bv);
        bv = x;
        bi = g0 + l;
      } else {
        sv = fmax(sv, x);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const double os = __shfl_xor_sync(0xffffffffu, sv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi >= 0 && (bi < 0 || oi < bi))) {
        sv = fmax(fmax(sv, os), bv);
        bv = ov;
        bi = oi;
      } else {
        sv = fmax(fmax(sv, os), ov);
      }
    }
    if (lane == 0) {
      s_red[warp] = bv;
      s_sec[warp] = sv;
      s_idx[warp] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      double b = s_red[0], s2 = s_sec[0];
      int ix = s_idx[0];
      for (int w = 1; w < nw; ++w) {
        const double ov = s_red[w];
        const int oi = s_idx[w];
        if (ov > b || (ov == b && oi >= 0 && (ix < 0 || oi < ix))) {
          s2 = fmax(fmax(s2, s_sec[w]), b);
          b = ov;
          ix = oi;
        } else {
          s2 = fmax(fmax(s2, s_sec[w]), ov);
        }
      }
      GridSlot gs;
      gs.best = b;
      gs.second = s2;
      gs.idx = ix;
      gs.pad = 0;
      slots[(step & 1) * G + crank] = gs;
    }
    ++nbar;
    if (!qr_grid_barrier(ctr, abort, nbar * G + (nbar == 1 ? t.wait_extra : 0), t.wait_limit)) {
      ok = false;
      break;
    }
    // the previous pivot column has been read by every CTA: store its R entries
    if (pend_l >= 0) {
      real_t* pc = t.A + (size_t)cols[pend_l] * ld;
      for (int i = pend_step + tid; i < m; i += kQrThreads) pc[i] = (i == pend_step) ? (real_t)pend_beta : (real_t)0.0;
      pend_l = -1;
    }
    // merge the CTAs' candidates
    double best = -1.0, sec = -1.0;
    int bidx = -1;
    grid_merge(slots + (step & 1) * G, G, reinterpret_cast<long long*>(s_red),
               reinterpret_cast<long long*>(s_sec), s_idx, &best, &sec, &bidx);
    if (bidx < 0) break;  // no candidate left (cannot happen for step < min(m, N))
    // the pivot column, in global memory (written by its owner before the barrier)
    int pseg = 0;
    {
      int a = 0, b = nseg - 1;
      while (a < b) {
        const int mid = (a + b + 1) >> 1;
        if (segoff[mid] <= bidx) a = mid;
        else b = mid - 1;
      }
      pseg = a;
    }
    const real_t* pc = t.A + (size_t)(segs[t.seg_begin + pseg].col + (bidx - segoff[pseg])) * ld;
    double nusq = best;
    if (sizeof(real_t) < sizeof(double)) {
      // FP32 storage: nu_0 and near-threshold decisions use the FP64 norm
      const bool nearthr = step == 0 || fabs(nusq - thr1 * nu0sq) <= 1e-4 * thr1 * nu0sq ||
                           (scheme == SPAND_SECOND_ORDER_SUPERFINE &&
                            fabs(nusq - thr2 * nu0sq) <= 1e-4 * thr2 * nu0sq);
      if (nearthr) {
        if (warp == 0) {
          double s64 = 0.0;
          for (int i = step + lane; i < m; i += kWarp) {
            const double a = (double)__ldcg(pc + i);
            s64 = fma(a, a, s64);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) s64 += __shfl_xor_sync(0xffffffffu, s64, o);
          if (lane == 0) s_nu64 = s64;
        }
        __syncthreads();
        nusq = s_nu64;
        __syncthreads();
      }
    }
    if (sec >= 0.0 && nusq > 0.0 && nusq - sec <= 1e-12 * nusq) flags |= 1;
    if (step == 0) {
      nu0sq = nusq;
      if (nu0sq == 0.0) {
        r = 0;
        break;
      }
    }
    if (fabs(nusq - thr1 * nu0sq) <= 1e-10 * thr1 * nu0sq) flags |= 2;
    if (scheme == SPAND_SECOND_ORDER_SUPERFINE && fabs(nusq - thr2 * nu0sq) <= 1e-10 * thr2 * nu0sq)
      flags |= 2;
    if (r < 0 && nusq < thr1 * nu0sq) {
      r = step;
      if (scheme != SPAND_SECOND_ORDER_SUPERFINE) break;
    }
    if (scheme == SPAND_SECOND_ORDER_SUPERFINE && nusq < thr2 * nu0sq) break;
    const double alpha = __ldcg(pc + step);
    const double normx = sqrt(nusq);
    double beta, tau;
    if (normx == 0.0) {
      beta = alpha;
      tau = 0.0;
    } else {
      beta = alpha >= 0.0 ? -normx : normx;
      tau = (beta - alpha) / beta;
    }
    const double den = alpha - beta;
    const bool owner = bidx >= g0 && bidx < g0 + nloc;
    for (int i = tid; i < m; i += kQrThreads) {
      real_t vi;
      if (i < step) vi = 0.0;
      else if (i == step) vi = 1.0;
      else vi = (normx == 0.0) ? 0.0 : (real_t)(__ldcg(pc + i) / den);
      v[i] = vi;
      if (owner) t.V[i + (size_t)step * m] = vi;
    }
    if (owner) {
      if (tid == 0) {
        t.tau[step] = tau;
        norms[bidx - g0] = -1.0;
        cand[bidx - g0] = -1.0;
      }
      pend_l = bidx - g0;
      pend_step = step;
      pend_beta = beta;
    }
    if (tid == 0) s_nm = 0;
    __syncthreads();
    // apply H_step to the other non-pivoted columns of this CTA; refresh their
    // norms (FP32) or downdate them (FP64)
    for (int l = warp; l < nloc; l += nw) {
      if (norms[l] < 0.0) continue;
      real_t* col = t.A + (size_t)cols[l] * ld;
      real_t d = 0.0;
      for (int i = step + lane; i < m; i += kWarp) d += v[i] * col[i];
      d = warp_sum(d);
      const real_t f = tau * d;
      real_t s = 0.0;
      for (int i = step + lane; i < m; i += kWarp) {
        const real_t a = col[i] - f * v[i];
        col[i] = a;
        if (!kDown && i > step) s += a * a;
      }
      if constexpr (kDown) {
        if (lane == 0) {  // lane 0 wrote the pivot-row entry itself
          const double x = col[step];
          const double dold = norms[l], eold = errb[l];
          const double dn = fmax(fma(-x, x, dold), 0.0);
          norms[l] = dn;
          errb[l] = eold + cst * (dold + eold) + 1.01 * u64 * dn;
          cand[l] = -1.0;
        }
      } else {
        s = warp_sum(s);
        if (lane == 0) {
          norms[l] = s;
          cand[l] = s;
        }
      }
    }
    __syncthreads();
    if constexpr (kDown) {
      // the columns whose exact norm may be the largest (or within 1e-12 of it)
      // are recomputed exactly and become this CTA's candidates
      double lbm = 0.0;
      for (int l = tid; l < nloc; l += kQrThreads) {
        const double dd = norms[l];
        if (dd < 0.0) continue;
        const double e = errb[l];
        lbm = fmax(lbm, dd - (e + gam * (dd + e)));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) lbm = fmax(lbm, __shfl_xor_sync(0xffffffffu, lbm, o));
      if (lane == 0) s_lbg[warp] = lbm;
      __syncthreads();
      double L = 0.0;
      for (int w = 0; w < nw; ++w) L = fmax(L, s_lbg[w]);
      const double Lthr = L * (1.0 - 4e-12);
      for (int l = tid; l < nloc; l += kQrThreads) {
        const double dd = norms[l];
        if (dd < 0.0) continue;
        const double e = errb[l];
        if (dd + (e + gam * (dd + e)) >= Lthr) memb[atomicAdd(&s_nm, 1)] = l;
      }
      __syncthreads();
      const int nm = s_nm;
      for (int q = warp; q < nm; q += nw) {
        const int l = memb[q];
        const real_t* col = t.A + (size_t)cols[l] * ld;
        real_t s2 = 0.0;
        for (int i = step + 1 + lane; i < m; i += kWarp) s2 += col[i] * col[i];
        s2 = warp_sum(s2);
        if (lane == 0) {
          norms[l] = s2;
          errb[l] = gam * s2;
          cand[l] = s2;
        }
      }
      __syncthreads();
    }
    nsteps = step + 1;
  }
  // every CTA has read the last pivot column once all pass this barrier
  if (ok) {
    ++nbar;
    ok = qr_grid_barrier(ctr, abort, nbar * G + (nbar == 1 ? t.wait_extra : 0), t.wait_limit);
  }
  if (!ok) {
    if (tid == 0) atomicExch(t.err + 1, 1);
    return;
  }
  if (pend_l >= 0) {
    real_t* pc = t.A + (size_t)cols[pend_l] * ld;
    for (int i = pend_step + tid; i < m; i += kQrThreads) pc[i] = (i == pend_step) ? (real_t)pend_beta : (real_t)0.0;
  }
  __syncthreads();
  if (r < 0) r = nsteps;
  // coarse rows of this CTA's columns -> the neighbours' rows (transposed)
  for (int e = tid; e < r * nloc; e += kQrThreads) {
    const int i = e % r, l = e / r;
    const int g = g0 + l;
    int a = 0, b = nseg - 1;
    while (a < b) {
      const int mid = (a + b + 1) >> 1;
      if (segoff[mid] <= g) a = mid;
      else b = mid - 1;
    }
    const RRQRSeg sg = segs[t.seg_begin + a];
    sg.mirror[(g - segoff[a]) + (size_t)i * sg.mirror_ld] = t.A[i + (size_t)cols[l] * ld];
  }
  if (crank == 0) {
    for (int e = tid; e < r * r; e += kQrThreads) {
      const int i = e % r, j = e / r;
      t.diag[i + (size_t)j * ld] = (i == j) ? 1.0 : 0.0;
    }
    if (tid == 0) {
      t.rank[t.id] = r;
      t.nref[t.id] = nsteps;
      t.flag[t.id] = flags;
      t.cur[t.id] = r;
    }
  }
}

// ---------------------------------------------------------------------------
// The same QR with the block held on chip: a thread-block cluster of C CTAs
// (C = 1, 2, 4, 8 or 16) per interface, each CTA keeping a contiguous slice of
// the columns in its shared memory for the whole factorization.  Per step the
// CTAs push their best candidates into each other's shared memory, one cluster
// barrier, then every CTA reads the pivot column from its owner's shared
// memory and forms the Householder vector itself.  The pivot rules are k_rrqr's.
// ---------------------------------------------------------------------------
namespace cg = cooperative_groups;

// Candidate keys.  The bit pattern of a non-negative real_t, read as a signed
// integer of the same width, orders like the value; the pivot search and the
// threshold tests of the step therefore compare integers.  (GB300's FP64 pipe
// is narrow: a warp-wide FP64 instruction costs tens of cycles, which the
// per-step decisions would otherwise pay in every warp, and FP32 storage needs
// no FP64 at all there.)  No candidate: the most negative integer.
template <typename R>
struct QrKeyOf;
template <>
struct QrKeyOf<double> {
  typedef long long key;
  typedef unsigned long long ukey;
  static __device__ __forceinline__ key of(double x) { return __double_as_longlong(x); }
  static __device__ __forceinline__ double val(key k) { return __longlong_as_double(k); }
  static __device__ __forceinline__ double rval(key k) { return __longlong_as_double(k); }
  // for x >= 0: value < x  <=>  key < above(x);  value <= x  <=>  key <= below(x)
  static __device__ __forceinline__ key above(double x) { return __double_as_longlong(x); }
  static __device__ __forceinline__ key below(double x) { return __double_as_longlong(x); }
};
template <>
struct QrKeyOf<float> {
  typedef int key;
  typedef unsigned ukey;
  static __device__ __forceinline__ key of(float x) { return __float_as_int(x); }
  static __device__ __forceinline__ double val(key k) { return (double)__int_as_float(k); }
  static __device__ __forceinline__ float rval(key k) { return __int_as_float(k); }
  static __device__ __forceinline__ key above(double x) { return __float_as_int(__double2float_ru(x)); }
  static __device__ __forceinline__ key below(double x) { return __float_as_int(__double2float_rd(x)); }
};
typedef QrKeyOf<real_t> QK;
typedef QK::key qkey_t;
typedef QK::ukey qukey_t;
constexpr qkey_t kNoKey = (qkey_t)(1ull << (8 * sizeof(qkey_t) - 1));

// Candidate exchange of one step: the largest squared norm's key, its column,
// its entry in the pivot row (the reflector's alpha), and the second largest key.
struct QrSlot {
  qkey_t best, second;
  real_t alpha;
  int idx;
};

__device__ __forceinline__ void slot_merge(QrSlot& a, const QrSlot& b) {
  const bool take = (b.best > a.best) || (b.best == a.best && b.idx < a.idx);
  if (take) {
    a.second = max(max(a.second, b.second), a.best);
    a.best = b.best;
    a.idx = b.idx;
    a.alpha = b.alpha;
  } else {
    a.second = max(max(a.second, b.second), b.best);
  }
}

// keys shifted to unsigned (no candidate -> 0) for the warp reductions
__device__ __forceinline__ qukey_t qk_up(qkey_t k) { return k < 0 ? (qukey_t)0 : (qukey_t)k + 1u; }
__device__ __forceinline__ qkey_t qk_down(qukey_t u) { return u == 0 ? kNoKey : (qkey_t)(u - 1u); }

__device__ __forceinline__ unsigned warp_max(unsigned x) { return __reduce_max_sync(0xffffffffu, x); }
__device__ __forceinline__ unsigned long long warp_max(unsigned long long x) {
  const unsigned hi = __reduce_max_sync(0xffffffffu, (unsigned)(x >> 32));
  const unsigned lo = __reduce_max_sync(0xffffffffu, (unsigned)(x >> 32) == hi ? (unsigned)x : 0u);
  return ((unsigned long long)hi << 32) | lo;
}

// The merge of the 32 lanes' slots, with the rules of slot_merge (largest key,
// ties to the lowest column; second = the largest key but the winner's),
// through warp-wide integer reductions instead of a shuffle tree.
__device__ __forceinline__ QrSlot warp_merge(const QrSlot& s) {
  const int lane = threadIdx.x & 31;
  const qukey_t ub = qk_up(s.best);
  const qukey_t mb = warp_max(ub);
  const bool top = ub == mb;
  const unsigned mi = __reduce_min_sync(0xffffffffu, top ? (unsigned)s.idx : 0xffffffffu);
  const int win = __ffs(__ballot_sync(0xffffffffu, top && (unsigned)s.idx == mi)) - 1;
  const qukey_t ms = warp_max(lane == win ? qk_up(s.second) : ub);
  QrSlot o;
  o.best = qk_down(mb);
  o.second = qk_down(ms);
  o.alpha = __shfl_sync(0xffffffffu, s.alpha, win);
  o.idx = (int)mi;
  return o;
}

// beta, tau and 1/(alpha - beta) of the Householder reflector that maps a
// column with pivot-row entry alpha and squared norm nsq (pivot row and below)
// onto beta e_1; called by a whole warp, the result lands in out[0..2] (out
// holds kReflScalars entries).  FP32 storage computes them in FP32; FP64 takes
// the square root once and three quotients in three lanes of the same
// instructions (IEEE division: the values are those of separate computations):
// also out[3] = alpha - beta, the pivot-row entry of the unscaled reflector
// x - beta e_1, and out[4] = tau / (alpha - beta)^2 = 1 / (beta (beta - alpha)),
// the coefficient of the update with that unscaled reflector.
constexpr int kReflScalars = 5;
__device__ __forceinline__ void reflector_scalars(real_t alpha, real_t nsq, int lane, real_t* out) {
  if constexpr (sizeof(real_t) < sizeof(double)) {
    if (lane == 0) {
      const float nx = sqrtf(nsq);
      float beta = alpha, tau = 0.f, inv = 0.f;
      if (nx != 0.f) {
        beta = alpha >= 0.f ? -nx : nx;
        tau = (beta - alpha) / beta;
        inv = 1.f / (alpha - beta);
      }
      out[0] = beta;
      out[1] = tau;
      out[2] = inv;
      out[3] = alpha - beta;
      out[4] = tau * inv * inv;
    }
  } else {
    if (lane < 3) {
      const double nx = sqrt((double)nsq);
      const double beta = (nx == 0.0) ? (double)alpha : (alpha >= 0.0 ? -nx : nx);
      const double num = lane == 0 ? beta - alpha : 1.0;
      const double den = lane == 0 ? beta : lane == 1 ? alpha - beta : beta * (beta - alpha);
      const double q = (nx == 0.0) ? 0.0 : num / den;
      if (lane == 0) {
        out[0] = beta;
        out[1] = q;
      } else if (lane == 1) {
        out[2] = q;
        out[3] = alpha - beta;
      } else {
        out[4] = q;
      }
    }
  }
}

// The same scalars formed by every thread (FP32 storage: a few FP32 instructions).
__device__ __forceinline__ void reflector_scalars_r(real_t alpha, real_t nsq, real_t* beta,
                                                    real_t* tau, real_t* inv) {
  const real_t nx = sqrt(nsq);
  *beta = alpha;
  *tau = 0;
  *inv = 0;
  if (nx != (real_t)0) {
    *beta = alpha >= (real_t)0 ? -nx : nx;
    *tau = (*beta - alpha) / *beta;
    *inv = (real_t)1 / (alpha - *beta);
  }
}

// Flags of one step: bit 0 a near tie of the two largest squared norms
// (relative gap <= 1e-12), bit 1 the pivot's squared norm within 1e-10 of a
// threshold.  FP32 norms: FP32 spacing (6e-8 relative) is far wider than either
// margin, so a near tie is equality and a margin holds at most one value,
// tested by key.  FP64 norms: the FP64 tests, reached only when the keys are
// close (a relative gap of 1e-12 spans fewer than 2^14 doubles, one of 1e-10
// fewer than 2^22).
__device__ __forceinline__ int qr_step_flags(bool near, qkey_t bk, qkey_t second, double nu64,
                                             double T1, double T2, double F1, double F2,
                                             qkey_t f1lo, qkey_t f1hi, qkey_t f2lo, qkey_t f2hi,
                                             bool superfine) {
  int fl = 0;
  if (sizeof(real_t) < sizeof(double) && !near) {
    if (bk > 0 && second == bk) fl |= 1;
    if ((bk >= f1lo && bk <= f1hi) || (superfine && bk >= f2lo && bk <= f2hi)) fl |= 2;
    return fl;
  }
  const double nusq = near ? nu64 : QK::val(bk);
  const long long k = __double_as_longlong(nusq);
  if (second >= 0 && nusq > 0.0) {
    const double sec = QK::val(second);
    if (k - __double_as_longlong(sec) <= (1ll << 14) && nusq - sec <= 1e-12 * nusq) fl |= 1;
  }
  if (llabs(k - __double_as_longlong(T1)) <= (1ll << 22) && fabs(nusq - T1) <= F1) fl |= 2;
  if (superfine && llabs(k - __double_as_longlong(T2)) <= (1ll << 22) && fabs(nusq - T2) <= F2)
    fl |= 2;
  return fl;
}

constexpr double kU64 = 1.1102230246251565e-16;  // 2^-53

// The downdated trailing norms of the FP64 RRQR kernels (d, its error bound E
// and the bound B = E + gam (d + E) on |d - exact|, described before
// qr_update_dd) in few FP64 instructions (each costs the narrow FP64 pipe its
// full warp width): since d_new <= d_old, one step's growth of E is
// bounded by E' = c1 E + c2 d_old, c1 = (1 + cst)(1 + 4u), c2 = (cst + 1.01 u)
// (1 + 4u) (the 1 + 4u factors absorb the rounding of the bound's own
// arithmetic); with s = d + E, the upper bound d + B = (1 + gam) s and the
// lower bound d - B = (d - E) - gam s.  The lower bounds' maximum and the
// membership test compare the bit patterns of the doubles as integers (the
// order of non-negative doubles; a negative value -- a pivoted column's
// marker, a negative lower bound -- sorts below every non-negative one).
struct QrDowndate {
  double c1, c2, g1, gam;
  __device__ __forceinline__ QrDowndate(int m) {
    const double cst = (8.0 * m + 64.0) * kU64;
    gam = 1.01 * (m + 2) * kU64;
    c1 = (1.0 + cst) * (1.0 + 4.0 * kU64);
    c2 = (cst + 1.01 * kU64) * (1.0 + 4.0 * kU64);
    g1 = (1.0 + gam) * (1.0 + 4.0 * kU64);
  }
};

// Two layouts of the on-chip block, one per storage precision.  FP32: column-
// major in 16-byte vectors (the update is bound by issue and shared-memory
// latency, which 128-bit accesses cut, and the pivot column is read in
// vectors).  FP64: row-major with scalar accesses (the update is bound by the
// FP64 pipe, and this layout measured faster there).
#ifdef SPAND_SINGLE
// The block on chip is column-major: each local column holds ldm = nch x kv
// entries (kv = 16 / sizeof(real_t), nch odd), so that a column is a run of
// 16-byte vectors and the lanes of a warp, on different columns, hit different
// 16-byte bank groups.  A thread of the tpc that share a column takes its
// vectors c0 + sl, c0 + sl + tpc, ... (c0: the vector holding the pivot row),
// four rows per pass, with four partial sums for the dot product v^T a and for
// the new trailing norm, over the nv = ceil(m / kv) vectors that hold rows; v is
// zero above the pivot row and below row m (so are the padding rows of the
// block), and entries above the pivot row are kept.
constexpr int kQv = 16 / (int)sizeof(real_t);  // entries per 16-byte vector
constexpr int kQu = 4 / kQv;                    // vectors per pass (four rows)
struct alignas(16) QVec {
  real_t x[kQv];
};

// the column's local layout: an odd number of vectors per column
__host__ __device__ inline int qr_cm_nvec(int m) {
  const int n = (m + kQv - 1) / kQv;
  return (n & 1) ? n : n + 1;
}

__device__ __forceinline__ real_t qr_dot(const QVec* a, const QVec* w, int c0, int nv, int sl,
                                         int tpc, unsigned gmask) {
  real_t d[4] = {0, 0, 0, 0};
  for (int c = c0 + sl; c < nv; c += kQu * tpc) {
#pragma unroll
    for (int u = 0; u < kQu; ++u) {
      const int cc = c + u * tpc;
      if (kQu == 1 || cc < nv) {
        const QVec x = a[cc], y = w[cc];
#pragma unroll
        for (int j = 0; j < kQv; ++j) d[u * kQv + j] = fma(y.x[j], x.x[j], d[u * kQv + j]);
      }
    }
  }
  real_t s = (d[0] + d[1]) + (d[2] + d[3]);
  for (int o = tpc >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o);
  return s;
}

// a -= f w on the thread's vectors (entries above the pivot row kept); returns
// the thread's part of the squared norm below the pivot row, reduced over the group
__device__ __forceinline__ real_t qr_axpy_norm(QVec* a, const QVec* w, real_t f, bool store, int c0,
                                               int nv, int step, int sl, int tpc, unsigned gmask) {
  real_t s[4] = {0, 0, 0, 0};
  for (int c = c0 + sl; c < nv; c += kQu * tpc) {
#pragma unroll
    for (int u = 0; u < kQu; ++u) {
      const int cc = c + u * tpc;
      if (kQu == 1 || cc < nv) {
        const QVec x = a[cc], y = w[cc];
        QVec z;
#pragma unroll
        for (int j = 0; j < kQv; ++j) {
          const int i = cc * kQv + j;
          z.x[j] = (i < step) ? x.x[j] : fma(-f, y.x[j], x.x[j]);
          if (i > step) s[u * kQv + j] = fma(z.x[j], z.x[j], s[u * kQv + j]);
        }
        if (store) a[cc] = z;
      }
    }
  }
  real_t t = (s[0] + s[1]) + (s[2] + s[3]);
  for (int o = tpc >> 1; o > 0; o >>= 1) t += __shfl_xor_sync(gmask, t, o);
  return t;
}

// One column's part of a step; the group's first thread records the new norm
// and offers the column as a candidate.
__device__ __forceinline__ void qr_update_one(real_t* col, const real_t* v, int c0, int nv, int step,
                                              int m, int sl, int tpc, unsigned gmask, real_t tau,
                                              int gidx, real_t* norm, QrSlot& mine) {
  QVec* a = reinterpret_cast<QVec*>(col);
  const QVec* w = reinterpret_cast<const QVec*>(v);
  const real_t f = tau * qr_dot(a, w, c0, nv, sl, tpc, gmask);
  const real_t s2 = qr_axpy_norm(a, w, f, true, c0, nv, step, sl, tpc, gmask);
  __syncwarp(gmask);  // the row step+1 entry was written by another thread of the group
  if (sl == 0) {
    *norm = s2;
    QrSlot c{QK::of(s2), kNoKey, step + 1 < m ? col[step + 1] : (real_t)0, gidx};
    slot_merge(mine, c);
  }
}

// Two columns in one pass (FP32: twice the independent chains per thread),
// each with exactly qr_update_one's arithmetic; a column that is not live
// (pivoted) is read but neither written nor offered.
__device__ __forceinline__ void qr_update_pair(real_t* ca, real_t* cb, bool ha, bool hb,
                                               const real_t* v, int c0, int nv, int step, int m,
                                               int sl, int tpc, unsigned gmask, real_t tau, int ia,
                                               int ib, real_t* na, real_t* nb, QrSlot& mine) {
  QVec* a = reinterpret_cast<QVec*>(ca);
  QVec* b = reinterpret_cast<QVec*>(cb);
  const QVec* w = reinterpret_cast<const QVec*>(v);
  real_t d[4] = {0, 0, 0, 0}, e[4] = {0, 0, 0, 0};
  for (int c = c0 + sl; c < nv; c += kQu * tpc) {
#pragma unroll
    for (int u = 0; u < kQu; ++u) {
      const int cc = c + u * tpc;
      if (kQu == 1 || cc < nv) {
        const QVec x = a[cc], y = b[cc], z = w[cc];
#pragma unroll
        for (int j = 0; j < kQv; ++j) {
          d[u * kQv + j] = fma(z.x[j], x.x[j], d[u * kQv + j]);
          e[u * kQv + j] = fma(z.x[j], y.x[j], e[u * kQv + j]);
        }
      }
    }
  }
  real_t sd = (d[0] + d[1]) + (d[2] + d[3]), se = (e[0] + e[1]) + (e[2] + e[3]);
  for (int o = tpc >> 1; o > 0; o >>= 1) {
    sd += __shfl_xor_sync(gmask, sd, o);
    se += __shfl_xor_sync(gmask, se, o);
  }
  const real_t f = tau * sd, g = tau * se;
  real_t s[4] = {0, 0, 0, 0}, r[4] = {0, 0, 0, 0};
  for (int c = c0 + sl; c < nv; c += kQu * tpc) {
#pragma unroll
    for (int u = 0; u < kQu; ++u) {
      const int cc = c + u * tpc;
      if (kQu == 1 || cc < nv) {
        const QVec x = a[cc], y = b[cc], z = w[cc];
        QVec p, q;
#pragma unroll
        for (int j = 0; j < kQv; ++j) {
          const int i = cc * kQv + j;
          p.x[j] = (i < step) ? x.x[j] : fma(-f, z.x[j], x.x[j]);
          q.x[j] = (i < step) ? y.x[j] : fma(-g, z.x[j], y.x[j]);
          if (i > step) {
            s[u * kQv + j] = fma(p.x[j], p.x[j], s[u * kQv + j]);
            r[u * kQv + j] = fma(q.x[j], q.x[j], r[u * kQv + j]);
          }
        }
        if (ha) a[cc] = p;
        if (hb) b[cc] = q;
      }
    }
  }
  real_t s2 = (s[0] + s[1]) + (s[2] + s[3]), t2 = (r[0] + r[1]) + (r[2] + r[3]);
  for (int o = tpc >> 1; o > 0; o >>= 1) {
    s2 += __shfl_xor_sync(gmask, s2, o);
    t2 += __shfl_xor_sync(gmask, t2, o);
  }
  __syncwarp(gmask);  // the row step+1 entries were written by another thread of the group
  if (sl == 0) {
    const bool nxt = step + 1 < m;
    if (ha) {
      *na = s2;
      QrSlot c{QK::of(s2), kNoKey, nxt ? ca[step + 1] : (real_t)0, ia};
      slot_merge(mine, c);
    }
    if (hb) {
      *nb = t2;
      QrSlot c{QK::of(t2), kNoKey, nxt ? cb[step + 1] : (real_t)0, ib};
      slot_merge(mine, c);
    }
  }
}

// the squared norm of a whole column, with the partial sums of qr_axpy_norm
__device__ __forceinline__ real_t qr_sumsq(const real_t* col, int nv, int sl, int tpc, unsigned gmask) {
  const QVec* a = reinterpret_cast<const QVec*>(col);
  real_t s[4] = {0, 0, 0, 0};
  for (int c = sl; c < nv; c += kQu * tpc) {
#pragma unroll
    for (int u = 0; u < kQu; ++u) {
      const int cc = c + u * tpc;
      if (kQu == 1 || cc < nv) {
        const QVec x = a[cc];
#pragma unroll
        for (int j = 0; j < kQv; ++j) s[u * kQv + j] = fma(x.x[j], x.x[j], s[u * kQv + j]);
      }
    }
  }
  real_t t = (s[0] + s[1]) + (s[2] + s[3]);
  for (int o = tpc >> 1; o > 0; o >>= 1) t += __shfl_xor_sync(gmask, t, o);
  return t;
}

// One thread per column (or a few, rows split among them): the dot product
// v^T a, the update a -= tau (v^T a) v and the new trailing norm are FMA chains
// in each thread; each thread also keeps the best candidate among its columns
// for the next step.  Per step: two block barriers (three for FP64, whose
// reflector scalars one warp forms) and one cluster barrier.  The owner keeps
// the pivot column intact until the next step's barrier, when every CTA has
// read it, and only then writes its R entries.
__global__ void __launch_bounds__(kQrcMaxThreads)
    k_rrqr_cluster(const RRQRTask* __restrict__ tasks, const RRQRSeg* __restrict__ segs,
                   int csize) {
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const RRQRTask t = tasks[blockIdx.x / csize];
  extern __shared__ real_t sm[];
  __shared__ QrSlot s_in[2][16];  // the cluster's candidates of a step, pushed by every CTA
  __shared__ QrSlot s_warp[kQrcMaxThreads / kWarp];
  __shared__ real_t s_refl[kReflScalars];  // beta, tau, 1/(alpha - beta), ..., formed by warp 0
  __shared__ double s_nu64;     // FP64 norm of the pivot column (FP32 storage only)
  __shared__ int s_N, s_flags;
  const int nthr = (int)blockDim.x;  // 256 or 512
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = nthr / kWarp;
  const int m = t.m;
  const size_t ld = t.ld;
  const int nseg = t.seg_end - t.seg_begin;
  const int ncl = (t.ncols_max + csize - 1) / csize;  // local column capacity
  // column stride: an odd number of vectors (bank spread); the arithmetic runs
  // over the nc vectors that hold rows
  const int nch = qr_cm_nvec(m), ldm = nch * kQv, nc = (m + kQv - 1) / kQv;
  real_t* v = reinterpret_cast<real_t*>((reinterpret_cast<uintptr_t>(sm) + 15) & ~(uintptr_t)15);
  real_t* A = v + ldm;                                 // ncl columns of ldm entries
  real_t* norms = A + (size_t)ncl * ldm;               // ncl
  int* pcol = reinterpret_cast<int*>(norms + ncl);     // ncl: column in the panel row
  int* segid = pcol + ncl;                             // ncl: segment of the column
  int* segoff = segid + ncl;                           // nseg + 1
  if (tid == 0) {
    int acc = 0;
    for (int g = 0; g < nseg; ++g) {
      segoff[g] = acc;
      acc += t.cur[segs[t.seg_begin + g].cl];
    }
    segoff[nseg] = acc;
    s_N = acc;
    s_flags = 0;
  }
  __syncthreads();
  const int N = s_N;
  const int cpb = (N + csize - 1) / csize;
  const int g0 = crank * cpb;
  const int nloc = max(0, min(N, g0 + cpb) - g0);
  // tpc threads share a column (its rows split among them), enough to keep all
  // warps busy when the CTA holds few columns
  int tpc = 1;
  while (tpc < 8 && nloc * tpc * 2 <= nthr) tpc *= 2;
  const int ngrp = nthr / tpc, grp = tid / tpc, sl = tid % tpc;
  const unsigned gmask = (tpc == 32) ? 0xffffffffu : (((1u << tpc) - 1u) << (lane & ~(tpc - 1)));
  for (int l = tid; l < nloc; l += nthr) {
    const int g = g0 + l;
    int lo = 0, hi = nseg - 1;  // last segment with segoff <= g
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (segoff[mid] <= g) lo = mid;
      else hi = mid - 1;
    }
    segid[l] = lo;
    pcol[l] = segs[t.seg_begin + lo].col + (g - segoff[lo]);
  }
  __syncthreads();
  for (int e = tid; e < ldm * nloc; e += nthr) {
    const int i = e % ldm, l = e / ldm;
    A[(size_t)l * ldm + i] = (i < m) ? t.A[i + (size_t)pcol[l] * ld] : (real_t)0;
  }
  __syncthreads();
  QrSlot mine{kNoKey, kNoKey, (real_t)0, 0x7fffffff};
  for (int l = grp; l < nloc; l += ngrp) {
    const real_t s2 = qr_sumsq(A + (size_t)l * ldm, nc, sl, tpc, gmask);
    if (sl == 0) {
      norms[l] = s2;
      QrSlot c{QK::of(s2), kNoKey, m > 0 ? A[(size_t)l * ldm] : (real_t)0, g0 + l};
      slot_merge(mine, c);
    }
  }
  const double eps = t.eps;
  const int scheme = t.scheme;
  const bool superfine = scheme == SPAND_SECOND_ORDER_SUPERFINE;
  const double thr1 = eps * eps;
  const double thr2 = thr1 * thr1;
  const int maxsteps = min(m, N);
  int r = -1, nsteps = 0, flags = 0;
  // thresholds, fixed once nu_0 is known: as doubles, as keys (value < T <=>
  // key < K), the FP32 windows in which the norm is recomputed in FP64, and the
  // near-threshold flag margins
  double nu0sq = 0.0, T1 = 0.0, T2 = 0.0, F1 = 0.0, F2 = 0.0;
  qkey_t K1 = 0, K2 = 0, lo1 = 1, hi1 = 0, lo2 = 1, hi2 = 0, f1lo = 1, f1hi = 0, f2lo = 1, f2hi = 0;
  // deferred R entries of the last pivot column (owner CTA only): other CTAs
  // read that column one step later, so it is overwritten after the next
  // exchange barrier
  int pend_l = -1, pend_step = 0;
  real_t pend_beta = 0;
  for (int step = 0; step < maxsteps; ++step) {
    mine = warp_merge(mine);
    if (lane == 0) s_warp[warp] = mine;
    __syncthreads();
    QrSlot gb{kNoKey, kNoKey, (real_t)0, 0x7fffffff};
    if (csize == 1) {
      // a lone CTA: every warp merges the warps' candidates itself (no exchange)
      if (lane < nw) gb = s_warp[lane];
      gb = warp_merge(gb);
    } else {
      QrSlot* in = s_in[step & 1];  // double-buffered: a CTA may push step s+1 while another reads s
      if (warp == 0) {
        QrSlot cta{kNoKey, kNoKey, (real_t)0, 0x7fffffff};
        if (lane < nw) cta = s_warp[lane];
        cta = warp_merge(cta);
        if (lane < csize) cluster.map_shared_rank(in, lane)[crank] = cta;
      }
      cluster.sync();
      if (lane < csize) gb = in[lane];
      gb = warp_merge(gb);  // every lane of every warp now holds the cluster's best
    }
    if (pend_l >= 0) {
      for (int i = pend_step + tid; i < m; i += nthr)
        A[(size_t)pend_l * ldm + i] = (i == pend_step) ? pend_beta : (real_t)0;
      pend_l = -1;
    }
    if (!(gb.idx >= 0 && gb.idx < N)) {  // no candidate left (N - step > 0 columns remain: not reached)
      if (r < 0) r = step;
      break;
    }
    const qkey_t bk = gb.best;
    const int owner = gb.idx / cpb;
    const int lp = gb.idx - owner * cpb;  // the pivot's column in the owner's slice
    // the pivot column in the owner's shared memory, read in 16-byte vectors
    // from the one holding the pivot row
    const QVec* pcv = reinterpret_cast<const QVec*>(cluster.map_shared_rank(A, owner) + (size_t)lp * ldm);
    QVec* vv = reinterpret_cast<QVec*>(v);
    const int c0 = step / kQv;
    // each thread's first vector of the column stays in registers from here to
    // the scaling below, the load in flight through the decisions; further
    // vectors (columns of more than nthr vectors) go through shared memory
    const int cme = c0 + tid;
    QVec pv;
    if (cme < nc) pv = pcv[cme];
    bool pulled = false;
    // FP32 storage: the decisions that set the rank (nu_0 and any step close to
    // a threshold) use the pivot column's norm recomputed in FP64
    bool near = false;
    double nu64 = 0.0;
    if constexpr (sizeof(real_t) < sizeof(double)) {
      near = step == 0 || (bk >= lo1 && bk <= hi1) || (superfine && bk >= lo2 && bk <= hi2);
      if (near) {
        if (cme < nc) vv[cme] = pv;
        for (int c = cme + nthr; c < nc; c += nthr) vv[c] = pcv[c];
        pulled = true;
        __syncthreads();
        if (warp == 0) {
          double s64 = 0.0;
          for (int i = step + lane; i < m; i += kWarp) {
            const double a = (double)v[i];
            s64 = fma(a, a, s64);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) s64 += __shfl_xor_sync(0xffffffffu, s64, o);
          if (lane == 0) s_nu64 = s64;
        }
        __syncthreads();
        nu64 = s_nu64;
      }
    }
    if (step == 0) {
      nu0sq = near ? nu64 : QK::val(bk);
      if (!(nu0sq > 0.0)) {
        r = 0;
        break;
      }
      T1 = thr1 * nu0sq;
      T2 = thr2 * nu0sq;
      K1 = QK::above(T1);
      K2 = QK::above(T2);
      F1 = 1e-10 * thr1 * nu0sq;
      F2 = 1e-10 * thr2 * nu0sq;
      if constexpr (sizeof(real_t) < sizeof(double)) {
        const double w1 = 1e-4 * thr1 * nu0sq, w2 = 1e-4 * thr2 * nu0sq;
        lo1 = QK::above(T1 - w1);
        hi1 = QK::below(T1 + w1);
        lo2 = QK::above(T2 - w2);
        hi2 = QK::below(T2 + w2);
        f1lo = QK::above(T1 - F1);
        f1hi = QK::below(T1 + F1);
        f2lo = QK::above(T2 - F2);
        f2hi = QK::below(T2 + F2);
      }
    }
    // the FP64 compares only on the rare near-threshold steps (a select would
    // run them, and the conversion below, in every thread of every step)
    bool lt1, lt2;
    real_t nsq;
    if (__builtin_expect(near, 0)) {
      lt1 = nu64 < T1;
      lt2 = nu64 < T2;
      nsq = (real_t)nu64;
    } else {
      lt1 = bk < K1;
      lt2 = bk < K2;
      nsq = QK::rval(bk);
    }
    if (r < 0 && lt1) {
      r = step;
      if (!superfine) {
        if (tid == 0 && crank == 0) flags |= qr_step_flags(near, bk, gb.second, nu64, T1, T2, F1, F2,
                                                         f1lo, f1hi, f2lo, f2hi, superfine);
        break;
      }
    }
    // the pivot column, read from its owner's shared memory (its rows at and
    // below the pivot row), becomes v in every CTA
    if (!pulled)
      for (int c = cme + nthr; c < nc; c += nthr) vv[c] = pcv[c];
    // flags (a near tie of the two largest norms; a norm within 1e-10 of a
    // threshold), kept in CTA 0 while the column is in flight
    if (tid == 0 && crank == 0)
      flags |= qr_step_flags(near, bk, gb.second, nu64, T1, T2, F1, F2, f1lo, f1hi, f2lo, f2hi, superfine);
    if (superfine && lt2) break;
    real_t beta, tau, inv;
    if constexpr (sizeof(real_t) < sizeof(double)) {
      // FP32: every warp forms the scalars itself
      reflector_scalars_r(gb.alpha, nsq, &beta, &tau, &inv);
    } else {
      if (warp == 0) reflector_scalars(gb.alpha, nsq, lane, s_refl);
      __syncthreads();  // s_refl, written by warp 0
      beta = s_refl[0];
      tau = s_refl[1];
      inv = s_refl[2];
    }
    const bool own = crank == owner;
    auto scale = [&](QVec x, int c) {
#pragma unroll
      for (int j = 0; j < kQv; ++j) {
        const int i = c * kQv + j;
        x.x[j] = (i < step || i >= m) ? (real_t)0 : (i == step) ? (real_t)1 : x.x[j] * inv;
        if (own && i >= step && i < m) t.V[i + (size_t)step * m] = x.x[j];
      }
      vv[c] = x;
    };
    if (cme < nc) scale(pv, cme);
    for (int c = cme + nthr; c < nc; c += nthr) scale(vv[c], c);  // the vectors this thread read
    if (own) {
      for (int i = tid; i < step; i += nthr) t.V[i + (size_t)step * m] = 0;
      if (tid == 0) {
        t.tau[step] = tau;
        norms[lp] = -1;
      }
      pend_l = lp;
      pend_step = step;
      pend_beta = beta;
    }
    __syncthreads();
    mine = QrSlot{kNoKey, kNoKey, (real_t)0, 0x7fffffff};
    // FP32: a thread with two columns (l, l + ngrp) updates both in one pass,
    // which doubles its independent chains; every column sees the same
    // arithmetic (four partial sums over the same rows) on either path
    constexpr bool kPairs = sizeof(real_t) < sizeof(double);
    for (int l = grp; l < nloc; l += (kPairs ? 2 : 1) * ngrp) {
      const int l2 = l + ngrp;
      if (kPairs && l2 < nloc) {
        const bool h1 = norms[l] >= (real_t)0, h2 = norms[l2] >= (real_t)0;
        if (h1 || h2) qr_update_pair(A + (size_t)l * ldm, A + (size_t)l2 * ldm, h1, h2, v, c0, nc, step, m, sl, tpc, gmask, tau,
                                     g0 + l, g0 + l2, norms + l, norms + l2, mine);
        continue;
      }
      if (norms[l] < (real_t)0) continue;  // the same l for the whole group
      qr_update_one(A + (size_t)l * ldm, v, c0, nc, step, m, sl, tpc, gmask, tau, g0 + l, norms + l, mine);
    }
    nsteps = step + 1;
  }
  if (r < 0) r = nsteps;
  if (tid == 0 && flags) atomicOr(cluster.map_shared_rank(&s_flags, 0), flags);
  cluster.sync();  // every CTA has also read the last pivot column
  if (pend_l >= 0)
    for (int i = pend_step + tid; i < m; i += nthr)
      A[(size_t)pend_l * ldm + i] = (i == pend_step) ? pend_beta : (real_t)0;
  __syncthreads();
  // write the columns back, mirror the coarse rows into the neighbours' rows
  for (int e = tid; e < m * nloc; e += nthr) {
    const int i = e % m, l = e / m;
    t.A[i + (size_t)pcol[l] * ld] = A[(size_t)l * ldm + i];
  }
  for (int e = tid; e < r * nloc; e += nthr) {
    const int i = e % r, l = e / r;
    const RRQRSeg g = segs[t.seg_begin + segid[l]];
    const int c = g0 + l - segoff[segid[l]];
    g.mirror[c + (size_t)i * g.mirror_ld] = A[(size_t)l * ldm + i];
  }
  if (crank == 0) {
    for (int e = tid; e < r * r; e += nthr) {
      const int i = e % r, j = e / r;
      t.diag[i + (size_t)j * ld] = (i == j) ? 1.0 : 0.0;
    }
    if (tid == 0) {
      t.rank[t.id] = r;
      t.nref[t.id] = nsteps;
      t.cur[t.id] = r;
      t.flag[t.id] = s_flags;
    }
  }
  cluster.sync();  // no CTA leaves while another may still read its shared memory
}
#else  // FP64 storage: row-major block
// One column's part of a step (a thread of the tpc that share the column):
// the dot product v^T a over four partial sums, the update a -= tau (v^T a) v
// four rows per pass with all loads ahead of the stores (a store to the block
// could alias the next loads of v, which would serialise them), and the new
// trailing norm over four partial sums.  The group's first thread records the
// norm and offers the column as a candidate.
__device__ __forceinline__ void qr_update_one(real_t* a, const real_t* v, int ncl, int step, int m,
                                              int sl, int tpc, unsigned gmask, real_t tau, int gidx,
                                              real_t* norm, QrSlot& mine) {
  real_t d0 = 0, d1 = 0, d2 = 0, d3 = 0;
  int i = step + sl;
#pragma unroll 2
  for (; i + 3 * tpc < m; i += 4 * tpc) {
    d0 = fma(v[i], a[(size_t)i * ncl], d0);
    d1 = fma(v[i + tpc], a[(size_t)(i + tpc) * ncl], d1);
    d2 = fma(v[i + 2 * tpc], a[(size_t)(i + 2 * tpc) * ncl], d2);
    d3 = fma(v[i + 3 * tpc], a[(size_t)(i + 3 * tpc) * ncl], d3);
  }
  for (; i < m; i += tpc) d0 = fma(v[i], a[(size_t)i * ncl], d0);
  real_t d = (d0 + d1) + (d2 + d3);
  for (int o = tpc >> 1; o > 0; o >>= 1) d += __shfl_xor_sync(gmask, d, o);
  const real_t f = tau * d;
  real_t s2a = 0, s2b = 0, s2c = 0, s2d = 0;
  i = step + sl;
  const size_t rs = (size_t)tpc * ncl;
  for (; i + 3 * tpc < m; i += 4 * tpc) {
    real_t* p0 = a + (size_t)i * ncl;
    const real_t v0 = v[i], v1 = v[i + tpc], v2 = v[i + 2 * tpc], v3 = v[i + 3 * tpc];
    const real_t a0 = p0[0], a1 = p0[rs], a2 = p0[2 * rs], a3 = p0[3 * rs];
    const real_t x0 = fma(-f, v0, a0), x1 = fma(-f, v1, a1);
    const real_t x2 = fma(-f, v2, a2), x3 = fma(-f, v3, a3);
    p0[0] = x0;
    p0[rs] = x1;
    p0[2 * rs] = x2;
    p0[3 * rs] = x3;
    if (i > step) s2a = fma(x0, x0, s2a);  // rows i + tpc, ... are below the pivot row
    s2b = fma(x1, x1, s2b);
    s2c = fma(x2, x2, s2c);
    s2d = fma(x3, x3, s2d);
  }
  for (; i < m; i += tpc) {
    const real_t x0 = fma(-f, v[i], a[(size_t)i * ncl]);
    a[(size_t)i * ncl] = x0;
    if (i > step) s2a = fma(x0, x0, s2a);
  }
  real_t s2 = (s2a + s2b) + (s2c + s2d);
  for (int o = tpc >> 1; o > 0; o >>= 1) s2 += __shfl_xor_sync(gmask, s2, o);
  __syncwarp(gmask);  // the row step+1 entry was written by another thread of the group
  if (sl == 0) {
    *norm = s2;
    QrSlot c{QK::of(s2), kNoKey, step + 1 < m ? a[(size_t)(step + 1) * ncl] : (real_t)0, gidx};
    slot_merge(mine, c);
  }
}

// Trailing norms by downdating.  Exact recomputation of every trailing column
// norm at every step (the pivot rule) costs a third FMA per entry on the narrow
// FP64 pipe.  Instead each live column carries d, its squared norm below the
// pivot row downdated by the new pivot-row entry after each update
// (||H x||^2 = ||x||^2 over the rows the reflector touches), and E, a bound on
// |d - T| where T is the sum of squares of the column's stored entries:
//   the initial sum of m squares:          E = gam d,  gam = 1.01 (m + 2) u;
//   one reflector (rounding of v, tau, the dot product and the update, and
//   the departure of the computed reflector from orthogonality, each a few m u
//   relative to the column's squared norm before the step):
//                                          E += cst (d_old + E),  cst = (8 m + 64) u;
//   the downdate itself (one FMA):         E += 1.01 u |d|.
// An exact recomputation of the sum of squares lies within gam T of T, so
// |d - exact| <= B = E + gam (d + E).  Per step, L = the CTA's largest d - B
// bounds the exact maximum from below; only the columns with d + B >= L (1 -
// 4e-12) can hold the exact maximum or a value within 1e-12 of it, so only
// they are recomputed exactly (and their d, E reset), and only they become
// candidates.  The pivot chosen is therefore the one exact recomputation of
// every norm would choose, with the same tie rule and the same near-tie flags.
// (kU64 and QrDowndate, the constants of these bounds, are defined above.)

// One column's part of a step without the norm: the dot product and the
// update of qr_update_one; the group's first thread (which holds the pivot row)
// downdates d, grows E, stores the upper bound d + B in *hb and returns the
// bit pattern of the lower bound d - B (0 in the other threads).  coef
// multiplies the unscaled reflector v twice: a -= coef (v^T a) v.
__device__ __forceinline__ long long qr_update_dd(real_t* a, const real_t* v, int ncl, int step, int m,
                                                  int sl, int tpc, unsigned gmask, real_t coef,
                                                  real_t* d, real_t* eb, real_t* hb,
                                                  const QrDowndate& q) {
#if SPAND_QR_ACC2
  // two partial sums, not four: the FMAs queue on the narrow FP64 pipe anyway,
  // and each extra partial sum costs an FP64 add per column and step
  real_t d0 = 0, d1 = 0;
  int i = step + sl;
#pragma unroll 2
  for (; i + 3 * tpc < m; i += 4 * tpc) {
    d0 = fma(v[i], a[(size_t)i * ncl], d0);
    d1 = fma(v[i + tpc], a[(size_t)(i + tpc) * ncl], d1);
    d0 = fma(v[i + 2 * tpc], a[(size_t)(i + 2 * tpc) * ncl], d0);
    d1 = fma(v[i + 3 * tpc], a[(size_t)(i + 3 * tpc) * ncl], d1);
  }
  for (; i < m; i += tpc) d0 = fma(v[i], a[(size_t)i * ncl], d0);
  real_t dd = d0 + d1;
#else
  real_t d0 = 0, d1 = 0, d2 = 0, d3 = 0;
  int i = step + sl;
#pragma unroll 2
  for (; i + 3 * tpc < m; i += 4 * tpc) {
    d0 = fma(v[i], a[(size_t)i * ncl], d0);
    d1 = fma(v[i + tpc], a[(size_t)(i + tpc) * ncl], d1);
    d2 = fma(v[i + 2 * tpc], a[(size_t)(i + 2 * tpc) * ncl], d2);
    d3 = fma(v[i + 3 * tpc], a[(size_t)(i + 3 * tpc) * ncl], d3);
  }
  for (; i < m; i += tpc) d0 = fma(v[i], a[(size_t)i * ncl], d0);
  real_t dd = (d0 + d1) + (d2 + d3);
#endif
  for (int o = tpc >> 1; o > 0; o >>= 1) dd += __shfl_xor_sync(gmask, dd, o);
  const real_t f = coef * dd;
  i = step + sl;
  const size_t rs = (size_t)tpc * ncl;
#pragma unroll 2
  for (; i + 3 * tpc < m; i += 4 * tpc) {
    real_t* p0 = a + (size_t)i * ncl;
    const real_t v0 = v[i], v1 = v[i + tpc], v2 = v[i + 2 * tpc], v3 = v[i + 3 * tpc];
    const real_t a0 = p0[0], a1 = p0[rs], a2 = p0[2 * rs], a3 = p0[3 * rs];
    p0[0] = fma(-f, v0, a0);
    p0[rs] = fma(-f, v1, a1);
    p0[2 * rs] = fma(-f, v2, a2);
    p0[3 * rs] = fma(-f, v3, a3);
  }
  for (; i < m; i += tpc) a[(size_t)i * ncl] = fma(-f, v[i], a[(size_t)i * ncl]);
  long long lk = 0;
  if (sl == 0) {
    const real_t x = a[(size_t)step * ncl];  // written by this thread above
    const real_t dold = *d, eold = *eb;
    real_t dn = fma(-x, x, dold);
    if (__double_as_longlong(dn) < 0) dn = 0.0;  // T >= 0: clamping stays in the bound
    const real_t en = fma(q.c2, dold, eold * q.c1);
    const real_t sb = dn + en;
    *d = dn;
    *eb = en;
    *hb = sb * q.g1;
    lk = __double_as_longlong(fma(-q.gam, sb, dn - en));
  }
  return lk;
}

// One thread per column (or a few, rows split among them): the dot product
// v^T a, the update a -= tau (v^T a) v and the new trailing norm are FMA chains
// in each thread; each thread also keeps the best candidate among its columns
// for the next step.  The block is stored row-major (row i of the local
// columns contiguous) so that a warp reads consecutive addresses.  Per step:
// three block barriers (candidates published; v and the reflector scalars,
// which one warp forms, ready; every column updated) and, for a cluster of
// several CTAs, one cluster barrier for the candidate exchange (a single CTA
// merges its warps' candidates in every warp instead).  The owner keeps the
// pivot column intact until the next step's barrier, when every CTA has read
// it, and only then writes its R entries.
__global__ void kQrcRegCap
    k_rrqr_cluster(const RRQRTask* __restrict__ tasks, const RRQRSeg* __restrict__ segs,
                   int csize) {
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const RRQRTask t = tasks[blockIdx.x / csize];
  extern __shared__ real_t sm[];
  __shared__ QrSlot s_in[2][16];  // the cluster's candidates of a step, pushed by every CTA
  __shared__ QrSlot s_warp[kQrcMaxThreads / kWarp];
  __shared__ real_t s_refl[kReflScalars];  // the reflector's scalars, formed by warp 0
  __shared__ int s_N, s_flags;
  const int nthr = (int)blockDim.x;  // 256 or 512
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = nthr / kWarp;
  const int m = t.m;
  const size_t ld = t.ld;
  const int nseg = t.seg_end - t.seg_begin;
  // local column capacity = row length of the row-major block, odd so that the
  // rows touched by one column's threads fall in different banks
  const int ncl = ((t.ncols_max + csize - 1) / csize) | 1;
  real_t* A = sm;                                      // m x ncl, row-major
  real_t* v = A + (size_t)m * ncl;                     // m
  real_t* norms = v + m;                               // ncl: d (downdated), -1 once pivoted
  real_t* errb = norms + ncl;                          // ncl: E, the bound on d's error
  real_t* hib = errb + ncl;                            // ncl: d + B, -1 once pivoted
  int* pcol = reinterpret_cast<int*>(hib + ncl);       // ncl: column in the panel row
  int* segid = pcol + ncl;                             // ncl: segment of the column
  int* segoff = segid + ncl;                           // nseg + 1
  __shared__ unsigned long long s_lb[kQrcMaxThreads / kWarp];
  const QrDowndate qd(m);
  const double gam = qd.gam;
  if (tid == 0) {
    int acc = 0;
    for (int g = 0; g < nseg; ++g) {
      segoff[g] = acc;
      acc += t.cur[segs[t.seg_begin + g].cl];
    }
    segoff[nseg] = acc;
    s_N = acc;
    s_flags = 0;
  }
  __syncthreads();
  const int N = s_N;
  const int cpb = (N + csize - 1) / csize;
  const int g0 = crank * cpb;
  const int nloc = max(0, min(N, g0 + cpb) - g0);
  // tpc threads share a column (its rows split among them), enough to keep all
  // warps busy when the CTA holds few columns
  int tpc = 1;
  while (tpc < 8 && nloc * tpc * 2 <= nthr) tpc *= 2;
  const int ngrp = nthr / tpc, grp = tid / tpc, sl = tid % tpc;
  const unsigned gmask = (tpc == 32) ? 0xffffffffu : (((1u << tpc) - 1u) << (lane & ~(tpc - 1)));
  for (int l = tid; l < nloc; l += nthr) {
    const int g = g0 + l;
    int lo = 0, hi = nseg - 1;  // last segment with segoff <= g
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (segoff[mid] <= g) lo = mid;
      else hi = mid - 1;
    }
    segid[l] = lo;
    pcol[l] = segs[t.seg_begin + lo].col + (g - segoff[lo]);
  }
  __syncthreads();
  for (int e = tid; e < m * nloc; e += nthr) {
    const int i = e % m, l = e / m;
    A[(size_t)i * ncl + l] = t.A[i + (size_t)pcol[l] * ld];
  }
  __syncthreads();
  QrSlot mine{kNoKey, kNoKey, (real_t)0, 0x7fffffff};
  for (int l = grp; l < nloc; l += ngrp) {
    real_t s2 = 0;
    for (int i = sl; i < m; i += tpc) {
      const real_t a = A[(size_t)i * ncl + l];
      s2 = fma(a, a, s2);
    }
    for (int o = tpc >> 1; o > 0; o >>= 1) s2 += __shfl_xor_sync(gmask, s2, o);
    if (sl == 0) {
      norms[l] = s2;
      errb[l] = gam * s2;
      QrSlot c{QK::of(s2), kNoKey, m > 0 ? A[l] : (real_t)0, g0 + l};
      slot_merge(mine, c);
    }
  }
  const double eps = t.eps;
  const int scheme = t.scheme;
  const bool superfine = scheme == SPAND_SECOND_ORDER_SUPERFINE;
  const double thr1 = eps * eps;
  const double thr2 = thr1 * thr1;
  const int maxsteps = min(m, N);
  int r = -1, nsteps = 0, flags = 0;
  // thresholds, fixed once nu_0 is known: as doubles, as keys (value < T <=>
  // key < K), and the near-threshold flag margins (FP64 norms)
  double nu0sq = 0.0, T1 = 0.0, T2 = 0.0, F1 = 0.0, F2 = 0.0;
  qkey_t K1 = 0, K2 = 0;
  const qkey_t f1lo = 1, f1hi = 0, f2lo = 1, f2hi = 0;  // margins of FP32 keys: not used here
  // deferred R entries of the last pivot column (owner CTA only): other CTAs
  // read that column one step later, so it is overwritten after the next
  // exchange barrier
  int pend_l = -1, pend_step = 0;
  real_t pend_beta = 0;
  for (int step = 0; step < maxsteps; ++step) {
    mine = warp_merge(mine);
    if (lane == 0) s_warp[warp] = mine;
    __syncthreads();
    QrSlot gb{kNoKey, kNoKey, (real_t)0, 0x7fffffff};
    if (csize == 1) {
      // one CTA: every warp merges the warps' candidates itself (no exchange)
      if (lane < nw) gb = s_warp[lane];
      gb = warp_merge(gb);
    } else {
      QrSlot* in = s_in[step & 1];  // double-buffered: a CTA may push step s+1 while another reads s
      if (warp == 0) {
        QrSlot cta{kNoKey, kNoKey, (real_t)0, 0x7fffffff};
        if (lane < nw) cta = s_warp[lane];
        cta = warp_merge(cta);
        if (lane < csize) cluster.map_shared_rank(in, lane)[crank] = cta;
      }
      cluster.sync();
      if (lane < csize) gb = in[lane];
      gb = warp_merge(gb);  // every lane of every warp now holds the cluster's best
    }
    if (pend_l >= 0) {
      for (int i = pend_step + tid; i < m; i += nthr)
        A[(size_t)i * ncl + pend_l] = (i == pend_step) ? pend_beta : (real_t)0;
      pend_l = -1;
    }
    if (!(gb.idx >= 0 && gb.idx < N)) {  // no candidate left (N - step > 0 columns remain: not reached)
      if (r < 0) r = step;
      break;
    }
    const qkey_t bk = gb.best;
    const int owner = gb.idx / cpb;
    const int lp = gb.idx - owner * cpb;  // the pivot's column in the owner's slice
    const real_t* pc = cluster.map_shared_rank(A, owner) + lp;
    // the pivot column, read from its owner's shared memory (its rows at and
    // below the pivot row) by warps 1.. from here on, through the decisions,
    // becomes v in every CTA; warp 0 forms the reflector scalars meanwhile (a
    // long dependent FP64 sequence).  v is not read before the next barrier.
    // v holds the reflector unscaled: x below the pivot row (read here) and
    // alpha - beta at it (written by warp 0 with the scalars); the scale
    // 1/(alpha - beta) enters the update's coefficient instead
    const int pt = tid - kWarp, pn = nthr - kWarp;
    if (warp > 0)
      for (int i = step + 1 + pt; i < m; i += pn) v[i] = pc[(size_t)i * ncl];
    // FP64 storage: the decisions take the norms as they are (the FP32
    // kernel's FP64 recomputation near the thresholds has no counterpart here)
    constexpr bool near = false;
    const double nu64 = 0.0;
    if (step == 0) {
      nu0sq = near ? nu64 : QK::val(bk);
      if (!(nu0sq > 0.0)) {
        r = 0;
        break;
      }
      T1 = thr1 * nu0sq;
      T2 = thr2 * nu0sq;
      K1 = QK::above(T1);
      K2 = QK::above(T2);
      F1 = 1e-10 * thr1 * nu0sq;
      F2 = 1e-10 * thr2 * nu0sq;
    }
    const bool lt1 = near ? nu64 < T1 : bk < K1;
    const bool lt2 = near ? nu64 < T2 : bk < K2;
    if (r < 0 && lt1) {
      r = step;
      if (!superfine) {
        if (tid == 0 && crank == 0) flags |= qr_step_flags(near, bk, gb.second, nu64, T1, T2, F1, F2,
                                                         f1lo, f1hi, f2lo, f2hi, superfine);
        break;
      }
    }
    // flags (a near tie of the two largest norms; a norm within 1e-10 of a
    // threshold), kept in CTA 0 while the column is in flight
    if (tid == 0 && crank == 0)
      flags |= qr_step_flags(near, bk, gb.second, nu64, T1, T2, F1, F2, f1lo, f1hi, f2lo, f2hi, superfine);
    if (superfine && lt2) break;
    const real_t nsq = near ? (real_t)nu64 : QK::rval(bk);
    if (warp == 0) {
      reflector_scalars(gb.alpha, nsq, lane, s_refl);
      __syncwarp();
      if (lane == 0) v[step] = s_refl[3];
    }
    __syncthreads();  // s_refl and v[step], written by warp 0; v below it by warps 1..
    const real_t beta = s_refl[0], tau = s_refl[1], inv = s_refl[2], coef = s_refl[4];
    const bool own = crank == owner;
    if (own) {  // the stored reflector, scaled: 1 at the pivot row, zero above
      for (int i = tid; i < m; i += nthr)
        t.V[i + (size_t)step * m] = i < step ? (real_t)0 : i == step ? (real_t)1 : v[i] * inv;
      if (tid == 0) {  // seen by the other threads after the next barrier; this
        t.tau[step] = tau;  // step's update skips the pivot column by its index
        norms[lp] = -1;
        hib[lp] = -1;
      }
      pend_l = lp;
      pend_step = step;
      pend_beta = beta;
    }
    const int lskip = own ? lp : -1;
    // the update with the unscaled v: tau (v^T a) v = (tau inv^2) (x^T a) x
    mine = QrSlot{kNoKey, kNoKey, (real_t)0, 0x7fffffff};
    long long lbk = 0;  // L: the largest lower bound d - B of the CTA's live columns (bits)
    for (int l = grp; l < nloc; l += ngrp) {
      // pivoted (now or before); the same l for the whole group
      if (l == lskip || __double_as_longlong(norms[l]) < 0) continue;
      lbk = max(lbk, qr_update_dd(A + l, v, ncl, step, m, sl, tpc, gmask, coef, norms + l,
                                  errb + l, hib + l, qd));
    }
    nsteps = step + 1;
    const unsigned long long lbw = warp_max((unsigned long long)lbk);
    if (lane == 0) s_lb[warp] = lbw;
    __syncthreads();  // every column updated, every warp's bound published
    unsigned long long Lk = 0;
    for (int w = 0; w < nw; ++w) Lk = max(Lk, s_lb[w]);
    // L (1 - 4e-12) or a little less, in integer arithmetic: 36030 steps of
    // the last bit lower a non-negative double by between 4.0e-12 and 8.0e-12
    // of its value (an ulp is between 2^-53 and 2^-52 of it)
    const long long Lthr = Lk > 36030ull ? (long long)Lk - 36030 : 0;
    // the columns that may hold the exact maximum (or a value within 1e-12 of
    // it): warp w tests columns 32 (w + nw j) + lane and recomputes its own
    // members' norms exactly, all lanes on one column; they are the candidates
    for (int c0 = warp * kWarp; c0 < nloc; c0 += nw * kWarp) {
      const int lc = c0 + lane;
      const bool mem = lc < nloc && __double_as_longlong(hib[lc]) >= Lthr;
      unsigned bal = __ballot_sync(0xffffffffu, mem);
      while (bal) {
        const int l = c0 + __ffs(bal) - 1;
        bal &= bal - 1;
        real_t s0 = 0, s1 = 0;
        int i = step + 1 + lane;
        for (; i + kWarp < m; i += 2 * kWarp) {
          const real_t x0 = A[(size_t)i * ncl + l], x1 = A[(size_t)(i + kWarp) * ncl + l];
          s0 = fma(x0, x0, s0);
          s1 = fma(x1, x1, s1);
        }
        if (i < m) {
          const real_t x0 = A[(size_t)i * ncl + l];
          s0 = fma(x0, x0, s0);
        }
        const real_t s2 = warp_sum(s0 + s1);
        if (lane == 0) {
          norms[l] = s2;
          errb[l] = gam * s2;
          QrSlot c{QK::of(s2), kNoKey, step + 1 < m ? A[(size_t)(step + 1) * ncl + l] : (real_t)0, g0 + l};
          slot_merge(mine, c);
        }
      }
    }
  }
  if (r < 0) r = nsteps;
  if (tid == 0 && flags) atomicOr(cluster.map_shared_rank(&s_flags, 0), flags);
  cluster.sync();  // every CTA has also read the last pivot column
  if (pend_l >= 0)
    for (int i = pend_step + tid; i < m; i += nthr)
      A[(size_t)i * ncl + pend_l] = (i == pend_step) ? pend_beta : (real_t)0;
  __syncthreads();
  // write the columns back, mirror the coarse rows into the neighbours' rows
  for (int e = tid; e < m * nloc; e += nthr) {
    const int i = e % m, l = e / m;
    t.A[i + (size_t)pcol[l] * ld] = A[(size_t)i * ncl + l];
  }
  for (int e = tid; e < r * nloc; e += nthr) {
    const int i = e % r, l = e / r;
    const RRQRSeg g = segs[t.seg_begin + segid[l]];
    const int c = g0 + l - segoff[segid[l]];
    g.mirror[c + (size_t)i * g.mirror_ld] = A[(size_t)i * ncl + l];
  }
  if (crank == 0) {
    for (int e = tid; e < r * r; e += nthr) {
      const int i = e % r, j = e / r;
      t.diag[i + (size_t)j * ld] = (i == j) ? 1.0 : 0.0;
    }
    if (tid == 0) {
      t.rank[t.id] = r;
      t.nref[t.id] = nsteps;
      t.cur[t.id] = r;
      t.flag[t.id] = s_flags;
    }
  }
  cluster.sync();  // no CTA leaves while another may still read its shared memory
}
#endif

// ---------------------------------------------------------------------------
// The multi-CTA QR with the block on chip: for interface blocks too large for
// the shared memory of one thread-block cluster but small enough for that of
// several SMs.  One cooperative launch; CTA k of a task keeps a contiguous
// slice of the block's columns in its shared memory for the whole
// factorization (row-major, as the FP64 cluster kernel).  Per step each CTA
// publishes its best candidate (exact squared norm, second best, column) and
// a copy of that column's rows from the pivot row down into a staging area in
// global memory (double-buffered by step parity), one bounded barrier, then
// every CTA merges the candidates, reads the winner's staged column (from L2)
// and forms v and the reflector scalars itself; the owner records v and tau and
// writes the R entries into its own slice at once (the others use the staged
// copy).  Pivot rule, ties, flags and thresholds are those of the other RRQR
// kernels; FP64 storage downdates the trailing norms (see k_rrqr_cluster),
// FP32 recomputes them.  A barrier wait that runs out raises the task's abort
// flag and the problem's error word, and every CTA of the task leaves.
// ---------------------------------------------------------------------------
__host__ __device__ inline int gsm_ncl(int cpb) { return cpb | 1; }

__global__ void kQrGsmRegCap
    k_rrqr_gsm(const RRQRGridTask* __restrict__ tasks, int ntasks, const RRQRSeg* __restrict__ segs) {
  extern __shared__ real_t sm[];
  constexpr int nw = kQrThreads / kWarp;
  __shared__ long long s_bv[nw], s_sv[nw];
  __shared__ unsigned long long s_lbg[nw];
  __shared__ int s_bi[nw];
  __shared__ long long s_best, s_sec;
  __shared__ double s_nu64;
  __shared__ int s_ix, s_N;
  __shared__ real_t s_refl[kReflScalars];
  int lo = 0, hi = ntasks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tasks[mid].cta0 <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const RRQRGridTask gt = tasks[lo];
  const RRQRTask& t = gt.t;
  const int crank = (int)blockIdx.x - gt.cta0, G = gt.ncta;
  int* ctr = gt.ws;
  int* abort = gt.ws + 1;
  GridSlot* slots = reinterpret_cast<GridSlot*>(gt.ws + 4);  // [2][G]
  real_t* stg = gt.stage;                                    // [2][G][m]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = t.m;
  const size_t ld = t.ld;
  const int nseg = t.seg_end - t.seg_begin;
  const int ncl = gsm_ncl((t.ncols_max + G - 1) / G);  // the slice's row length
  real_t* A = sm;                                     // m x ncl, row-major
  real_t* v = A + (size_t)m * ncl;                    // m
  real_t* norms = v + m;                              // ncl: d (FP64) or the norm (FP32); -1 once pivoted
  real_t* errb = norms + ncl;                         // ncl: FP64 E
  real_t* cand = errb + ncl;                          // ncl: exact norms of the candidates, else -1
  real_t* hib = cand + ncl;                           // ncl: FP64 d + B, -1 once pivoted
  int* pcol = reinterpret_cast<int*>(hib + ncl);      // ncl
  int* segid = pcol + ncl;                            // ncl
  int* segoff = segid + ncl;                          // nseg + 1
  constexpr bool kDown = sizeof(real_t) == sizeof(double);
  const QrDowndate qd(m);
  const double gam = qd.gam;
  if (tid == 0) {
    int acc = 0;
    for (int g = 0; g < nseg; ++g) {
      segoff[g] = acc;
      acc += t.cur[segs[t.seg_begin + g].cl];
    }
    segoff[nseg] = acc;
    s_N = acc;
  }
  __syncthreads();
  const int N = s_N;
  const int cpb = (N + G - 1) / G;
  const int g0 = crank * cpb, nloc = max(0, min(N, g0 + cpb) - g0);
  int tpc = 1;
  while (tpc < 32 && nloc * tpc * 2 <= kQrThreads) tpc *= 2;
  const int ngrp = kQrThreads / tpc, grp = tid / tpc, sl = tid % tpc;
  const unsigned gmask = (tpc == 32) ? 0xffffffffu : (((1u << tpc) - 1u) << (lane & ~(tpc - 1)));
  for (int l = tid; l < nloc; l += kQrThreads) {
    const int g = g0 + l;
    int a = 0, b = nseg - 1;  // last segment with segoff <= g
    while (a < b) {
      const int mid = (a + b + 1) >> 1;
      if (segoff[mid] <= g) a = mid;
      else b = mid - 1;
    }
    segid[l] = a;
    pcol[l] = segs[t.seg_begin + a].col + (g - segoff[a]);
  }
  __syncthreads();
  for (int e = tid; e < m * nloc; e += kQrThreads) {
    const int i = e % m, l = e / m;
    A[(size_t)i * ncl + l] = t.A[i + (size_t)pcol[l] * ld];
  }
  __syncthreads();
  for (int l = warp; l < nloc; l += nw) {
    real_t s0 = 0, s1 = 0;
    int i = lane;
    for (; i + kWarp < m; i += 2 * kWarp) {
      const real_t x0 = A[(size_t)i * ncl + l], x1 = A[(size_t)(i + kWarp) * ncl + l];
      s0 = fma(x0, x0, s0);
      s1 = fma(x1, x1, s1);
    }
    if (i < m) s0 = fma(A[(size_t)i * ncl + l], A[(size_t)i * ncl + l], s0);
    const real_t s2 = warp_sum(s0 + s1);
    if (lane == 0) {
      norms[l] = s2;
      cand[l] = s2;
      errb[l] = gam * s2;
    }
  }
  __syncthreads();
  const double eps = t.eps;
  const int scheme = t.scheme;
  const bool superfine = scheme == SPAND_SECOND_ORDER_SUPERFINE;
  const double thr1 = eps * eps;
  const double thr2 = thr1 * thr1;
  const int maxsteps = min(m, N);
  int r = -1, nsteps = 0, flags = 0, nbar = 0;
  bool ok = true;
  double nu0sq = 0.0, T1 = 0.0, T2 = 0.0;
  for (int step = 0; step < maxsteps; ++step) {
    // the CTA's best candidate (ties to the lowest column) and second best, as
    // the bit patterns of the norms as doubles (the FP32 norms widen exactly):
    // integer comparisons, no FP64 instruction; -1 = none
    long long bv = -1, sv = -1;
    int bi = -1;
    for (int l = tid; l < nloc; l += kQrThreads) {  // l rises: an equal key keeps the lower column
      const long long x = __double_as_longlong((double)cand[l]);
      if (x < 0) continue;
      if (x > bv) {
        sv = max(sv, bv);
        bv = x;
        bi = g0 + l;
      } else {
        sv = max(sv, x);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const long long os = __shfl_xor_sync(0xffffffffu, sv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi >= 0 && (bi < 0 || oi < bi))) {
        sv = max(max(sv, os), bv);
        bv = ov;
        bi = oi;
      } else {
        sv = max(max(sv, os), ov);
      }
    }
    if (lane == 0) {
      s_bv[warp] = bv;
      s_sv[warp] = sv;
      s_bi[warp] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      long long b = s_bv[0], s2 = s_sv[0];
      int ix = s_bi[0];
      for (int w = 1; w < nw; ++w) {
        const long long ov = s_bv[w];
        const int oi = s_bi[w];
        if (ov > b || (ov == b && oi >= 0 && (ix < 0 || oi < ix))) {
          s2 = max(max(s2, s_sv[w]), b);
          b = ov;
          ix = oi;
        } else {
          s2 = max(max(s2, s_sv[w]), ov);
        }
      }
      s_best = b;
      s_sec = s2;
      s_ix = ix;
    }
    __syncthreads();
    // publish the candidate and a copy of its column (rows step .. m-1)
    const int par = step & 1;
    {
      const int ix = s_ix;
      real_t* dst = stg + ((size_t)par * G + crank) * m;
      if (ix >= 0)
        for (int i = step + tid; i < m; i += kQrThreads) dst[i] = A[(size_t)i * ncl + (ix - g0)];
      if (tid == 0) {
        GridSlot gs;
        gs.best = s_best >= 0 ? __longlong_as_double(s_best) : -1.0;
        gs.second = s_sec >= 0 ? __longlong_as_double(s_sec) : -1.0;
        gs.idx = ix;
        gs.pad = 0;
        slots[par * G + crank] = gs;
      }
    }
    ++nbar;
    if (!qr_grid_barrier(ctr, abort, nbar * G + (nbar == 1 ? t.wait_extra : 0), t.wait_limit)) {
      ok = false;
      break;
    }
    // merge the CTAs' candidates
    double best = -1.0, sec = -1.0;
    int bidx = -1;
    grid_merge(slots + par * G, G, s_bv, s_sv, s_bi, &best, &sec, &bidx);
    if (bidx < 0) break;  // no candidate left (cannot happen for step < min(m, N))
    const int owner = bidx / cpb;
    const real_t* pcs = stg + ((size_t)par * G + owner) * m;  // the pivot column, rows step..
    double nusq = best;
    if (sizeof(real_t) < sizeof(double)) {
      // FP32 storage: nu_0 and near-threshold decisions use the FP64 norm
      const bool nearthr = step == 0 || fabs(nusq - thr1 * nu0sq) <= 1e-4 * thr1 * nu0sq ||
                           (superfine && fabs(nusq - thr2 * nu0sq) <= 1e-4 * thr2 * nu0sq);
      if (nearthr) {
        if (warp == 0) {
          double s64 = 0.0;
          for (int i = step + lane; i < m; i += kWarp) {
            const double a = (double)__ldcg(pcs + i);
            s64 = fma(a, a, s64);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) s64 += __shfl_xor_sync(0xffffffffu, s64, o);
          if (lane == 0) s_nu64 = s64;
        }
        __syncthreads();
        nusq = s_nu64;
        __syncthreads();
      }
    }
    if (step == 0) {
      nu0sq = nusq;
      if (nu0sq == 0.0) {
        r = 0;
        break;
      }
      T1 = thr1 * nu0sq;
      T2 = thr2 * nu0sq;
    }
    // the flags (kept by thread 0 only) and the stop decisions: FP64 work in
    // one thread, integer comparisons of non-negative doubles in the others
    if (tid == 0) {
      if (sec >= 0.0 && nusq > 0.0 && nusq - sec <= 1e-12 * nusq) flags |= 1;
      if (fabs(nusq - T1) <= 1e-10 * T1) flags |= 2;
      if (superfine && fabs(nusq - T2) <= 1e-10 * T2) flags |= 2;
    }
    const long long nk = __double_as_longlong(nusq);
    if (r < 0 && nk < __double_as_longlong(T1)) {
      r = step;
      if (!superfine) break;
    }
    if (superfine && nk < __double_as_longlong(T2)) break;
    // warp 0 forms the reflector scalars while the other warps read the pivot
    // column (a long dependent FP64 sequence against an L2 read)
    if (warp == 0) {
      reflector_scalars(__ldcg(pcs + step), (real_t)nusq, lane, s_refl);
    } else {
      for (int i = step + 1 + tid - kWarp; i < m; i += kQrThreads - kWarp) v[i] = __ldcg(pcs + i);
    }
    __syncthreads();
    const real_t beta = s_refl[0], tau = s_refl[1], inv = s_refl[2];
    const bool own = crank == owner;
    const int lp = bidx - g0;
    for (int i = tid; i < m; i += kQrThreads) {
      real_t vi;
      if (i < step) vi = 0;
      else if (i == step) vi = 1;
      else vi = v[i] * inv;
      v[i] = vi;
      if (own) {
        t.V[i + (size_t)step * m] = vi;
        if (i >= step) A[(size_t)i * ncl + lp] = (i == step) ? beta : (real_t)0;  // R entries
      }
    }
    if (own && tid == 0) {
      t.tau[step] = tau;
      norms[lp] = -1;
      cand[lp] = -1;
      hib[lp] = -1;
    }
    __syncthreads();
    // apply H_step to the CTA's other live columns
    long long lbk = 0;  // FP64: the largest lower bound d - B of the CTA's live columns (bits)
    for (int l = grp; l < nloc; l += ngrp) {
      if (norms[l] < (real_t)0) continue;  // the same l for the whole group
      real_t* a = A + l;
      real_t d0 = 0, d1 = 0;
      int i = step + sl;
      for (; i + tpc < m; i += 2 * tpc) {
        d0 = fma(v[i], a[(size_t)i * ncl], d0);
        d1 = fma(v[i + tpc], a[(size_t)(i + tpc) * ncl], d1);
      }
      if (i < m) d0 = fma(v[i], a[(size_t)i * ncl], d0);
      real_t dd = d0 + d1;
      for (int o = tpc >> 1; o > 0; o >>= 1) dd += __shfl_xor_sync(gmask, dd, o);
      const real_t f = tau * dd;
      real_t q0 = 0, q1 = 0;
      i = step + sl;
      for (; i + tpc < m; i += 2 * tpc) {
        const real_t x0 = fma(-f, v[i], a[(size_t)i * ncl]);
        const real_t x1 = fma(-f, v[i + tpc], a[(size_t)(i + tpc) * ncl]);
        a[(size_t)i * ncl] = x0;
        a[(size_t)(i + tpc) * ncl] = x1;
        if (!kDown) {
          if (i > step) q0 = fma(x0, x0, q0);
          q1 = fma(x1, x1, q1);
        }
      }
      if (i < m) {
        const real_t x0 = fma(-f, v[i], a[(size_t)i * ncl]);
        a[(size_t)i * ncl] = x0;
        if (!kDown && i > step) q0 = fma(x0, x0, q0);
      }
      if constexpr (kDown) {
        if (sl == 0) {  // this thread wrote the pivot-row entry
          const double x = a[(size_t)step * ncl];
          const double dold = norms[l], eold = errb[l];
          double dn = fma(-x, x, dold);
          if (__double_as_longlong(dn) < 0) dn = 0.0;  // T >= 0: clamping stays in the bound
          const double en = fma(qd.c2, dold, eold * qd.c1);
          const double sb = dn + en;
          norms[l] = dn;
          errb[l] = en;
          hib[l] = sb * qd.g1;
          cand[l] = -1;
          lbk = max(lbk, __double_as_longlong(fma(-qd.gam, sb, dn - en)));
        }
      } else {
        real_t q = q0 + q1;
        for (int o = tpc >> 1; o > 0; o >>= 1) q += __shfl_xor_sync(gmask, q, o);
        if (sl == 0) {
          norms[l] = q;
          cand[l] = q;
        }
      }
    }
    __syncthreads();
    if constexpr (kDown) {
      // the columns that may hold the exact maximum (upper bound d + B at least
      // L (1 - 4e-12), L the largest lower bound; see the cluster kernel) are
      // recomputed exactly and become the candidates; integer comparisons
      const unsigned long long lbw = warp_max((unsigned long long)lbk);
      if (lane == 0) s_lbg[warp] = lbw;
      __syncthreads();
      unsigned long long Lk = 0;
      for (int w = 0; w < nw; ++w) Lk = max(Lk, s_lbg[w]);
      const long long Lthr = Lk > 36030ull ? (long long)Lk - 36030 : 0;  // L (1 - 4e-12) or less
      for (int c0 = warp * kWarp; c0 < nloc; c0 += nw * kWarp) {
        const int lc = c0 + lane;
        const bool mem = lc < nloc && __double_as_longlong((double)hib[lc]) >= Lthr;
        unsigned bal = __ballot_sync(0xffffffffu, mem);
        while (bal) {
          const int l = c0 + __ffs(bal) - 1;
          bal &= bal - 1;
          real_t s0 = 0, s1 = 0;
          int i = step + 1 + lane;
          for (; i + kWarp < m; i += 2 * kWarp) {
            const real_t x0 = A[(size_t)i * ncl + l], x1 = A[(size_t)(i + kWarp) * ncl + l];
            s0 = fma(x0, x0, s0);
            s1 = fma(x1, x1, s1);
          }
          if (i < m) s0 = fma(A[(size_t)i * ncl + l], A[(size_t)i * ncl + l], s0);
          const real_t s2 = warp_sum(s0 + s1);
          if (lane == 0) {
            norms[l] = s2;
            errb[l] = gam * s2;
            cand[l] = s2;
          }
        }
      }
      __syncthreads();
    }
    nsteps = step + 1;
  }
  if (!ok) {
    if (tid == 0) atomicExch(t.err + 1, 1);
    return;
  }
  if (r < 0) r = nsteps;
  __syncthreads();
  // write the slice back, mirror the coarse rows into the neighbours' rows
  for (int e = tid; e < m * nloc; e += kQrThreads) {
    const int i = e % m, l = e / m;
    t.A[i + (size_t)pcol[l] * ld] = A[(size_t)i * ncl + l];
  }
  for (int e = tid; e < r * nloc; e += kQrThreads) {
    const int i = e % r, l = e / r;
    const RRQRSeg g = segs[t.seg_begin + segid[l]];
    const int c = g0 + l - segoff[segid[l]];
    g.mirror[c + (size_t)i * g.mirror_ld] = A[(size_t)i * ncl + l];
  }
  if (crank == 0) {
    for (int e = tid; e < r * r; e += kQrThreads) {
      const int i = e % r, j = e / r;
      t.diag[i + (size_t)j * ld] = (i == j) ? 1.0 : 0.0;
    }
    if (tid == 0) {
      t.rank[t.id] = r;
      t.nref[t.id] = nsteps;
      t.flag[t.id] = flags;
      t.cur[t.id] = r;
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
constexpr int kSmemBudget = 200 * 1024;  // dynamic shared memory per CTA we allow

// Errors of the grant surface through cudaGetLastError, which the callers check
// after each stage's launches.
static void set_smem(const void* fn, int bytes) { (void)grant_smem(fn, bytes); }

void launch_copy(const CopyTask* t, int ntasks, cudaStream_t s) {
  if (ntasks > 0) k_copy<<<ntasks, 256, 0, s>>>(t);
}

void launch_scatter(const double* val, const int64_t* dst_index, real_t* base_lo,
                    real_t* base_hi, int64_t split, int64_t nnz, cudaStream_t s) {
  if (nnz <= 0) return;
  const int64_t nb = std::min<int64_t>((nnz + 255) / 256, 152 * 32);
  k_scatter<<<(int)nb, 256, 0, s>>>(val, dst_index, base_lo, base_hi, split, nnz);
}

void launch_set_identity(const PotrfTask* t, int ntasks, cudaStream_t s) {
  if (ntasks > 0) k_set_identity<<<ntasks, 256, 0, s>>>(t);
}

void launch_potrf(const PotrfTask* t, int ntasks, int max_m, cudaStream_t s) {
  if (ntasks <= 0) return;
  int cap = max_m * max_m;
  int bytes = cap * (int)sizeof(real_t);
  if (bytes > kSmemBudget) {
    cap = kSmemBudget / (int)sizeof(real_t);
    bytes = kSmemBudget;
  }
  set_smem((const void*)k_potrf, bytes);
  k_potrf<<<ntasks, 256, bytes, s>>>(t, cap);
}

void launch_trsm(const TrsmTask* t, int ntasks, int max_m, cudaStream_t s) {
  if (ntasks <= 0) return;
  int rows = max_m;
  int bytes = rows * kTrsmNC * (int)sizeof(real_t);
  if (bytes > kSmemBudget) {
    rows = kSmemBudget / (kTrsmNC * (int)sizeof(real_t));
    bytes = rows * kTrsmNC * (int)sizeof(real_t);
  }
  set_smem((const void*)k_trsm, bytes);
  k_trsm<<<ntasks, kTrsmThreads, bytes, s>>>(t, rows);
}

void launch_form_qt(const FormQtTask* t, int ntasks, int max_m, cudaStream_t s) {
  if (ntasks <= 0) return;
  int rows = max_m;
  const int extra = 4 * kTrsmNC * (int)sizeof(real_t);
  int bytes = rows * kTrsmNC * (int)sizeof(real_t) + extra;
  if (bytes > kSmemBudget) {
    rows = (kSmemBudget - extra) / (kTrsmNC * (int)sizeof(real_t));
    bytes = rows * kTrsmNC * (int)sizeof(real_t) + extra;
  }
  set_smem((const void*)k_form_qt, bytes);
  k_form_qt<<<ntasks, kFqThreads, bytes, s>>>(t, rows);
}

void launch_schur(const SchurTile* tiles, int ntiles, const SchurContrib* c, cudaStream_t s) {
  if (ntiles > 0) k_schur<<<ntiles, 256, 0, s>>>(tiles, c);
}

bool schur_tc_available() {
#ifdef SPAND_SINGLE
  return true;
#else
  return false;
#endif
}

cudaError_t launch_schur_tc(const SchurTile* tiles, int ntiles, const SchurContrib* c, int* err,
                            cudaStream_t s) {
#ifdef SPAND_SINGLE
  if (ntiles <= 0) return cudaSuccess;
  const cudaError_t e = grant_smem((const void*)k_schur_tc, kTcSmem);
  if (e != cudaSuccess) return e;
  k_schur_tc<<<ntiles, kTcThreads, kTcSmem, s>>>(tiles, c, err);
  return cudaGetLastError();
#else
  (void)tiles;
  (void)ntiles;
  (void)c;
  (void)err;
  (void)s;
  return cudaErrorNotSupported;
#endif
}

int rrqr_cluster_smem_bytes(int m, int ncols_max, int nseg, int csize) {
  const long e = (long)sizeof(real_t);
#ifdef SPAND_SINGLE
  const long ncl = (ncols_max + csize - 1) / csize;
  const long ldm = (long)qr_cm_nvec(m) * kQv;
  const long b = 16 + e * ldm * (ncl + 1) + e * ncl + 8L * ncl + 4L * (nseg + 2) + 16;
#else
  const long ncl = ((ncols_max + csize - 1) / csize) | 1;
  const long b = e * m * ncl + e * m + 3 * e * ncl + 8L * ncl + 4L * (nseg + 2) + 16;
#endif
  return (int)std::min<long>(b, 1L << 30);
}

cudaError_t launch_rrqr_cluster(const RRQRTask* t, int ntasks, const RRQRSeg* segs, int csize,
                                int smem_bytes, int threads, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  cudaError_t e = grant_smem((const void*)k_rrqr_cluster, smem_bytes);
  if (e == cudaSuccess && csize > 8) e = allow_wide_clusters((const void*)k_rrqr_cluster);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(ntasks * csize));
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = (size_t)smem_bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_rrqr_cluster, t, segs, csize);
}

int rrqr_cluster_active(int csize, int smem_bytes, int threads) {
  cudaError_t e = grant_smem((const void*)k_rrqr_cluster, smem_bytes);
  if (e == cudaSuccess && csize > 8) e = allow_wide_clusters((const void*)k_rrqr_cluster);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)csize);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = (size_t)smem_bytes;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (const void*)k_rrqr_cluster, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

int rrqr_smem_bytes(int max_m, int max_cols, int max_segs) {
  // norms (real_t) + v (real_t) + cols (int) + segoff (int)
  return max_cols * (int)sizeof(real_t) + max_m * (int)sizeof(real_t) + max_cols * 4 +
         (max_segs + 2) * 4 + 16;
}

void launch_rrqr(const RRQRTask* t, int ntasks, const RRQRSeg* segs,
                 int max_m, int max_cols, int max_segs, cudaStream_t s) {
  if (ntasks <= 0) return;
  const int bytes = rrqr_smem_bytes(max_m, max_cols, max_segs);
  set_smem((const void*)k_rrqr, bytes);
  k_rrqr<<<ntasks, kQrThreads, bytes, s>>>(t, segs);
}

int rrqr_grid_smem_bytes(int max_m, int max_cpb, int max_segs) {
  // v (real_t) + norms, bounds, candidates (real_t) + cols, members (int) + segoff (int)
  return max_m * (int)sizeof(real_t) + 3 * max_cpb * (int)sizeof(real_t) + 2 * max_cpb * 4 +
         (max_segs + 2) * 4 + 16;
}

int rrqr_gsm_smem_bytes(int m, int cpb, int nseg) {
  const long ncl = gsm_ncl(cpb), e = (long)sizeof(real_t);
  // the slice, v, then d, E, the candidates' norms and d + B (real_t), the
  // columns' panel positions and segments (int), the segment offsets
  const long b = e * m * ncl + e * m + 4 * e * ncl + 8L * ncl + 4L * (nseg + 2) + 16;
  return (int)std::min<long>(b, 1L << 30);
}

cudaError_t launch_rrqr_gsm(const RRQRGridTask* t, int ntasks, int nctas, const RRQRSeg* segs,
                            int smem_bytes, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  const cudaError_t e = grant_smem((const void*)k_rrqr_gsm, smem_bytes);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nctas);
  cfg.blockDim = dim3(kQrThreads);
  cfg.dynamicSmemBytes = (size_t)smem_bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident, or the launch fails
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_rrqr_gsm, t, ntasks, segs);
}

cudaError_t launch_rrqr_grid(const RRQRGridTask* t, int ntasks, int nctas, const RRQRSeg* segs,
                             int smem_bytes, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  const cudaError_t e = grant_smem((const void*)k_rrqr_grid, smem_bytes);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nctas);
  cfg.blockDim = dim3(kQrThreads);
  cfg.dynamicSmemBytes = (size_t)smem_bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident, or the launch fails
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_rrqr_grid, t, ntasks, segs);
}

}  // namespace SPAND_NS
}  // namespace spand
