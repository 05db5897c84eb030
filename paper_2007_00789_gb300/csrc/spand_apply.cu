// Preconditioner apply M = L^{-T} L^{-1} (§3, Algorithm 2 caption).
//
// L^{-1} is the product, in processing order, of the elimination operators
// G_s, the scalings D_p and the sparsification operators E_p Q_p^T of
// Algorithm 2.  The forward sweep applies them in that order to the n-vector
// z; the backward sweep applies their transposes in reverse.  Every variable
// has a fixed position ("slot") in z; after Q_p^T the coarse coordinates of p
// occupy its first r slots and the fine ones the rest.  Each phase below is
// one launch batched over the operators of one stage (or one colour), which
// touch disjoint slots except for the accumulation into neighbour slots, done
// with atomics.  An item of a launch may carry several vectors (right-hand
// sides of one problem, ldz apart): the operator is then read once for up to
// NV of them at a time.
#include <cooperative_groups.h>

#include "spand_real.h"

namespace spand {
namespace SPAND_NS {

namespace {

constexpr int kApThreads = 256;
constexpr int kApWarps = kApThreads / 32;
// Four resident CTAs per SM stated (registers capped to fit): measured on the
// batch of 64 problems, FP64 128.9 solves/s against 119.1 with two CTAs, FP32
// 296.9 against 282.9 with the compiler's own choice (three: 125.8 and 281.0)
#ifndef SPAND_AP_MINB
#define SPAND_AP_MINB 4
#endif
#if SPAND_AP_MINB > 0
#define AP_BOUNDS __launch_bounds__(kApThreads, SPAND_AP_MINB)
#else
#define AP_BOUNDS __launch_bounds__(kApThreads)
#endif

namespace cg = cooperative_groups;

// Matrix-vector products for NV vectors at once, written for memory-level
// parallelism: the operators are read once from HBM, so each warp keeps many
// independent coalesced loads in flight.  Each matrix element loaded feeds NV
// FMAs (one per vector).  The vectors sit in shared memory, vector v at
// x + v * xs.

// One 64-row tile starting at rt of gemv_n below; TWO = false when the tile's
// second half holds no row, so that no instruction is spent on it (an FP64
// instruction costs its full warp width on the narrow FP64 pipe whatever the
// active lanes).
template <int NV, bool TWO, class Out>
__device__ __forceinline__ void gemv_n_tile(const real_t* __restrict__ M, size_t ld, int r0, int r1,
                                            int rt, int C, const real_t* __restrict__ x, int xs,
                                            real_t* red, Out& out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ra = rt + lane, rb = rt + 32 + lane;
  const bool va = ra < r1, vb = TWO && rb < r1;
  const int per = (((C + kApWarps - 1) / kApWarps) + 3) & ~3;
  const int cb = warp * per, ce = min(C, cb + per);
  real_t sa[NV], sb[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) sa[v] = sb[v] = 0.0;
  const real_t* Ma = M + (va ? ra : r0);
  const real_t* Mb = M + (vb ? rb : r0);
  int c = cb;
#pragma unroll 2
  for (; c + 3 < ce; c += 4) {
    real_t a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a[u] = va ? Ma[(size_t)(c + u) * ld] : (real_t)0.0;
      if (TWO) b[u] = vb ? Mb[(size_t)(c + u) * ld] : (real_t)0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const real_t xv = x[v * xs + c + u];
        sa[v] = fma(a[u], xv, sa[v]);
        if (TWO) sb[v] = fma(b[u], xv, sb[v]);
      }
  }
  for (; c < ce; ++c) {
    const real_t a = va ? Ma[(size_t)c * ld] : (real_t)0.0;
    const real_t b = vb ? Mb[(size_t)c * ld] : (real_t)0.0;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      sa[v] = fma(a, x[v * xs + c], sa[v]);
      if (TWO) sb[v] = fma(b, x[v * xs + c], sb[v]);
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    red[(v * kApWarps + warp) * 64 + lane] = sa[v];
    if (TWO) red[(v * kApWarps + warp) * 64 + 32 + lane] = sb[v];
  }
  __syncthreads();
  if (warp < (TWO ? 2 : 1)) {
    const int r = rt + warp * 32 + lane;
    if (r < r1) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        real_t t = 0.0;
        for (int w = 0; w < kApWarps; ++w) t += red[(v * kApWarps + w) * 64 + warp * 32 + lane];
        out(r, v, t);
      }
    }
  }
  __syncthreads();
}

// out(r, v, sum_{c < C(rt)} M[r + c*ld] x_v[c]) for rows r in [r0, r1); ccap(rt)
// bounds the columns a 64-row tile starting at rt needs (C for a full matrix,
// rt + 64 for a lower-triangular one whose strict upper part is zero).  A
// warp reads columns of a 64-row tile (lane = rows rt+lane and rt+32+lane,
// four columns per step: eight 128-byte loads in flight per lane pair), the
// warps split the columns, and warp 0 and 1 add the warps' partial sums.
template <int NV, class Cap, class Out>
__device__ void gemv_n(const real_t* __restrict__ M, size_t ld, int r0, int r1, Cap ccap,
                       const real_t* __restrict__ x, int xs, real_t* red, Out out) {
  for (int rt = r0; rt < r1; rt += 64) {
    // FP32 keeps one code path (the skipped half costs little on the FP32 pipe)
    if (sizeof(real_t) == sizeof(float) || rt + 32 < r1)
      gemv_n_tile<NV, true>(M, ld, r0, r1, rt, ccap(rt), x, xs, red, out);
    else
      gemv_n_tile<NV, false>(M, ld, r0, r1, rt, ccap(rt), x, xs, red, out);
  }
}

// out(c, v, sum_{r in [rlo(c), R)} M[r + c*ld] x_v[r]) for columns c in [c0, c1);
// rlo(c) is the first row column c needs (0 for a full matrix, c for the
// transpose of a lower-triangular one).  A warp reduces four columns at a time
// over a range of rows: its lanes read consecutive rows of each (coalesced, four
// loads in flight per lane), then the partial sums are added across the warp.
// When the columns are too few to give every warp four (a thin slice of a
// large operator), the rows are split into chunks as well, so that all warps
// work, and the chunks' partial sums are added in a fixed order in shared
// memory (red: at least 32 * NV entries).
template <int NV, class Lo, class Out>
__device__ void gemv_t(const real_t* __restrict__ M, size_t ld, int c0, int c1, int R, Lo rlo,
                       const real_t* __restrict__ x, int xs, real_t* red, Out out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ncol = c1 - c0;
  if (ncol <= 0) {
    __syncthreads();
    return;
  }
  const int ncg = (ncol + 3) / 4;                              // groups of four columns
  const int nrc = ncg >= kApWarps ? 1 : (kApWarps + ncg - 1) / ncg;  // row chunks per group
  const int chunk = nrc == 1 ? R : (((R + nrc - 1) / nrc) + 31) & ~31;
  for (int item = warp; item < ncg * nrc; item += kApWarps) {
    const int g = item % ncg, rc = item / ncg;
    const int cq = c0 + 4 * g;
    real_t s[4][NV];
    int lo4[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      lo4[u] = cq + u < c1 ? rlo(cq + u) : R;
#pragma unroll
      for (int v = 0; v < NV; ++v) s[u][v] = 0.0;
    }
    const int rb = rc * chunk, re = min(R, rb + chunk);
    const int rs = max(rb, min(min(lo4[0], lo4[1]), min(lo4[2], lo4[3])));
#pragma unroll 2
    for (int r = rs + lane; r < re; r += 32) {
      real_t a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        a[u] = (r >= lo4[u]) ? M[(size_t)(cq + u) * ld + r] : (real_t)0.0;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const real_t xv = x[v * xs + r];
#pragma unroll
        for (int u = 0; u < 4; ++u) s[u][v] = fma(a[u], xv, s[u][v]);
      }
    }
    // the four columns' sums across the warp, transposed as they are reduced:
    // after the xor-16 and xor-8 exchanges each lane carries one column
    // (u = 2 * bit 4 + bit 3 of the lane), so 6 additions replace 20
    const bool h16 = lane & 16, h8 = lane & 8;
    const int uq = (h16 ? 2 : 0) + (h8 ? 1 : 0);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      real_t k0 = h16 ? s[2][v] : s[0][v], k1 = h16 ? s[3][v] : s[1][v];
      const real_t g0 = h16 ? s[0][v] : s[2][v], g1 = h16 ? s[1][v] : s[3][v];
      k0 += __shfl_xor_sync(0xffffffffu, g0, 16);
      k1 += __shfl_xor_sync(0xffffffffu, g1, 16);
      real_t t = h8 ? k1 : k0;
      t += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
      t += __shfl_xor_sync(0xffffffffu, t, 4);
      t += __shfl_xor_sync(0xffffffffu, t, 2);
      t += __shfl_xor_sync(0xffffffffu, t, 1);
      if ((lane & 7) == 0 && cq + uq < c1) {
        if (nrc == 1) out(cq + uq, v, t);
        else red[((rc * ncg + g) * 4 + uq) * NV + v] = t;
      }
    }
  }
  __syncthreads();
  if (nrc > 1) {
    for (int e = threadIdx.x; e < ncol * NV; e += blockDim.x) {
      const int c = e / NV, v = e - c * NV;
      real_t t = 0.0;
      for (int rc = 0; rc < nrc; ++rc) t += red[((rc * ncg + (c >> 2)) * 4 + (c & 3)) * NV + v];
      out(c0 + c, v, t);
    }
    __syncthreads();
  }
}

// out(r, v, sum_{c < C} M[r + c*ld] x_v[c]) for rows r in [r0, r1), one thread
// per row: for a matrix of few columns (C up to a few dozen) whose rows are the
// long dimension, every thread keeps C independent loads in flight, the warp's
// loads of one column are consecutive, and no partial sums cross threads.
template <int NV, class Out>
__device__ void gemv_rows(const real_t* __restrict__ M, size_t ld, int r0, int r1, int C,
                          const real_t* __restrict__ x, int xs, Out out) {
  for (int r = r0 + (int)threadIdx.x; r < r1; r += blockDim.x) {
    real_t s[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) s[v] = 0.0;
    const real_t* p = M + r;
#pragma unroll 8
    for (int c = 0; c < C; ++c) {
      const real_t a = p[(size_t)c * ld];
#pragma unroll
      for (int v = 0; v < NV; ++v) s[v] = fma(a, x[v * xs + c], s[v]);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) out(r, v, s[v]);
  }
}

// Every operator is applied by a thread-block cluster of K CTAs (K from the
// launch; 1 for small operators); CTA k produces the contiguous slice
// [n k / K, n (k+1) / K) of each output.  When a later step needs a whole
// intermediate vector, each CTA stores its slice into every CTA's shared
// memory and the cluster synchronises.  Shared memory per vector: x (m),
// y (m), gathered neighbour values (ncols); and the warps' partial sums.
__device__ __forceinline__ int part_lo(int n, int k, int K) { return (int)(((long)n * k) / K); }

__device__ __forceinline__ void share(cg::cluster_group& cl, int K, real_t* buf, int i, real_t val) {
  for (int c = 0; c < K; ++c) cl.map_shared_rank(buf, c)[i] = val;
}

// The item that holds launch-wide operator `task` (items are sorted by `first`).
__device__ __forceinline__ ApItem find_item(const ApItem* __restrict__ items, int nitems, int task) {
  int lo = 0, hi = nitems - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].first <= task) lo = mid;
    else hi = mid - 1;
  }
  return items[lo];
}

template <int NV>
__global__ void AP_BOUNDS
    k_ap_interior(const ApItem* __restrict__ items, int nitems, real_t* __restrict__ z, int forward) {
  cg::cluster_group cl = cg::this_cluster();
  const int K = (int)cl.num_blocks(), k = (int)cl.block_rank();
  extern __shared__ real_t sh[];
  __shared__ real_t red[2 * kApThreads * NV];
  const int task = (int)(blockIdx.x / K);
  const ApItem it = find_item(items, nitems, task);
  const ApInterior t = ((const ApInterior*)it.ops)[task - it.first];
  const int m = t.m, nc = t.ncols;
  real_t* xs = sh;               // NV x m
  real_t* ys = sh + NV * m;      // NV x m
  real_t* zw = sh + 2 * NV * m;  // NV x nc
  const int lo = part_lo(m, k, K), hi = part_lo(m, k + 1, K);
  const size_t ldz = (size_t)it.ldz;
  for (int v0 = 0; v0 < it.nvec; v0 += NV) {
    const int nv = min(NV, it.nvec - v0);
    real_t* zb = z + it.zoff + (size_t)v0 * ldz;
    for (int e = threadIdx.x; e < NV * m; e += blockDim.x) {
      const int v = e / m, i = e - v * m;
      xs[e] = v < nv ? zb[v * ldz + t.slots[i]] : (real_t)0.0;
    }
    if (!forward)
      for (int e = threadIdx.x; e < NV * nc; e += blockDim.x) {
        const int v = e / nc, c = e - v * nc;
        const int ws = t.wslots[c];
        // the diagonal segment (ws < 0) contributes nothing
        zw[e] = (v < nv && ws >= 0) ? zb[v * ldz + ws] : (real_t)0.0;
      }
    __syncthreads();
    if (forward) {
      // y = L_s^{-1} x, then z_s = y and z_w -= W_s y (column c of the panel row is W_s^T[:, c])
      gemv_n<NV>(t.Linv, m, lo, hi, [&](int rt) { return min(m, rt + 64); }, xs, m, red,
                 [&](int r, int v, real_t val) { share(cl, K, ys + v * m, r, val); });
      cl.sync();
      for (int e = threadIdx.x; e < nv * (hi - lo); e += blockDim.x) {
        const int v = e / (hi - lo), i = lo + e - v * (hi - lo);
        zb[v * ldz + t.slots[i]] = ys[v * m + i];
      }
      gemv_t<NV>(t.WT, m, part_lo(nc, k, K), part_lo(nc, k + 1, K), m, [](int) { return 0; }, ys, m,
                 red, [&](int c, int v, real_t val) {
                   const int ws = t.wslots[c];
                   if (ws >= 0 && v < nv) atomicAdd(zb + v * ldz + ws, -val);
                 });
    } else {
      // y = x - W_s^T z_w, then z_s = L_s^{-T} y
      gemv_n<NV>(t.WT, m, lo, hi, [&](int) { return nc; }, zw, nc, red,
                 [&](int r, int v, real_t val) { share(cl, K, ys + v * m, r, xs[v * m + r] - val); });
      cl.sync();
      gemv_t<NV>(t.Linv, m, lo, hi, m, [](int ct) { return ct; }, ys, m, red,
                 [&](int j, int v, real_t val) {
                   if (v < nv) zb[v * ldz + t.slots[j]] = val;
                 });
    }
    if (v0 + NV < it.nvec) cl.sync();  // no CTA refills ys while another still reads it
  }
}

template <int NV>
__global__ void AP_BOUNDS
    k_ap_scale(const ApItem* __restrict__ items, int nitems, real_t* __restrict__ z, int forward) {
  cg::cluster_group cl = cg::this_cluster();
  const int K = (int)cl.num_blocks(), k = (int)cl.block_rank();
  extern __shared__ real_t sh[];
  __shared__ real_t red[2 * kApThreads * NV];
  const int task = (int)(blockIdx.x / K);
  const ApItem it = find_item(items, nitems, task);
  const ApScale t = ((const ApScale*)it.ops)[task - it.first];
  const int m = t.m;
  real_t* xs = sh;  // NV x m
  const int lo = part_lo(m, k, K), hi = part_lo(m, k + 1, K);
  const size_t ldz = (size_t)it.ldz;
  for (int v0 = 0; v0 < it.nvec; v0 += NV) {
    const int nv = min(NV, it.nvec - v0);
    real_t* zb = z + it.zoff + (size_t)v0 * ldz;
    for (int e = threadIdx.x; e < NV * m; e += blockDim.x) {
      const int v = e / m, i = e - v * m;
      xs[e] = v < nv ? zb[v * ldz + t.slots[i]] : (real_t)0.0;
    }
    cl.sync();  // every CTA has read z_p before any CTA overwrites part of it
    if (forward)
      gemv_n<NV>(t.Zinv, m, lo, hi, [&](int rt) { return min(m, rt + 64); }, xs, m, red,
                 [&](int r, int v, real_t val) {
                   if (v < nv) zb[v * ldz + t.slots[r]] = val;
                 });
    else
      gemv_t<NV>(t.Zinv, m, lo, hi, m, [](int ct) { return ct; }, xs, m, red,
                 [&](int j, int v, real_t val) {
                   if (v < nv) zb[v * ldz + t.slots[j]] = val;
                 });
    if (v0 + NV < it.nvec) __syncthreads();
  }
}

template <int NV>
__global__ void AP_BOUNDS
    k_ap_qe(const ApItem* __restrict__ items, int nitems, real_t* __restrict__ z, int forward) {
  cg::cluster_group cl = cg::this_cluster();
  const int K = (int)cl.num_blocks(), k = (int)cl.block_rank();
  extern __shared__ real_t sh[];
  __shared__ real_t red[2 * kApThreads * NV];
  const int task = (int)(blockIdx.x / K);
  const ApItem it = find_item(items, nitems, task);
  const ApQE t = ((const ApQE*)it.ops)[task - it.first];
  const int m = t.m, nc = t.ncols, nE = t.nE;
  real_t* xs = sh;               // NV x m
  real_t* ys = sh + NV * m;      // NV x m
  real_t* zw = sh + 2 * NV * m;  // NV x nc
  const int lo = part_lo(m, k, K), hi = part_lo(m, k + 1, K);
  const size_t ldz = (size_t)it.ldz;
  for (int v0 = 0; v0 < it.nvec; v0 += NV) {
    const int nv = min(NV, it.nvec - v0);
    real_t* zb = z + it.zoff + (size_t)v0 * ldz;
    for (int e = threadIdx.x; e < NV * m; e += blockDim.x) {
      const int v = e / m, i = e - v * m;
      xs[e] = v < nv ? zb[v * ldz + t.slots[i]] : (real_t)0.0;
    }
    if (!forward && nE > 0)
      for (int e = threadIdx.x; e < NV * nc; e += blockDim.x) {
        const int v = e / nc, c = e - v * nc;
        zw[e] = v < nv ? zb[v * ldz + t.eslots[c]] : (real_t)0.0;
      }
    __syncthreads();
    if (forward) {
      // y = Q^T x; z_p = y; z_w -= E-tilde^T y_f
      gemv_n<NV>(t.Qt, m, lo, hi, [&](int) { return m; }, xs, m, red,
                 [&](int r, int v, real_t val) { share(cl, K, ys + v * m, r, val); });
      cl.sync();
      for (int e = threadIdx.x; e < nv * (hi - lo); e += blockDim.x) {
        const int v = e / (hi - lo), i = lo + e - v * (hi - lo);
        zb[v * ldz + t.slots[i]] = ys[v * m + i];
      }
      // (E-tilde is row-major: column c of E-tilde is row c of a column-major
      // ncols x nE matrix with leading dimension ncols)
      if (nE > 0)
        gemv_rows<NV>(t.E, nc, part_lo(nc, k, K), part_lo(nc, k + 1, K), nE, ys + t.r, m,
                      [&](int c, int v, real_t val) {
                        if (v < nv) atomicAdd(zb + v * ldz + t.eslots[c], -val);
                      });
    } else {
      // x_f -= E-tilde z_w, then z_p = Q x
      for (int e = threadIdx.x; e < NV * (hi - lo); e += blockDim.x) {
        const int v = e / (hi - lo), i = lo + e - v * (hi - lo);
        if (i < t.r || i >= t.r + nE) share(cl, K, ys + v * m, i, xs[v * m + i]);
      }
      if (nE > 0) {
        const int flo = max(lo, t.r) - t.r, fhi = min(hi, t.r + nE) - t.r;
        // row i of E-tilde is contiguous: a warp reduces four rows at a time
        if (fhi > flo)
          gemv_t<NV>(t.E, nc, flo, fhi, nc, [](int) { return 0; }, zw, nc, red,
                     [&](int i, int v, real_t val) {
                       share(cl, K, ys + v * m, t.r + i, xs[v * m + t.r + i] - val);
                     });
      }
      cl.sync();
      gemv_t<NV>(t.Qt, m, lo, hi, m, [](int) { return 0; }, ys, m, red,
                 [&](int j, int v, real_t val) {
                   if (v < nv) zb[v * ldz + t.slots[j]] = val;
                 });
    }
    if (v0 + NV < it.nvec) cl.sync();  // no CTA refills ys while another still reads it
  }
}

// ---------------------------------------------------------------------------
// The whole preconditioner sweep of one problem and one right-hand side as
// one persistent cooperative launch.  The sweep is a list of sub-phases; a
// sub-phase is a list of items -- one operator and a range of its rows or
// columns -- that the CTAs take in turn, and a grid-wide barrier separates
// dependent sub-phases.  An operator too large for one CTA is thereby spread
// over as many CTAs as its size asks for (a thread-block cluster holds at most
// 16), and a stage's few large operators no longer leave most SMs idle.  Where
// an operator's product needs all of an intermediate vector (y = L^{-1} x
// before the W_s update, y = Q^T x before the E-tilde one, ...), the
// intermediate goes to the scratch vector Y at the operator's own slots (the
// slots of the operators of one sub-phase are disjoint) and the next
// sub-phase reads it there.  Reads of z and Y go through L2 (__ldcg): they
// were written by other SMs before the barrier.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool sweep_barrier(int* ctr, int* abort, int target, long long limit) {
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
      __nanosleep(32);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Resident CTAs per SM the sweep is compiled for (registers capped to fit):
// measured on the 128^3 diffusion problem, one FP64 apply 14.3 / 13.1 / 13.5 ms
// for 2 / 3 / 4, one FP32 apply 10.0 / 8.1 / 7.5 ms.  (One warp per item for
// sub-phases of many small items, instead of the whole CTA, measured no faster:
// 13.8 against 13.2 ms FP64, 7.67 against 7.61 ms FP32.)
#ifndef SPAND_SWEEP_MINB
#ifdef SPAND_SINGLE
#define SPAND_SWEEP_MINB 4
#else
#define SPAND_SWEEP_MINB 3
#endif
#endif
__global__ void __launch_bounds__(kApThreads, SPAND_SWEEP_MINB)
    k_ap_sweep(const SwPhase* __restrict__ phases, int nph, const SwItem* __restrict__ items,
               const ApInterior* __restrict__ api, const ApScale* __restrict__ aps,
               const ApQE* __restrict__ apq, real_t* __restrict__ z, real_t* __restrict__ Y,
               int* ctr, int* abort, long long limit, long long* trace) {
  extern __shared__ real_t sh[];
  __shared__ real_t red[2 * kApThreads];
  // optional clock trace: CTA 0's SM clock at the start and as it leaves each
  // sub-phase's barrier (when every CTA has finished that sub-phase)
  if (trace && blockIdx.x == 0 && threadIdx.x == 0) trace[0] = clock64();
  const int tid = threadIdx.x, nt = blockDim.x;
  auto ld = [](const real_t* p) { return __ldcg(p); };
  for (int ph = 0; ph < nph; ++ph) {
    const SwPhase P = phases[ph];
    for (int q = blockIdx.x; q < P.nitems; q += gridDim.x) {
      const SwItem it = items[P.item0 + q];
      switch (P.kind) {
        case SW_FI_A: {  // rows of y = L_s^{-1} x_s into Y
          const ApInterior t = api[it.op];
          const int m = t.m;
          for (int i = tid; i < m; i += nt) sh[i] = ld(z + t.slots[i]);
          __syncthreads();
          gemv_n<1>(t.Linv, m, it.lo, it.hi, [&](int rt) { return min(m, rt + 64); }, sh, m, red,
                    [&](int r, int, real_t v) { Y[t.slots[r]] = v; });
          break;
        }
        case SW_FI_B: {  // z_s = y; z_w -= W_s y over a range of neighbour columns
          const ApInterior t = api[it.op];
          const int m = t.m;
          for (int i = tid; i < m; i += nt) sh[i] = ld(Y + t.slots[i]);
          __syncthreads();
          if (it.aux)
            for (int i = tid; i < m; i += nt) z[t.slots[i]] = sh[i];
          gemv_t<1>(t.WT, m, it.lo, it.hi, m, [](int) { return 0; }, sh, m, red,
                    [&](int c, int, real_t v) {
                      const int ws = t.wslots[c];
                      if (ws >= 0) atomicAdd(z + ws, -v);
                    });
          break;
        }
        case SW_FS_A: {  // rows of Z_p^{-1} x_p into Y
          const ApScale t = aps[it.op];
          const int m = t.m;
          for (int i = tid; i < m; i += nt) sh[i] = ld(z + t.slots[i]);
          __syncthreads();
          gemv_n<1>(t.Zinv, m, it.lo, it.hi, [&](int rt) { return min(m, rt + 64); }, sh, m, red,
                    [&](int r, int, real_t v) { Y[t.slots[r]] = v; });
          break;
        }
        case SW_COPY: {  // z = Y on a scaling's slots
          const ApScale t = aps[it.op];
          for (int i = it.lo + tid; i < it.hi; i += nt) z[t.slots[i]] = ld(Y + t.slots[i]);
          break;
        }
        case SW_FQ_A: {  // rows of y = Q_p^T x_p into Y
          const ApQE t = apq[it.op];
          const int m = t.m;
          for (int i = tid; i < m; i += nt) sh[i] = ld(z + t.slots[i]);
          __syncthreads();
          gemv_n<1>(t.Qt, m, it.lo, it.hi, [&](int) { return m; }, sh, m, red,
                    [&](int r, int, real_t v) { Y[t.slots[r]] = v; });
          break;
        }
        case SW_FQ_B: {  // z_p = y; z_w -= E-tilde^T y_f over a range of neighbour columns
          const ApQE t = apq[it.op];
          for (int i = tid; i < t.nE; i += nt) sh[i] = ld(Y + t.slots[t.r + i]);
          if (it.aux)
            for (int i = tid; i < t.m; i += nt) z[t.slots[i]] = ld(Y + t.slots[i]);
          __syncthreads();
          if (t.nE > 0)
            gemv_rows<1>(t.E, t.ncols, it.lo, it.hi, t.nE, sh, 0,
                         [&](int c, int, real_t v) { atomicAdd(z + t.eslots[c], -v); });
          break;
        }
        case SW_BQ_A: {  // y_f = x_f - E-tilde z_w over a range of fine rows, the rest copied, into Y
          const ApQE t = apq[it.op];
          const int nc = t.ncols;
          for (int c = tid; c < nc && t.nE > 0; c += nt) sh[c] = ld(z + t.eslots[c]);
          if (it.aux)
            for (int i = tid; i < t.m; i += nt)
              if (i < t.r || i >= t.r + t.nE) Y[t.slots[i]] = ld(z + t.slots[i]);
          __syncthreads();
          gemv_t<1>(t.E, nc, it.lo, it.hi, nc, [](int) { return 0; }, sh, nc, red,
                    [&](int i, int, real_t v) { Y[t.slots[t.r + i]] = ld(z + t.slots[t.r + i]) - v; });
          break;
        }
        case SW_BQ_B: {  // z_p = Q y over a range of output rows (columns of Q^T)
          const ApQE t = apq[it.op];
          const int m = t.m;
          for (int i = tid; i < m; i += nt) sh[i] = ld(Y + t.slots[i]);
          __syncthreads();
          gemv_t<1>(t.Qt, m, it.lo, it.hi, m, [](int) { return 0; }, sh, m, red,
                    [&](int j, int, real_t v) { z[t.slots[j]] = v; });
          break;
        }
        case SW_BS_A: {  // Z_p^{-T} x_p over a range of outputs, into Y
          const ApScale t = aps[it.op];
          const int m = t.m;
          for (int i = tid; i < m; i += nt) sh[i] = ld(z + t.slots[i]);
          __syncthreads();
          gemv_t<1>(t.Zinv, m, it.lo, it.hi, m, [](int c) { return c; }, sh, m, red,
                    [&](int j, int, real_t v) { Y[t.slots[j]] = v; });
          break;
        }
        case SW_BI_A: {  // rows of y = x_s - W_s^T z_w into Y (the diagonal segment skipped)
          const ApInterior t = api[it.op];
          const int m = t.m, nc = t.ncols, dc = it.aux;
          for (int c = tid; c < nc; c += nt) {
            const int ws = t.wslots[c];
            sh[c] = ws >= 0 ? ld(z + ws) : (real_t)0;
          }
          __syncthreads();
          gemv_n<1>(t.WT, m, it.lo, it.hi, [&](int) { return dc; }, sh, nc, red,
                    [&](int r, int, real_t v) { Y[t.slots[r]] = ld(z + t.slots[r]) - v; });
          const int c1 = dc + m;
          gemv_n<1>(t.WT + (size_t)c1 * m, m, it.lo, it.hi, [&](int) { return nc - c1; }, sh + c1,
                    nc, red, [&](int r, int, real_t v) { Y[t.slots[r]] -= v; });
          break;
        }
        case SW_BI_B: {  // z_s = L_s^{-T} y over a range of outputs
          const ApInterior t = api[it.op];
          const int m = t.m;
          for (int i = tid; i < m; i += nt) sh[i] = ld(Y + t.slots[i]);
          __syncthreads();
          gemv_t<1>(t.Linv, m, it.lo, it.hi, m, [](int c) { return c; }, sh, m, red,
                    [&](int j, int, real_t v) { z[t.slots[j]] = v; });
          break;
        }
        default:
          break;
      }
      __syncthreads();  // the shared vectors are refilled by the next item
    }
    if (ph + 1 < nph && !sweep_barrier(ctr, abort, (ph + 1) * (int)gridDim.x, limit)) return;
    if (trace && blockIdx.x == 0 && threadIdx.x == 0) trace[ph + 1] = clock64();
  }
}

}  // namespace

// The dynamic shared memory a launch may use beyond the 48 KB default must be
// granted per kernel; the static part (the partial-sum buffer) counts too, so
// the grant is made for any dynamic size above 16 KB (grant_smem only raises it).

__global__ void k_copy_real(int n, const real_t* __restrict__ s, real_t* __restrict__ d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) d[i] = s[i];
}

void launch_copy_real(int n, const real_t* src, real_t* dst, cudaStream_t s) {
  k_copy_real<<<std::max(1, std::min((n + 255) / 256, 152 * 16)), 256, 0, s>>>(n, src, dst);
}

typedef void (*ApKernel)(const ApItem*, int, real_t*, int);

// Attribute and launch errors are left for cudaGetLastError, which the apply
// checks after its launches.
static void launch_ap(ApKernel kern, const ApItem* items, int nitems, int ntasks, int K, int bytes,
                      real_t* z, bool forward, cudaStream_t s) {
  if (ntasks <= 0) return;
  if (grant_smem((const void*)kern, bytes) != cudaSuccess) return;
  if (K > 8 && allow_wide_clusters((const void*)kern) != cudaSuccess) return;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(ntasks * K));
  cfg.blockDim = dim3(kApThreads);
  cfg.dynamicSmemBytes = (size_t)bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)K;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, items, nitems, z, forward ? 1 : 0);
}

// Vectors per pass for a launch whose items carry up to max_nvec vectors and
// whose shared memory is per_vec bytes per vector: 1, 2 or 4.  Several
// vectors only while the CTA's shared memory stays under 96 KB, so that the
// thread-block clusters of the single-vector launch shape stay schedulable.
// Up to 4 vectors per pass: wider passes (8, 16 in FP32) measured slower, the
// extra registers and shared memory costing more resident warps than the
// fewer operator reads save.
constexpr int kApMaxVectors = 4;

static int ap_vectors(int max_nvec, int per_vec) {
  int nv = 1;
  while (nv * 2 <= std::min(max_nvec, kApMaxVectors)) nv *= 2;
  while (nv > 1 && (size_t)nv * per_vec > (size_t)96 * 1024) nv >>= 1;
  return nv;
}

template <template <int> class Pick>
static ApKernel pick(int nv) {
  if constexpr (kApMaxVectors >= 16) {
    if (nv == 16) return Pick<16>::k;
    if (nv == 8) return Pick<8>::k;
  }
  return nv == 4 ? Pick<4>::k : nv == 2 ? Pick<2>::k : Pick<1>::k;
}
template <int NV> struct PickInterior { static constexpr ApKernel k = k_ap_interior<NV>; };
template <int NV> struct PickScale { static constexpr ApKernel k = k_ap_scale<NV>; };
template <int NV> struct PickQE { static constexpr ApKernel k = k_ap_qe<NV>; };

int sweep_ctas(int smem_bytes) {
  if (grant_smem((const void*)k_ap_sweep, smem_bytes) != cudaSuccess) return 0;
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ap_sweep, kApThreads, smem_bytes) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return sms * per;
}

cudaError_t launch_ap_sweep(const SwPhase* phases, int nph, const SwItem* items,
                            const ApInterior* api, const ApScale* aps, const ApQE* apq, real_t* z,
                            real_t* Y, int* ws, int nctas, int smem_bytes, long long limit,
                            long long* trace, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ws, 0, sizeof(int), s);  // the barrier counter
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nctas);
  cfg.blockDim = dim3(kApThreads);
  cfg.dynamicSmemBytes = (size_t)smem_bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident, or the launch fails
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_ap_sweep, phases, nph, items, api, aps, apq, z, Y, ws, ws + 1,
                            limit, trace);
}

void launch_ap_interior(const ApItem* items, int nitems, int ntasks, int K, int max_m,
                        int max_cols, int max_nvec, real_t* z, bool forward, cudaStream_t s) {
  const int per = std::max(2 * max_m + max_cols, 1) * (int)sizeof(real_t);
  const int nv = ap_vectors(max_nvec, per);
  launch_ap(pick<PickInterior>(nv), items, nitems, ntasks, K, nv * per, z, forward, s);
}

void launch_ap_scale(const ApItem* items, int nitems, int ntasks, int K, int max_m, int max_nvec,
                     real_t* z, bool forward, cudaStream_t s) {
  const int per = std::max(max_m, 1) * (int)sizeof(real_t);
  const int nv = ap_vectors(max_nvec, per);
  launch_ap(pick<PickScale>(nv), items, nitems, ntasks, K, nv * per, z, forward, s);
}

void launch_ap_qe(const ApItem* items, int nitems, int ntasks, int K, int max_m, int max_cols,
                  int max_nvec, real_t* z, bool forward, cudaStream_t s) {
  const int per = std::max(2 * max_m + max_cols, 1) * (int)sizeof(real_t);
  const int nv = ap_vectors(max_nvec, per);
  launch_ap(pick<PickQE>(nv), items, nitems, ntasks, K, nv * per, z, forward, s);
}

}  // namespace SPAND_NS
}  // namespace spand
