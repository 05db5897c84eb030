// Preconditioner apply M = L^{-T} L^{-1} and PCG vector kernels (FP64).
//
// L^{-1} is the product, in processing order, of the elimination operators
// G_s, the scalings D_p and the sparsification operators E_p Q_p^T of
// Algorithm 2 (§3).  The forward sweep applies them in that order to the
// n-vector z; the backward sweep applies their transposes in reverse.  Every
// variable has a fixed position ("slot") in z; after Q_p^T the coarse
// coordinates of p occupy its first r slots and the fine ones the rest.
// Each phase below is one launch batched over the operators of one stage (or
// one colour), which touch disjoint slots except for the accumulation into
// neighbour slots, done with atomics.
#include <cooperative_groups.h>

#include "spand_real.h"

namespace spand {
namespace SPAND_NS {

namespace {

constexpr int kApThreads = 256;

namespace cg = cooperative_groups;

// Tiled matrix-vector products used by every apply step.  A CTA works on 32
// outputs at a time (lane = output); its warps split the reduction dimension,
// each keeping 4 partial sums, and warp 0 adds the warps' results from shared
// memory.  The serial chain per thread is reduction length / (4 warps-worth),
// not the full length, which is what bounds the latency of the large
// operators of the upper levels.
constexpr int kApWarps = kApThreads / 32;

// out(r, sum_{c < C(r0)} M[r + c*ld] x[c]) for rows r in [r0, r1); ccap(rt) bounds
// the columns a 32-row tile starting at rt needs (C for a full matrix, rt + 32
// for a lower-triangular one whose strict upper part is zero).
template <class Cap, class Out>
__device__ void gemv_n(const real_t* __restrict__ M, size_t ld, int r0, int r1, Cap ccap,
                       const real_t* __restrict__ x, real_t* red, Out out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int rt = r0; rt < r1; rt += 32) {
    const int r = rt + lane;
    const int C = ccap(rt);
    const int per = (C + kApWarps - 1) / kApWarps;
    const int cb = warp * per, ce = min(C, cb + per);
    real_t s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    if (r < r1) {
      const real_t* Mr = M + r;
      int c = cb;
      for (; c + 3 < ce; c += 4) {
        s0 = fma(Mr[(size_t)c * ld], x[c], s0);
        s1 = fma(Mr[(size_t)(c + 1) * ld], x[c + 1], s1);
        s2 = fma(Mr[(size_t)(c + 2) * ld], x[c + 2], s2);
        s3 = fma(Mr[(size_t)(c + 3) * ld], x[c + 3], s3);
      }
      for (; c < ce; ++c) s0 = fma(Mr[(size_t)c * ld], x[c], s0);
    }
    red[warp * 32 + lane] = (s0 + s1) + (s2 + s3);
    __syncthreads();
    if (warp == 0 && r < r1) {
      real_t t = 0.0;
      for (int w = 0; w < kApWarps; ++w) t += red[w * 32 + lane];
      out(r, t);
    }
    __syncthreads();
  }
}

// out(c, sum_{r in [rlo(ct), R)} M[r + c*ld] x[r]) for columns c in [c0, c1);
// rlo(ct) is the first row a 32-column tile starting at ct needs (0 for a full
// matrix, ct for the transpose of a lower-triangular one).
template <class Lo, class Out>
__device__ void gemv_t(const real_t* __restrict__ M, size_t ld, int c0, int c1, int R, Lo rlo,
                       const real_t* __restrict__ x, real_t* red, Out out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int ct = c0; ct < c1; ct += 32) {
    const int c = ct + lane;
    const int rb0 = rlo(ct);
    const int per = (R - rb0 + kApWarps - 1) / kApWarps;
    const int rb = rb0 + warp * per, re = min(R, rb + per);
    real_t s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    if (c < c1) {
      const real_t* col = M + (size_t)c * ld;
      int r = rb;
      for (; r + 3 < re; r += 4) {
        s0 = fma(col[r], x[r], s0);
        s1 = fma(col[r + 1], x[r + 1], s1);
        s2 = fma(col[r + 2], x[r + 2], s2);
        s3 = fma(col[r + 3], x[r + 3], s3);
      }
      for (; r < re; ++r) s0 = fma(col[r], x[r], s0);
    }
    red[warp * 32 + lane] = (s0 + s1) + (s2 + s3);
    __syncthreads();
    if (warp == 0 && c < c1) {
      real_t t = 0.0;
      for (int w = 0; w < kApWarps; ++w) t += red[w * 32 + lane];
      out(c, t);
    }
    __syncthreads();
  }
}

namespace cg = cooperative_groups;

// Every operator is applied by a thread-block cluster of K CTAs (K from the
// launch; 1 for small operators); CTA k produces the contiguous slice
// [n k / K, n (k+1) / K) of each output.  When a later step needs a whole
// intermediate vector, each CTA stores its slice into every CTA's shared
// memory and the cluster synchronises.  Shared memory: x (m), y (m),
// gathered neighbour values (ncols), and the warps' partial sums.
__device__ __forceinline__ int part_lo(int n, int k, int K) { return (int)(((long)n * k) / K); }

__device__ __forceinline__ void share(cg::cluster_group& cl, int K, real_t* buf, int i, real_t val) {
  for (int c = 0; c < K; ++c) cl.map_shared_rank(buf, c)[i] = val;
}

// The operator of global task index `task`: the item whose range holds it
// (items are sorted by `first`), and the vector of that item's problem.
__device__ __forceinline__ const void* item_op(const ApItem* __restrict__ items, int nitems,
                                               int task, size_t op_bytes, int64_t* zoff) {
  int lo = 0, hi = nitems - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].first <= task) lo = mid;
    else hi = mid - 1;
  }
  const ApItem it = items[lo];
  *zoff = it.zoff;
  return (const char*)it.ops + (size_t)(task - it.first) * op_bytes;
}

__global__ void __launch_bounds__(kApThreads)
    k_ap_interior(const ApItem* __restrict__ items, int nitems, real_t* __restrict__ z, int forward) {
  cg::cluster_group cl = cg::this_cluster();
  const int K = (int)cl.num_blocks(), k = (int)cl.block_rank();
  extern __shared__ real_t sh[];
  __shared__ real_t red[kApThreads];
  int64_t zoff;
  const ApInterior t = *(const ApInterior*)item_op(items, nitems, (int)(blockIdx.x / K), sizeof(ApInterior), &zoff);
  z += zoff;
  const int m = t.m, nc = t.ncols;
  real_t* xs = sh;
  real_t* ys = sh + m;
  real_t* zw = sh + 2 * m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) xs[i] = z[t.slots[i]];
  if (!forward)
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      const int ws = t.wslots[c];
      zw[c] = ws >= 0 ? z[ws] : 0.0;  // the diagonal segment contributes nothing
    }
  __syncthreads();
  const int lo = part_lo(m, k, K), hi = part_lo(m, k + 1, K);
  if (forward) {
    // y = L_s^{-1} x, then z_s = y and z_w -= W_s y (column c of the panel row is W_s^T[:, c])
    gemv_n(t.Linv, m, lo, hi, [&](int rt) { return min(m, rt + 32); }, xs, red,
           [&](int r, real_t v) { share(cl, K, ys, r, v); });
    cl.sync();
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) z[t.slots[i]] = ys[i];
    gemv_t(t.WT, m, part_lo(nc, k, K), part_lo(nc, k + 1, K), m, [](int) { return 0; }, ys, red,
           [&](int c, real_t v) {
             const int ws = t.wslots[c];
             if (ws >= 0) atomicAdd(z + ws, -v);
           });
  } else {
    // y = x - W_s^T z_w, then z_s = L_s^{-T} y
    gemv_n(t.WT, m, lo, hi, [&](int) { return nc; }, zw, red,
           [&](int r, real_t v) { share(cl, K, ys, r, xs[r] - v); });
    cl.sync();
    gemv_t(t.Linv, m, lo, hi, m, [](int ct) { return ct; }, ys, red,
           [&](int j, real_t v) { z[t.slots[j]] = v; });
  }
}

__global__ void __launch_bounds__(kApThreads)
    k_ap_scale(const ApItem* __restrict__ items, int nitems, real_t* __restrict__ z, int forward) {
  cg::cluster_group cl = cg::this_cluster();
  const int K = (int)cl.num_blocks(), k = (int)cl.block_rank();
  extern __shared__ real_t sh[];
  __shared__ real_t red[kApThreads];
  int64_t zoff;
  const ApScale t = *(const ApScale*)item_op(items, nitems, (int)(blockIdx.x / K), sizeof(ApScale), &zoff);
  z += zoff;
  const int m = t.m;
  real_t* xs = sh;
  for (int i = threadIdx.x; i < m; i += blockDim.x) xs[i] = z[t.slots[i]];
  cl.sync();  // every CTA has read z_p before any CTA overwrites part of it
  const int lo = part_lo(m, k, K), hi = part_lo(m, k + 1, K);
  if (forward)
    gemv_n(t.Zinv, m, lo, hi, [&](int rt) { return min(m, rt + 32); }, xs, red,
           [&](int r, real_t v) { z[t.slots[r]] = v; });
  else
    gemv_t(t.Zinv, m, lo, hi, m, [](int ct) { return ct; }, xs, red,
           [&](int j, real_t v) { z[t.slots[j]] = v; });
}

__global__ void __launch_bounds__(kApThreads)
    k_ap_qe(const ApItem* __restrict__ items, int nitems, real_t* __restrict__ z, int forward) {
  cg::cluster_group cl = cg::this_cluster();
  const int K = (int)cl.num_blocks(), k = (int)cl.block_rank();
  extern __shared__ real_t sh[];
  __shared__ real_t red[kApThreads];
  int64_t zoff;
  const ApQE t = *(const ApQE*)item_op(items, nitems, (int)(blockIdx.x / K), sizeof(ApQE), &zoff);
  z += zoff;
  const int m = t.m, nc = t.ncols, nE = t.nE;
  real_t* xs = sh;
  real_t* ys = sh + m;
  real_t* zw = sh + 2 * m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) xs[i] = z[t.slots[i]];
  if (!forward && nE > 0)
    for (int c = threadIdx.x; c < nc; c += blockDim.x) zw[c] = z[t.eslots[c]];
  __syncthreads();
  const int lo = part_lo(m, k, K), hi = part_lo(m, k + 1, K);
  if (forward) {
    // y = Q^T x; z_p = y; z_w -= E-tilde^T y_f
    gemv_n(t.Qt, m, lo, hi, [&](int) { return m; }, xs, red,
           [&](int r, real_t v) { share(cl, K, ys, r, v); });
    cl.sync();
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) z[t.slots[i]] = ys[i];
    if (nE > 0)
      gemv_t(t.E, nE, part_lo(nc, k, K), part_lo(nc, k + 1, K), nE, [](int) { return 0; },
             ys + t.r, red, [&](int c, real_t v) { atomicAdd(z + t.eslots[c], -v); });
  } else {
    // x_f -= E-tilde z_w, then z_p = Q x
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x)
      if (i < t.r || i >= t.r + nE) share(cl, K, ys, i, xs[i]);
    if (nE > 0) {
      const int flo = max(lo, t.r) - t.r, fhi = min(hi, t.r + nE) - t.r;
      if (fhi > flo)
        gemv_n(t.E, nE, flo, fhi, [&](int) { return nc; }, zw, red,
               [&](int r, real_t v) { share(cl, K, ys, t.r + r, xs[t.r + r] - v); });
    }
    cl.sync();
    gemv_t(t.Qt, m, lo, hi, m, [](int) { return 0; }, ys, red,
           [&](int j, real_t v) { z[t.slots[j]] = v; });
  }
}

}  // namespace


static void smem_attr(const void* fn, int bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

__global__ void k_copy_real(int n, const real_t* __restrict__ s, real_t* __restrict__ d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) d[i] = s[i];
}

void launch_copy_real(int n, const real_t* src, real_t* dst, cudaStream_t s) {
  k_copy_real<<<std::max(1, std::min((n + 255) / 256, 152 * 16)), 256, 0, s>>>(n, src, dst);
}

static void launch_ap(void (*kern)(const ApItem*, int, real_t*, int), const ApItem* items,
                      int nitems, int ntasks, int K, int bytes, real_t* z, bool forward,
                      cudaStream_t s) {
  if (ntasks <= 0) return;
  smem_attr((const void*)kern, bytes);
  if (K > 8) cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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

void launch_ap_interior(const ApItem* items, int nitems, int ntasks, int K, int max_m,
                        int max_cols, real_t* z, bool forward, cudaStream_t s) {
  launch_ap(k_ap_interior, items, nitems, ntasks, K,
            std::max(2 * max_m + max_cols, 1) * (int)sizeof(real_t), z, forward, s);
}

void launch_ap_scale(const ApItem* items, int nitems, int ntasks, int K, int max_m, real_t* z,
                     bool forward, cudaStream_t s) {
  launch_ap(k_ap_scale, items, nitems, ntasks, K, std::max(max_m, 1) * (int)sizeof(real_t), z,
            forward, s);
}

void launch_ap_qe(const ApItem* items, int nitems, int ntasks, int K, int max_m, int max_cols,
                  real_t* z, bool forward, cudaStream_t s) {
  launch_ap(k_ap_qe, items, nitems, ntasks, K,
            std::max(2 * max_m + max_cols, 1) * (int)sizeof(real_t), z, forward, s);
}

}  // namespace SPAND_NS
}  // namespace spand
