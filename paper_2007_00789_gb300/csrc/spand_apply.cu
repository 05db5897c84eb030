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
#include "spand_internal.h"

namespace spand {

namespace {

constexpr int kApThreads = 128;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

// z <- L^{-1} z (lower, column oriented) on a shared-memory vector.
__device__ void trsv_lower(const double* L, int m, size_t ld, double* zs) {
  for (int j = 0; j < m; ++j) {
    if (threadIdx.x == 0) zs[j] /= L[j + j * ld];
    __syncthreads();
    const double zj = zs[j];
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) zs[i] -= L[i + j * ld] * zj;
    __syncthreads();
  }
}

// z <- L^{-T} z.
__device__ void trsv_lower_t(const double* L, int m, size_t ld, double* zs) {
  for (int j = m - 1; j >= 0; --j) {
    if (threadIdx.x == 0) zs[j] /= L[j + j * ld];
    __syncthreads();
    const double zj = zs[j];
    for (int i = threadIdx.x; i < j; i += blockDim.x) zs[i] -= L[j + i * ld] * zj;
    __syncthreads();
  }
}

__global__ void k_ap_interior(const ApInterior* __restrict__ tasks, double* __restrict__ z,
                              int forward) {
  extern __shared__ double zs[];
  const ApInterior t = tasks[blockIdx.x];
  const int m = t.m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < m; i += blockDim.x) zs[i] = z[t.slots[i]];
  __syncthreads();
  if (forward) {
    trsv_lower(t.L, m, t.ldL, zs);
    for (int i = threadIdx.x; i < m; i += blockDim.x) z[t.slots[i]] = zs[i];
    // z_w -= W_s z_s with W_s = (W_s^T)^T stored as the panel row
    for (int c = warp; c < t.ncols; c += nw) {
      const int ws = t.wslots[c];
      if (ws < 0) continue;
      const double* col = t.WT + (size_t)c * m;
      double s = 0.0;
      for (int i = lane; i < m; i += 32) s += col[i] * zs[i];
      s = warp_sum(s);
      if (lane == 0) atomicAdd(z + ws, -s);
    }
  } else {
    // z_s -= W_s^T z_w, then z_s <- L_s^{-T} z_s
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      double s = 0.0;
      for (int c = 0; c < t.ncols; ++c) {
        const int ws = t.wslots[c];
        if (ws >= 0) s += t.WT[i + (size_t)c * m] * z[ws];
      }
      zs[i] -= s;
    }
    __syncthreads();
    trsv_lower_t(t.L, m, t.ldL, zs);
    for (int i = threadIdx.x; i < m; i += blockDim.x) z[t.slots[i]] = zs[i];
  }
}

__global__ void k_ap_scale(const ApScale* __restrict__ tasks, double* __restrict__ z,
                           int forward) {
  extern __shared__ double zs[];
  const ApScale t = tasks[blockIdx.x];
  const int m = t.m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) zs[i] = z[t.slots[i]];
  __syncthreads();
  if (forward) trsv_lower(t.Z, m, m, zs);
  else trsv_lower_t(t.Z, m, m, zs);
  for (int i = threadIdx.x; i < m; i += blockDim.x) z[t.slots[i]] = zs[i];
}

__global__ void k_ap_qe(const ApQE* __restrict__ tasks, double* __restrict__ z, int forward) {
  extern __shared__ double zs[];
  __shared__ double red[32];
  const ApQE t = tasks[blockIdx.x];
  const int m = t.m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < m; i += blockDim.x) zs[i] = z[t.slots[i]];
  __syncthreads();
  if (forward) {
    // z_p <- Q^T z_p = H_{nref-1} ... H_0 z_p
    for (int s = 0; s < t.nref; ++s) {
      const double* v = t.V + (size_t)s * m;
      double d = 0.0;
      for (int i = s + threadIdx.x; i < m; i += blockDim.x) d += v[i] * zs[i];
      d = block_sum(d, red);
      const double f = t.tau[s] * d;
      for (int i = s + threadIdx.x; i < m; i += blockDim.x) zs[i] -= f * v[i];
      __syncthreads();
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) z[t.slots[i]] = zs[i];
    // z_w -= E-tilde^T z_f
    if (t.nE > 0) {
      for (int c = warp; c < t.ncols; c += nw) {
        const double* col = t.E + (size_t)c * t.nE;
        double s = 0.0;
        for (int i = lane; i < t.nE; i += 32) s += col[i] * zs[t.r + i];
        s = warp_sum(s);
        if (lane == 0) atomicAdd(z + t.eslots[c], -s);
      }
    }
  } else {
    // z_f -= E-tilde z_w
    if (t.nE > 0) {
      for (int i = threadIdx.x; i < t.nE; i += blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < t.ncols; ++c) s += t.E[i + (size_t)c * t.nE] * z[t.eslots[c]];
        zs[t.r + i] -= s;
      }
      __syncthreads();
    }
    // z_p <- Q z_p = H_0 ... H_{nref-1} z_p
    for (int s = t.nref - 1; s >= 0; --s) {
      const double* v = t.V + (size_t)s * m;
      double d = 0.0;
      for (int i = s + threadIdx.x; i < m; i += blockDim.x) d += v[i] * zs[i];
      d = block_sum(d, red);
      const double f = t.tau[s] * d;
      for (int i = s + threadIdx.x; i < m; i += blockDim.x) zs[i] -= f * v[i];
      __syncthreads();
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) z[t.slots[i]] = zs[i];
  }
}

// ---------------------------------------------------------------------------
// PCG kernels.
// ---------------------------------------------------------------------------
__global__ void k_spmv(int n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                       const double* __restrict__ val, const double* __restrict__ x,
                       double* __restrict__ y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) s += val[e] * x[colind[e]];
    y[i] = s;
  }
}

constexpr int kDotBlocks = 304;
constexpr int kDotThreads = 256;

__global__ void k_dot_partial(int n, const double* __restrict__ x, const double* __restrict__ y,
                              double* __restrict__ partial) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    s += x[i] * y[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_dot_final(const double* __restrict__ partial, int np, double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += partial[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}

// scal layout: 0 rz, 1 pq, 2 rz_new, 3 rr
__global__ void k_pcg_init(int n, const double* __restrict__ b, double* __restrict__ x,
                           double* __restrict__ r) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    x[i] = 0.0;
    r[i] = b[i];
  }
}

__global__ void k_pcg_step_x(int n, const double* __restrict__ scal, const double* __restrict__ p,
                             const double* __restrict__ q, double* __restrict__ x,
                             double* __restrict__ r) {
  const double alpha = scal[0] / scal[1];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    r[i] -= alpha * q[i];
  }
}

__global__ void k_pcg_step_p(int n, const double* __restrict__ scal, const double* __restrict__ z,
                             double* __restrict__ p) {
  const double beta = scal[2] / scal[0];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

__global__ void k_pcg_scalars(double* scal, int which) {
  if (which == 0) scal[0] = scal[2];  // rz <- rz_new
}

__global__ void k_residual(int n, const double* __restrict__ b, const double* __restrict__ ax,
                           double* __restrict__ r) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    r[i] = b[i] - ax[i];
}

__global__ void k_copy_vec(int n, const double* __restrict__ s, double* __restrict__ d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) d[i] = s[i];
}

inline int vec_blocks(int n) { return std::max(1, std::min((n + 255) / 256, 152 * 16)); }

}  // namespace

static void smem_attr(const void* fn, int bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

void launch_ap_interior(const ApInterior* t, int ntasks, int max_m, double* z, bool forward,
                        cudaStream_t s) {
  if (ntasks <= 0) return;
  const int bytes = std::max(max_m, 1) * 8;
  smem_attr((const void*)k_ap_interior, bytes);
  k_ap_interior<<<ntasks, kApThreads, bytes, s>>>(t, z, forward ? 1 : 0);
}

void launch_ap_scale(const ApScale* t, int ntasks, int max_m, double* z, bool forward,
                     cudaStream_t s) {
  if (ntasks <= 0) return;
  const int bytes = std::max(max_m, 1) * 8;
  smem_attr((const void*)k_ap_scale, bytes);
  k_ap_scale<<<ntasks, kApThreads, bytes, s>>>(t, z, forward ? 1 : 0);
}

void launch_ap_qe(const ApQE* t, int ntasks, int max_m, double* z, bool forward, cudaStream_t s) {
  if (ntasks <= 0) return;
  const int bytes = std::max(max_m, 1) * 8;
  smem_attr((const void*)k_ap_qe, bytes);
  k_ap_qe<<<ntasks, kApThreads, bytes, s>>>(t, z, forward ? 1 : 0);
}

void launch_spmv(int n, const int32_t* rowptr, const int32_t* colind, const double* val,
                 const double* x, double* y, cudaStream_t s) {
  k_spmv<<<vec_blocks(n), 256, 0, s>>>(n, rowptr, colind, val, x, y);
}

int dot_partials(int n) {
  (void)n;
  return kDotBlocks;
}

void launch_dot(int n, const double* x, const double* y, double* partial, double* out,
                cudaStream_t s) {
  k_dot_partial<<<kDotBlocks, kDotThreads, 0, s>>>(n, x, y, partial);
  k_dot_final<<<1, kDotThreads, 0, s>>>(partial, kDotBlocks, out);
}

void launch_pcg_init(int n, const double* b, double* x, double* r, cudaStream_t s) {
  k_pcg_init<<<vec_blocks(n), 256, 0, s>>>(n, b, x, r);
}
void launch_pcg_step_x(int n, const double* scal, const double* p, const double* q, double* x,
                       double* r, cudaStream_t s) {
  k_pcg_step_x<<<vec_blocks(n), 256, 0, s>>>(n, scal, p, q, x, r);
}
void launch_pcg_step_p(int n, const double* scal, const double* z, double* p, cudaStream_t s) {
  k_pcg_step_p<<<vec_blocks(n), 256, 0, s>>>(n, scal, z, p);
}
void launch_pcg_scalars(double* scal, int which, cudaStream_t s) {
  k_pcg_scalars<<<1, 1, 0, s>>>(scal, which);
}
void launch_residual(int n, const double* b, const double* ax, double* r, cudaStream_t s) {
  k_residual<<<vec_blocks(n), 256, 0, s>>>(n, b, ax, r);
}
void launch_copy_vec(int n, const double* src, double* dst, cudaStream_t s) {
  k_copy_vec<<<vec_blocks(n), 256, 0, s>>>(n, src, dst);
}

}  // namespace spand
