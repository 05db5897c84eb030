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

constexpr int kApThreads = 256;

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

// y = T x for a lower-triangular T (ld m), thread per row: FMA chains only.
__device__ void lower_mv(const double* T, int m, const double* x, double* y) {
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double s0 = 0.0, s1 = 0.0;
    int j = 0;
    for (; j + 1 <= i; j += 2) {
      s0 = fma(T[i + (size_t)j * m], x[j], s0);
      s1 = fma(T[i + (size_t)(j + 1) * m], x[j + 1], s1);
    }
    if (j <= i) s0 = fma(T[i + (size_t)j * m], x[j], s0);
    y[i] = s0 + s1;
  }
}

// y = T^T x for a lower-triangular T: thread j walks column j of T.
__device__ void lower_tmv(const double* T, int m, const double* x, double* y) {
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const double* col = T + (size_t)j * m;
    double s0 = 0.0, s1 = 0.0;
    int i = j;
    for (; i + 1 < m; i += 2) {
      s0 = fma(col[i], x[i], s0);
      s1 = fma(col[i + 1], x[i + 1], s1);
    }
    if (i < m) s0 = fma(col[i], x[i], s0);
    y[j] = s0 + s1;
  }
}

// s = sum_c M[row + c*ld] * x[c] over c < n, 4 partial sums to keep loads in flight.
__device__ __forceinline__ double row_dot(const double* __restrict__ M, size_t ld, int n,
                                          const double* __restrict__ x) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int c = 0;
  for (; c + 3 < n; c += 4) {
    s0 = fma(M[(size_t)c * ld], x[c], s0);
    s1 = fma(M[(size_t)(c + 1) * ld], x[c + 1], s1);
    s2 = fma(M[(size_t)(c + 2) * ld], x[c + 2], s2);
    s3 = fma(M[(size_t)(c + 3) * ld], x[c + 3], s3);
  }
  for (; c < n; ++c) s0 = fma(M[(size_t)c * ld], x[c], s0);
  return (s0 + s1) + (s2 + s3);
}

// s = sum_i col[i] * x[i] over i < n (a contiguous column).
__device__ __forceinline__ double col_dot(const double* __restrict__ col, int n,
                                          const double* __restrict__ x) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int i = 0;
  for (; i + 3 < n; i += 4) {
    s0 = fma(col[i], x[i], s0);
    s1 = fma(col[i + 1], x[i + 1], s1);
    s2 = fma(col[i + 2], x[i + 2], s2);
    s3 = fma(col[i + 3], x[i + 3], s3);
  }
  for (; i < n; ++i) s0 = fma(col[i], x[i], s0);
  return (s0 + s1) + (s2 + s3);
}

// Shared memory of the apply kernels: x (m), y (m), gathered neighbour values (ncols).
__global__ void k_ap_interior(const ApInterior* __restrict__ tasks, double* __restrict__ z,
                              int forward) {
  extern __shared__ double sh[];
  const ApInterior t = tasks[blockIdx.x];
  const int m = t.m;
  double* xs = sh;
  double* ys = sh + m;
  double* zw = sh + 2 * m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) xs[i] = z[t.slots[i]];
  if (!forward)
    for (int c = threadIdx.x; c < t.ncols; c += blockDim.x) {
      const int ws = t.wslots[c];
      zw[c] = ws >= 0 ? z[ws] : 0.0;  // the diagonal segment contributes nothing
    }
  __syncthreads();
  if (forward) {
    // z_s <- L_s^{-1} z_s, then z_w -= W_s z_s (column c of the panel row holds W_s^T[:, c])
    lower_mv(t.Linv, m, xs, ys);
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) z[t.slots[i]] = ys[i];
    for (int c = threadIdx.x; c < t.ncols; c += blockDim.x) {
      const int ws = t.wslots[c];
      if (ws < 0) continue;
      atomicAdd(z + ws, -col_dot(t.WT + (size_t)c * m, m, ys));
    }
  } else {
    // z_s -= W_s^T z_w, then z_s <- L_s^{-T} z_s
    for (int i = threadIdx.x; i < m; i += blockDim.x) ys[i] = xs[i] - row_dot(t.WT + i, m, t.ncols, zw);
    __syncthreads();
    lower_tmv(t.Linv, m, ys, xs);
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) z[t.slots[i]] = xs[i];
  }
}

__global__ void k_ap_scale(const ApScale* __restrict__ tasks, double* __restrict__ z,
                           int forward) {
  extern __shared__ double sh[];
  const ApScale t = tasks[blockIdx.x];
  const int m = t.m;
  double* xs = sh;
  double* ys = sh + m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) xs[i] = z[t.slots[i]];
  __syncthreads();
  if (forward) lower_mv(t.Zinv, m, xs, ys);
  else lower_tmv(t.Zinv, m, xs, ys);
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) z[t.slots[i]] = ys[i];
}

__global__ void k_ap_qe(const ApQE* __restrict__ tasks, double* __restrict__ z, int forward) {
  extern __shared__ double sh[];
  const ApQE t = tasks[blockIdx.x];
  const int m = t.m;
  double* xs = sh;
  double* ys = sh + m;
  double* zw = sh + 2 * m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) xs[i] = z[t.slots[i]];
  if (!forward && t.nE > 0)
    for (int c = threadIdx.x; c < t.ncols; c += blockDim.x) zw[c] = z[t.eslots[c]];
  __syncthreads();
  if (forward) {
    // z_p <- Q^T z_p (row i of Q^T: Qt[i + j m] over j)
    for (int i = threadIdx.x; i < m; i += blockDim.x) ys[i] = row_dot(t.Qt + i, m, m, xs);
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) z[t.slots[i]] = ys[i];
    // z_w -= E-tilde^T z_f
    if (t.nE > 0)
      for (int c = threadIdx.x; c < t.ncols; c += blockDim.x)
        atomicAdd(z + t.eslots[c], -col_dot(t.E + (size_t)c * t.nE, t.nE, ys + t.r));
  } else {
    // z_f -= E-tilde z_w
    if (t.nE > 0) {
      for (int i = threadIdx.x; i < t.nE; i += blockDim.x)
        xs[t.r + i] -= row_dot(t.E + i, t.nE, t.ncols, zw);
      __syncthreads();
    }
    // z_p <- Q z_p = (Q^T)^T z_p: thread j walks column j of Q^T
    for (int j = threadIdx.x; j < m; j += blockDim.x) ys[j] = col_dot(t.Qt + (size_t)j * m, m, xs);
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) z[t.slots[i]] = ys[i];
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

void launch_ap_interior(const ApInterior* t, int ntasks, int max_m, int max_cols, double* z,
                        bool forward, cudaStream_t s) {
  if (ntasks <= 0) return;
  const int bytes = std::max(2 * max_m + max_cols, 1) * 8;
  smem_attr((const void*)k_ap_interior, bytes);
  k_ap_interior<<<ntasks, kApThreads, bytes, s>>>(t, z, forward ? 1 : 0);
}

void launch_ap_scale(const ApScale* t, int ntasks, int max_m, double* z, bool forward,
                     cudaStream_t s) {
  if (ntasks <= 0) return;
  const int bytes = std::max(max_m, 1) * 16;
  smem_attr((const void*)k_ap_scale, bytes);
  k_ap_scale<<<ntasks, kApThreads, bytes, s>>>(t, z, forward ? 1 : 0);
}

void launch_ap_qe(const ApQE* t, int ntasks, int max_m, int max_cols, double* z, bool forward,
                  cudaStream_t s) {
  if (ntasks <= 0) return;
  const int bytes = std::max(2 * max_m + max_cols, 1) * 8;
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
