// FP64 vector kernels of PCG (§4): CSR SpMV, deterministic two-pass dot
// products, the CG vector updates with device-resident scalars, and the
// FP64 <-> FP32 conversions around an FP32 preconditioner apply.
#include "spand_internal.h"

namespace spand {

namespace {

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


__global__ void k_d2f(int n, const double* __restrict__ s, float* __restrict__ d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) d[i] = (float)s[i];
}

__global__ void k_f2d(int n, const float* __restrict__ s, double* __restrict__ d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) d[i] = (double)s[i];
}

}  // namespace

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

void launch_d2f(int n, const double* src, float* dst, cudaStream_t s) {
  k_d2f<<<vec_blocks(n), 256, 0, s>>>(n, src, dst);
}
void launch_f2d(int n, const float* src, double* dst, cudaStream_t s) {
  k_f2d<<<vec_blocks(n), 256, 0, s>>>(n, src, dst);
}

}  // namespace spand
