// FP64 vector kernels of PCG (§4): CSR SpMV, deterministic two-pass dot
// products, the CG vector updates with device-resident scalars, and the
// FP64 <-> FP32 conversions around an FP32 preconditioner apply.
#include <map>
#include <mutex>
#include <utility>

#include "spand_internal.h"

namespace spand {

namespace {
std::mutex g_attr_mu;
std::map<std::pair<int, const void*>, int> g_smem_granted;  // (device, kernel) -> bytes
std::map<std::pair<int, const void*>, int> g_wide_clusters;
}  // namespace

cudaError_t grant_smem(const void* fn, int bytes) {
  if (bytes <= 16 * 1024) return cudaSuccess;  // the static part needs no grant below 48 KB in all
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_attr_mu);
  int& have = g_smem_granted[{dev, fn}];
  if (bytes <= have) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) have = bytes;
  return e;
}

cudaError_t allow_wide_clusters(const void* fn) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_attr_mu);
  int& done = g_wide_clusters[{dev, fn}];
  if (done) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess) done = 1;
  return e;
}

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


// dst = sc .* src (the diagonal prescaling of the preconditioner apply)
__global__ void k_scale(int n, const double* __restrict__ sc, const double* __restrict__ s,
                        double* __restrict__ d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) d[i] = sc[i] * s[i];
}

__global__ void k_d2f_scaled(int n, const double* __restrict__ sc, const double* __restrict__ s,
                             float* __restrict__ d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    d[i] = (float)(sc[i] * s[i]);
}

__global__ void k_f2d_scaled(int n, const double* __restrict__ sc, const float* __restrict__ s,
                             double* __restrict__ d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    d[i] = sc[i] * (double)s[i];
}

__global__ void k_d2f(int n, const double* __restrict__ s, float* __restrict__ d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) d[i] = (float)s[i];
}

__global__ void k_f2d(int n, const float* __restrict__ s, double* __restrict__ d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) d[i] = (double)s[i];
}

// ---- segmented kernels: many independent vectors in one concatenated array.
// Each CTA works on one chunk (a range inside one segment); chunk boundaries
// are fixed relative to the segment start and every reduction has a fixed
// order, so a segment's results do not depend on the other segments.
constexpr int kSegThreads = 256;

__global__ void __launch_bounds__(kSegThreads)
    k_seg_spmv(const VChunk* __restrict__ ch, const VSeg* __restrict__ segs,
               const double* __restrict__ x, double* __restrict__ y) {
  const VChunk c = ch[blockIdx.x];
  const VSeg g = segs[c.seg];
  const double* xs = x + g.off;
  for (int64_t i = c.begin + threadIdx.x; i < c.end; i += blockDim.x) {
    const int il = (int)(i - g.off);
    double s = 0.0;
    for (int e = g.rowptr[il]; e < g.rowptr[il + 1]; ++e) s += g.val[e] * xs[g.colind[e]];
    y[i] = s;
  }
}

__global__ void __launch_bounds__(kSegThreads)
    k_seg_dot(const VChunk* __restrict__ ch, const double* __restrict__ x,
              const double* __restrict__ y, double* __restrict__ partial) {
  __shared__ double red[32];
  const VChunk c = ch[blockIdx.x];
  double s = 0.0;
  for (int64_t i = c.begin + threadIdx.x; i < c.end; i += blockDim.x) s += x[i] * y[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// One thread per segment of the list: the sum of its chunks' partials, in order.
__global__ void k_seg_dot_final(const VSegRef* __restrict__ refs, int nref,
                                const double* __restrict__ partial, double* __restrict__ sc,
                                int slot) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nref) return;
  const VSegRef r = refs[j];
  double s = 0.0;
  for (int c = 0; c < r.nchunks; ++c) s += partial[r.chunk0 + c];
  sc[kSegScal * r.seg + slot] = s;
}

__global__ void __launch_bounds__(kSegThreads)
    k_seg_init(const VChunk* __restrict__ ch, const double* __restrict__ b, double* __restrict__ x,
               double* __restrict__ r) {
  const VChunk c = ch[blockIdx.x];
  for (int64_t i = c.begin + threadIdx.x; i < c.end; i += blockDim.x) {
    x[i] = 0.0;
    r[i] = b[i];
  }
}

__global__ void __launch_bounds__(kSegThreads)
    k_seg_step_x(const VChunk* __restrict__ ch, const double* __restrict__ sc,
                 const double* __restrict__ p, const double* __restrict__ q, double* __restrict__ x,
                 double* __restrict__ r) {
  const VChunk c = ch[blockIdx.x];
  const double alpha = sc[kSegScal * c.seg + 0] / sc[kSegScal * c.seg + 1];
  for (int64_t i = c.begin + threadIdx.x; i < c.end; i += blockDim.x) {
    x[i] += alpha * p[i];
    r[i] -= alpha * q[i];
  }
}

// mode (c.mode) 0: p = z + (rz_new / rz) p; 1: p = z (start or restart)
__global__ void __launch_bounds__(kSegThreads)
    k_seg_step_p(const VChunk* __restrict__ ch, const double* __restrict__ sc,
                 const double* __restrict__ z, double* __restrict__ p) {
  const VChunk c = ch[blockIdx.x];
  if (c.mode == 1) {
    for (int64_t i = c.begin + threadIdx.x; i < c.end; i += blockDim.x) p[i] = z[i];
  } else {
    const double beta = sc[kSegScal * c.seg + 2] / sc[kSegScal * c.seg + 0];
    for (int64_t i = c.begin + threadIdx.x; i < c.end; i += blockDim.x) p[i] = z[i] + beta * p[i];
  }
}

__global__ void k_seg_rz(const VSegRef* __restrict__ refs, int nref, double* __restrict__ sc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nref) sc[kSegScal * refs[j].seg + 0] = sc[kSegScal * refs[j].seg + 2];
}

__global__ void __launch_bounds__(kSegThreads)
    k_seg_residual(const VChunk* __restrict__ ch, const double* __restrict__ b,
                   const double* __restrict__ ax, double* __restrict__ r) {
  const VChunk c = ch[blockIdx.x];
  for (int64_t i = c.begin + threadIdx.x; i < c.end; i += blockDim.x) r[i] = b[i] - ax[i];
}

// The copies around a preconditioner apply; a segment whose problem is
// prescaled multiplies by its D^{-1/2} (g.scale) on the way.
__global__ void __launch_bounds__(kSegThreads)
    k_seg_copy(const VChunk* __restrict__ ch, const VSeg* __restrict__ segs,
               const double* __restrict__ s, double* __restrict__ d) {
  const VChunk c = ch[blockIdx.x];
  const double* sc = segs[c.seg].scale;
  const int64_t off = segs[c.seg].off;
  for (int64_t i = c.begin + threadIdx.x; i < c.end; i += blockDim.x)
    d[i] = sc ? sc[i - off] * s[i] : s[i];
}

__global__ void __launch_bounds__(kSegThreads)
    k_seg_rescale(const VChunk* __restrict__ ch, const VSeg* __restrict__ segs, double* __restrict__ d) {
  const VChunk c = ch[blockIdx.x];
  const double* sc = segs[c.seg].scale;
  if (!sc) return;
  const int64_t off = segs[c.seg].off;
  for (int64_t i = c.begin + threadIdx.x; i < c.end; i += blockDim.x) d[i] *= sc[i - off];
}

__global__ void __launch_bounds__(kSegThreads)
    k_seg_d2f(const VChunk* __restrict__ ch, const VSeg* __restrict__ segs,
              const double* __restrict__ s, float* __restrict__ d) {
  const VChunk c = ch[blockIdx.x];
  const double* sc = segs[c.seg].scale;
  const int64_t off = segs[c.seg].off;
  for (int64_t i = c.begin + threadIdx.x; i < c.end; i += blockDim.x)
    d[i] = (float)(sc ? sc[i - off] * s[i] : s[i]);
}

__global__ void __launch_bounds__(kSegThreads)
    k_seg_f2d(const VChunk* __restrict__ ch, const VSeg* __restrict__ segs,
              const float* __restrict__ s, double* __restrict__ d) {
  const VChunk c = ch[blockIdx.x];
  const double* sc = segs[c.seg].scale;
  const int64_t off = segs[c.seg].off;
  for (int64_t i = c.begin + threadIdx.x; i < c.end; i += blockDim.x)
    d[i] = sc ? sc[i - off] * (double)s[i] : (double)s[i];
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

void launch_seg_spmv(const VChunk* ch, int nch, const VSeg* segs, const double* x, double* y,
                     cudaStream_t s) {
  if (nch > 0) k_seg_spmv<<<nch, kSegThreads, 0, s>>>(ch, segs, x, y);
}
void launch_seg_dot(const VChunk* ch, int nch, const VSegRef* refs, int nref, const double* x,
                    const double* y, double* partial, double* sc, int slot, cudaStream_t s) {
  if (nch <= 0 || nref <= 0) return;
  k_seg_dot<<<nch, kSegThreads, 0, s>>>(ch, x, y, partial);
  k_seg_dot_final<<<(nref + 127) / 128, 128, 0, s>>>(refs, nref, partial, sc, slot);
}
void launch_seg_init(const VChunk* ch, int nch, const double* b, double* x, double* r,
                     cudaStream_t s) {
  if (nch > 0) k_seg_init<<<nch, kSegThreads, 0, s>>>(ch, b, x, r);
}
void launch_seg_step_x(const VChunk* ch, int nch, const double* sc, const double* p,
                       const double* q, double* x, double* r, cudaStream_t s) {
  if (nch > 0) k_seg_step_x<<<nch, kSegThreads, 0, s>>>(ch, sc, p, q, x, r);
}
void launch_seg_step_p(const VChunk* ch, int nch, const VSegRef* refs, int nref, double* sc,
                       const double* z, double* p, cudaStream_t s) {
  if (nch <= 0) return;
  k_seg_step_p<<<nch, kSegThreads, 0, s>>>(ch, sc, z, p);
  k_seg_rz<<<(nref + 127) / 128, 128, 0, s>>>(refs, nref, sc);
}
void launch_seg_residual(const VChunk* ch, int nch, const double* b, const double* ax, double* r,
                         cudaStream_t s) {
  if (nch > 0) k_seg_residual<<<nch, kSegThreads, 0, s>>>(ch, b, ax, r);
}
void launch_seg_copy(const VChunk* ch, int nch, const VSeg* segs, const double* src, double* dst,
                     cudaStream_t s) {
  if (nch > 0) k_seg_copy<<<nch, kSegThreads, 0, s>>>(ch, segs, src, dst);
}
void launch_seg_rescale(const VChunk* ch, int nch, const VSeg* segs, double* dst, cudaStream_t s) {
  if (nch > 0) k_seg_rescale<<<nch, kSegThreads, 0, s>>>(ch, segs, dst);
}
void launch_seg_d2f(const VChunk* ch, int nch, const VSeg* segs, const double* src, float* dst,
                    cudaStream_t s) {
  if (nch > 0) k_seg_d2f<<<nch, kSegThreads, 0, s>>>(ch, segs, src, dst);
}
void launch_seg_f2d(const VChunk* ch, int nch, const VSeg* segs, const float* src, double* dst,
                    cudaStream_t s) {
  if (nch > 0) k_seg_f2d<<<nch, kSegThreads, 0, s>>>(ch, segs, src, dst);
}
void launch_scale(int n, const double* sc, const double* src, double* dst, cudaStream_t s) {
  k_scale<<<vec_blocks(n), 256, 0, s>>>(n, sc, src, dst);
}
void launch_d2f_scaled(int n, const double* sc, const double* src, float* dst, cudaStream_t s) {
  k_d2f_scaled<<<vec_blocks(n), 256, 0, s>>>(n, sc, src, dst);
}
void launch_f2d_scaled(int n, const double* sc, const float* src, double* dst, cudaStream_t s) {
  k_f2d_scaled<<<vec_blocks(n), 256, 0, s>>>(n, sc, src, dst);
}

}  // namespace spand
