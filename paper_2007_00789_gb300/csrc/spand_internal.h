// Internal declarations of the spaND library: symbolic structures, device
// task descriptors and kernel launchers.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <exception>
#include <functional>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "spand.h"

namespace spand {

// ---------------------------------------------------------------------------
// Symbolic phase (host): geometric nested dissection and per-stage clusters.
// ---------------------------------------------------------------------------

// work(w) for w in [0, nth): w = 0 on the calling thread, the others on the
// library's kept host threads; false (nothing run) while the threads serve
// another loop.
bool host_pool_run(int nth, const std::function<void(int)>& work);

// fn(i, w) for i in [0, n) on up to 16 host threads, at least grain items a
// thread (a loop of few cheap items runs on the calling thread alone); w is
// the worker index (for per-worker scratch).  The items must be independent.
template <class F>
inline void parallel_for(int n, F&& fn, int grain = 1) {
  const int hw = std::max(1, (int)std::thread::hardware_concurrency());
  const int nth = std::max(1, std::min((n + grain - 1) / std::max(1, grain), std::min(16, hw)));
  if (nth <= 1) {
    for (int i = 0; i < n; ++i) fn(i, 0);
    return;
  }
  // items are drawn in chunks (about 16 per thread), so that many small items
  // do not serialise on the shared counter
  const int chunk = std::max(1, n / (nth * 16));
  std::atomic<int> next(0);
  // an exception (a failed allocation) stops the loop and is rethrown on the
  // calling thread once every thread has left it
  std::exception_ptr error;
  std::mutex error_m;
  const std::function<void(int)> work = [&](int w) {
    try {
      for (int i0; (i0 = next.fetch_add(chunk)) < n;)
        for (int i = i0; i < std::min(n, i0 + chunk); ++i) fn(i, w);
    } catch (...) {
      std::lock_guard<std::mutex> g(error_m);
      if (!error) error = std::current_exception();
      next.store(n);
    }
  };
  if (!host_pool_run(nth, work)) {
    // the kept threads are busy (a loop inside a loop, or another caller's)
    std::vector<std::thread> th;
    for (int w = 1; w < nth; ++w) th.emplace_back(work, w);
    work(0);
    for (auto& x : th) x.join();
  }
  if (error) std::rethrow_exception(error);
}

// Allocator that leaves trivially constructible elements uninitialised on
// resize, so that a large host array is first touched by the parallel loop
// that fills it rather than by a serial zero fill.
template <class T>
struct uninit_alloc : std::allocator<T> {
  using value_type = T;
  template <class U>
  struct rebind {
    using other = uninit_alloc<U>;
  };
  uninit_alloc() noexcept = default;
  template <class U>
  uninit_alloc(const uninit_alloc<U>&) noexcept {}
  template <class U>
  void construct(U* p) noexcept {
    ::new ((void*)p) U;
  }
  template <class U, class... A>
  void construct(U* p, A&&... a) {
    ::new ((void*)p) U(std::forward<A>(a)...);
  }
};
template <class T>
using host_vec = std::vector<T, uninit_alloc<T>>;

// dst[0..n) = src[0..n), in 1 MiB pieces on the host threads
template <class T>
inline void parallel_copy(T* dst, const T* src, int64_t n) {
  constexpr int64_t kPiece = (int64_t(1) << 20) / sizeof(T);
  parallel_for((int)((n + kPiece - 1) / kPiece), [&](int c, int) {
    const int64_t b = c * kPiece, e = std::min(n, b + kPiece);
    std::memcpy(dst + b, src + b, (size_t)(e - b) * sizeof(T));
  });
}

// Nested-dissection tree to depth nlevels-1.  Node i has children 2i+1
// (coordinate below the cut) and 2i+2 (above); internal nodes are i < nint.
struct Tree {
  int n = 0, dim = 0, nlevels = 0;
  int algebraic = 0;            // 0: geometric bisection of coordinates; 1: of the graph of A
  host_vec<double> coords;      // n x dim (geometric)
  std::vector<int> cut_dim;     // per internal node (geometric)
  std::vector<double> cut_val;  // per internal node (geometric)
  std::vector<int> node_of;     // vertex -> separator node or leaf
  std::vector<int> level_of;    // vertex -> level (leaves 0, root nlevels-1)
  // algebraic: the reach of every vertex (leaves connected to it through
  // vertices of lower level), CSR over vertices, ascending; width = the
  // largest reach (>= 1)
  std::vector<int> reach_ptr, reach;
  int width = 1;
};

// Structure of one stage that does not depend on numerical ranks.
struct StageSym {
  int ncl = 0;                             // clusters alive at the stage start
  std::vector<int> level;                  // per cluster
  std::vector<uint8_t> interior;           // per cluster: 1 if eliminated at this stage
  std::vector<int> interiors, ifaces;      // ascending ids
  std::vector<std::vector<int>> adj0;      // neighbours at the stage start (no self)
  std::vector<std::vector<int>> adj1;      // interfaces: neighbours after the interior
                                           // eliminations, fill included (no self)
  std::vector<int> colour;                 // interfaces: greedy colour, else -1
  int ncolours = 0;
  std::vector<std::vector<int>> by_colour; // interface ids of each colour, ascending
  std::vector<int> parent;                 // interfaces: cluster id at stage k+1
  std::vector<std::vector<int>> children;  // k >= 1: stage k-1 clusters merged into it
  std::vector<std::vector<int>> members0;  // k == 0: vertices of each cluster, ascending
  std::vector<std::vector<int>> rowsegs;   // blocks stored in each cluster's panel row:
                                           // adj0 + self for interiors, adj1 + self otherwise
  // Schur targets (q, r), q >= r, of the interior eliminations with their
  // contributing interiors s (ascending): CSR over targets.
  std::vector<int> schur_q, schur_r, schur_ptr, schur_s;
  bool sparsify = false;
};

int build_tree(const double* coords, int n, int dim, int nlevels, Tree& t, std::string& err);
// Algebraic nested dissection of the (symmetric) CSR pattern.
int build_tree_graph(const int32_t* rowptr, const int32_t* colind, int n, int nlevels, Tree& t,
                     std::string& err);
// Stage-0 cluster of every vertex; returns the number of clusters.
int stage0_cluster_map(const Tree& t, std::vector<int>& cl);

int build_stages(const Tree& t, const int32_t* rowptr, const int32_t* colind, int skip,
                 std::vector<StageSym>& st, std::string& err);

// ---------------------------------------------------------------------------
// FP64 vector kernels of PCG (spand_pcg.cu).
// ---------------------------------------------------------------------------
void launch_spmv(int n, const int32_t* rowptr, const int32_t* colind, const double* val,
                 const double* x, double* y, cudaStream_t s);
// Deterministic dot product: out[0] = sum x_i y_i (two passes, fixed order).
void launch_dot(int n, const double* x, const double* y, double* partial, double* out,
                cudaStream_t s);
int dot_partials(int n);

// PCG vector updates, scalars read from device memory.
void launch_pcg_init(int n, const double* b, double* x, double* r, cudaStream_t s);
void launch_pcg_step_x(int n, const double* scal, const double* p, const double* q, double* x,
                       double* r, cudaStream_t s);
void launch_pcg_step_p(int n, const double* scal, const double* z, double* p, cudaStream_t s);
void launch_pcg_scalars(double* scal, int which, cudaStream_t s);
void launch_residual(int n, const double* b, const double* ax, double* r, cudaStream_t s);
void launch_copy_vec(int n, const double* src, double* dst, cudaStream_t s);
// precision conversions around an FP32 preconditioner apply
void launch_d2f(int n, const double* src, float* dst, cudaStream_t s);
void launch_f2d(int n, const float* src, double* dst, cudaStream_t s);

// ---------------------------------------------------------------------------
// Segmented FP64 vector kernels (spand_pcg.cu): the PCG of many independent
// problems (or right-hand sides) whose vectors are concatenated.  A segment
// is one vector; a chunk is a range of at most kSegChunk entries inside one
// segment, at a fixed offset from the segment start; each kernel runs one CTA
// per chunk of the list it is given.  Per-segment scalars live in
// sc[kSegScal * seg + j]: j = 0 rz, 1 pq, 2 rz_new, 3 rr, 4 bb.
// ---------------------------------------------------------------------------
constexpr int kSegChunk = 4096;
constexpr int kSegScal = 8;
struct VSeg {
  const int32_t* rowptr;  // the segment's matrix (CSR, device)
  const int32_t* colind;
  const double* val;
  const double* scale;    // D^{-1/2} of a prescaled problem (n entries), else null
  int64_t off;            // first entry of the segment in the concatenated vectors
  int n, pad;
};
struct VChunk {
  int64_t begin, end;     // absolute positions, inside one segment
  int seg, mode;          // mode: per-kernel flag (step_p: 1 = restart the direction)
};
struct VSegRef {          // one segment of a list: its chunks in that list
  int seg, chunk0, nchunks, pad;
};
void launch_seg_spmv(const VChunk* ch, int nch, const VSeg* segs, const double* x, double* y,
                     cudaStream_t s);
void launch_seg_dot(const VChunk* ch, int nch, const VSegRef* refs, int nref, const double* x,
                    const double* y, double* partial, double* sc, int slot, cudaStream_t s);
void launch_seg_init(const VChunk* ch, int nch, const double* b, double* x, double* r,
                     cudaStream_t s);
void launch_seg_step_x(const VChunk* ch, int nch, const double* sc, const double* p,
                       const double* q, double* x, double* r, cudaStream_t s);
// p update per chunk mode, then rz <- rz_new for the listed segments
void launch_seg_step_p(const VChunk* ch, int nch, const VSegRef* refs, int nref, double* sc,
                       const double* z, double* p, cudaStream_t s);
void launch_seg_residual(const VChunk* ch, int nch, const double* b, const double* ax, double* r,
                         cudaStream_t s);
// copies around an apply, scaled by the segment's D^{-1/2} where it has one
void launch_seg_copy(const VChunk* ch, int nch, const VSeg* segs, const double* src, double* dst,
                     cudaStream_t s);
void launch_seg_rescale(const VChunk* ch, int nch, const VSeg* segs, double* dst, cudaStream_t s);
void launch_seg_d2f(const VChunk* ch, int nch, const VSeg* segs, const double* src, float* dst,
                    cudaStream_t s);
void launch_seg_f2d(const VChunk* ch, int nch, const VSeg* segs, const float* src, double* dst,
                    cudaStream_t s);
// dst = sc .* src (and with an FP32 side), for the prescaled apply
void launch_scale(int n, const double* sc, const double* src, double* dst, cudaStream_t s);
void launch_d2f_scaled(int n, const double* sc, const double* src, float* dst, cudaStream_t s);
void launch_f2d_scaled(int n, const double* sc, const float* src, double* dst, cudaStream_t s);

}  // namespace spand
