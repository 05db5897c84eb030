// Internal declarations of the spaND library: symbolic structures, device
// task descriptors and kernel launchers.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "spand.h"

namespace spand {

// ---------------------------------------------------------------------------
// Symbolic phase (host): geometric nested dissection and per-stage clusters.
// ---------------------------------------------------------------------------

// Nested-dissection tree to depth nlevels-1.  Node i has children 2i+1
// (coordinate below the cut) and 2i+2 (above); internal nodes are i < nint.
struct Tree {
  int n = 0, dim = 0, nlevels = 0;
  std::vector<double> coords;   // n x dim
  std::vector<int> cut_dim;     // per internal node
  std::vector<double> cut_val;  // per internal node
  std::vector<int> node_of;     // vertex -> separator node or leaf
  std::vector<int> level_of;    // vertex -> level (leaves 0, root nlevels-1)
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
// Cluster ids of every vertex at stage k (-1 if eliminated); returns #clusters.
int cluster_map(const Tree& t, int k, std::vector<int>& cl, std::vector<int>* level_of_cluster);
int build_stages(const Tree& t, const int32_t* rowptr, const int32_t* colind, int skip,
                 std::vector<StageSym>& st, std::string& err);

// ---------------------------------------------------------------------------
// Device task descriptors (plain structs copied to the device in one blob).
// ---------------------------------------------------------------------------

// dst[i + j*dst_ld] = (trans ? src[j + i*src_ld] : src[i + j*src_ld]); i < rows, j < cols.
struct CopyTask {
  const double* src;
  double* dst;
  int src_ld, dst_ld, rows, cols, trans, pad;
};

// In-place lower Cholesky of an m x m column-major block (ld), id for errors.
struct PotrfTask {
  double* a;
  int m, ld, id, pad;
};

// trans == 0: X (m x ncols, ld ldx) <- L^{-1} X.
// trans == 1: B (ncols x m, ld ldx) <- B L^{-T}, i.e. B^T <- L^{-1} B^T.
// ident >= 0: X <- L^{-1} [e_ident .. e_{ident+ncols-1}] (columns of L^{-1}; X's
// previous contents are ignored).
struct TrsmTask {
  const double* L;
  double* X;
  int m, ldl, ldx, ncols, trans, pad;  // pad: ident (first identity column) or -1
};

// Columns c0 .. c0+ncols-1 of Q^T = H_{nref-1} ... H_0 (m x m, ld m).
struct FormQtTask {
  const double* V;
  const double* tau;
  double* Qt;  // already offset to column c0
  int m, nref, c0, ncols;
};

// One output tile (rows x cols <= 32 x 32) of a Schur target block:
// T -= sum_c A_c^T B_c, written at dst (ld) and, unless mirror == nullptr,
// transposed at mirror (ld_mirror).
struct SchurTile {
  double* dst;
  double* mirror;
  int ld, ld_mirror, rows, cols, cbegin, cend, i0, j0;
};
// A_c: K x (i0 + rows) at a (lda), B_c: K x (j0 + cols) at b (ldb); the tile
// uses columns i0.. of A_c and j0.. of B_c.  pad = 0: element (k, i) at
// k + i*ld (column-major); pad = 1: at k*ld + i (the transposed storage, e.g.
// a column panel P whose product P P^T is wanted).
struct SchurContrib {
  const double* a;
  const double* b;
  int K, lda, ldb, pad;
};

// One segment (neighbour block) of an interface's panel row.
struct RRQRSeg {
  double* mirror;  // origin of the transposed block in the neighbour's row
  int col;         // first column of the segment in the row
  int cl;          // neighbour cluster id (its live width is cur_size[cl])
  int mirror_ld;   // leading dimension of the neighbour's row
  int pad;
};

struct RRQRTask {
  double* A;       // panel row of interface p, column-major, ld
  double* diag;    // origin of the diagonal segment (set to I_r afterwards)
  double* V;       // reflectors, m x maxref, ld m
  double* tau;     // maxref
  int m, ld, seg_begin, seg_end, id, maxref, ncols_max, nseg_max;
};

// Preconditioner apply descriptors.  The triangular factors and Q_p are
// applied through explicit matrices formed at the end of each stage
// (L_s^{-1}, Z_p^{-1}, Q_p^T), so every apply step is a dense product.
struct ApInterior {
  const double* Linv;   // m x m lower, L_s^{-1}, ld m
  const double* WT;     // panel row, m x ncols (ld = m); diag columns skipped via wslot < 0
  const int* slots;     // m vector positions
  const int* wslots;    // ncols vector positions (-1 for the diagonal segment)
  int m, ncols;
};
struct ApScale {
  const double* Zinv;  // m x m lower, Z_p^{-1}, ld m
  const int* slots;
  int m, pad;
};
struct ApQE {
  const double* Qt;   // m x m, Q_p^T, ld m
  const double* E;    // nE x ncols, ld nE
  const int* slots;   // m positions (before sparsification)
  const int* eslots;  // ncols positions
  int m, r, nE, ncols;
};

// ---------------------------------------------------------------------------
// Kernel launchers (spand_kernels.cu / spand_apply.cu).
// ---------------------------------------------------------------------------
void launch_copy(const CopyTask* t, int ntasks, cudaStream_t s);
// base_lo[d] = val[e] for 0 <= d < split, base_hi[d - split] for d >= split, skip d < 0.
void launch_scatter(const double* val, const int64_t* dst_index, double* base_lo,
                    double* base_hi, int64_t split, int64_t nnz, cudaStream_t s);
void launch_potrf(const PotrfTask* t, int ntasks, int max_m, int* err, cudaStream_t s);
void launch_trsm(const TrsmTask* t, int ntasks, int max_m, cudaStream_t s);
void launch_schur(const SchurTile* tiles, int ntiles, const SchurContrib* c, cudaStream_t s);
void launch_form_qt(const FormQtTask* t, int ntasks, int max_m, cudaStream_t s);
void launch_set_identity(const PotrfTask* t, int ntasks, cudaStream_t s);
int rrqr_smem_bytes(int max_m, int max_cols, int max_segs);
// On-chip variant: C CTAs per interface (a thread-block cluster), the block in shared memory.
int rrqr_cluster_smem_bytes(int m, int ncols_max, int nseg, int csize);
// Clusters of this shape that can be resident at once (0: cannot be launched).
int rrqr_cluster_active(int csize, int smem_bytes);
void launch_rrqr_cluster(const RRQRTask* t, int ntasks, const RRQRSeg* segs, int* cur_size,
                         int* rank_out, int* nref_out, int* flag_out, double eps, int scheme,
                         int csize, int smem_bytes, cudaStream_t s);
void launch_rrqr(const RRQRTask* t, int ntasks, const RRQRSeg* segs, int* cur_size,
                 int* rank_out, int* nref_out, int* flag_out, double eps, int scheme, int max_m,
                 int max_cols, int max_segs, cudaStream_t s);

// K: CTAs per operator (a thread-block cluster), 1..16.
void launch_ap_interior(const ApInterior* t, int ntasks, int K, int max_m, int max_cols, double* z,
                        bool forward, cudaStream_t s);
void launch_ap_scale(const ApScale* t, int ntasks, int K, int max_m, double* z, bool forward,
                     cudaStream_t s);
void launch_ap_qe(const ApQE* t, int ntasks, int K, int max_m, int max_cols, double* z,
                  bool forward, cudaStream_t s);

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

}  // namespace spand
