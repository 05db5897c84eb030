// Precision-dependent declarations: task descriptors and kernel launchers of
// the factorization and the apply, written against real_t.  This header is
// included by the translation units that are compiled twice, once with
// SPAND_REAL=double / SPAND_NS=f64 and once with SPAND_REAL=float /
// SPAND_NS=f32, so every name lives in namespace spand::SPAND_NS.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "spand.h"

#ifndef SPAND_REAL
#define SPAND_REAL double
#define SPAND_NS f64
#endif

namespace spand {

// ---------------------------------------------------------------------------
// Kernel attributes (spand_pcg.cu).  The dynamic shared memory a kernel may
// use beyond 48 KB is a per-function limit on the current device; graphs
// captured earlier can hold launches of the same kernel with more dynamic
// shared memory than a later launch asks for, so the limit is only ever
// raised, never lowered.  Both return the CUDA error of the attribute call.
// ---------------------------------------------------------------------------
cudaError_t grant_smem(const void* fn, int bytes);
cudaError_t allow_wide_clusters(const void* fn);  // thread-block clusters of more than 8 CTAs

namespace SPAND_NS {

typedef SPAND_REAL real_t;

// ---------------------------------------------------------------------------
// Device task descriptors (plain structs copied to the device in one blob).
// ---------------------------------------------------------------------------

// dst[i + j*dst_ld] = (trans ? src[j + i*src_ld] : src[i + j*src_ld]); i < rows, j < cols.
struct CopyTask {
  const real_t* src;
  real_t* dst;
  int src_ld, dst_ld, rows, cols, trans, pad;
};

// In-place lower Cholesky of an m x m column-major block (ld).  A non-positive
// pivot stores id + 1 in *err (the first failure wins).
struct PotrfTask {
  real_t* a;
  int* err;
  int m, ld, id, pad;
};

// trans == 0: X (m x ncols, ld ldx) <- L^{-1} X.
// trans == 1: B (ncols x m, ld ldx) <- B L^{-T}, i.e. B^T <- L^{-1} B^T.
// ident >= 0: X <- L^{-1} [e_ident .. e_{ident+ncols-1}] (columns of L^{-1}; X's
// previous contents are ignored).
struct TrsmTask {
  const real_t* L;
  real_t* X;
  int m, ldl, ldx, ncols, trans, pad;  // pad: ident (first identity column) or -1
};

// Columns c0 .. c0+ncols-1 of Q^T = H_{nref-1} ... H_0 (m x m, ld m).
struct FormQtTask {
  const real_t* V;
  const real_t* tau;
  real_t* Qt;  // already offset to column c0
  int m, nref, c0, ncols;
};

// One output tile (rows x cols <= 32 x 32) of a Schur target block:
// T -= sum_c A_c^T B_c, written at dst (ld) and, unless mirror == nullptr,
// transposed at mirror (ld_mirror).
struct SchurTile {
  real_t* dst;
  real_t* mirror;
  int ld, ld_mirror, rows, cols, cbegin, cend, i0, j0;
};
// A_c: K x (i0 + rows) at a (lda), B_c: K x (j0 + cols) at b (ldb); the tile
// uses columns i0.. of A_c and j0.. of B_c.  pad = 0: element (k, i) at
// k + i*ld (column-major); pad = 1: at k*ld + i (the transposed storage, e.g.
// a column panel P whose product P P^T is wanted).
struct SchurContrib {
  const real_t* a;
  const real_t* b;
  int K, lda, ldb, pad;
};

// One segment (neighbour block) of an interface's panel row.
struct RRQRSeg {
  real_t* mirror;  // origin of the transposed block in the neighbour's row
  int col;         // first column of the segment in the row
  int cl;          // neighbour cluster id (its live width is cur_size[cl])
  int mirror_ld;   // leading dimension of the neighbour's row
  int pad;
};

struct RRQRTask {
  real_t* A;       // panel row of interface p, column-major, ld
  real_t* diag;    // origin of the diagonal segment (set to I_r afterwards)
  real_t* V;       // reflectors, m x maxref, ld m
  real_t* tau;     // maxref
  int* cur;        // live width of every cluster of the problem (read, and cur[id] = r)
  int* rank;       // outputs, indexed by cluster id: rank r, reflectors taken, near-tie flags
  int* nref;
  int* flag;
  int* err;        // the problem's error words: err[1] = 1 if a multi-CTA QR lost synchronisation
  double eps;      // relative tolerance of the problem (Algorithm 1)
  int scheme;      // SPAND_FIRST_ORDER, SPAND_SECOND_ORDER_FULL or SPAND_SECOND_ORDER_SUPERFINE
  int m, ld, seg_begin, seg_end, id, maxref, ncols_max, nseg_max;
  int wait_extra;        // multi-CTA QR: added to the first barrier's target (testing hook, else 0)
  long long wait_limit;  // multi-CTA QR: polls of a barrier counter before the wait gives up
};

// An interface QR spread over ncta CTAs of one cooperative launch (CTAs
// cta0 .. cta0+ncta-1), for blocks too large for a thread-block cluster's
// shared memory.  ws: the task's workspace of kQrGridWs(ncta) ints, zero at
// launch (barrier counter, abort flag, candidate slots).
struct RRQRGridTask {
  RRQRTask t;
  int* ws;
  real_t* stage;  // on-chip variant: [2][ncta][m] staged candidate columns
  int cta0, ncta;
};
inline size_t qr_grid_ws_ints(int ncta) { return 4 + 2 * (size_t)ncta * 6; }

// Preconditioner apply descriptors.  The triangular factors and Q_p are
// applied through explicit matrices formed at the end of each stage
// (L_s^{-1}, Z_p^{-1}, Q_p^T), so every apply step is a dense product.
struct ApInterior {
  const real_t* Linv;   // m x m lower, L_s^{-1}, ld m
  const real_t* WT;     // panel row, m x ncols (ld = m); diag columns skipped via wslot < 0
  const int* slots;     // m vector positions
  const int* wslots;    // ncols vector positions (-1 for the diagonal segment)
  int m, ncols;
};
struct ApScale {
  const real_t* Zinv;  // m x m lower, Z_p^{-1}, ld m
  const int* slots;
  int m, pad;
};
struct ApQE {
  const real_t* Qt;   // m x m, Q_p^T, ld m
  const real_t* E;    // nE x ncols, row-major: E[i, c] at i * ncols + c
  const int* slots;   // m positions (before sparsification)
  const int* eslots;  // ncols positions
  int m, r, nE, ncols;
};

// A run of `count` operators of one problem (descriptors at ops, of the
// launch's kind) applied to the nvec vectors z + zoff + j * ldz; in a launch
// the items are sorted by `first`, the launch-wide index of their first
// operator.  One launch can so cover the operators of several problems and
// several right-hand sides of each.
struct ApItem {
  const void* ops;
  int64_t zoff, ldz;
  int count, first, nvec, pad;
};

// ---------------------------------------------------------------------------
// Kernel launchers (spand_kernels.cu / spand_apply.cu).
// ---------------------------------------------------------------------------
void launch_copy(const CopyTask* t, int ntasks, cudaStream_t s);
// base_lo[d] = val[e] for 0 <= d < split, base_hi[d - split] for d >= split, skip d < 0.
void launch_scatter(const double* val, const int64_t* dst_index, real_t* base_lo,
                    real_t* base_hi, int64_t split, int64_t nnz, cudaStream_t s);
void launch_potrf(const PotrfTask* t, int ntasks, int max_m, cudaStream_t s);
void launch_trsm(const TrsmTask* t, int ntasks, int max_m, cudaStream_t s);
void launch_schur(const SchurTile* tiles, int ntiles, const SchurContrib* c, cudaStream_t s);
// Tensor-core Schur tiles of up to 128 x 128 (FP32 storage; contributions in the
// K-major storage, pad = 0): available in the FP32 build only; err: set to 1 if
// a bounded wait for the tensor cores ran out.
bool schur_tc_available();
constexpr int kSchurTcTile = 128;
cudaError_t launch_schur_tc(const SchurTile* tiles, int ntiles, const SchurContrib* c, int* err,
                            cudaStream_t s);
void launch_copy_real(int n, const real_t* src, real_t* dst, cudaStream_t s);
void launch_form_qt(const FormQtTask* t, int ntasks, int max_m, cudaStream_t s);
void launch_set_identity(const PotrfTask* t, int ntasks, cudaStream_t s);
int rrqr_smem_bytes(int max_m, int max_cols, int max_segs);
// On-chip variant: C CTAs per interface (a thread-block cluster), the block in shared memory.
int rrqr_cluster_smem_bytes(int m, int ncols_max, int nseg, int csize);
// Clusters of this shape that can be resident at once (0: cannot be launched).
int rrqr_cluster_active(int csize, int smem_bytes, int threads);
// threads: CTA size, 256, 512 or 1024
cudaError_t launch_rrqr_cluster(const RRQRTask* t, int ntasks, const RRQRSeg* segs, int csize,
                                int smem_bytes, int threads, cudaStream_t s);
void launch_rrqr(const RRQRTask* t, int ntasks, const RRQRSeg* segs, int max_m, int max_cols,
                 int max_segs, cudaStream_t s);
// Cooperative multi-CTA QR: nctas CTAs in all (at most one per SM), each task
// its range of them; returns a CUDA error code of the launch.
int rrqr_grid_smem_bytes(int max_m, int max_cpb, int max_segs);
cudaError_t launch_rrqr_grid(const RRQRGridTask* t, int ntasks, int nctas, const RRQRSeg* segs,
                             int smem_bytes, cudaStream_t s);
// The same with every CTA's slice of columns in its shared memory (at most one
// CTA per SM); rrqr_gsm_smem_bytes: the dynamic shared memory of a CTA holding
// cpb columns of m rows.
int rrqr_gsm_smem_bytes(int m, int cpb, int nseg);
cudaError_t launch_rrqr_gsm(const RRQRGridTask* t, int ntasks, int nctas, const RRQRSeg* segs,
                            int smem_bytes, cudaStream_t s);

// The persistent single-vector sweep (k_ap_sweep): sub-phases of items, each
// item one operator (index into the descriptor array of its kind) and a range
// [lo, hi) of its rows or columns; aux: per kind (SW_FI_B, SW_FQ_B, SW_BQ_A: 1
// if the item also copies the operator's vector; SW_BI_A: the first column of
// the diagonal segment of the panel row).
enum SweepKind {
  SW_FI_A = 0, SW_FI_B, SW_FS_A, SW_COPY, SW_FQ_A, SW_FQ_B, SW_BQ_A, SW_BQ_B, SW_BS_A, SW_BI_A,
  SW_BI_B
};
struct SwPhase {
  int kind, item0, nitems, pad;
};
struct SwItem {
  int op, lo, hi, aux;
};
// CTAs of one cooperative sweep launch (all resident) for this shared memory; 0 if none.
int sweep_ctas(int smem_bytes);
// ws: 2 ints (barrier counter, abort flag); the counter is cleared by the launch.
// trace: NULL, or nph clock readings of CTA 0 (debugging: SPAND_DEBUG_SWEEP=1).
cudaError_t launch_ap_sweep(const SwPhase* phases, int nph, const SwItem* items,
                            const ApInterior* api, const ApScale* aps, const ApQE* apq, real_t* z,
                            real_t* Y, int* ws, int nctas, int smem_bytes, long long limit,
                            long long* trace, cudaStream_t s);

// K: CTAs per operator (a thread-block cluster), 1..16; ntasks: operators
// over all nitems items (device array); max_nvec: the most vectors of an item.
void launch_ap_interior(const ApItem* items, int nitems, int ntasks, int K, int max_m,
                        int max_cols, int max_nvec, real_t* z, bool forward, cudaStream_t s);
void launch_ap_scale(const ApItem* items, int nitems, int ntasks, int K, int max_m, int max_nvec,
                     real_t* z, bool forward, cudaStream_t s);
void launch_ap_qe(const ApItem* items, int nitems, int ntasks, int K, int max_m, int max_cols,
                  int max_nvec, real_t* z, bool forward, cudaStream_t s);


}  // namespace SPAND_NS
}  // namespace spand
