// Orchestration of the spaND factorization (Algorithm 2, §3) and of the
// preconditioner apply, written against real_t and compiled once per
// precision (namespace spand::f64 and spand::f32).
//
// Stage k = 0 .. ell-1 of the multilevel partition runs as batched kernels on
// one stream:
//   pack (k = 0) or merge (k > 0) the live blocks into panel rows;
//   eliminate the interiors: POTRF of A_ss, TRSM W_s^T = L_s^{-1} A_sw,
//     Schur tiles A_qr -= W_q W_r^T (each target written once, mirrored);
//   if skip <= k < ell-1: scale the interfaces (POTRF A_pp = Z_p Z_p^T, left
//     and right triangular solves on every off-diagonal block, A_pp = I), then
//     for each colour of the interface graph one batched RRQR launch
//     (Algorithm 1) that also writes the coarse rows into the neighbours;
//   read the ranks back (the one host sync of the stage) and lay out stage k+1.
// Interior panel rows are allocated in the persistent factor arena (they
// become L_s and W_s^T in place); interface rows live in two ping-pong scratch
// buffers.  Each stage's task tables are built on the host and uploaded in
// one copy.
#include <atomic>

#include "spand_handle.h"
#include "spand_real.h"

namespace spand {
namespace SPAND_NS {

int plan_multi(const ApSeg* segs, int nseg, MultiApply& M, cudaStream_t s);

namespace {

struct ApInteriorP {
  const real_t* Linv;
  const real_t* WT;
  int64_t slots, wslots;
  int m, ncols;
  int dc;  // first column of the diagonal segment in the panel row
};
struct ApScaleP {
  const real_t* Zinv;
  int64_t slots;
  int m;
};
struct ApQEP {
  const real_t* Qt;
  const real_t* E;
  int64_t slots, eslots;
  int m, r, nE, ncols;
};


// SPAND_DEBUG_PLAN=1 in the environment prints every interface's RRQR shape and
// kernel choice to stderr while a stage is laid out (for tuning; off by default).
bool debug_plan() {
  static const bool on = [] {
    const char* e = getenv("SPAND_DEBUG_PLAN");
    return e && e[0] == '1';
  }();
  return on;
}

// SPAND_DEBUG_SWEEP=1: every persistent apply sweep records CTA 0's clock per
// sub-phase and prints, per sub-phase, its kind, items and cycles (stderr).
bool debug_sweep() {
  static const bool on = [] {
    const char* e = getenv("SPAND_DEBUG_SWEEP");
    return e && e[0] == '1';
  }();
  return on;
}

// SPAND_DEBUG_TIME=1: a full factorization prints, per stage, the host time of
// its planning, of its upload, capture and launch, of the wait for its ranks
// and of the bookkeeping after them (stderr, milliseconds).
bool debug_time() {
  static const bool on = [] {
    const char* e = getenv("SPAND_DEBUG_TIME");
    return e && e[0] == '1';
  }();
  return on;
}

// Appends pool[off, off + len) to the pool (a range that lies before its end;
// the copy indexes the pool after it has grown, so a reallocation is harmless).
inline void pool_append(std::vector<int>& pool, int64_t off, int len) {
  const size_t old = pool.size();
  pool.resize(old + (size_t)len);
  std::copy(pool.begin() + off, pool.begin() + off + len, pool.begin() + old);
}

inline int segcol_of(const std::vector<int>& segs, const std::vector<int>& cols, int d) {
  auto it = std::lower_bound(segs.begin(), segs.end(), d);
  return cols[it - segs.begin()];
}

// Split a copy into column chunks so that large blocks use several CTAs.
void push_copy(std::vector<CopyTask>& v, const real_t* src, real_t* dst, int src_ld, int dst_ld,
               int rows, int cols, int trans) {
  if (rows <= 0 || cols <= 0) return;
  const int chunk = std::max(1, 8192 / std::max(rows, 1));
  for (int j0 = 0; j0 < cols; j0 += chunk) {
    const int w = std::min(chunk, cols - j0);
    CopyTask t;
    t.dst = dst + (size_t)j0 * dst_ld;
    t.src = trans ? src + j0 : src + (size_t)j0 * src_ld;
    t.src_ld = src_ld;
    t.dst_ld = dst_ld;
    t.rows = rows;
    t.cols = w;
    t.trans = trans;
    t.pad = 0;
    v.push_back(t);
  }
}

// ident: X <- L^{-1} I (explicit inverse of the lower-triangular L, m x m).
void push_trsm(std::vector<TrsmTask>& v, const real_t* L, int ldl, real_t* X, int m, int ldx,
               int ncols, int trans, bool ident = false) {
  if (m <= 0 || ncols <= 0) return;
  for (int c0 = 0; c0 < ncols; c0 += 32) {
    TrsmTask t;
    t.L = L;
    t.ldl = ldl;
    t.m = m;
    t.ldx = ldx;
    t.ncols = std::min(32, ncols - c0);
    t.trans = trans;
    t.pad = ident ? c0 : -1;
    t.X = trans ? X + c0 : X + (size_t)c0 * ldx;
    v.push_back(t);
  }
}

double copy_bytes(const std::vector<CopyTask>& v) {
  double b = 0.0;
  for (auto& t : v) b += 16.0 * t.rows * t.cols;
  return b;
}
double potrf_bytes(const std::vector<PotrfTask>& v) {
  double b = 0.0;
  for (auto& t : v) b += 16.0 * t.m * t.m;
  return b;
}
double trsm_flops(const std::vector<TrsmTask>& v) {
  double f = 0.0;
  for (auto& t : v) f += (double)t.m * t.m * t.ncols;
  return f;
}
double trtri_flops(const std::vector<TrsmTask>& v) {
  double f = 0.0;  // columns c0.. of L^{-1}: sum over columns of (m - c)^2 / 2 FMAs
  for (auto& t : v)
    for (int c = t.pad; c < t.pad + t.ncols; ++c) f += (double)(t.m - c) * (t.m - c);
  return f;
}
double formqt_flops(const std::vector<FormQtTask>& v) {
  double f = 0.0;
  for (auto& t : v)
    for (int s = 0; s < t.nref; ++s) f += 4.0 * (t.m - s) * t.ncols;
  return f;
}
double trsm_bytes(const std::vector<TrsmTask>& v) {
  double b = 0.0;
  for (auto& t : v) b += 16.0 * t.m * t.ncols;
  return b;
}
// Algorithmic Schur work: 2 K rows cols per off-diagonal tile, K rows (rows+1)
// for a tile on the diagonal of a diagonal block (only its lower half is needed).
void schur_work(const std::vector<SchurTile>& tiles, const std::vector<SchurContrib>& c,
                double* flops, double* bytes, bool full_tiles = false) {
  double f = 0.0, b = 0.0;
  for (auto& t : tiles) {
    const bool diag = (t.mirror == nullptr) && !full_tiles;
    for (int i = t.cbegin; i < t.cend; ++i) {
      const double K = c[i].K;
      f += diag ? K * t.rows * (t.rows + 1) : 2.0 * K * t.rows * t.cols;
      b += 8.0 * K * (t.rows + t.cols);
    }
    b += 16.0 * t.rows * t.cols;
  }
  *flops = f;
  *bytes = b;
}

// Batched Cholesky of variable-size blocks.  Blocks of up to kPotrfSmall rows
// are factored by one CTA each in shared memory; larger ones by a tiled
// right-looking algorithm, all of them advancing one kPanel-column panel per
// step: Cholesky of the diagonal tile, triangular solve of the panel below it,
// and the update of the trailing lower triangle with Schur tiles.
constexpr int kPotrfSmall = 128;
constexpr int kPanel = 64;

struct PotrfPlan {
  std::vector<PotrfTask> small;
  int small_max = 0;
  struct Step {
    std::vector<PotrfTask> diag;
    std::vector<TrsmTask> trsm;
    std::vector<SchurTile> tiles;
    std::vector<SchurContrib> contribs;
    size_t o_diag = 0, o_trsm = 0, o_tiles = 0, o_contribs = 0;
  };
  std::vector<Step> steps;
  double flops = 0.0, bytes = 0.0;
  size_t o_small = 0;
};

PotrfPlan plan_potrf(const std::vector<PotrfTask>& tasks) {
  PotrfPlan P;
  int nsteps = 0;
  for (const auto& t : tasks) {
    P.flops += (double)t.m * t.m * t.m / 3.0;
    P.bytes += 16.0 * t.m * t.m;
    if (t.m <= kPotrfSmall) {
      P.small.push_back(t);
      P.small_max = std::max(P.small_max, t.m);
    } else {
      nsteps = std::max(nsteps, (t.m + kPanel - 1) / kPanel);
    }
  }
  P.steps.resize(nsteps);
  for (const auto& t : tasks) {
    if (t.m <= kPotrfSmall) continue;
    for (int k = 0; k * kPanel < t.m; ++k) {
      auto& st = P.steps[k];
      const int k0 = k * kPanel, b = std::min(kPanel, t.m - k0), below = t.m - k0 - b;
      real_t* dg = t.a + k0 + (size_t)k0 * t.ld;
      st.diag.push_back({dg, t.err, b, t.ld, t.id, 0});
      if (below <= 0) continue;
      real_t* panel = dg + b;
      push_trsm(st.trsm, dg, t.ld, panel, b, t.ld, below, 1);
      const int cb = (int)st.contribs.size();
      SchurContrib c;
      c.a = panel;
      c.b = panel;
      c.K = b;
      c.lda = t.ld;
      c.ldb = t.ld;
      c.pad = 1;
      st.contribs.push_back(c);
      real_t* trail = panel + (size_t)b * t.ld;
      for (int i0 = 0; i0 < below; i0 += 32)
        for (int j0 = 0; j0 <= i0; j0 += 32) {
          SchurTile tl;
          tl.dst = trail + i0 + (size_t)j0 * t.ld;
          tl.mirror = nullptr;
          tl.ld = t.ld;
          tl.ld_mirror = 0;
          tl.rows = std::min(32, below - i0);
          tl.cols = std::min(32, below - j0);
          tl.cbegin = cb;
          tl.cend = cb + 1;
          tl.i0 = i0;
          tl.j0 = j0;
          st.tiles.push_back(tl);
        }
    }
  }
  return P;
}

void plan_to_blob(PotrfPlan& P, Blob& blob) {
  P.o_small = blob.add(P.small);
  for (auto& st : P.steps) {
    st.o_diag = blob.add(st.diag);
    st.o_trsm = blob.add(st.trsm);
    st.o_tiles = blob.add(st.tiles);
    st.o_contribs = blob.add(st.contribs);
  }
}

struct StageLayout {
  std::vector<int> m;                      // size at stage start
  std::vector<real_t*> row;                // panel row origin
  std::vector<int> ncols;
  std::vector<std::vector<int>> segcol;    // column offset of every block in the row
  std::vector<int64_t> slot_off;           // offset of the cluster's slots in the pool
  std::vector<real_t*> Z, V, tau;
  std::vector<int> maxref, ncols_ub;       // interfaces: reflector capacity, sum of widths
  std::vector<uint8_t> qr_grid;            // interfaces: 1 if the multi-CTA RRQR factors it
};

// Whether a cluster of cs CTAs with the largest shared-memory slice can be resident.
bool cluster_ok(spand_s* h, int cs) {
  if (h->rrqr_path == 1 || h->rrqr_path == 3 || h->rrqr_path == 4 || (h->rrqr_path == 2 && cs > 8))
    return false;
  int lc = 0;
  while ((1 << lc) < cs) ++lc;
  int& st = h->cluster_state[sizeof(real_t) == 4 ? 1 : 0][lc];
  if (st < 0) st = rrqr_cluster_active(cs, kQrClusterSmem, 256) > 0 ? 1 : 0;
  return st == 1;
}

// The multi-CTA RRQR keeps the block on chip when some number of CTAs, at
// most one per SM, holds it in shared memory: the fewest CTAs that do (0 if
// none).  kQrOnChip marks such tasks (a flag bit beside the testing hook in
// wait_extra, cleared before the launch).
constexpr int kGsmSmem = 220 * 1024;
constexpr int kQrOnChip = 1 << 20;
int gsm_need(int m, int ncols, int nseg) {
  if (m <= 0 || ncols <= 0) return 1;
  for (int nc = std::max(1, (int)(((int64_t)m * ncols * (int64_t)sizeof(real_t)) / kGsmSmem));
       nc <= kNumSMs; ++nc)
    if (rrqr_gsm_smem_bytes(m, (ncols + nc - 1) / nc, nseg) <= kGsmSmem) return nc;
  return 0;
}

// Per-problem state of a factorization in progress.
struct Run {
  spand_s* h = nullptr;
  int ell = 0;
  std::vector<StageLayout> L;
  std::vector<int> pool;  // slot pool (vector positions), uploaded at the end
  std::vector<ApInteriorP> api;
  std::vector<ApScaleP> aps;
  std::vector<ApQEP> apq;
  std::vector<Phase> phases;
  int64_t nnzf = 0;
  // work of the previous stage that runs with the next stage's launches:
  // E-tilde compaction and the explicit apply operators L^{-1}, Z^{-1}, Q^T
  std::vector<CopyTask> pending_e;
  std::vector<TrsmTask> pending_inv;
  std::vector<FormQtTask> pending_qt;
  int pending_inv_m = 0, pending_qt_m = 0;
  // scratch generations seen by each captured stage; a later reallocation of a
  // buffer that an earlier graph uses leaves that graph pointing at freed memory
  std::vector<std::pair<int, int>> used_gen;
  size_t ioff = 0;  // offset of the problem's counters in the running stage's table
};

// Counters of one problem in a stage: widths, ranks, reflector counts and
// near-tie flags of its ncl clusters, then the error word of its Cholesky
// factorizations (and one spare word).
inline size_t counters_of(int ncl) { return 4 * (size_t)ncl + 2; }

// The task tables of one stage of a group of problems, concatenated.  Every
// task carries its own pointers, so the tasks of different problems share
// each launch.
struct StageWork {
  std::vector<CopyTask> pend_e;
  std::vector<TrsmTask> pend_inv;
  std::vector<FormQtTask> pend_qt;
  int pend_inv_m = 0, pend_qt_m = 0;
  std::vector<std::pair<void*, size_t>> zero;  // cleared before the pack or the merge
  struct Pack {
    const double* val;
    const int64_t* idx;
    real_t *lo, *hi;
    int64_t split, nnz;
  };
  std::vector<Pack> packs;
  std::vector<CopyTask> merge;
  std::vector<PotrfTask> potrf_int;
  std::vector<TrsmTask> trsm_int;
  int max_m_int = 0;
  std::vector<SchurTile> tiles;
  std::vector<SchurTile> tiles_tc;  // 128 x 128 tiles for the tensor cores (FP32)
  int* tc_err = nullptr;            // error word the tensor-core tiles report a timeout in
  std::vector<SchurContrib> contribs;
  std::vector<CopyTask> zcopy, mirror;
  std::vector<PotrfTask> zpotrf, ident;
  std::vector<TrsmTask> ltrsm, rtrsm;
  int max_m_if = 0;
  struct QrGroup {
    std::vector<RRQRTask> tasks;
    int max_m = 0, max_cols = 0, max_segs = 0, smem = 0;
    int bucket = 0, threads = 256, base = 0;
  };
  // (colour, bucket * 4096 + CTA size) -> tasks; bucket b >= 1: thread-block
  // clusters of 2^(b-1) CTAs, bucket 0: the global-memory kernel
  std::map<std::pair<int, int>, QrGroup> qr;
  std::vector<RRQRSeg> qr_segs;
  std::vector<int> ints;  // pristine counters of every problem of the stage
};

void take_pending(Run& R, StageWork& W) {
  W.pend_e.insert(W.pend_e.end(), R.pending_e.begin(), R.pending_e.end());
  W.pend_inv.insert(W.pend_inv.end(), R.pending_inv.begin(), R.pending_inv.end());
  W.pend_qt.insert(W.pend_qt.end(), R.pending_qt.begin(), R.pending_qt.end());
  W.pend_inv_m = std::max(W.pend_inv_m, R.pending_inv_m);
  W.pend_qt_m = std::max(W.pend_qt_m, R.pending_qt_m);
  R.pending_e.clear();
  R.pending_inv.clear();
  R.pending_qt.clear();
  R.pending_inv_m = R.pending_qt_m = 0;
}

// Lays out stage k of one problem and appends its tasks to W.  d_cnt: the
// problem's counters on the device (counters_of(ncl) ints).
int build_stage(Run& R, int k, StageWork& W, int* d_cnt) {
  spand_s* h = R.h;
  const StageSym& S = h->st[k];
  StageLayout& Ly = R.L[k];
  std::vector<int>& pool = R.pool;
  const int ncl = S.ncl;
  take_pending(R, W);
  // ---- sizes and slots at the stage start
  Ly.m.assign(ncl, 0);
  Ly.slot_off.assign(ncl, 0);
  if (k == 0) {
    for (int c = 0; c < ncl; ++c) {
      Ly.m[c] = (int)S.members0[c].size();
      Ly.slot_off[c] = (int64_t)pool.size();
      pool.insert(pool.end(), S.members0[c].begin(), S.members0[c].end());
    }
  } else {
    const StageSym& P = h->st[k - 1];
    const StageLayout& Lp = R.L[k - 1];
    for (int c = 0; c < ncl; ++c) {
      Ly.slot_off[c] = (int64_t)pool.size();
      int m = 0;
      for (int p : S.children[c]) {
        const int live = P.sparsify ? h->ranks[k - 1][p] : Lp.m[p];
        pool_append(pool, Lp.slot_off[p], live);
        m += live;
      }
      Ly.m[c] = m;
    }
  }
  h->sizes[k] = Ly.m;
  // ---- panel layout
  Ly.row.assign(ncl, nullptr);
  Ly.ncols.assign(ncl, 0);
  Ly.segcol.assign(ncl, {});
  size_t fbytes = 0, sbytes = 0;
  std::vector<size_t> roff(ncl);
  for (int c = 0; c < ncl; ++c) {
    const auto& rs = S.rowsegs[c];
    auto& sc = Ly.segcol[c];
    sc.resize(rs.size());
    int acc = 0;
    for (size_t i = 0; i < rs.size(); ++i) {
      sc[i] = acc;
      acc += Ly.m[rs[i]];
    }
    Ly.ncols[c] = acc;
    // every row region starts on a multiple of 4 elements (the same layout
    // rule as the analyze-time pack map, whatever the element size)
    const size_t bytes = (((size_t)Ly.m[c] * acc + 3) & ~size_t(3)) * sizeof(real_t);
    if (S.interior[c]) {
      roff[c] = fbytes;
      fbytes += bytes;
    } else {
      roff[c] = sbytes;
      sbytes += bytes;
    }
  }
  void* fptr = nullptr;
  RET(h->farena.alloc(std::max<size_t>(fbytes, 16), &fptr));
  DevBuf& scr = h->scratch[k & 1];
  RET(scr.ensure(std::max<size_t>(sbytes, 16)));
  for (int c = 0; c < ncl; ++c)
    Ly.row[c] = reinterpret_cast<real_t*>((S.interior[c] ? (char*)fptr : scr.p) + roff[c]);
  if (k == 0 && h->pack_split != (int64_t)(fbytes / sizeof(real_t))) {
    // the analyze-time pack map assumed the same layout
    return fail(SPAND_ECUDA, "internal: stage-0 layout mismatch");
  }
  if (fbytes) W.zero.push_back({fptr, fbytes});
  if (sbytes) W.zero.push_back({scr.p, sbytes});
  if (k == 0)
    W.packs.push_back({h->d_fval, h->d_pack, (real_t*)fptr, (real_t*)scr.p, h->pack_split, h->nnz});
  auto segc = [&](int c, int d) { return segcol_of(S.rowsegs[c], Ly.segcol[c], d); };
  int* d_err = d_cnt + 4 * ncl;

  // ---- merge of the previous stage's live blocks
  if (k > 0) {
    const StageSym& P = h->st[k - 1];
    const StageLayout& Lp = R.L[k - 1];
    // offsets of each child inside its parent
    std::vector<int> off_in_parent(P.ncl, 0);
    for (int c = 0; c < ncl; ++c) {
      int acc = 0;
      for (int p : S.children[c]) {
        off_in_parent[p] = acc;
        acc += P.sparsify ? h->ranks[k - 1][p] : Lp.m[p];
      }
    }
    for (int p : P.ifaces) {
      const int Pc = P.parent[p];
      const int lp = P.sparsify ? h->ranks[k - 1][p] : Lp.m[p];
      const auto& rs = P.rowsegs[p];
      for (size_t i = 0; i < rs.size(); ++i) {
        const int q = rs[i];
        const int Qc = P.parent[q];
        const int lq = P.sparsify ? h->ranks[k - 1][q] : Lp.m[q];
        const real_t* src = Lp.row[p] + (size_t)Lp.segcol[p][i] * Lp.m[p];
        // an interface row holds no interior columns: that block reaches the
        // interior's row through the transposed child block (q, p)
        if (S.interior[Qc] && !S.interior[Pc]) continue;
        const auto& prs = S.rowsegs[Pc];
        auto it = std::lower_bound(prs.begin(), prs.end(), Qc);
        if (it == prs.end() || *it != Qc) return fail(SPAND_ECUDA, "internal: merge target missing");
        real_t* dst = Ly.row[Pc] + off_in_parent[p] +
                      (size_t)(Ly.segcol[Pc][it - prs.begin()] + off_in_parent[q]) * Ly.m[Pc];
        push_copy(W.merge, src, dst, Lp.m[p], Ly.m[Pc], lp, lq, 0);
      }
    }
  }
  // ---- interiors
  for (int sidx : S.interiors) {
    const int m = Ly.m[sidx];
    W.max_m_int = std::max(W.max_m_int, m);
    const int dc = segc(sidx, sidx);
    W.potrf_int.push_back({Ly.row[sidx] + (size_t)dc * m, d_err, m, m, sidx, 0});
    push_trsm(W.trsm_int, Ly.row[sidx] + (size_t)dc * m, m, Ly.row[sidx], m, m, dc, 0);
    push_trsm(W.trsm_int, Ly.row[sidx] + (size_t)dc * m, m, Ly.row[sidx] + (size_t)(dc + m) * m, m,
              m, Ly.ncols[sidx] - dc - m, 0);
  }
  for (size_t tg = 0; tg < S.schur_q.size(); ++tg) {
    const int q = S.schur_q[tg], r = S.schur_r[tg];
    const int mq = Ly.m[q], mr = Ly.m[r];
    if (mq == 0 || mr == 0) continue;
    const int cb = (int)W.contribs.size();
    for (int e = S.schur_ptr[tg]; e < S.schur_ptr[tg + 1]; ++e) {
      const int sidx = S.schur_s[e];
      const int ms = Ly.m[sidx];
      if (ms == 0) continue;
      SchurContrib c;
      c.a = Ly.row[sidx] + (size_t)segc(sidx, q) * ms;
      c.b = Ly.row[sidx] + (size_t)segc(sidx, r) * ms;
      c.K = ms;
      c.lda = ms;
      c.ldb = ms;
      c.pad = 0;
      W.contribs.push_back(c);
    }
    const int ce = (int)W.contribs.size();
    if (ce == cb) continue;
    real_t* blk = Ly.row[q] + (size_t)segc(q, r) * mq;
    real_t* mir = (q != r) ? Ly.row[r] + (size_t)segc(r, q) * mr : nullptr;
    // FP32: large blocks with a deep contribution go to the tensor cores
    int ksum = 0;
    for (int e = cb; e < ce; ++e) ksum += W.contribs[e].K;
    const bool tc = schur_tc_available() && !h->schur_simt && mq >= 64 && mr >= 64 && ksum >= 96;
    const int tile = tc ? kSchurTcTile : 32;
    if (tc) W.tc_err = d_err + 1;
    for (int i0 = 0; i0 < mq; i0 += tile)
      for (int j0 = 0; j0 < mr; j0 += tile) {
        if (q == r && j0 > i0) continue;  // diagonal block: lower tiles only, mirrored below
        SchurTile t;
        t.dst = blk + i0 + (size_t)j0 * mq;
        t.ld = mq;
        t.rows = std::min(tile, mq - i0);
        t.cols = std::min(tile, mr - j0);
        t.cbegin = cb;
        t.cend = ce;
        t.i0 = i0;
        t.j0 = j0;
        if (q != r) {
          t.mirror = mir + j0 + (size_t)i0 * mr;
          t.ld_mirror = mr;
        } else if (j0 < i0) {
          t.mirror = blk + j0 + (size_t)i0 * mq;
          t.ld_mirror = mq;
        } else {
          t.mirror = nullptr;
          t.ld_mirror = 0;
        }
        (tc ? W.tiles_tc : W.tiles).push_back(t);
      }
  }
  // ---- interfaces: scaling and sparsification
  Ly.Z.assign(ncl, nullptr);
  Ly.V.assign(ncl, nullptr);
  Ly.tau.assign(ncl, nullptr);
  Ly.maxref.assign(ncl, 0);
  Ly.ncols_ub.assign(ncl, 0);
  Ly.qr_grid.assign(ncl, 0);
  if (S.sparsify) {
    for (int p : S.ifaces) {
      const int m = Ly.m[p];
      W.max_m_if = std::max(W.max_m_if, m);
      void* zp = nullptr;
      RET(h->farena.alloc(std::max<size_t>((size_t)m * m * sizeof(real_t), 16), &zp));
      Ly.Z[p] = (real_t*)zp;
      int nub = 0;
      for (int q : S.adj1[p]) nub += Ly.m[q];
      Ly.ncols_ub[p] = nub;
      const int mr = std::min(m, nub);
      Ly.maxref[p] = mr;
      void *vp = nullptr, *tp = nullptr;
      RET(h->farena.alloc(std::max<size_t>((size_t)m * mr * sizeof(real_t), 16), &vp));
      RET(h->farena.alloc(std::max<size_t>((size_t)mr * sizeof(real_t), 16), &tp));
      Ly.V[p] = (real_t*)vp;
      Ly.tau[p] = (real_t*)tp;
      const int dc = segc(p, p);
      push_copy(W.zcopy, Ly.row[p] + (size_t)dc * m, Ly.Z[p], m, m, m, m, 0);
      W.zpotrf.push_back({Ly.Z[p], d_err, m, m, p, 0});
      push_trsm(W.ltrsm, Ly.Z[p], m, Ly.row[p], m, m, dc, 0);
      const auto& rs = S.rowsegs[p];
      for (size_t i = 0; i < rs.size(); ++i) {
        const int q = rs[i];
        if (q >= p) break;
        const int mq = Ly.m[q];
        real_t* B = Ly.row[p] + (size_t)Ly.segcol[p][i] * m;
        push_trsm(W.rtrsm, Ly.Z[q], mq, B, mq, m, m, 1);
        push_copy(W.mirror, B, Ly.row[q] + (size_t)segc(q, p) * mq, m, mq, mq, m, 1);
      }
      W.ident.push_back({Ly.row[p] + (size_t)dc * m, nullptr, m, m, p, 0});
    }
    for (int col = 0; col < S.ncolours; ++col) {
      for (int p : S.by_colour[col]) {
        const int m = Ly.m[p];
        RRQRTask t;
        t.A = Ly.row[p];
        t.ld = m;
        t.m = m;
        t.diag = Ly.row[p] + (size_t)segc(p, p) * m;
        t.V = Ly.V[p];
        t.tau = Ly.tau[p];
        t.cur = d_cnt;
        t.rank = d_cnt + ncl;
        t.nref = d_cnt + 2 * ncl;
        t.flag = d_cnt + 3 * ncl;
        t.err = d_err;
        t.eps = h->eps;
        t.scheme = h->scheme;
        t.id = p;
        t.maxref = Ly.maxref[p];
        t.ncols_max = Ly.ncols_ub[p];
        t.wait_extra = h->qr_wait_extra;
        t.wait_limit = h->qr_wait_limit;
        t.seg_begin = (int)W.qr_segs.size();
        const auto& rs = S.rowsegs[p];
        for (size_t i = 0; i < rs.size(); ++i) {
          const int q = rs[i];
          if (q == p) continue;
          RRQRSeg g;
          g.col = Ly.segcol[p][i];
          g.cl = q;
          g.mirror = Ly.row[q] + (size_t)segc(q, p) * Ly.m[q];
          g.mirror_ld = Ly.m[q];
          g.pad = 0;
          W.qr_segs.push_back(g);
        }
        t.seg_end = (int)W.qr_segs.size();
        t.nseg_max = t.seg_end - t.seg_begin;
        // Cluster size: the smallest that fits shared memory, raised until the
        // colour's interfaces fill about two CTAs per SM, while keeping at least
        // 32 columns per CTA.
        // The base bucket b0 (the smallest cluster whose shared memory holds the
        // block) keys the tuned choices of spand_tune: a growth factor for the
        // cluster size and the CTA size.
        const int ntask = (int)S.by_colour[col].size();
        int b0 = 0;
        for (int lc = 0; lc <= 4 && !b0; ++lc)
          if (rrqr_cluster_smem_bytes(m, t.ncols_max, t.nseg_max, 1 << lc) <= kQrClusterSmem &&
              cluster_ok(h, 1 << lc))
            b0 = lc + 1;
        const int grow = b0 ? std::max(1, h->tune_grow[b0]) : 1;
        int want = 1;
        while (want < 16 && want * ntask < 2 * kNumSMs && (2 * want) * 32 <= t.ncols_max) want *= 2;
        want = std::min(16, want * grow);
        int b = 0;
        int bytes_b = 0;
        if (b0) {
          int lw = b0 - 1;
          while ((1 << lw) < want && lw < 4 && cluster_ok(h, 1 << (lw + 1))) ++lw;
          b = lw + 1;
          bytes_b = rrqr_cluster_smem_bytes(m, t.ncols_max, t.nseg_max, 1 << lw);
        }
        // CTA size: the handle's choice, else the tuned one, else 256 threads
        int thr = 256;
        const int want_thr = h->rrqr_threads > 0 ? h->rrqr_threads : (b0 ? h->tune_thr[b0] : 0);
        if (b > 0 && want_thr > 0) {
          thr = want_thr;
          const int cs = 1 << (b - 1);
          if (rrqr_cluster_active(cs, bytes_b, thr) <= 0) thr = 256;
        }
        // too wide for a cluster: spread over several CTAs of a cooperative
        // launch (bucket 6), unless the single-CTA streamed kernel is asked for
        if ((b == 0 && h->rrqr_path != 1) || h->rrqr_path == 3 || h->rrqr_path == 4) b = 6;
        Ly.qr_grid[p] = b == 6 ? 1 : 0;
        // multi-CTA: on chip where the block fits the shared memory of at most
        // one CTA per SM, else streamed (rrqr_path 3: always streamed)
        if (b == 6) t.wait_extra |= (h->rrqr_path != 3 && h->rrqr_path != 5 &&
                                     gsm_need(m, t.ncols_max, t.nseg_max) > 0)
                                        ? kQrOnChip : 0;
        if (debug_plan())
          fprintf(stderr, "spand plan: stage %d colour %d iface %d m %d ncols_ub %d nseg %d bucket %d thr %d\n",
                  k, col, p, m, t.ncols_max, t.nseg_max, b, thr);
        // while tuning, each base bucket launches on its own so that its time can
        // be read from its launches; otherwise equal shapes share a launch
        auto& g = W.qr[{col, ((h->tuning ? b0 : 0) * 8 + b) * 4096 + thr}];
        g.threads = thr;
        g.bucket = b;
        g.base = b0;
        g.tasks.push_back(t);
        g.max_m = std::max(g.max_m, m);
        g.max_cols = std::max(g.max_cols, t.ncols_max);
        g.max_segs = std::max(g.max_segs, t.nseg_max);
        g.smem = std::max(g.smem, bytes_b);
        if (b == 0 && rrqr_smem_bytes(g.max_m, g.max_cols, g.max_segs) > 220 * 1024)
          return fail(SPAND_ENOMEM, "interface block too wide for the RRQR workspace (stage " +
                                        std::to_string(k) + ")");
        if (b == 6 && !(t.wait_extra & kQrOnChip) && rrqr_grid_smem_bytes(m, 32, t.nseg_max) > 200 * 1024)
          return fail(SPAND_ENOMEM, "interface too tall for the multi-CTA RRQR (stage " +
                                        std::to_string(k) + ")");
      }
    }
  }
  // pristine counters: widths at the stage start, then -1 for ranks,
  // reflectors and flags, then the error words
  W.ints.insert(W.ints.end(), Ly.m.begin(), Ly.m.end());
  W.ints.insert(W.ints.end(), 3 * (size_t)ncl, -1);
  W.ints.push_back(0);
  W.ints.push_back(0);
  return SPAND_OK;
}

// Offsets of a stage's tables in its uploaded blob.
struct StageBlob {
  size_t e, inv, fq, merge, ti, tiles, tiles_tc, contr, zc, lt, rt, mi, id, seg, ints;
  PotrfPlan pint, pz;
  std::vector<size_t> qr;
  // multi-CTA QR launches: grid-task arrays (patched with workspace pointers
  // once the blob's device address is known) and the zeroed workspace
  struct GridLaunch {
    size_t off;        // RRQRGridTask array in the blob
    int ntasks, nctas, smem;
    size_t group;      // index of the QrGroup
    bool onchip;       // k_rrqr_gsm (the slices in shared memory) or k_rrqr_grid
  };
  std::vector<GridLaunch> grid;
  std::vector<std::vector<size_t>> grid_ws;  // per launch: workspace int offset of each task
  std::vector<std::vector<size_t>> grid_stage;  // per launch: staging byte offset of each task
  size_t ws = 0, ws_ints = 0;
  // staging of the on-chip multi-CTA QR: the blob's tail, never uploaded
  // (always written before it is read)
  size_t stage = 0, stage_bytes = 0, upload = 0;
};

// Tasks of one launch in decreasing cost (stable: equal tasks keep their
// order, e.g. the column blocks of one operator stay together): CTAs are handed
// out in task order as SMs free up, so a launch ends on its short tasks.
template <class T, class C>
void longest_first(std::vector<T>& v, C cost) {
  std::stable_sort(v.begin(), v.end(), [&](const T& a, const T& b) { return cost(a) > cost(b); });
}

StageBlob pack_blob(StageWork& W, Blob& blob) {
  StageBlob o;
  // the explicit inverses and Q^T of the apply operators, longest first (measured:
  // 23.7 -> 21.8 and 38.4 -> 35.4 ms per 128^3 factorization; the same order for
  // the triangular solves and Schur tiles of the factorization measured no gain)
  longest_first(W.pend_inv, [](const TrsmTask& t) {
    const double rows = t.pad >= 0 ? (double)(t.m - t.pad) : (double)t.m;  // identity: rows below it
    return rows * rows * t.ncols;
  });
  longest_first(W.pend_qt, [](const FormQtTask& t) { return (double)t.m * t.m * t.nref; });
  o.e = blob.add(W.pend_e);
  o.inv = blob.add(W.pend_inv);
  o.fq = blob.add(W.pend_qt);
  o.merge = blob.add(W.merge);
  o.pint = plan_potrf(W.potrf_int);
  plan_to_blob(o.pint, blob);
  o.pz = plan_potrf(W.zpotrf);
  plan_to_blob(o.pz, blob);
  o.ti = blob.add(W.trsm_int);
  o.tiles = blob.add(W.tiles);
  o.tiles_tc = blob.add(W.tiles_tc);
  o.contr = blob.add(W.contribs);
  o.zc = blob.add(W.zcopy);
  o.lt = blob.add(W.ltrsm);
  o.rt = blob.add(W.rtrsm);
  o.mi = blob.add(W.mirror);
  o.id = blob.add(W.ident);
  size_t gi = 0;
  for (auto& kv : W.qr) {
    auto& g = kv.second;
    // the longest QRs first (cost ~ m N min(m, N) of the block; measured: 400 ->
    // 377 ms FP64, 143 -> 130 ms FP32 per 128^3 factorization)
    if (g.bucket != 6)
      longest_first(g.tasks, [](const RRQRTask& t) {
        return (double)t.m * t.ncols_max * std::min(t.m, t.ncols_max);
      });
    o.qr.push_back(blob.add(g.tasks));
    if (g.bucket == 6) {
      std::vector<RRQRTask> onchip, streamed;
      for (RRQRTask t : g.tasks) {
        const bool oc = (t.wait_extra & kQrOnChip) != 0;
        t.wait_extra &= ~kQrOnChip;
        (oc ? onchip : streamed).push_back(t);
      }
      // on chip: launches of tasks whose fewest CTAs fit in one CTA per SM; the
      // spare SMs go to the tasks by their work m x ncols
      for (size_t t0 = 0; t0 < onchip.size();) {
        size_t t1 = t0;
        int used = 0;
        while (t1 < onchip.size()) {
          const RRQRTask& t = onchip[t1];
          const int need = gsm_need(t.m, t.ncols_max, t.nseg_max);
          if (t1 > t0 && used + need > kNumSMs) break;
          used += need;
          ++t1;
        }
        double wsum = 0.0;
        for (size_t i = t0; i < t1; ++i) wsum += (double)onchip[i].m * onchip[i].ncols_max;
        const int spare = std::max(0, kNumSMs - used);
        std::vector<RRQRGridTask> gts;
        std::vector<size_t> wsoff, stoff;
        int cta = 0, smem = 0;
        for (size_t i = t0; i < t1; ++i) {
          const RRQRTask& t = onchip[i];
          const double w = (double)t.m * t.ncols_max;
          int nc = gsm_need(t.m, t.ncols_max, t.nseg_max) + (wsum > 0.0 ? (int)(spare * w / wsum) : 0);
          nc = std::max(1, std::min(nc, std::max(1, t.ncols_max)));
          RRQRGridTask gt;
          gt.t = t;
          gt.ws = nullptr;
          gt.stage = nullptr;
          gt.cta0 = cta;
          gt.ncta = nc;
          gts.push_back(gt);
          wsoff.push_back(o.ws_ints);
          o.ws_ints += qr_grid_ws_ints(nc);
          stoff.push_back(o.stage_bytes);
          o.stage_bytes += ((size_t)2 * nc * std::max(t.m, 1) * sizeof(real_t) + 255) & ~size_t(255);
          cta += nc;
          smem = std::max(smem, rrqr_gsm_smem_bytes(t.m, (t.ncols_max + nc - 1) / nc, t.nseg_max));
        }
        StageBlob::GridLaunch gl;
        gl.off = blob.add(gts);
        gl.ntasks = (int)gts.size();
        gl.nctas = cta;
        gl.smem = smem;
        gl.group = gi;
        gl.onchip = true;
        o.grid.push_back(gl);
        o.grid_ws.push_back(wsoff);
        o.grid_stage.push_back(stoff);
        t0 = t1;
      }
      // streamed: at most one CTA per SM per launch; tasks share the SMs by their work
      for (size_t t0 = 0; t0 < streamed.size(); t0 += kNumSMs) {
        const size_t t1 = std::min(streamed.size(), t0 + (size_t)kNumSMs);
        double wsum = 0.0;
        for (size_t i = t0; i < t1; ++i) wsum += (double)streamed[i].m * streamed[i].ncols_max;
        const int spare = kNumSMs - (int)(t1 - t0);
        std::vector<RRQRGridTask> gts;
        std::vector<size_t> wsoff;
        int cta = 0, smem = 0;
        for (size_t i = t0; i < t1; ++i) {
          const RRQRTask& t = streamed[i];
          const double w = (double)t.m * t.ncols_max;
          int nc = 1 + (wsum > 0.0 ? (int)(spare * w / wsum) : 0);
          nc = std::max(1, std::min(nc, (t.ncols_max + 31) / 32));  // at least 32 columns per CTA
          RRQRGridTask gt;
          gt.t = t;
          gt.ws = nullptr;
          gt.stage = nullptr;
          gt.cta0 = cta;
          gt.ncta = nc;
          gts.push_back(gt);
          wsoff.push_back(o.ws_ints);
          o.ws_ints += qr_grid_ws_ints(nc);
          cta += nc;
          smem = std::max(smem, rrqr_grid_smem_bytes(t.m, (t.ncols_max + nc - 1) / nc, t.nseg_max));
        }
        StageBlob::GridLaunch gl;
        gl.off = blob.add(gts);
        gl.ntasks = (int)gts.size();
        gl.nctas = cta;
        gl.smem = smem;
        gl.group = gi;
        gl.onchip = false;
        o.grid.push_back(gl);
        o.grid_ws.push_back(wsoff);
        o.grid_stage.push_back({});
      }
    }
    ++gi;
  }
  o.seg = blob.add(W.qr_segs);
  o.ints = blob.add(W.ints);
  o.ws = blob.add(std::vector<int>(std::max<size_t>(o.ws_ints, 4), 0));
  o.upload = blob.h.size();
  if (o.stage_bytes) {
    o.stage = (blob.h.size() + 255) & ~size_t(255);
    blob.h.resize(o.stage + o.stage_bytes);
  }
  return o;
}

// The grid tasks' workspace pointers, once the blob sits at device address D.
void patch_grid(const StageBlob& o, Blob& blob, char* D) {
  for (size_t L = 0; L < o.grid.size(); ++L) {
    RRQRGridTask* gt = (RRQRGridTask*)(blob.h.data() + o.grid[L].off);
    for (int i = 0; i < o.grid[L].ntasks; ++i) {
      gt[i].ws = (int*)(D + o.ws) + o.grid_ws[L][i];
      gt[i].stage = o.grid[L].onchip ? (real_t*)(D + o.stage + o.grid_stage[L][i]) : nullptr;
    }
  }
}

// All launches of one stage on stream cs; D: the uploaded blob, cnt: the live
// counters (reset from the blob's pristine copy first).  Returns the number of
// kernel launches through *nl.
int launch_stage(StageWork& W, const StageBlob& O, char* D, int* cnt, Prof& P, cudaStream_t cs,
                 int* nl, FactorGroup& G, int stage) {
  auto run = [&](int kind, size_t ntasks, double flops, double bytes, auto&& launch) {
    if (ntasks == 0) return;
    ++*nl;
    P.run(kind, cs, flops, bytes, launch);
  };
  if (!W.ints.empty())
    CK(cudaMemcpyAsync(cnt, D + O.ints, W.ints.size() * sizeof(int), cudaMemcpyDeviceToDevice, cs));
  // The previous stage's apply operators read only that stage's data (its
  // interface rows in the other scratch buffer, the factor arena), which this
  // stage does not write: they run on a side branch (a parallel graph branch
  // when captured) and fill the SMs this stage's latency-bound launches leave
  // idle.  The branch joins at the end of the stage, before the next stage
  // clears that scratch buffer.  With profiling, everything stays on cs.
  const bool pend = !W.pend_e.empty() || !W.pend_inv.empty() || !W.pend_qt.empty();
  cudaStream_t ps = cs;
  if (pend && G.side && !P.on) {
    CK(cudaEventRecord(G.ev_fork, cs));
    CK(cudaStreamWaitEvent(G.side, G.ev_fork, 0));
    ps = G.side;
  }
  run(KK_ECOPY, W.pend_e.size(), 0.0, copy_bytes(W.pend_e),
      [&] { launch_copy((const CopyTask*)(D + O.e), (int)W.pend_e.size(), ps); });
  run(KK_TRTRI, W.pend_inv.size(), trtri_flops(W.pend_inv), trsm_bytes(W.pend_inv), [&] {
    launch_trsm((const TrsmTask*)(D + O.inv), (int)W.pend_inv.size(), W.pend_inv_m, ps);
  });
  run(KK_FORMQ, W.pend_qt.size(), formqt_flops(W.pend_qt), 0.0, [&] {
    launch_form_qt((const FormQtTask*)(D + O.fq), (int)W.pend_qt.size(), W.pend_qt_m, ps);
  });
  if (ps != cs) CK(cudaEventRecord(G.ev_join, ps));
  auto join = [&]() -> int {
    if (ps != cs) CK(cudaStreamWaitEvent(cs, G.ev_join, 0));
    return SPAND_OK;
  };
  for (auto& z : W.zero) CK(cudaMemsetAsync(z.first, 0, z.second, cs));
  for (auto& pk : W.packs)
    run(KK_PACK, 1, 0.0, 16.0 * pk.nnz,
        [&] { launch_scatter(pk.val, pk.idx, pk.lo, pk.hi, pk.split, pk.nnz, cs); });
  run(KK_MERGE, W.merge.size(), 0.0, copy_bytes(W.merge),
      [&] { launch_copy((const CopyTask*)(D + O.merge), (int)W.merge.size(), cs); });
  auto run_potrf = [&](int kind, const PotrfPlan& PP) {
    bool first = true;
    auto fl = [&]() { double f = first ? PP.flops : 0.0; first = false; return f; };
    run(kind, PP.small.size(), fl(), PP.bytes, [&] {
      launch_potrf((const PotrfTask*)(D + PP.o_small), (int)PP.small.size(), PP.small_max, cs);
    });
    for (auto& st : PP.steps) {
      run(kind, st.diag.size(), fl(), 0.0, [&] {
        launch_potrf((const PotrfTask*)(D + st.o_diag), (int)st.diag.size(), kPanel, cs);
      });
      run(kind, st.trsm.size(), 0.0, 0.0, [&] {
        launch_trsm((const TrsmTask*)(D + st.o_trsm), (int)st.trsm.size(), kPanel, cs);
      });
      run(kind, st.tiles.size(), 0.0, 0.0, [&] {
        launch_schur((const SchurTile*)(D + st.o_tiles), (int)st.tiles.size(),
                     (const SchurContrib*)(D + st.o_contribs), cs);
      });
    }
  };
  run_potrf(KK_POTRF, O.pint);
  run(KK_TRSM, W.trsm_int.size(), trsm_flops(W.trsm_int), trsm_bytes(W.trsm_int), [&] {
    launch_trsm((const TrsmTask*)(D + O.ti), (int)W.trsm_int.size(), W.max_m_int, cs);
  });
  {
    double fl = 0.0, by = 0.0;
    schur_work(W.tiles, W.contribs, &fl, &by);
    run(KK_SCHUR, W.tiles.size(), fl, by, [&] {
      launch_schur((const SchurTile*)(D + O.tiles), (int)W.tiles.size(),
                   (const SchurContrib*)(D + O.contr), cs);
    });
    schur_work(W.tiles_tc, W.contribs, &fl, &by, true);
    cudaError_t te = cudaSuccess;
    run(KK_SCHUR_TC, W.tiles_tc.size(), fl, by, [&] {
      te = launch_schur_tc((const SchurTile*)(D + O.tiles_tc), (int)W.tiles_tc.size(),
                           (const SchurContrib*)(D + O.contr), W.tc_err, cs);
    });
    if (te != cudaSuccess) {
      join();
      return fail(SPAND_ECUDA, std::string("tensor-core Schur launch: ") + cudaGetErrorString(te));
    }
  }
  run(KK_SCALE_COPY, W.zcopy.size(), 0.0, copy_bytes(W.zcopy),
      [&] { launch_copy((const CopyTask*)(D + O.zc), (int)W.zcopy.size(), cs); });
  run_potrf(KK_SCALE_POTRF, O.pz);
  run(KK_SCALE_TRSM, W.ltrsm.size(), trsm_flops(W.ltrsm), trsm_bytes(W.ltrsm),
      [&] { launch_trsm((const TrsmTask*)(D + O.lt), (int)W.ltrsm.size(), W.max_m_if, cs); });
  run(KK_SCALE_TRSM, W.rtrsm.size(), trsm_flops(W.rtrsm), trsm_bytes(W.rtrsm),
      [&] { launch_trsm((const TrsmTask*)(D + O.rt), (int)W.rtrsm.size(), W.max_m_if, cs); });
  run(KK_SCALE_COPY, W.mirror.size(), 0.0, copy_bytes(W.mirror),
      [&] { launch_copy((const CopyTask*)(D + O.mi), (int)W.mirror.size(), cs); });
  run(KK_SCALE_COPY, W.ident.size(), 0.0, potrf_bytes(W.ident) / 2,
      [&] { launch_set_identity((const PotrfTask*)(D + O.id), (int)W.ident.size(), cs); });
  if (O.ws_ints) CK(cudaMemsetAsync(D + O.ws, 0, O.ws_ints * sizeof(int), cs));
  size_t gi = 0;
  cudaError_t gerr = cudaSuccess;
  for (auto& kv : W.qr) {
    const auto& g = kv.second;
    const int b = g.bucket;
    const size_t off = O.qr[gi];
    if (b == 6) {
      for (const auto& gl : O.grid) {
        if (gl.group != gi) continue;
        P.tag = stage * 100;
        run(KK_RRQR_GRID, (size_t)gl.ntasks, 0.0, 0.0, [&] {
          const cudaError_t e =
              gl.onchip ? launch_rrqr_gsm((const RRQRGridTask*)(D + gl.off), gl.ntasks, gl.nctas,
                                          (const RRQRSeg*)(D + O.seg), gl.smem, cs)
                        : launch_rrqr_grid((const RRQRGridTask*)(D + gl.off), gl.ntasks, gl.nctas,
                                           (const RRQRSeg*)(D + O.seg), gl.smem, cs);
          if (e != cudaSuccess && gerr == cudaSuccess) gerr = e;
        });
      }
    } else {
      P.tag = stage * 100 + g.base;  // the autotuner reads the base bucket (tag % 100)
      run(KK_RRQR, g.tasks.size(), 0.0, 0.0, [&] {
        if (b == 0)
          launch_rrqr((const RRQRTask*)(D + off), (int)g.tasks.size(), (const RRQRSeg*)(D + O.seg),
                      g.max_m, g.max_cols, g.max_segs, cs);
        else {
          const cudaError_t e =
              launch_rrqr_cluster((const RRQRTask*)(D + off), (int)g.tasks.size(),
                                  (const RRQRSeg*)(D + O.seg), 1 << (b - 1), g.smem, g.threads, cs);
          if (e != cudaSuccess && gerr == cudaSuccess) gerr = e;
        }
      });
    }
    ++gi;
  }
  RET(join());
  if (gerr != cudaSuccess)
    return fail(SPAND_ECUDA, std::string("RRQR launch: ") + cudaGetErrorString(gerr));
  CK(cudaGetLastError());
  return SPAND_OK;
}

// After the stage's counters came back (hp: this problem's counters): record
// the ranks and lay out the apply operators of the stage, whose explicit
// inverses, Q^T and E-tilde copies run with the next stage's launches.
int finish_stage(Run& R, int k, const int* hp, Prof& P) {
  spand_s* h = R.h;
  const StageSym& S = h->st[k];
  StageLayout& Ly = R.L[k];
  std::vector<int>& pool = R.pool;
  const int ncl = S.ncl;
  h->ranks[k].assign(hp + ncl, hp + 2 * ncl);
  h->nrefs[k].assign(hp + 2 * ncl, hp + 3 * ncl);
  h->flags[k].assign(hp + 3 * ncl, hp + 4 * ncl);
  auto segc = [&](int c, int d) { return segcol_of(S.rowsegs[c], Ly.segcol[c], d); };
  if (P.on && S.sparsify) {
    double fl[2] = {0.0, 0.0}, by[2] = {0.0, 0.0};
    for (int p : S.ifaces) {
      const int m = Ly.m[p], nref = h->nrefs[k][p];
      const int w = Ly.qr_grid[p];
      int N = 0;
      for (int q : S.adj1[p]) N += (S.colour[q] < S.colour[p]) ? h->ranks[k][q] : Ly.m[q];
      for (int t = 0; t < nref; ++t) fl[w] += 6.0 * (double)(m - t) * (double)(N - t);
      by[w] += 16.0 * (double)m * N;  // the block is read and written once
    }
    P.stat[KK_RRQR].flops += fl[0];
    P.stat[KK_RRQR].bytes += by[0];
    P.stat[KK_RRQR_GRID].flops += fl[1];
    P.stat[KK_RRQR_GRID].bytes += by[1];
  }
  auto explicit_inverse = [&](const real_t* Lb, int m, real_t** out) -> int {
    void* ip = nullptr;
    RET(h->farena.alloc(std::max<size_t>((size_t)m * m * sizeof(real_t), 16), &ip));
    *out = (real_t*)ip;
    push_trsm(R.pending_inv, Lb, m, *out, m, m, m, 0, true);
    R.pending_inv_m = std::max(R.pending_inv_m, m);
    return SPAND_OK;
  };
  {
    Phase ph{PH_INTERIOR, (int)R.api.size(), 0, 0, 0.0, 0.0};
    ph.stage = k;
    std::vector<int> Ks, ms, cols;
    std::vector<double> fl, by;
    for (int sidx : S.interiors) {
      const int m = Ly.m[sidx];
      ApInteriorP a;
      a.m = m;
      a.ncols = Ly.ncols[sidx];
      const int dc = segc(sidx, sidx);
      real_t* Linv = nullptr;
      if (m > 0) RET(explicit_inverse(Ly.row[sidx] + (size_t)dc * m, m, &Linv));
      a.Linv = Linv;
      a.WT = Ly.row[sidx];
      a.dc = dc;
      a.slots = Ly.slot_off[sidx];
      a.wslots = (int64_t)pool.size();
      for (int d : S.rowsegs[sidx]) {
        if (d == sidx) {
          pool.insert(pool.end(), (size_t)Ly.m[d], -1);
        } else {
          pool_append(pool, Ly.slot_off[d], Ly.m[d]);
        }
      }
      R.api.push_back(a);
      const double fm = (double)m * (m + 1) / 2 + (double)m * (a.ncols - m);
      Ks.push_back(ap_cluster(fm));
      ms.push_back(m);
      cols.push_back(a.ncols);
      fl.push_back(2.0 * fm);
      by.push_back(8.0 * fm + 24.0 * a.ncols);
      R.nnzf += (int64_t)m * (m + 1) / 2 + (int64_t)m * (a.ncols - m);
    }
    ph.end = (int)R.api.size();
    if (ph.end > ph.begin) split_phase(R.phases, R.api, ph, Ks, fl, by, ms, cols);
  }
  if (!S.sparsify) return SPAND_OK;
  {
    Phase ph{PH_SCALE, (int)R.aps.size(), 0, 0, 0.0, 0.0};
    ph.stage = k;
    std::vector<int> Ks, ms, cols;
    std::vector<double> fl, by;
    for (int p : S.ifaces) {
      const int m = Ly.m[p];
      real_t* Zinv = nullptr;
      if (m > 0) RET(explicit_inverse(Ly.Z[p], m, &Zinv));
      R.aps.push_back({Zinv, Ly.slot_off[p], m});
      const double fm = (double)m * (m + 1) / 2;
      Ks.push_back(ap_cluster(fm));
      ms.push_back(m);
      cols.push_back(0);
      fl.push_back(2.0 * fm);
      by.push_back(8.0 * fm + 16.0 * m);
      R.nnzf += (int64_t)m * (m + 1) / 2;
    }
    ph.end = (int)R.aps.size();
    if (ph.end > ph.begin) split_phase(R.phases, R.aps, ph, Ks, fl, by, ms, cols);
  }
  for (int col = 0; col < S.ncolours; ++col) {
    Phase pq{PH_QE, (int)R.apq.size(), 0, 0, 0.0, 0.0};
    pq.stage = k;
    pq.colour = col;
    std::vector<int> Ks, ms, cols;
    std::vector<double> fl, by;
    for (int p : S.by_colour[col]) {
      const int m = Ly.m[p];
      const int r = h->ranks[k][p], nref = h->nrefs[k][p];
      int nE = 0;
      if (h->scheme == SPAND_SECOND_ORDER_FULL) nE = m - r;
      else if (h->scheme == SPAND_SECOND_ORDER_SUPERFINE) nE = nref - r;
      ApQEP a;
      a.m = m;
      a.r = r;
      a.nE = nE;
      a.Qt = nullptr;
      if (m > 0) {
        void* qp = nullptr;
        RET(h->farena.alloc((size_t)m * m * sizeof(real_t), &qp));
        a.Qt = (real_t*)qp;
        for (int c0 = 0; c0 < m; c0 += 32) {
          FormQtTask ft;
          ft.V = Ly.V[p];
          ft.tau = Ly.tau[p];
          ft.Qt = (real_t*)a.Qt + (size_t)c0 * m;
          ft.m = m;
          ft.nref = nref;
          ft.c0 = c0;
          ft.ncols = std::min(32, m - c0);
          R.pending_qt.push_back(ft);
        }
        R.pending_qt_m = std::max(R.pending_qt_m, m);
      }
      a.slots = Ly.slot_off[p];
      a.eslots = (int64_t)pool.size();
      int ncols = 0;
      const auto& rs = S.rowsegs[p];
      std::vector<std::pair<int, int>> segw;  // (column in row, width)
      for (size_t i = 0; i < rs.size(); ++i) {
        const int q = rs[i];
        if (q == p) continue;
        const int w = (S.colour[q] < S.colour[p]) ? h->ranks[k][q] : Ly.m[q];
        pool_append(pool, Ly.slot_off[q], w);
        segw.push_back({Ly.segcol[p][i], w});
        ncols += w;
      }
      a.ncols = ncols;
      a.E = nullptr;
      if (nE > 0 && ncols > 0) {
        void* ep = nullptr;
        RET(h->farena.alloc((size_t)nE * ncols * sizeof(real_t), &ep));
        real_t* Edst = (real_t*)ep;
        a.E = Edst;
        int acc = 0;
        // E-tilde row-major (row i at i * ncols): rows r .. r + nE - 1 of each
        // neighbour segment of the panel row, transposed into place
        for (auto& sw : segw) {
          push_copy(R.pending_e, Ly.row[p] + r + (size_t)sw.first * m, Edst + acc, m, ncols,
                    sw.second, nE, 1);
          acc += sw.second;
        }
      } else {
        a.nE = 0;
      }
      R.apq.push_back(a);
      const double fm = (double)m * m + (double)a.nE * ncols;
      Ks.push_back(ap_cluster(fm));
      ms.push_back(m);
      cols.push_back(a.nE > 0 ? ncols : 0);
      fl.push_back(2.0 * fm);
      by.push_back(8.0 * fm + 16.0 * (m + ncols));
      R.nnzf += (int64_t)m * nref + nref + (int64_t)a.nE * ncols;
    }
    pq.end = (int)R.apq.size();
    if (pq.end > pq.begin) split_phase(R.phases, R.apq, pq, Ks, fl, by, ms, cols);
  }
  return SPAND_OK;
}

// Uploads the problem's apply plan: slot pool and descriptors into its arena.
int upload_apply_plan(Run& R, cudaStream_t s) {
  spand_s* h = R.h;
  void *pp = nullptr, *pa = nullptr, *ps = nullptr, *pq = nullptr;
  RET(h->farena.alloc(std::max<size_t>(R.pool.size() * 4, 16), &pp));
  RET(h->farena.alloc(std::max<size_t>(R.api.size() * sizeof(ApInterior), 16), &pa));
  RET(h->farena.alloc(std::max<size_t>(R.aps.size() * sizeof(ApScale), 16), &ps));
  RET(h->farena.alloc(std::max<size_t>(R.apq.size() * sizeof(ApQE), 16), &pq));
  const int* dpool = (const int*)pp;
  std::vector<ApInterior> vi(R.api.size());
  for (size_t i = 0; i < R.api.size(); ++i) {
    const auto& a = R.api[i];
    vi[i] = {a.Linv, a.WT, dpool + a.slots, dpool + a.wslots, a.m, a.ncols};
  }
  std::vector<ApScale> vs(R.aps.size());
  for (size_t i = 0; i < R.aps.size(); ++i) vs[i] = {R.aps[i].Zinv, dpool + R.aps[i].slots, R.aps[i].m, 0};
  std::vector<ApQE> vq(R.apq.size());
  for (size_t i = 0; i < R.apq.size(); ++i) {
    const auto& a = R.apq[i];
    vq[i] = {a.Qt, a.E, dpool + a.slots, dpool + a.eslots, a.m, a.r, a.nE, a.ncols};
  }
  // the host vectors must outlive the copies: synchronise before returning
  if (!R.pool.empty())
    CK(cudaMemcpyAsync(pp, R.pool.data(), R.pool.size() * 4, cudaMemcpyHostToDevice, s));
  if (!vi.empty()) CK(cudaMemcpyAsync(pa, vi.data(), vi.size() * sizeof(ApInterior), cudaMemcpyHostToDevice, s));
  if (!vs.empty()) CK(cudaMemcpyAsync(ps, vs.data(), vs.size() * sizeof(ApScale), cudaMemcpyHostToDevice, s));
  if (!vq.empty()) CK(cudaMemcpyAsync(pq, vq.data(), vq.size() * sizeof(ApQE), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  h->d_api = pa;
  h->d_aps = ps;
  h->d_apq = pq;
  h->phases = R.phases;
  h->nnz_factor = R.nnzf;
  return SPAND_OK;
}

// The program of the persistent single-vector sweep (k_ap_sweep), from the
// problem's apply phases: per (stage, kind, colour) two sub-phases forward
// and two backward (one for a scaling's copy back), items of about kSwItem
// matrix entries.  Program, scratch vector and barrier words go into the
// factor arena, so that applying allocates nothing.
constexpr int kSwItem = 16384;

int build_sweep(Run& R, cudaStream_t s) {
  spand_s* h = R.h;
  h->sweep_valid = false;
  // untuned: the persistent form for FP32 factors from kSweepMinN unknowns up
  // (FP64: the per-phase launches measured faster at every size)
  const bool want = h->apply_mode == 2 ||
                    (h->apply_mode == 0 &&
                     (h->sweep_pref == 0 || (h->sweep_pref < 0 && sizeof(real_t) == sizeof(float) &&
                                             (int64_t)h->n >= spand_s::kSweepMinN)));
  if (!want) return SPAND_OK;
  struct Grp {
    int stage, kind, colour;
    std::vector<std::pair<int, int>> ranges;
  };
  std::vector<Grp> groups;
  for (const Phase& ph : R.phases) {
    if (!groups.empty() && groups.back().stage == ph.stage && groups.back().kind == ph.kind &&
        groups.back().colour == ph.colour)
      groups.back().ranges.push_back({ph.begin, ph.end});
    else
      groups.push_back({ph.stage, ph.kind, ph.colour, {{ph.begin, ph.end}}});
  }
  std::vector<SwPhase> P;
  std::vector<SwItem> I;
  int max_vec = 1;
  auto phase = [&](int kind, auto&& gen) {
    SwPhase p{kind, (int)I.size(), 0, 0};
    gen();
    p.nitems = (int)I.size() - p.item0;
    if (p.nitems) P.push_back(p);
  };
  // row blocks of a GEMV over C columns (multiples of 64 rows), column blocks
  // of a transposed one over R rows (multiples of 4 columns)
  auto rows = [&](int op, int m, int C, int aux) {
    const int step = 64 * std::max(1, kSwItem / (64 * std::max(C, 1)));
    for (int lo = 0; lo < m; lo += step) I.push_back({op, lo, std::min(m, lo + step), aux});
  };
  auto cols = [&](int op, int c0, int c1, int Rr, int& aux) {
    const int step = 4 * std::max(1, kSwItem / (4 * std::max(Rr, 1)));
    for (int lo = c0; lo < c1; lo += step) {
      I.push_back({op, lo, std::min(c1, lo + step), aux});
      aux = 0;
    }
  };
  auto each = [&](const Grp& g, auto&& f) {
    for (auto& rg : g.ranges)
      for (int i = rg.first; i < rg.second; ++i) f(i);
  };
  for (const Grp& g : groups) {
    if (g.kind == PH_INTERIOR) {
      phase(SW_FI_A, [&] {
        each(g, [&](int i) {
          max_vec = std::max(max_vec, R.api[i].m);
          if (R.api[i].m) rows(i, R.api[i].m, R.api[i].m / 2 + 1, 0);
        });
      });
      phase(SW_FI_B, [&] {
        each(g, [&](int i) {
          const auto& a = R.api[i];
          if (!a.m) return;
          max_vec = std::max(max_vec, a.m);
          int aux = 1;
          cols(i, 0, a.dc, a.m, aux);
          cols(i, a.dc + a.m, a.ncols, a.m, aux);
          if (aux) I.push_back({i, 0, 0, 1});  // no neighbour: the copy alone
        });
      });
    } else if (g.kind == PH_SCALE) {
      phase(SW_FS_A, [&] {
        each(g, [&](int i) {
          max_vec = std::max(max_vec, R.aps[i].m);
          if (R.aps[i].m) rows(i, R.aps[i].m, R.aps[i].m / 2 + 1, 0);
        });
      });
      phase(SW_COPY, [&] {
        each(g, [&](int i) {
          for (int lo = 0; lo < R.aps[i].m; lo += 4096) I.push_back({i, lo, std::min(R.aps[i].m, lo + 4096), 0});
        });
      });
    } else {
      phase(SW_FQ_A, [&] {
        each(g, [&](int i) {
          max_vec = std::max(max_vec, R.apq[i].m);
          if (R.apq[i].m) rows(i, R.apq[i].m, R.apq[i].m, 0);
        });
      });
      phase(SW_FQ_B, [&] {
        each(g, [&](int i) {
          const auto& a = R.apq[i];
          if (!a.m) return;
          max_vec = std::max(max_vec, a.m);
          if (a.nE > 0 && a.ncols > 0) {
            const int step = 256 * std::max(1, kSwItem / (256 * a.nE));
            for (int lo = 0; lo < a.ncols; lo += step) I.push_back({i, lo, std::min(a.ncols, lo + step), lo == 0});
          } else {
            I.push_back({i, 0, 0, 1});
          }
        });
      });
    }
  }
  for (auto gi = groups.rbegin(); gi != groups.rend(); ++gi) {
    const Grp& g = *gi;
    if (g.kind == PH_QE) {
      phase(SW_BQ_A, [&] {
        each(g, [&](int i) {
          const auto& a = R.apq[i];
          if (!a.m) return;
          max_vec = std::max(max_vec, a.ncols);
          int aux = 1;
          if (a.nE > 0 && a.ncols > 0) cols(i, 0, a.nE, a.ncols, aux);
          if (aux) I.push_back({i, 0, 0, 1});
        });
      });
      phase(SW_BQ_B, [&] {
        each(g, [&](int i) {
          int aux = 0;
          if (R.apq[i].m) cols(i, 0, R.apq[i].m, R.apq[i].m, aux);
        });
      });
    } else if (g.kind == PH_SCALE) {
      phase(SW_BS_A, [&] {
        each(g, [&](int i) {
          int aux = 0;
          if (R.aps[i].m) cols(i, 0, R.aps[i].m, R.aps[i].m / 2 + 1, aux);
        });
      });
      phase(SW_COPY, [&] {
        each(g, [&](int i) {
          for (int lo = 0; lo < R.aps[i].m; lo += 4096) I.push_back({i, lo, std::min(R.aps[i].m, lo + 4096), 0});
        });
      });
    } else {
      phase(SW_BI_A, [&] {
        each(g, [&](int i) {
          const auto& a = R.api[i];
          if (!a.m) return;
          max_vec = std::max(max_vec, a.ncols);
          rows(i, a.m, std::max(a.ncols - a.m, 1), a.dc);
        });
      });
      phase(SW_BI_B, [&] {
        each(g, [&](int i) {
          int aux = 0;
          if (R.api[i].m) cols(i, 0, R.api[i].m, R.api[i].m / 2 + 1, aux);
        });
      });
    }
  }
  const int smem = (max_vec + 16) * (int)sizeof(real_t);
  const int nctas = sweep_ctas(smem);
  if (nctas <= 0 || P.empty()) return SPAND_OK;  // the per-phase launches stay in use
  void *pp = nullptr, *pi = nullptr, *py = nullptr, *pw = nullptr;
  RET(h->farena.alloc(P.size() * sizeof(SwPhase), &pp));
  RET(h->farena.alloc(std::max<size_t>(I.size(), 1) * sizeof(SwItem), &pi));
  RET(h->farena.alloc(std::max<size_t>((size_t)h->n, 1) * sizeof(real_t), &py));
  RET(h->farena.alloc(16, &pw));
  void* ptr = nullptr;
  if (debug_sweep()) RET(h->farena.alloc((P.size() + 1) * sizeof(long long), &ptr));
  CK(cudaMemcpyAsync(pp, P.data(), P.size() * sizeof(SwPhase), cudaMemcpyHostToDevice, s));
  if (!I.empty()) CK(cudaMemcpyAsync(pi, I.data(), I.size() * sizeof(SwItem), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(pw, 0, 16, s));
  CK(cudaStreamSynchronize(s));  // the host tables must outlive the copies
  h->sweep_phases = pp;
  h->sweep_items = pi;
  h->sweep_y = py;
  h->sweep_ws = (int*)pw;
  h->sweep_trace = (long long*)ptr;
  h->sweep_trace_kinds.clear();
  h->sweep_trace_items.clear();
  if (ptr)
    for (const SwPhase& p : P) {
      h->sweep_trace_kinds.push_back(p.kind);
      h->sweep_trace_items.push_back(p.nitems);
    }
  h->sweep_nph = (int)P.size();
  h->sweep_ctas = nctas;
  h->sweep_smem = smem;
  double fl = 0.0, by = 0.0;
  for (const Phase& ph : R.phases) {
    fl += 2.0 * ph.flops;
    by += 2.0 * ph.bytes;
  }
  h->sweep_flops = fl;
  h->sweep_bytes = by;
  h->sweep_valid = true;
  return SPAND_OK;
}

int ensure_pinned(FactorGroup& G, size_t n) {
  if (n <= G.h_cap) return SPAND_OK;
  if (G.h_ints) cudaFreeHost(G.h_ints);
  G.h_ints = nullptr;
  G.h_cap = 0;
  CK(cudaMallocHost(&G.h_ints, 2 * n * sizeof(int)));
  G.h_cap = 2 * n;
  return SPAND_OK;
}

uint64_t next_layout_id() {
  static std::atomic<uint64_t> counter{0};  // distinct handles may be factored by different threads
  return ++counter;
}

}  // namespace

// ---------------------------------------------------------------------------
// The refactorization chain.  Check-table layout per stage (ints): for every
// problem of the stage: counter offset, cluster count, offset of its expected
// ranks and reflector counts (2 ncl ints) in the chain buffer, offset of its
// flags there.  Status block (4 ints): kind (0 ok, 1 ranks differ, 2
// non-positive Cholesky pivot, 3 a multi-CTA RRQR timed out), stage, problem
// (index in the stage's list), cluster.
// ---------------------------------------------------------------------------
__global__ void k_stage_check(const int* __restrict__ cnt, const int* __restrict__ tab, int nprob,
                              int* __restrict__ buf, int stage, cudaGraphConditionalHandle next,
                              int has_next) {
  __shared__ int s_bad;
  int* status = buf;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  const bool live = *(volatile int*)status == 0;  // an earlier stage failed: compare nothing
  if (live) {
    for (int j = 0; j < nprob; ++j) {
      const int ioff = tab[4 * j], ncl = tab[4 * j + 1], eo = tab[4 * j + 2], fo = tab[4 * j + 3];
      const int* c = cnt + ioff;
      for (int i = threadIdx.x; i < 2 * ncl; i += blockDim.x)
        if (c[ncl + i] != buf[eo + i]) s_bad = 1;
      for (int i = threadIdx.x; i < ncl; i += blockDim.x) buf[fo + i] = c[3 * ncl + i];
      if (threadIdx.x == 0 && status[0] == 0) {
        if (c[4 * ncl + 1] != 0) {
          status[0] = 3;
          status[1] = stage;
          status[2] = j;
        } else if (c[4 * ncl] != 0) {
          status[0] = 2;
          status[1] = stage;
          status[2] = j;
          status[3] = c[4 * ncl] - 1;
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (live && s_bad && status[0] == 0) {
      status[0] = 1;
      status[1] = stage;
    }
    if (has_next) cudaGraphSetConditional(next, status[0] == 0 ? 1u : 0u);
  }
}

int build_chain(FactorGroup& G, cudaStream_t s) {
  const size_t ns = G.sg.size();
  // host image of the chain buffer: status, tables, expected ranks, flags
  std::vector<int> img(4, 0);
  std::vector<size_t> toff(ns);
  std::vector<int> nprob(ns);
  G.chain_foff.assign(ns, {});
  std::vector<std::vector<size_t>> eoff(ns);
  for (size_t k = 0; k < ns; ++k) {
    const auto& g = G.sg[k];
    nprob[k] = (int)g.who.size();
    toff[k] = img.size();
    img.resize(img.size() + 4 * g.who.size(), 0);
  }
  for (size_t k = 0; k < ns; ++k) {
    const auto& g = G.sg[k];
    size_t e = 0;
    for (size_t j = 0; j < g.who.size(); ++j) {
      const int ncl = g.ncl[j];
      eoff[k].push_back(img.size());
      img.insert(img.end(), g.expect.begin() + e, g.expect.begin() + e + 2 * (size_t)ncl);
      e += 2 * (size_t)ncl;
    }
  }
  G.chain_flags = img.size();
  for (size_t k = 0; k < ns; ++k) {
    const auto& g = G.sg[k];
    for (size_t j = 0; j < g.who.size(); ++j) {
      G.chain_foff[k].push_back(img.size());
      img.resize(img.size() + g.ncl[j], 0);
    }
  }
  for (size_t k = 0; k < ns; ++k)
    for (size_t j = 0; j < G.sg[k].who.size(); ++j) {
      int* t = img.data() + toff[k] + 4 * j;
      t[0] = (int)G.sg[k].ioff[j];
      t[1] = G.sg[k].ncl[j];
      t[2] = (int)eoff[k][j];
      t[3] = (int)G.chain_foff[k][j];
    }
  G.chain_ints = img.size();
  RET(G.chain_buf.ensure(img.size() * sizeof(int)));
  int* D = (int*)G.chain_buf.p;
  CK(cudaMemcpyAsync(D, img.data(), img.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));

  cudaGraph_t chain = nullptr;
  CK(cudaGraphCreate(&chain, 0));
  auto fail_out = [&](cudaError_t e) {
    cudaGraphDestroy(chain);
    return fail(SPAND_ECUDA, std::string("building the refactorization chain: ") + cudaGetErrorString(e));
  };
  cudaGraphNode_t prev = nullptr;
  {
    cudaMemsetParams mp = {};
    mp.dst = D;
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = 4;
    mp.height = 1;
    const cudaError_t e = cudaGraphAddMemsetNode(&prev, chain, nullptr, 0, &mp);
    if (e != cudaSuccess) return fail_out(e);
  }
  cudaGraphConditionalHandle next = 0;
  for (size_t k = 0; k < ns; ++k) {
    const auto& g = G.sg[k];
    cudaGraph_t body = chain;
    if (k > 0) {  // enabled by the previous stage's check
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = next;
      cp.conditional.type = cudaGraphCondTypeIf;
      cp.conditional.size = 1;
      cudaGraphNode_t cn = nullptr;
      const cudaError_t e = cudaGraphAddNode(&cn, chain, &prev, nullptr, 1, &cp);
      if (e != cudaSuccess) return fail_out(e);
      body = cp.conditional.phGraph_out[0];
      prev = cn;
    }
    if (g.graph) {
      cudaGraphNode_t child = nullptr;
      const cudaError_t e = cudaGraphAddChildGraphNode(&child, body, k > 0 ? nullptr : &prev,
                                                       k > 0 ? 0 : 1, g.graph);
      if (e != cudaSuccess) return fail_out(e);
      if (k == 0) prev = child;
    }
    if (k + 1 < ns) {
      cudaError_t e = cudaGraphConditionalHandleCreate(&next, chain, 0, cudaGraphCondAssignDefault);
      if (e != cudaSuccess) return fail_out(e);
      const int* cnt = (const int*)G.ints.p;
      const int* tab = D + toff[k];
      int np = nprob[k];
      int* buf = D;
      int stage = (int)k;
      int has_next = 1;
      void* args[] = {(void*)&cnt, (void*)&tab, (void*)&np, (void*)&buf, (void*)&stage, (void*)&next,
                      (void*)&has_next};
      cudaKernelNodeParams kp = {};
      kp.func = (void*)k_stage_check;
      kp.gridDim = dim3(1);
      kp.blockDim = dim3(256);
      kp.sharedMemBytes = 0;
      kp.kernelParams = args;
      cudaGraphNode_t kn = nullptr;
      e = cudaGraphAddKernelNode(&kn, chain, &prev, 1, &kp);
      if (e != cudaSuccess) return fail_out(e);
      prev = kn;
    }
  }
  const cudaError_t ie = cudaGraphInstantiate(&G.chain, chain, 0);
  cudaGraphDestroy(chain);
  if (ie != cudaSuccess) {
    G.chain = nullptr;
    return fail(SPAND_ECUDA, std::string("instantiating the refactorization chain: ") + cudaGetErrorString(ie));
  }
  CK(cudaGraphUpload(G.chain, s));  // the device-side setup now, not in the first launch
  return SPAND_OK;
}

// One launch of the chain, one readback of its status and flags.
int chain_replay(spand_s* const* hs, FactorGroup& G, cudaStream_t s) {
  CK(cudaGraphLaunch(G.chain, s));
  RET(ensure_pinned(G, G.chain_ints));
  int* hp = G.h_ints;
  CK(cudaMemcpyAsync(hp, G.chain_buf.p, G.chain_ints * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const int kind = hp[0], stage = hp[1];
  if (kind == 1) return 1;  // other ranks: the caller rebuilds
  if (kind == 3)
    return fail(SPAND_ETIMEOUT, "a multi-CTA RRQR timed out waiting for its CTAs (stage " +
                                    std::to_string(stage) + ")");
  if (kind == 2)
    return fail(SPAND_ENOTSPD, "non-positive Cholesky pivot in problem " +
                                   std::to_string(G.sg[stage].who[hp[2]]) + " at stage " +
                                   std::to_string(stage) + ", cluster " + std::to_string(hp[3]));
  for (size_t k = 0; k < G.sg.size(); ++k) {
    const auto& g = G.sg[k];
    for (size_t j = 0; j < g.who.size(); ++j) {
      const int* f = hp + G.chain_foff[k][j];
      hs[g.who[j]]->flags[k].assign(f, f + g.ncl[j]);
    }
  }
  return SPAND_OK;
}

// Replays the stage graphs of the group's previous factorization; returns 1 if
// a stage produced other ranks than the ones the graphs were built with (the
// caller then rebuilds), SPAND_OK on success, or an error code.
int factor_replay(spand_s* const* hs, int count, FactorGroup& G, cudaStream_t s) {
  // the stage graphs chained into one graph; if that fails, replay falls back
  // to launching the stage graphs one by one
  if (!G.chain && !G.chain_failed && build_chain(G, s) != SPAND_OK) {
    cudaGetLastError();
    G.chain_failed = true;
  }
  if (G.chain) return chain_replay(hs, G, s);
  for (size_t k = 0; k < G.sg.size(); ++k) {
    auto& g = G.sg[k];
    if (g.exec) CK(cudaGraphLaunch(g.exec, s));
    if (g.nints == 0) continue;
    RET(ensure_pinned(G, g.nints));
    int* hp = G.h_ints;
    CK(cudaMemcpyAsync(hp, G.ints.p, g.nints * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    size_t e = 0;
    for (size_t j = 0; j < g.who.size(); ++j) {
      const int ncl = g.ncl[j];
      const int* c = hp + g.ioff[j];
      if (c[4 * ncl + 1] != 0)
        return fail(SPAND_ETIMEOUT, "a multi-CTA RRQR timed out waiting for its CTAs (stage " +
                                     std::to_string(k) + ")");
      if (c[4 * ncl] != 0)
        return fail(SPAND_ENOTSPD, "non-positive Cholesky pivot in problem " +
                                       std::to_string(g.who[j]) + " at stage " + std::to_string(k) +
                                       ", cluster " + std::to_string(c[4 * ncl] - 1));
      if (!std::equal(c + ncl, c + 3 * ncl, g.expect.begin() + e)) return 1;
      e += 2 * (size_t)ncl;
    }
    for (size_t j = 0; j < g.who.size(); ++j) {
      const int ncl = g.ncl[j];
      const int* c = hp + g.ioff[j];
      hs[g.who[j]]->flags[k].assign(c + 3 * ncl, c + 4 * ncl);
    }
  }
  CK(cudaStreamSynchronize(s));
  return SPAND_OK;
}

int factor_group(spand_s* const* hs, int count, FactorGroup& G, Prof& P, cudaStream_t s) {
  auto t0 = std::chrono::steady_clock::now();
  if (count <= 0) return SPAND_OK;
  const int precision = sizeof(real_t) == 4 ? 1 : 0;
  bool no_graph = false;
  for (int i = 0; i < count; ++i) {
    RET(ensure_device(hs[i]));
    no_graph = no_graph || hs[i]->no_graph;
  }
  auto stamp = [&]() {
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    for (int i = 0; i < count; ++i) hs[i]->factor_ms = ms;
  };
  bool replay = G.valid && G.prec == precision && !P.on && (int)G.layouts.size() == count;
  for (int i = 0; replay && i < count; ++i)
    replay = hs[i]->factored && hs[i]->layout_id == G.layouts[i];
  if (replay) {
    const int rc = factor_replay(hs, count, G, s);
    if (rc == SPAND_OK) {
      stamp();
      return SPAND_OK;
    }
    if (rc != 1) {
      for (int i = 0; i < count; ++i) hs[i]->factored = false;
      return rc;
    }
  }
  // full factorization; stage graphs are (re)built unless profiling is on
  G.drop();
  const bool capture = !P.on && !no_graph;
  if (capture && !G.cap_stream) CK(cudaStreamCreateWithFlags(&G.cap_stream, cudaStreamNonBlocking));
  if (!G.side) {
    CK(cudaStreamCreateWithFlags(&G.side, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&G.ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&G.ev_join, cudaEventDisableTiming));
  }
  G.prec = precision;
  int maxell = 0;
  std::vector<Run> runs(count);
  for (int i = 0; i < count; ++i) {
    spand_s* h = hs[i];
    h->drop_graphs();  // its own graphs and its apply graph point into the old layout
    h->factored = false;
    h->farena.reset();
    h->launches = 0;
    h->layout_id = next_layout_id();
    const int ell = h->nlevels;
    h->sizes.assign(ell, {});
    h->ranks.assign(ell, {});
    h->nrefs.assign(ell, {});
    h->flags.assign(ell, {});
    runs[i].h = h;
    runs[i].ell = ell;
    runs[i].L.resize(ell);
    maxell = std::max(maxell, ell);
  }
  // device counters: room for the widest stage
  size_t nints_max = 16;
  for (int k = 0; k < maxell; ++k) {
    size_t c = 0;
    for (int i = 0; i < count; ++i)
      if (k < runs[i].ell) c += counters_of(hs[i]->st[k].ncl);
    nints_max = std::max(nints_max, c);
  }
  RET(G.ints.ensure(nints_max * sizeof(int)));
  RET(ensure_pinned(G, nints_max));
  int* dcnt = (int*)G.ints.p;
  if (capture) G.sg.resize(maxell + 1);
  int64_t launches = 0;

  using clk = std::chrono::steady_clock;
  auto ms_since = [](clk::time_point a) {
    return std::chrono::duration<double, std::milli>(clk::now() - a).count();
  };
  for (int k = 0; k <= maxell; ++k) {
    clk::time_point tk = clk::now();
    double t_plan = 0, t_launch = 0, t_wait = 0;
    StageWork W;
    std::vector<int> who, ncls;
    std::vector<size_t> ioffs;
    size_t ioff = 0;
    for (int i = 0; i < count; ++i) {
      Run& R = runs[i];
      if (k < R.ell) {
        R.ioff = ioff;
        RET(build_stage(R, k, W, dcnt + ioff));
        who.push_back(i);
        ncls.push_back(hs[i]->st[k].ncl);
        ioffs.push_back(ioff);
        ioff += counters_of(hs[i]->st[k].ncl);
      } else if (k == R.ell) {
        take_pending(R, W);  // the operators of the problem's last stage
      }
    }
    Blob blob;
    StageBlob O = pack_blob(W, blob);
    t_plan = ms_since(tk);
    tk = clk::now();
    char* D = nullptr;
    if (capture) {
      auto& g = G.sg[k];
      if (g.cap < blob.h.size() + 16) {
        if (g.d_blob) cudaFree(g.d_blob);
        g.d_blob = nullptr;
        g.cap = 0;
        CK(cudaMalloc(&g.d_blob, blob.h.size() + 16));
        g.cap = blob.h.size() + 16;
      }
      D = g.d_blob;
    } else {
      RET(G.tables.ensure(blob.h.size() + 16));
      D = G.tables.p;
    }
    patch_grid(O, blob, D);
    CK(cudaMemcpyAsync(D, blob.h.data(), O.upload, cudaMemcpyHostToDevice, s));
    // launches go to the capture stream (recorded into the stage graph) or to s
    cudaStream_t cs = s;
    if (capture) {
      for (int i : who) runs[i].used_gen.push_back({hs[i]->scratch[0].gen, hs[i]->scratch[1].gen});
      CK(cudaStreamSynchronize(s));
      CK(cudaStreamBeginCapture(G.cap_stream, cudaStreamCaptureModeThreadLocal));
      cs = G.cap_stream;
    }
    int nl = 0;
    const int lrc = launch_stage(W, O, D, dcnt, P, cs, &nl, G, k);
    if (capture) {
      cudaGraph_t graph = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(G.cap_stream, &graph);
      RET(lrc);
      CK(ce);
      cudaGraphExec_t exec = nullptr;
      const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
      if (ie != cudaSuccess) cudaGraphDestroy(graph);
      CK(ie);
      auto& g = G.sg[k];
      g.exec = exec;
      g.graph = graph;  // kept for the chain of the whole refactorization
      g.who = who;
      g.ncl = ncls;
      g.ioff = ioffs;
      g.nints = ioff;
      g.expect.clear();
      CK(cudaGraphLaunch(exec, s));
    } else {
      RET(lrc);
    }
    launches += nl;
    t_launch = ms_since(tk);
    tk = clk::now();
    if (ioff == 0) continue;
    // ---- read back ranks and the error words (the sync of this stage)
    int* hp = G.h_ints;
    CK(cudaMemcpyAsync(hp, dcnt, ioff * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    t_wait = ms_since(tk);
    tk = clk::now();
    for (size_t j = 0; j < who.size(); ++j) {
      const int* c = hp + ioffs[j];
      if (c[4 * ncls[j] + 1] != 0) {
        for (int i = 0; i < count; ++i) hs[i]->factored = false;
        G.drop();
        return fail(SPAND_ETIMEOUT, "a multi-CTA RRQR timed out waiting for its CTAs (stage " +
                                     std::to_string(k) + ")");
      }
      if (c[4 * ncls[j]] != 0) {
        for (int i = 0; i < count; ++i) hs[i]->factored = false;
        G.drop();
        return fail(SPAND_ENOTSPD, "non-positive Cholesky pivot" +
                                       (count > 1 ? " in problem " + std::to_string(who[j]) : std::string()) +
                                       " at stage " + std::to_string(k) + ", cluster " +
                                       std::to_string(c[4 * ncls[j]] - 1));
      }
    }
    if (P.on) P.resolve();
    for (size_t j = 0; j < who.size(); ++j) {
      const int* c = hp + ioffs[j];
      if (capture) G.sg[k].expect.insert(G.sg[k].expect.end(), c + ncls[j], c + 3 * ncls[j]);
      RET(finish_stage(runs[who[j]], k, c, P));
    }
    if (debug_time())
      fprintf(stderr, "spand time: stage %d plan %.2f launch %.2f wait %.2f finish %.2f ms (%d launches%s)\n",
              k, t_plan, t_launch, t_wait, ms_since(tk), nl, capture ? ", captured" : "");
  }
  CK(cudaStreamSynchronize(s));
  clk::time_point tt = clk::now();
  if (P.on) P.resolve();
  for (int i = 0; i < count; ++i) {
    RET(upload_apply_plan(runs[i], s));
    RET(build_sweep(runs[i], s));
    hs[i]->launches = launches;
    hs[i]->factored = true;
    // the plan of the problem's own apply, so that applying allocates nothing
    ApSeg seg{hs[i], 0};
    RET(plan_multi(&seg, 1, hs[i]->self_ma, s));
  }
  CK(cudaGetLastError());
  if (debug_time()) fprintf(stderr, "spand time: apply plans %.2f ms\n", ms_since(tt));
  G.valid = capture;
  G.layouts.resize(count);
  for (int i = 0; i < count; ++i) {
    G.layouts[i] = hs[i]->layout_id;
    for (const auto& g : runs[i].used_gen)
      if (g.first != hs[i]->scratch[0].gen || g.second != hs[i]->scratch[1].gen) G.valid = false;
  }
  // the stage graphs become one chain at the first refactorization (a one-off
  // factorization never pays for it)
  stamp();
  return SPAND_OK;
}

int factor(spand_s* h, cudaStream_t s) { return factor_group(&h, 1, h->fg, h->prof, s); }

// The apply of one problem: the merged apply over that problem alone (one
// launch per phase; with graphs, the cluster-size groups of a phase run as
// parallel graph branches).
int apply(spand_s* h, const real_t* r, real_t* z, cudaStream_t s) {
  if (r != z)
    h->prof.run(KK_VEC, s, 0.0, 2.0 * sizeof(real_t) * h->n, [&] { launch_copy_real(h->n, r, z, s); });
  if (h->sweep_valid) {  // the whole sweep as one persistent launch
    cudaError_t e = cudaSuccess;
    h->prof.run(KK_AP_SWEEP, s, h->sweep_flops, h->sweep_bytes, [&] {
      e = launch_ap_sweep((const SwPhase*)h->sweep_phases, h->sweep_nph,
                          (const SwItem*)h->sweep_items, (const ApInterior*)h->d_api,
                          (const ApScale*)h->d_aps, (const ApQE*)h->d_apq, z, (real_t*)h->sweep_y,
                          h->sweep_ws, h->sweep_ctas, h->sweep_smem, spand_s::kSweepWait,
                          h->sweep_trace, s);
    });
    if (e != cudaSuccess) return fail(SPAND_ECUDA, std::string("apply sweep launch: ") + cudaGetErrorString(e));
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (h->sweep_trace && cudaStreamIsCapturing(s, &cap) == cudaSuccess &&
        cap == cudaStreamCaptureStatusNone) {
      std::vector<long long> tr(h->sweep_nph + 1, 0);
      if (cudaMemcpyAsync(tr.data(), h->sweep_trace, tr.size() * sizeof(long long), cudaMemcpyDeviceToHost, s) ==
              cudaSuccess &&
          cudaStreamSynchronize(s) == cudaSuccess)
        for (int p = 0; p < h->sweep_nph; ++p)
          fprintf(stderr, "spand sweep: phase %d kind %d items %d cycles %lld\n", p,
                  h->sweep_trace_kinds[p], h->sweep_trace_items[p],
                  p + 1 < h->sweep_nph ? tr[p + 1] - tr[p] : -1ll);
    }
    return SPAND_OK;
  }
  ApSeg seg{h, 0};
  return apply_multi(&seg, 1, z, h->self_ma, h->prof, !h->no_graph, s);
}

// The launch plan of a merged apply (rebuilt when the problems, their
// offsets or their factorizations changed).
int plan_multi(const ApSeg* segs, int nseg, MultiApply& M, cudaStream_t s) {
  bool same = (int)M.key.size() == nseg;
  for (int i = 0; same && i < nseg; ++i)
    same = M.key[i].first == segs[i].h && M.key[i].second == segs[i].zoff &&
           M.layouts[i] == segs[i].h->layout_id;
  if (!same) {
    M.drop();
    M.key.resize(nseg);
    M.layouts.resize(nseg);
    // vectors of one problem at a constant stride form one run (an item with
    // nvec vectors, whose operators are read once for several of them)
    struct Run {
      const spand_s* h;
      int64_t zoff, ldz;
      int nvec;
    };
    std::vector<int> order(nseg);
    for (int i = 0; i < nseg; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      if (segs[a].h != segs[b].h) return segs[a].h < segs[b].h;
      return segs[a].zoff < segs[b].zoff;
    });
    std::vector<Run> runs;
    for (int i : order) {
      const spand_s* h = segs[i].h;
      if (!h->factored) return fail(SPAND_ESTATE, "apply before a successful factorization");
      M.key[i] = {h, segs[i].zoff};
      M.layouts[i] = h->layout_id;
      if (!runs.empty()) {
        Run& q = runs.back();
        const int64_t d = segs[i].zoff - q.zoff;
        if (q.h == h && ((q.nvec == 1 && d >= h->n) || (q.nvec > 1 && d == q.ldz * q.nvec))) {
          if (q.nvec == 1) q.ldz = d;
          ++q.nvec;
          continue;
        }
      }
      runs.push_back({h, segs[i].zoff, (int64_t)h->n, 1});
    }
    struct Ent {
      int stage, kind, colour, K, run;
      size_t phase;
    };
    std::vector<Ent> ents;
    for (int i = 0; i < (int)runs.size(); ++i) {
      const spand_s* h = runs[i].h;
      for (size_t j = 0; j < h->phases.size(); ++j) {
        const Phase& ph = h->phases[j];
        ents.push_back({ph.stage, ph.kind, ph.colour, ph.K, i, j});
      }
    }
    std::stable_sort(ents.begin(), ents.end(), [](const Ent& a, const Ent& b) {
      if (a.stage != b.stage) return a.stage < b.stage;
      if (a.kind != b.kind) return a.kind < b.kind;
      if (a.colour != b.colour) return a.colour < b.colour;
      return a.K < b.K;
    });
    std::vector<ApItem> items;
    M.launches.clear();
    for (size_t e = 0; e < ents.size();) {
      MultiApply::Launch L{};
      const Ent& h0 = ents[e];
      L.kind = h0.kind;
      L.K = h0.K;
      L.stage = h0.stage;
      L.colour = h0.colour;
      L.item0 = items.size();
      for (; e < ents.size() && ents[e].stage == h0.stage && ents[e].kind == h0.kind &&
             ents[e].colour == h0.colour && ents[e].K == h0.K;
           ++e) {
        const Run& ru = runs[ents[e].run];
        const spand_s* h = ru.h;
        const Phase& ph = h->phases[ents[e].phase];
        ApItem item;
        item.ops = nullptr;
        item.zoff = ru.zoff;
        item.ldz = ru.ldz;
        item.nvec = ru.nvec;
        item.pad = 0;
        item.count = ph.end - ph.begin;
        item.first = L.ntasks;
        // the descriptor base is the handle's table for the phase's kind
        const char* base = ph.kind == PH_INTERIOR ? (const char*)h->d_api
                           : ph.kind == PH_SCALE  ? (const char*)h->d_aps
                                                  : (const char*)h->d_apq;
        const size_t esz = ph.kind == PH_INTERIOR ? sizeof(ApInterior)
                           : ph.kind == PH_SCALE  ? sizeof(ApScale)
                                                  : sizeof(ApQE);
        item.ops = base + (size_t)ph.begin * esz;
        items.push_back(item);
        L.ntasks += item.count;
        L.max_m = std::max(L.max_m, ph.max_m);
        L.max_cols = std::max(L.max_cols, ph.max_cols);
        L.max_nvec = std::max(L.max_nvec, ru.nvec);
        L.flops += ph.flops * ru.nvec;
        L.bytes += ph.bytes * ((ru.nvec + 3) / 4);  // operators read once per pass of <= 4 vectors
      }
      L.nitems = (int)(items.size() - L.item0);
      M.launches.push_back(L);
    }
    RET(M.items.ensure(std::max<size_t>(items.size() * sizeof(ApItem), 16)));
    if (!items.empty())
      CK(cudaMemcpyAsync(M.items.p, items.data(), items.size() * sizeof(ApItem),
                         cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));  // the host table must outlive the copy
  }
  return SPAND_OK;
}

// Merged apply over several problems (see apply_multi in spand_handle.h).
int apply_multi(const ApSeg* segs, int nseg, real_t* z, MultiApply& M, Prof& P, bool graph,
                cudaStream_t s) {
  RET(plan_multi(segs, nseg, M, s));
  const ApItem* items = (const ApItem*)M.items.p;
  auto one = [&](const MultiApply::Launch& L, bool fwd, cudaStream_t cs) {
    const int kind = L.kind == PH_INTERIOR ? KK_AP_INTERIOR : L.kind == PH_SCALE ? KK_AP_SCALE : KK_AP_QE;
    P.tag = (fwd ? 0 : 10000) + L.stage * 100 + L.K;
    P.run(kind, cs, L.flops, L.bytes, [&] {
      const ApItem* it = items + L.item0;
      if (L.kind == PH_INTERIOR)
        launch_ap_interior(it, L.nitems, L.ntasks, L.K, L.max_m, L.max_cols, L.max_nvec, z, fwd, cs);
      else if (L.kind == PH_SCALE)
        launch_ap_scale(it, L.nitems, L.ntasks, L.K, L.max_m, L.max_nvec, z, fwd, cs);
      else launch_ap_qe(it, L.nitems, L.ntasks, L.K, L.max_m, L.max_cols, L.max_nvec, z, fwd, cs);
    });
  };
  // groups of consecutive launches with equal (stage, kind, colour): independent
  std::vector<std::pair<size_t, size_t>> groups;
  for (size_t i = 0; i < M.launches.size();) {
    size_t j = i + 1;
    const auto& a = M.launches[i];
    while (j < M.launches.size() && M.launches[j].stage == a.stage && M.launches[j].kind == a.kind &&
           M.launches[j].colour == a.colour)
      ++j;
    groups.push_back({i, j});
    i = j;
  }
  auto launch_all = [&](cudaStream_t cs, bool forked) {
    auto group = [&](size_t b, size_t e, bool fwd) {
      if (!forked || e - b == 1) {
        for (size_t i = b; i < e; ++i) one(M.launches[i], fwd, cs);
        return;
      }
      cudaEventRecord(M.fork, cs);
      const int nb = (int)std::min<size_t>(e - b, MultiApply::kSide);
      for (int q = 0; q < nb; ++q) cudaStreamWaitEvent(M.side[q], M.fork, 0);
      for (size_t i = b; i < e; ++i) one(M.launches[i], fwd, M.side[(i - b) % MultiApply::kSide]);
      for (int q = 0; q < nb; ++q) {
        cudaEventRecord(M.join[q], M.side[q]);
        cudaStreamWaitEvent(cs, M.join[q], 0);
      }
    };
    for (const auto& g : groups) group(g.first, g.second, true);
    for (auto it = groups.rbegin(); it != groups.rend(); ++it) group(it->first, it->second, false);
  };
  if (!graph || P.on) {
    launch_all(s, false);
    CK(cudaGetLastError());
    return SPAND_OK;
  }
  if (!M.fork) {
    CK(cudaEventCreateWithFlags(&M.fork, cudaEventDisableTiming));
    for (int q = 0; q < MultiApply::kSide; ++q) {
      CK(cudaStreamCreateWithFlags(&M.side[q], cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&M.join[q], cudaEventDisableTiming));
    }
  }
  if (!(M.exec && M.gz == (const void*)z)) {
    if (M.exec) cudaGraphExecDestroy(M.exec);
    M.exec = nullptr;
    if (!M.cap_stream) CK(cudaStreamCreateWithFlags(&M.cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(M.cap_stream, cudaStreamCaptureModeThreadLocal));
    launch_all(M.cap_stream, true);
    cudaGraph_t g = nullptr;
    const cudaError_t le = cudaGetLastError();
    const cudaError_t ce = cudaStreamEndCapture(M.cap_stream, &g);
    CK(le);
    CK(ce);
    const cudaError_t ie = cudaGraphInstantiate(&M.exec, g, 0);
    cudaGraphDestroy(g);
    CK(ie);
    M.gz = z;
  }
  CK(cudaGraphLaunch(M.exec, s));
  return SPAND_OK;
}

}  // namespace SPAND_NS
}  // namespace spand
