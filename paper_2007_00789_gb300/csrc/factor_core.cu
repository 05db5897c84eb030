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
#include "spand_handle.h"
#include "spand_real.h"

namespace spand {
namespace SPAND_NS {

namespace {

struct ApInteriorP {
  const real_t* Linv;
  const real_t* WT;
  int64_t slots, wslots;
  int m, ncols;
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
double potrf_flops(const std::vector<PotrfTask>& v) {
  double f = 0.0;
  for (auto& t : v) f += (double)t.m * t.m * t.m / 3.0;
  return f;
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
                double* flops, double* bytes) {
  double f = 0.0, b = 0.0;
  for (auto& t : tiles) {
    const bool diag = (t.mirror == nullptr);
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
      st.diag.push_back({dg, b, t.ld, t.id, 0});
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
};

// Whether a cluster of cs CTAs with the largest shared-memory slice can be resident.
bool cluster_ok(spand_s* h, int cs) {
  if (h->rrqr_path == 1) return false;
  int lc = 0;
  while ((1 << lc) < cs) ++lc;
  int& st = h->cluster_state[sizeof(real_t) == 4 ? 1 : 0][lc];
  if (st < 0) st = rrqr_cluster_active(cs, kQrClusterSmem) > 0 ? 1 : 0;
  return st == 1;
}

}  // namespace

// Replays the stage graphs of the previous factorization; returns 1 if a
// stage produced other ranks than the ones the graphs were built with (the
// caller then rebuilds), SPAND_OK on success, or an error code.
int factor_replay(spand_s* h, cudaStream_t s) {
  const int ell = h->nlevels;
  CK(cudaMemsetAsync(h->d_err, 0, 2 * sizeof(int), s));
  for (int k = 0; k <= ell; ++k) {
    auto& g = h->sgraph[k];
    if (g.exec) CK(cudaGraphLaunch(g.exec, s));
    if (k == ell) break;
    int* hp = h->h_pinned;
    const int ncl = g.ncl;
    CK(cudaMemcpyAsync(hp, g.d_blob + g.o_rank, ncl * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hp + ncl, g.d_blob + g.o_nref, ncl * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hp + 2 * ncl, g.d_blob + g.o_flag, ncl * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hp + 3 * ncl, h->d_err, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hp[3 * ncl] != 0)
      return fail(SPAND_ENOTSPD, "non-positive Cholesky pivot at stage " + std::to_string(k) +
                                     ", cluster " + std::to_string(hp[3 * ncl] - 1));
    if (!std::equal(g.ranks.begin(), g.ranks.end(), hp) ||
        !std::equal(g.nrefs.begin(), g.nrefs.end(), hp + ncl))
      return 1;
    h->flags[k].assign(hp + 2 * ncl, hp + 3 * ncl);
  }
  CK(cudaStreamSynchronize(s));
  return SPAND_OK;
}

int factor(spand_s* h, cudaStream_t s) {
  auto t0 = std::chrono::steady_clock::now();
  RET(ensure_device(h));
  const int precision = sizeof(real_t) == 4 ? 1 : 0;
  if (h->graph_valid && h->graph_prec == precision && !h->prof.on && h->factored) {
    const int rc = factor_replay(h, s);
    if (rc == SPAND_OK) {
      h->factor_ms =
          std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      return SPAND_OK;
    }
    if (rc != 1) {
      h->factored = false;
      return rc;
    }
  }
  // full factorization; stage graphs are (re)built unless profiling is on
  h->drop_graphs();
  const bool capture = !h->prof.on;
  if (capture && !h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  if (capture) h->sgraph.resize(h->nlevels + 1);
  h->graph_prec = precision;
  h->factored = false;
  h->farena.reset();
  h->launches = 0;
  // scratch generations seen by each stage's graph; a later reallocation of a
  // buffer that an earlier graph uses leaves that graph pointing at freed memory
  std::vector<std::pair<int, int>> used_gen;
  const int ell = h->nlevels;
  std::vector<StageLayout> L(ell);
  std::vector<int> pool;  // slot pool (vector positions), uploaded at the end
  std::vector<ApInteriorP> api;
  std::vector<ApScaleP> aps;
  std::vector<ApQEP> apq;
  std::vector<Phase> phases;
  h->sizes.assign(ell, {});
  h->ranks.assign(ell, {});
  h->nrefs.assign(ell, {});
  h->flags.assign(ell, {});
  int64_t nnzf = 0;
  CK(cudaMemsetAsync(h->d_err, 0, 2 * sizeof(int), s));
  // work of the previous stage that runs with the next stage's launches:
  // E-tilde compaction and the explicit apply operators L^{-1}, Z^{-1}, Q^T
  std::vector<CopyTask> pending_e;
  std::vector<TrsmTask> pending_inv;
  std::vector<FormQtTask> pending_qt;
  int pending_inv_m = 0, pending_qt_m = 0;

  for (int k = 0; k < ell; ++k) {
    const StageSym& S = h->st[k];
    StageLayout& Ly = L[k];
    const int ncl = S.ncl;
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
      const StageLayout& Lp = L[k - 1];
      for (int c = 0; c < ncl; ++c) {
        Ly.slot_off[c] = (int64_t)pool.size();
        int m = 0;
        for (int p : S.children[c]) {
          const int live = P.sparsify ? h->ranks[k - 1][p] : Lp.m[p];
          for (int i = 0; i < live; ++i) pool.push_back(pool[Lp.slot_off[p] + i]);
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
    auto segc = [&](int c, int d) { return segcol_of(S.rowsegs[c], Ly.segcol[c], d); };

    // ---- task tables
    Blob blob;
    std::vector<CopyTask> merge;
    if (k > 0) {
      const StageSym& P = h->st[k - 1];
      const StageLayout& Lp = L[k - 1];
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
          push_copy(merge, src, dst, Lp.m[p], Ly.m[Pc], lp, lq, 0);
        }
      }
    }
    // interiors
    std::vector<PotrfTask> potrf_int;
    std::vector<TrsmTask> trsm_int;
    int max_m_int = 0;
    for (int sidx : S.interiors) {
      const int m = Ly.m[sidx];
      max_m_int = std::max(max_m_int, m);
      const int dc = segc(sidx, sidx);
      potrf_int.push_back({Ly.row[sidx] + (size_t)dc * m, m, m, sidx, 0});
      push_trsm(trsm_int, Ly.row[sidx] + (size_t)dc * m, m, Ly.row[sidx], m, m, dc, 0);
      push_trsm(trsm_int, Ly.row[sidx] + (size_t)dc * m, m, Ly.row[sidx] + (size_t)(dc + m) * m, m,
                m, Ly.ncols[sidx] - dc - m, 0);
    }
    std::vector<SchurTile> tiles;
    std::vector<SchurContrib> contribs;
    for (size_t tg = 0; tg < S.schur_q.size(); ++tg) {
      const int q = S.schur_q[tg], r = S.schur_r[tg];
      const int mq = Ly.m[q], mr = Ly.m[r];
      if (mq == 0 || mr == 0) continue;
      const int cb = (int)contribs.size();
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
        contribs.push_back(c);
      }
      const int ce = (int)contribs.size();
      if (ce == cb) continue;
      real_t* blk = Ly.row[q] + (size_t)segc(q, r) * mq;
      real_t* mir = (q != r) ? Ly.row[r] + (size_t)segc(r, q) * mr : nullptr;
      for (int i0 = 0; i0 < mq; i0 += 32)
        for (int j0 = 0; j0 < mr; j0 += 32) {
          if (q == r && j0 > i0) continue;
          SchurTile t;
          t.dst = blk + i0 + (size_t)j0 * mq;
          t.ld = mq;
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
          t.rows = std::min(32, mq - i0);
          t.cols = std::min(32, mr - j0);
          t.cbegin = cb;
          t.cend = ce;
          t.i0 = i0;
          t.j0 = j0;
          tiles.push_back(t);
        }
    }
    // interfaces: scaling and sparsification
    std::vector<CopyTask> zcopy, mirror;
    std::vector<PotrfTask> zpotrf, ident;
    std::vector<TrsmTask> ltrsm, rtrsm;
    std::vector<std::vector<RRQRTask>> qr_tasks;
    std::vector<RRQRSeg> qr_segs;
    std::vector<int> qr_max_m, qr_max_cols, qr_max_segs, qr_csize, qr_smem;
    int max_m_if = 0;
    Ly.Z.assign(ncl, nullptr);
    Ly.V.assign(ncl, nullptr);
    Ly.tau.assign(ncl, nullptr);
    Ly.maxref.assign(ncl, 0);
    Ly.ncols_ub.assign(ncl, 0);
    if (S.sparsify) {
      for (int p : S.ifaces) {
        const int m = Ly.m[p];
        max_m_if = std::max(max_m_if, m);
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
        push_copy(zcopy, Ly.row[p] + (size_t)dc * m, Ly.Z[p], m, m, m, m, 0);
        zpotrf.push_back({Ly.Z[p], m, m, p, 0});
        push_trsm(ltrsm, Ly.Z[p], m, Ly.row[p], m, m, dc, 0);
        const auto& rs = S.rowsegs[p];
        for (size_t i = 0; i < rs.size(); ++i) {
          const int q = rs[i];
          if (q >= p) break;
          const int mq = Ly.m[q];
          real_t* B = Ly.row[p] + (size_t)Ly.segcol[p][i] * m;
          push_trsm(rtrsm, Ly.Z[q], mq, B, mq, m, m, 1);
          push_copy(mirror, B, Ly.row[q] + (size_t)segc(q, p) * mq, m, mq, mq, m, 1);
        }
        ident.push_back({Ly.row[p] + (size_t)dc * m, m, m, p, 0});
      }
      // one bucket per (colour, cluster size); cluster size 0 = the global-memory kernel
      for (int col = 0; col < S.ncolours; ++col) {
        std::vector<RRQRTask> bucket[6];
        int bm[6] = {0}, bc[6] = {0}, bs[6] = {0}, bsm[6] = {0};
        for (int p : S.by_colour[col]) {
          const int m = Ly.m[p];
          RRQRTask t;
          t.A = Ly.row[p];
          t.ld = m;
          t.m = m;
          t.diag = Ly.row[p] + (size_t)segc(p, p) * m;
          t.V = Ly.V[p];
          t.tau = Ly.tau[p];
          t.id = p;
          t.maxref = Ly.maxref[p];
          t.ncols_max = Ly.ncols_ub[p];
          t.seg_begin = (int)qr_segs.size();
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
            qr_segs.push_back(g);
          }
          t.seg_end = (int)qr_segs.size();
          t.nseg_max = t.seg_end - t.seg_begin;
          // Cluster size: the smallest that fits shared memory, raised until the
          // colour's interfaces fill about two CTAs per SM, while keeping at least
          // 32 columns per CTA.
          const int ntask = (int)S.by_colour[col].size();
          int want = 1;
          while (want < 16 && want * ntask < 2 * kNumSMs && (2 * want) * 32 <= t.ncols_max) want *= 2;
          int b = 0;  // bucket: 1..5 for cluster sizes 1, 2, 4, 8, 16; 0 = fallback
          for (int lc = 0; lc <= 4; ++lc) {
            const int cs = 1 << lc;
            const int bytes = rrqr_cluster_smem_bytes(m, t.ncols_max, t.nseg_max, cs);
            if (bytes <= kQrClusterSmem && cluster_ok(h, cs)) {
              int lw = lc;
              while ((1 << lw) < want && lw < 4 && cluster_ok(h, 1 << (lw + 1))) ++lw;
              b = lw + 1;
              bsm[b] = std::max(bsm[b], rrqr_cluster_smem_bytes(m, t.ncols_max, t.nseg_max, 1 << lw));
              break;
            }
          }
          bucket[b].push_back(t);
          bm[b] = std::max(bm[b], m);
          bc[b] = std::max(bc[b], t.ncols_max);
          bs[b] = std::max(bs[b], t.nseg_max);
        }
        for (int b = 0; b < 6; ++b) {
          if (bucket[b].empty()) continue;
          qr_tasks.push_back(bucket[b]);
          qr_csize.push_back(b == 0 ? 0 : 1 << (b - 1));
          qr_max_m.push_back(bm[b]);
          qr_max_cols.push_back(bc[b]);
          qr_max_segs.push_back(bs[b]);
          qr_smem.push_back(bsm[b]);
          if (b == 0 && rrqr_smem_bytes(bm[b], bc[b], bs[b]) > 220 * 1024)
            return fail(SPAND_ENOMEM, "interface block too wide for the RRQR workspace (stage " +
                                          std::to_string(k) + ")");
        }
      }
    }
    std::vector<int> cur_size(Ly.m.begin(), Ly.m.end());
    std::vector<int> rank_init(ncl, -1);

    // ---- upload
    const size_t o_e = blob.add(pending_e);
    const size_t o_inv = blob.add(pending_inv);
    const size_t o_fq = blob.add(pending_qt);
    const size_t o_merge = blob.add(merge);
    PotrfPlan plan_int = plan_potrf(potrf_int);
    plan_to_blob(plan_int, blob);
    PotrfPlan plan_z = plan_potrf(zpotrf);
    plan_to_blob(plan_z, blob);
    const size_t o_ti = blob.add(trsm_int);
    const size_t o_tiles = blob.add(tiles);
    const size_t o_contr = blob.add(contribs);
    const size_t o_zc = blob.add(zcopy);

    const size_t o_lt = blob.add(ltrsm);
    const size_t o_rt = blob.add(rtrsm);
    const size_t o_mi = blob.add(mirror);
    const size_t o_id = blob.add(ident);
    std::vector<size_t> o_qr(qr_tasks.size());
    for (size_t c = 0; c < qr_tasks.size(); ++c) o_qr[c] = blob.add(qr_tasks[c]);
    const size_t o_seg = blob.add(qr_segs);
    const size_t o_cur = blob.add(cur_size);
    const size_t o_cur0 = blob.add(cur_size);
    const size_t o_rank = blob.add(rank_init);
    const size_t o_nref = blob.add(rank_init);
    const size_t o_flag = blob.add(rank_init);
    char* D = nullptr;
    if (capture) {
      auto& g = h->sgraph[k];
      if (g.cap < blob.h.size() + 16) {
        if (g.d_blob) cudaFree(g.d_blob);
        g.d_blob = nullptr;
        g.cap = 0;
        CK(cudaMalloc(&g.d_blob, blob.h.size() + 16));
        g.cap = blob.h.size() + 16;
      }
      D = g.d_blob;
    } else {
      RET(h->tables.ensure(blob.h.size() + 16));
      D = h->tables.p;
    }
    CK(cudaMemcpyAsync(D, blob.h.data(), blob.h.size(), cudaMemcpyHostToDevice, s));
    // launches go to the capture stream (recorded into the stage graph) or to s
    cudaStream_t cs = s;
    if (capture) {
      used_gen.push_back({h->scratch[0].gen, h->scratch[1].gen});
      CK(cudaStreamSynchronize(s));
      CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
      cs = h->cap_stream;
      // the RRQR kernels shrink the widths in place: start from the pristine copy
      CK(cudaMemcpyAsync(D + o_cur, D + o_cur0, cur_size.size() * sizeof(int),
                         cudaMemcpyDeviceToDevice, cs));
    }

    // ---- kernels
    int nl = 0;
    Prof& P = h->prof;
    auto run = [&](int kind, size_t ntasks, double flops, double bytes, auto&& launch) {
      if (ntasks == 0) return;
      ++nl;
      P.run(kind, cs, flops, bytes, launch);
    };
    run(KK_ECOPY, pending_e.size(), 0.0, copy_bytes(pending_e),
        [&] { launch_copy((const CopyTask*)(D + o_e), (int)pending_e.size(), cs); });
    run(KK_TRTRI, pending_inv.size(), trtri_flops(pending_inv), trsm_bytes(pending_inv), [&] {
      launch_trsm((const TrsmTask*)(D + o_inv), (int)pending_inv.size(), pending_inv_m, cs);
    });
    run(KK_FORMQ, pending_qt.size(), formqt_flops(pending_qt), 0.0, [&] {
      launch_form_qt((const FormQtTask*)(D + o_fq), (int)pending_qt.size(), pending_qt_m, cs);
    });
    if (fbytes) CK(cudaMemsetAsync(fptr, 0, fbytes, cs));
    if (sbytes) CK(cudaMemsetAsync(scr.p, 0, sbytes, cs));
    if (k == 0) {
      run(KK_PACK, 1, 0.0, 16.0 * h->nnz, [&] {
        launch_scatter(h->d_val, h->d_pack, (real_t*)fptr, (real_t*)scr.p, h->pack_split, h->nnz, cs);
      });
    } else {
      run(KK_MERGE, merge.size(), 0.0, copy_bytes(merge),
          [&] { launch_copy((const CopyTask*)(D + o_merge), (int)merge.size(), cs); });
    }
    auto run_potrf = [&](int kind, PotrfPlan& PP) {
      bool first = true;
      auto fl = [&]() { double f = first ? PP.flops : 0.0; first = false; return f; };
      run(kind, PP.small.size(), fl(), PP.bytes, [&] {
        launch_potrf((const PotrfTask*)(D + PP.o_small), (int)PP.small.size(), PP.small_max, h->d_err, cs);
      });
      for (auto& st : PP.steps) {
        run(kind, st.diag.size(), fl(), 0.0, [&] {
          launch_potrf((const PotrfTask*)(D + st.o_diag), (int)st.diag.size(), kPanel, h->d_err, cs);
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
    run_potrf(KK_POTRF, plan_int);
    run(KK_TRSM, trsm_int.size(), trsm_flops(trsm_int), trsm_bytes(trsm_int),
        [&] { launch_trsm((const TrsmTask*)(D + o_ti), (int)trsm_int.size(), max_m_int, cs); });
    {
      double fl = 0.0, by = 0.0;
      schur_work(tiles, contribs, &fl, &by);
      run(KK_SCHUR, tiles.size(), fl, by, [&] {
        launch_schur((const SchurTile*)(D + o_tiles), (int)tiles.size(),
                     (const SchurContrib*)(D + o_contr), cs);
      });
    }
    if (S.sparsify) {
      run(KK_SCALE_COPY, zcopy.size(), 0.0, copy_bytes(zcopy),
          [&] { launch_copy((const CopyTask*)(D + o_zc), (int)zcopy.size(), cs); });
      run_potrf(KK_SCALE_POTRF, plan_z);
      run(KK_SCALE_TRSM, ltrsm.size(), trsm_flops(ltrsm), trsm_bytes(ltrsm),
          [&] { launch_trsm((const TrsmTask*)(D + o_lt), (int)ltrsm.size(), max_m_if, cs); });
      run(KK_SCALE_TRSM, rtrsm.size(), trsm_flops(rtrsm), trsm_bytes(rtrsm),
          [&] { launch_trsm((const TrsmTask*)(D + o_rt), (int)rtrsm.size(), max_m_if, cs); });
      run(KK_SCALE_COPY, mirror.size(), 0.0, copy_bytes(mirror),
          [&] { launch_copy((const CopyTask*)(D + o_mi), (int)mirror.size(), cs); });
      run(KK_SCALE_COPY, ident.size(), 0.0, potrf_bytes(ident) / 2,
          [&] { launch_set_identity((const PotrfTask*)(D + o_id), (int)ident.size(), cs); });
      for (size_t c = 0; c < qr_tasks.size(); ++c) {
        run(KK_RRQR, qr_tasks[c].size(), 0.0, 0.0, [&] {
          if (qr_csize[c] == 0)
            launch_rrqr((const RRQRTask*)(D + o_qr[c]), (int)qr_tasks[c].size(),
                        (const RRQRSeg*)(D + o_seg), (int*)(D + o_cur), (int*)(D + o_rank),
                        (int*)(D + o_nref), (int*)(D + o_flag), h->eps, h->scheme, qr_max_m[c],
                        qr_max_cols[c], qr_max_segs[c], cs);
          else
            launch_rrqr_cluster((const RRQRTask*)(D + o_qr[c]), (int)qr_tasks[c].size(),
                                (const RRQRSeg*)(D + o_seg), (int*)(D + o_cur), (int*)(D + o_rank),
                                (int*)(D + o_nref), (int*)(D + o_flag), h->eps, h->scheme,
                                qr_csize[c], qr_smem[c], cs);
        });
      }
    }
    CK(cudaGetLastError());
    h->launches += nl;
    if (capture) {
      cudaGraph_t graph = nullptr;
      CK(cudaStreamEndCapture(h->cap_stream, &graph));
      cudaGraphExec_t exec = nullptr;
      const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      CK(ie);
      auto& g = h->sgraph[k];
      g.exec = exec;
      g.o_rank = o_rank;
      g.o_nref = o_nref;
      g.o_flag = o_flag;
      g.ncl = ncl;
      CK(cudaGraphLaunch(exec, s));
    }
    // ---- read back ranks and the error flag (the sync of this stage)
    const size_t need = 3 * (size_t)ncl + 2;
    if (need > h->h_pinned_cap) {
      if (h->h_pinned) cudaFreeHost(h->h_pinned);
      h->h_pinned = nullptr;
      CK(cudaMallocHost(&h->h_pinned, need * 2 * sizeof(int)));
      h->h_pinned_cap = need * 2;
    }
    int* hp = h->h_pinned;
    CK(cudaMemcpyAsync(hp, D + o_rank, ncl * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hp + ncl, D + o_nref, ncl * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hp + 2 * ncl, D + o_flag, ncl * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hp + 3 * ncl, h->d_err, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hp[3 * ncl] != 0) {
      const int cid = hp[3 * ncl] - 1;
      return fail(SPAND_ENOTSPD, "non-positive Cholesky pivot at stage " + std::to_string(k) +
                                     ", cluster " + std::to_string(cid));
    }
    h->ranks[k].assign(hp, hp + ncl);
    h->nrefs[k].assign(hp + ncl, hp + 2 * ncl);
    h->flags[k].assign(hp + 2 * ncl, hp + 3 * ncl);
    if (capture) {
      h->sgraph[k].ranks = h->ranks[k];
      h->sgraph[k].nrefs = h->nrefs[k];
    }
    if (P.on) {
      P.resolve();
      if (S.sparsify) {
        double fl = 0.0, by = 0.0;
        for (int p : S.ifaces) {
          const int m = Ly.m[p], nref = h->nrefs[k][p];
          int N = 0;
          for (int q : S.adj1[p]) N += (S.colour[q] < S.colour[p]) ? h->ranks[k][q] : Ly.m[q];
          for (int t = 0; t < nref; ++t) fl += 6.0 * (double)(m - t) * (double)(N - t);
          by += 16.0 * (double)m * N;  // the block is read and written once
        }
        P.stat[KK_RRQR].flops += fl;
        P.stat[KK_RRQR].bytes += by;
      }
    }

    // ---- apply operators of this stage (explicit inverses and Q^T are formed
    //      by tasks that run with the next stage's launches)
    pending_e.clear();
    pending_inv.clear();
    pending_qt.clear();
    pending_inv_m = pending_qt_m = 0;
    auto explicit_inverse = [&](const real_t* L, int m, real_t** out) -> int {
      void* ip = nullptr;
      RET(h->farena.alloc(std::max<size_t>((size_t)m * m * sizeof(real_t), 16), &ip));
      *out = (real_t*)ip;
      push_trsm(pending_inv, L, m, *out, m, m, m, 0, true);
      pending_inv_m = std::max(pending_inv_m, m);
      return SPAND_OK;
    };
    {
      Phase ph{PH_INTERIOR, (int)api.size(), 0, 0, 0.0, 0.0};
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
        a.slots = Ly.slot_off[sidx];
        a.wslots = (int64_t)pool.size();
        for (int d : S.rowsegs[sidx]) {
          for (int i = 0; i < Ly.m[d]; ++i)
            pool.push_back(d == sidx ? -1 : pool[Ly.slot_off[d] + i]);
        }
        api.push_back(a);
        const double fm = (double)m * (m + 1) / 2 + (double)m * (a.ncols - m);
        Ks.push_back(ap_cluster(fm));
        ms.push_back(m);
        cols.push_back(a.ncols);
        fl.push_back(2.0 * fm);
        by.push_back(8.0 * fm + 24.0 * a.ncols);
        nnzf += (int64_t)m * (m + 1) / 2 + (int64_t)m * (a.ncols - m);
      }
      ph.end = (int)api.size();
      if (ph.end > ph.begin) split_phase(phases, api, ph, Ks, fl, by, ms, cols);
    }
    if (S.sparsify) {
      Phase ph{PH_SCALE, (int)aps.size(), 0, 0, 0.0, 0.0};
      std::vector<int> Ks, ms, cols;
      std::vector<double> fl, by;
      for (int p : S.ifaces) {
        const int m = Ly.m[p];
        real_t* Zinv = nullptr;
        if (m > 0) RET(explicit_inverse(Ly.Z[p], m, &Zinv));
        aps.push_back({Zinv, Ly.slot_off[p], m});
        const double fm = (double)m * (m + 1) / 2;
        Ks.push_back(ap_cluster(fm));
        ms.push_back(m);
        cols.push_back(0);
        fl.push_back(2.0 * fm);
        by.push_back(8.0 * fm + 16.0 * m);
        nnzf += (int64_t)m * (m + 1) / 2;
      }
      ph.end = (int)aps.size();
      if (ph.end > ph.begin) split_phase(phases, aps, ph, Ks, fl, by, ms, cols);
      for (int col = 0; col < S.ncolours; ++col) {
        Phase pq{PH_QE, (int)apq.size(), 0, 0, 0.0, 0.0};
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
              pending_qt.push_back(ft);
            }
            pending_qt_m = std::max(pending_qt_m, m);
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
            for (int j = 0; j < w; ++j) pool.push_back(pool[Ly.slot_off[q] + j]);
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
            for (auto& sw : segw) {
              push_copy(pending_e, Ly.row[p] + r + (size_t)sw.first * m, Edst + (size_t)acc * nE, m,
                        nE, nE, sw.second, 0);
              acc += sw.second;
            }
          } else {
            a.nE = 0;
          }
          apq.push_back(a);
          const double fm = (double)m * m + (double)a.nE * ncols;
          Ks.push_back(ap_cluster(fm));
          ms.push_back(m);
          cols.push_back(a.nE > 0 ? ncols : 0);
          fl.push_back(2.0 * fm);
          by.push_back(8.0 * fm + 16.0 * (m + ncols));
          nnzf += (int64_t)m * nref + nref + (int64_t)a.nE * ncols;
        }
        pq.end = (int)apq.size();
        if (pq.end > pq.begin) split_phase(phases, apq, pq, Ks, fl, by, ms, cols);
      }
    }
  }
  // ---- final upload: E compaction of the last sparsified stage (if any was pending)
  {
    Blob blob;
    const size_t o_e = blob.add(pending_e);
    const size_t o_inv = blob.add(pending_inv);
    const size_t o_fq = blob.add(pending_qt);
    char* D = nullptr;
    if (capture) {
      auto& g = h->sgraph[ell];
      if (g.cap < blob.h.size() + 16) {
        if (g.d_blob) cudaFree(g.d_blob);
        g.d_blob = nullptr;
        g.cap = 0;
        CK(cudaMalloc(&g.d_blob, blob.h.size() + 16));
        g.cap = blob.h.size() + 16;
      }
      D = g.d_blob;
    } else {
      RET(h->tables.ensure(blob.h.size() + 16));
      D = h->tables.p;
    }
    CK(cudaMemcpyAsync(D, blob.h.data(), blob.h.size(), cudaMemcpyHostToDevice, s));
    const bool any = !pending_e.empty() || !pending_inv.empty() || !pending_qt.empty();
    cudaStream_t cs = s;
    if (capture && any) {
      CK(cudaStreamSynchronize(s));
      CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
      cs = h->cap_stream;
    }
    if (!pending_e.empty()) {
      h->prof.run(KK_ECOPY, cs, 0.0, copy_bytes(pending_e), [&] {
        launch_copy((const CopyTask*)(D + o_e), (int)pending_e.size(), cs);
      });
      h->launches += 1;
    }
    if (!pending_inv.empty()) {
      h->prof.run(KK_TRTRI, cs, trtri_flops(pending_inv), trsm_bytes(pending_inv), [&] {
        launch_trsm((const TrsmTask*)(D + o_inv), (int)pending_inv.size(), pending_inv_m, cs);
      });
      h->launches += 1;
    }
    if (!pending_qt.empty()) {
      h->prof.run(KK_FORMQ, cs, formqt_flops(pending_qt), 0.0, [&] {
        launch_form_qt((const FormQtTask*)(D + o_fq), (int)pending_qt.size(), pending_qt_m, cs);
      });
      h->launches += 1;
    }
    if (capture && any) {
      cudaGraph_t graph = nullptr;
      CK(cudaStreamEndCapture(h->cap_stream, &graph));
      cudaGraphExec_t exec = nullptr;
      const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      CK(ie);
      h->sgraph[ell].exec = exec;
      CK(cudaGraphLaunch(exec, s));
    }
  }
  // ---- apply plan: slot pool + descriptors into the factor arena
  void *pp = nullptr, *pa = nullptr, *ps = nullptr, *pq = nullptr;
  RET(h->farena.alloc(std::max<size_t>(pool.size() * 4, 16), &pp));
  RET(h->farena.alloc(std::max<size_t>(api.size() * sizeof(ApInterior), 16), &pa));
  RET(h->farena.alloc(std::max<size_t>(aps.size() * sizeof(ApScale), 16), &ps));
  RET(h->farena.alloc(std::max<size_t>(apq.size() * sizeof(ApQE), 16), &pq));
  const int* dpool = (const int*)pp;
  std::vector<ApInterior> vi(api.size());
  for (size_t i = 0; i < api.size(); ++i)
    vi[i] = {api[i].Linv, api[i].WT, dpool + api[i].slots, dpool + api[i].wslots, api[i].m,
             api[i].ncols};
  std::vector<ApScale> vs(aps.size());
  for (size_t i = 0; i < aps.size(); ++i) vs[i] = {aps[i].Zinv, dpool + aps[i].slots, aps[i].m, 0};
  std::vector<ApQE> vq(apq.size());
  for (size_t i = 0; i < apq.size(); ++i)
    vq[i] = {apq[i].Qt, apq[i].E, dpool + apq[i].slots, dpool + apq[i].eslots, apq[i].m,
             apq[i].r, apq[i].nE, apq[i].ncols};
  if (!pool.empty()) CK(cudaMemcpyAsync(pp, pool.data(), pool.size() * 4, cudaMemcpyHostToDevice, s));
  if (!vi.empty()) CK(cudaMemcpyAsync(pa, vi.data(), vi.size() * sizeof(ApInterior), cudaMemcpyHostToDevice, s));
  if (!vs.empty()) CK(cudaMemcpyAsync(ps, vs.data(), vs.size() * sizeof(ApScale), cudaMemcpyHostToDevice, s));
  if (!vq.empty()) CK(cudaMemcpyAsync(pq, vq.data(), vq.size() * sizeof(ApQE), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  if (h->prof.on) h->prof.resolve();
  h->d_api = pa;
  h->d_aps = ps;
  h->d_apq = pq;
  h->phases = phases;
  h->nnz_factor = nnzf;
  h->factored = true;
  h->graph_valid = capture;
  for (const auto& g : used_gen)
    if (g.first != h->scratch[0].gen || g.second != h->scratch[1].gen) h->graph_valid = false;
  h->factor_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return SPAND_OK;
}

int apply_launches(spand_s* h, const real_t* r, real_t* z, cudaStream_t s);

// The whole apply as one CUDA graph (built on first use for these vectors),
// or as plain launches while profiling.
int apply(spand_s* h, const real_t* r, real_t* z, cudaStream_t s) {
  if (h->prof.on || h->no_graph) return apply_launches(h, r, z, s);
  if (!(h->apply_exec && h->apply_r == (const void*)r && h->apply_z == (void*)z)) {
    if (h->apply_exec) cudaGraphExecDestroy(h->apply_exec);
    h->apply_exec = nullptr;
    if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = apply_launches(h, r, z, h->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &graph);
    RET(rc);
    CK(ce);
    const cudaError_t ie = cudaGraphInstantiate(&h->apply_exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(ie);
    h->apply_r = r;
    h->apply_z = z;
  }
  CK(cudaGraphLaunch(h->apply_exec, s));
  return SPAND_OK;
}

int apply_launches(spand_s* h, const real_t* r, real_t* z, cudaStream_t s) {
  Prof& P = h->prof;
  const int n = h->n;
  if (r != z) P.run(KK_VEC, s, 0.0, 2.0 * sizeof(real_t) * n, [&] { launch_copy_real(n, r, z, s); });
  auto one = [&](const Phase& ph, bool fwd) {
    const int nt = ph.end - ph.begin;
    const int kind = ph.kind == PH_INTERIOR ? KK_AP_INTERIOR : ph.kind == PH_SCALE ? KK_AP_SCALE : KK_AP_QE;
    P.run(kind, s, ph.flops, ph.bytes, [&] {
      if (ph.kind == PH_INTERIOR)
        launch_ap_interior((const ApInterior*)h->d_api + ph.begin, nt, ph.K, ph.max_m, ph.max_cols, z, fwd, s);
      else if (ph.kind == PH_SCALE)
        launch_ap_scale((const ApScale*)h->d_aps + ph.begin, nt, ph.K, ph.max_m, z, fwd, s);
      else launch_ap_qe((const ApQE*)h->d_apq + ph.begin, nt, ph.K, ph.max_m, ph.max_cols, z, fwd, s);
    });
  };
  for (const Phase& ph : h->phases) one(ph, true);
  for (auto it = h->phases.rbegin(); it != h->phases.rend(); ++it) one(*it, false);
  CK(cudaGetLastError());
  return SPAND_OK;
}

}  // namespace SPAND_NS
}  // namespace spand
