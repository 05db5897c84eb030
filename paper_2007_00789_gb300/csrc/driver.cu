// Host orchestration of the spaND factorization, apply and PCG, and the C
// ABI of include/spand.h.
//
// Factorization (Algorithm 2, §3).  Stage k = 0 .. ell-1 of the multilevel
// partition runs as batched kernels on one stream:
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
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "spand_internal.h"

using namespace spand;

static thread_local std::string g_last_error;

static int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define CK(call)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail(e_ == cudaErrorMemoryAllocation ? SPAND_ENOMEM : SPAND_ECUDA,     \
                  std::string(#call) + ": " + cudaGetErrorString(e_));              \
  } while (0)

#define RET(call)                  \
  do {                             \
    int rc_ = (call);              \
    if (rc_ != SPAND_OK) return rc_; \
  } while (0)

namespace {

// Bump allocator over device chunks; pointers stay valid until release().
struct DevArena {
  struct Chunk {
    char* p;
    size_t cap, used;
  };
  std::vector<Chunk> chunks;
  size_t cur = 0;
  size_t min_chunk = size_t(256) << 20;

  int alloc(size_t bytes, void** out) {
    bytes = (bytes + 255) & ~size_t(255);
    while (cur < chunks.size()) {
      Chunk& c = chunks[cur];
      if (c.used + bytes <= c.cap) {
        *out = c.p + c.used;
        c.used += bytes;
        return SPAND_OK;
      }
      ++cur;
    }
    const size_t cap = std::max(bytes, min_chunk);
    char* p = nullptr;
    cudaError_t e = cudaMalloc(&p, cap);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(SPAND_ENOMEM, "device allocation of " + std::to_string(cap) + " bytes failed");
    }
    chunks.push_back({p, cap, bytes});
    cur = chunks.size() - 1;
    *out = p;
    return SPAND_OK;
  }
  void reset() {
    for (auto& c : chunks) c.used = 0;
    cur = 0;
  }
  void release() {
    for (auto& c : chunks) cudaFree(c.p);
    chunks.clear();
    cur = 0;
  }
  size_t held() const {
    size_t s = 0;
    for (auto& c : chunks) s += c.cap;
    return s;
  }
};

// Growable device buffer (contents not preserved on growth).
struct DevBuf {
  char* p = nullptr;
  size_t cap = 0;
  int ensure(size_t bytes) {
    if (bytes <= cap) return SPAND_OK;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    size_t want = std::max(bytes, size_t(1) << 20);
    want = want + want / 4;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(SPAND_ENOMEM, "device allocation of " + std::to_string(want) + " bytes failed");
    }
    cap = want;
    return SPAND_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

// Host staging of one stage's task tables.
struct Blob {
  std::vector<char> h;
  template <class T>
  size_t add(const std::vector<T>& v) {
    size_t off = (h.size() + 15) & ~size_t(15);
    h.resize(off + v.size() * sizeof(T));
    if (!v.empty()) memcpy(h.data() + off, v.data(), v.size() * sizeof(T));
    return off;
  }
  void clear() { h.clear(); }
};

// Per-kernel profiling: CUDA events around every launch group on the caller's
// stream, resolved after the stream is synchronised; algorithmic FLOPs and
// bytes are counted on the host from the task sizes.
enum KernelKind {
  KK_PACK, KK_MERGE, KK_POTRF, KK_TRSM, KK_SCHUR, KK_SCALE_POTRF, KK_SCALE_TRSM, KK_SCALE_COPY,
  KK_RRQR, KK_ECOPY, KK_TRTRI, KK_FORMQ, KK_AP_INTERIOR, KK_AP_SCALE, KK_AP_QE, KK_SPMV, KK_DOT,
  KK_VEC, KK_COUNT
};
const char* const kKindName[KK_COUNT] = {
    "pack", "merge", "potrf", "trsm", "schur", "scale_potrf", "scale_trsm", "scale_copy",
    "rrqr", "e_copy", "trtri", "form_qt", "apply_interior", "apply_scale", "apply_qe", "spmv",
    "dot", "vector"};

struct Prof {
  bool on = false;
  struct Pend {
    int kind;
    cudaEvent_t a, b;
    double flops, bytes;
  };
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<Pend> pend;
  spand_kernel_stat stat[KK_COUNT];
  Prof() { clear(); }
  void clear() {
    for (int k = 0; k < KK_COUNT; ++k) {
      memset(&stat[k], 0, sizeof(stat[k]));
      snprintf(stat[k].name, sizeof(stat[k].name), "%s", kKindName[k]);
    }
  }
  cudaEvent_t ev() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  template <class F>
  void run(int kind, cudaStream_t s, double flops, double bytes, F&& launch) {
    if (!on) {
      launch();
      return;
    }
    Pend p{kind, ev(), ev(), flops, bytes};
    cudaEventRecord(p.a, s);
    launch();
    cudaEventRecord(p.b, s);
    pend.push_back(p);
  }
  void add_flops(int kind, double flops) {
    if (on) stat[kind].flops += flops;
  }
  // call after the stream has been synchronised
  void resolve() {
    for (auto& p : pend) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, p.a, p.b);
      stat[p.kind].launches += 1;
      stat[p.kind].total_ms += ms;
      stat[p.kind].flops += p.flops;
      stat[p.kind].bytes += p.bytes;
    }
    pend.clear();
    used = 0;
  }
  void release() {
    for (auto e : pool) cudaEventDestroy(e);
    pool.clear();
    used = 0;
  }
};

constexpr int kQrClusterSmem = 200 * 1024;  // shared-memory slice per CTA of the on-chip RRQR
constexpr int kNumSMs = 152;                 // GB300

enum PhaseKind { PH_INTERIOR = 0, PH_SCALE = 1, PH_QE = 2 };
struct Phase {
  int kind, begin, end, max_m;
  double flops, bytes;  // algorithmic, forward sweep (the backward one is the same)
  int max_cols = 0;     // widest neighbour gather
  int K = 1;            // CTAs per operator (thread-block cluster)
};

// CTAs per apply operator: enough that each handles about 12k FMAs.
inline int ap_cluster(double fmas) {
  int K = 1;
  while (K < 16 && fmas / K > 12288.0) K *= 2;
  return K;
}

// Split [ph.begin, ph.end) of the descriptor vector v into one phase per
// cluster size; the operators of a phase are independent, so their order
// within the phase is free.
template <class T>
void split_phase(std::vector<Phase>& phases, std::vector<T>& v, const Phase& ph,
                 const std::vector<int>& Ks, const std::vector<double>& fl,
                 const std::vector<double>& by, const std::vector<int>& ms,
                 const std::vector<int>& cols) {
  std::vector<int> order(ph.end - ph.begin);
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return Ks[a] < Ks[b]; });
  std::vector<T> seg(order.size());
  for (size_t i = 0; i < order.size(); ++i) seg[i] = v[ph.begin + order[i]];
  std::copy(seg.begin(), seg.end(), v.begin() + ph.begin);
  size_t i = 0;
  while (i < order.size()) {
    Phase q = ph;
    q.K = Ks[order[i]];
    q.begin = ph.begin + (int)i;
    q.max_m = 0;
    q.max_cols = 0;
    q.flops = q.bytes = 0.0;
    while (i < order.size() && Ks[order[i]] == q.K) {
      q.max_m = std::max(q.max_m, ms[order[i]]);
      q.max_cols = std::max(q.max_cols, cols[order[i]]);
      q.flops += fl[order[i]];
      q.bytes += by[order[i]];
      ++i;
    }
    q.end = ph.begin + (int)i;
    phases.push_back(q);
  }
}

struct ApInteriorP {
  const double* Linv;
  const double* WT;
  int64_t slots, wslots;
  int m, ncols;
};
struct ApScaleP {
  const double* Zinv;
  int64_t slots;
  int m;
};
struct ApQEP {
  const double* Qt;
  const double* E;
  int64_t slots, eslots;
  int m, r, nE, ncols;
};

}  // namespace

struct spand_s {
  int n = 0, dim = 0, nlevels = 0, scheme = 0, skip = 0;
  int64_t nnz = 0;
  double eps = 0.0;
  int maxit = 500, true_every = 50, max_restarts = 2;
  Tree tree;
  std::vector<StageSym> st;
  std::vector<int32_t> h_rowptr, h_colind;
  std::vector<double> h_val;
  // device copy of A
  int32_t* d_rowptr = nullptr;
  int32_t* d_colind = nullptr;
  double* d_val = nullptr;
  int64_t* d_pack = nullptr;     // stage-0 destination of every nonzero
  int64_t pack_split = 0;        // interior part / interface part of the stage-0 layout
  std::vector<int64_t> h_pack;
  // memory
  DevArena farena;
  DevBuf scratch[2];
  DevBuf tables;
  int* d_err = nullptr;
  int* h_pinned = nullptr;       // rank/nref/err readback
  size_t h_pinned_cap = 0;
  // factor results
  bool factored = false;
  std::vector<std::vector<int>> sizes, ranks, nrefs, flags;
  std::vector<Phase> phases;
  ApInterior* d_api = nullptr;
  ApScale* d_aps = nullptr;
  ApQE* d_apq = nullptr;
  int64_t nnz_factor = 0;
  int64_t launches = 0;
  double factor_ms = 0.0;
  // pcg
  double *d_r = nullptr, *d_z = nullptr, *d_p = nullptr, *d_q = nullptr, *d_b = nullptr,
         *d_x = nullptr;
  double* d_scal = nullptr;
  double* d_partial = nullptr;
  double* h_scal = nullptr;
  double pcg_ms = 0.0, pcg_relres = 0.0;
  int pcg_iters = 0;
  Prof prof;
  int rrqr_path = 0;  // 0: choose per interface; 1: always the global-memory kernel
  int cluster_state[5] = {-1, -1, -1, -1, -1};
  // whether a cluster of cs CTAs with the largest shared-memory slice can be resident
  bool cluster_ok(int cs) {
    if (rrqr_path == 1) return false;
    int lc = 0;
    while ((1 << lc) < cs) ++lc;
    if (cluster_state[lc] < 0) cluster_state[lc] = rrqr_cluster_active(cs, kQrClusterSmem) > 0 ? 1 : 0;
    return cluster_state[lc] == 1;
  }
};

namespace {

inline int segcol_of(const std::vector<int>& segs, const std::vector<int>& cols, int d) {
  auto it = std::lower_bound(segs.begin(), segs.end(), d);
  return cols[it - segs.begin()];
}

// Split a copy into column chunks so that large blocks use several CTAs.
void push_copy(std::vector<CopyTask>& v, const double* src, double* dst, int src_ld, int dst_ld,
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
void push_trsm(std::vector<TrsmTask>& v, const double* L, int ldl, double* X, int m, int ldx,
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
      double* dg = t.a + k0 + (size_t)k0 * t.ld;
      st.diag.push_back({dg, b, t.ld, t.id, 0});
      if (below <= 0) continue;
      double* panel = dg + b;
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
      double* trail = panel + (size_t)b * t.ld;
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
  std::vector<double*> row;                // panel row origin
  std::vector<int> ncols;
  std::vector<std::vector<int>> segcol;    // column offset of every block in the row
  std::vector<int64_t> slot_off;           // offset of the cluster's slots in the pool
  std::vector<double*> Z, V, tau;
  std::vector<int> maxref, ncols_ub;       // interfaces: reflector capacity, sum of widths
};

// First device use of a handle: upload A and the stage-0 pack map.
int ensure_device(spand_s* h) {
  if (h->d_rowptr) return SPAND_OK;
  const size_t n = (size_t)h->n, nnz = (size_t)std::max<int64_t>(h->nnz, 1);
  CK(cudaMalloc(&h->d_rowptr, (n + 1) * 4));
  CK(cudaMalloc(&h->d_colind, nnz * 4));
  CK(cudaMalloc(&h->d_val, nnz * 8));
  CK(cudaMalloc(&h->d_pack, nnz * 8));
  CK(cudaMalloc(&h->d_err, 4 * sizeof(int)));
  CK(cudaMemcpy(h->d_rowptr, h->h_rowptr.data(), (n + 1) * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->d_colind, h->h_colind.data(), (size_t)h->nnz * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->d_val, h->h_val.data(), (size_t)h->nnz * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->d_pack, h->h_pack.data(), (size_t)h->nnz * 8, cudaMemcpyHostToDevice));
  return SPAND_OK;
}

int factor_impl(spand_s* h, cudaStream_t s) {
  auto t0 = std::chrono::steady_clock::now();
  RET(ensure_device(h));
  h->factored = false;
  h->farena.reset();
  h->launches = 0;
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
      const size_t bytes = (size_t)Ly.m[c] * acc * sizeof(double);
      if (S.interior[c]) {
        roff[c] = fbytes;
        fbytes += (bytes + 15) & ~size_t(15);
      } else {
        roff[c] = sbytes;
        sbytes += (bytes + 15) & ~size_t(15);
      }
    }
    void* fptr = nullptr;
    RET(h->farena.alloc(std::max<size_t>(fbytes, 16), &fptr));
    DevBuf& scr = h->scratch[k & 1];
    RET(scr.ensure(std::max<size_t>(sbytes, 16)));
    for (int c = 0; c < ncl; ++c)
      Ly.row[c] = reinterpret_cast<double*>((S.interior[c] ? (char*)fptr : scr.p) + roff[c]);
    if (k == 0 && h->pack_split != (int64_t)(fbytes / sizeof(double))) {
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
          const double* src = Lp.row[p] + (size_t)Lp.segcol[p][i] * Lp.m[p];
          // an interface row holds no interior columns: that block reaches the
          // interior's row through the transposed child block (q, p)
          if (S.interior[Qc] && !S.interior[Pc]) continue;
          const auto& prs = S.rowsegs[Pc];
          auto it = std::lower_bound(prs.begin(), prs.end(), Qc);
          if (it == prs.end() || *it != Qc) return fail(SPAND_ECUDA, "internal: merge target missing");
          double* dst = Ly.row[Pc] + off_in_parent[p] +
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
      double* blk = Ly.row[q] + (size_t)segc(q, r) * mq;
      double* mir = (q != r) ? Ly.row[r] + (size_t)segc(r, q) * mr : nullptr;
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
        RET(h->farena.alloc(std::max<size_t>((size_t)m * m * 8, 16), &zp));
        Ly.Z[p] = (double*)zp;
        int nub = 0;
        for (int q : S.adj1[p]) nub += Ly.m[q];
        Ly.ncols_ub[p] = nub;
        const int mr = std::min(m, nub);
        Ly.maxref[p] = mr;
        void *vp = nullptr, *tp = nullptr;
        RET(h->farena.alloc(std::max<size_t>((size_t)m * mr * 8, 16), &vp));
        RET(h->farena.alloc(std::max<size_t>((size_t)mr * 8, 16), &tp));
        Ly.V[p] = (double*)vp;
        Ly.tau[p] = (double*)tp;
        const int dc = segc(p, p);
        push_copy(zcopy, Ly.row[p] + (size_t)dc * m, Ly.Z[p], m, m, m, m, 0);
        zpotrf.push_back({Ly.Z[p], m, m, p, 0});
        push_trsm(ltrsm, Ly.Z[p], m, Ly.row[p], m, m, dc, 0);
        const auto& rs = S.rowsegs[p];
        for (size_t i = 0; i < rs.size(); ++i) {
          const int q = rs[i];
          if (q >= p) break;
          const int mq = Ly.m[q];
          double* B = Ly.row[p] + (size_t)Ly.segcol[p][i] * m;
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
            if (bytes <= kQrClusterSmem && h->cluster_ok(cs)) {
              int lw = lc;
              while ((1 << lw) < want && lw < 4 && h->cluster_ok(1 << (lw + 1))) ++lw;
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
    const size_t o_rank = blob.add(rank_init);
    const size_t o_nref = blob.add(rank_init);
    const size_t o_flag = blob.add(rank_init);
    RET(h->tables.ensure(blob.h.size() + 16));
    char* D = h->tables.p;
    CK(cudaMemcpyAsync(D, blob.h.data(), blob.h.size(), cudaMemcpyHostToDevice, s));

    // ---- kernels
    int nl = 0;
    Prof& P = h->prof;
    auto run = [&](int kind, size_t ntasks, double flops, double bytes, auto&& launch) {
      if (ntasks == 0) return;
      ++nl;
      P.run(kind, s, flops, bytes, launch);
    };
    run(KK_ECOPY, pending_e.size(), 0.0, copy_bytes(pending_e),
        [&] { launch_copy((const CopyTask*)(D + o_e), (int)pending_e.size(), s); });
    run(KK_TRTRI, pending_inv.size(), trtri_flops(pending_inv), trsm_bytes(pending_inv), [&] {
      launch_trsm((const TrsmTask*)(D + o_inv), (int)pending_inv.size(), pending_inv_m, s);
    });
    run(KK_FORMQ, pending_qt.size(), formqt_flops(pending_qt), 0.0, [&] {
      launch_form_qt((const FormQtTask*)(D + o_fq), (int)pending_qt.size(), pending_qt_m, s);
    });
    if (fbytes) CK(cudaMemsetAsync(fptr, 0, fbytes, s));
    if (sbytes) CK(cudaMemsetAsync(scr.p, 0, sbytes, s));
    if (k == 0) {
      run(KK_PACK, 1, 0.0, 16.0 * h->nnz, [&] {
        launch_scatter(h->d_val, h->d_pack, (double*)fptr, (double*)scr.p, h->pack_split, h->nnz, s);
      });
    } else {
      run(KK_MERGE, merge.size(), 0.0, copy_bytes(merge),
          [&] { launch_copy((const CopyTask*)(D + o_merge), (int)merge.size(), s); });
    }
    auto run_potrf = [&](int kind, PotrfPlan& PP) {
      bool first = true;
      auto fl = [&]() { double f = first ? PP.flops : 0.0; first = false; return f; };
      run(kind, PP.small.size(), fl(), PP.bytes, [&] {
        launch_potrf((const PotrfTask*)(D + PP.o_small), (int)PP.small.size(), PP.small_max, h->d_err, s);
      });
      for (auto& st : PP.steps) {
        run(kind, st.diag.size(), fl(), 0.0, [&] {
          launch_potrf((const PotrfTask*)(D + st.o_diag), (int)st.diag.size(), kPanel, h->d_err, s);
        });
        run(kind, st.trsm.size(), 0.0, 0.0, [&] {
          launch_trsm((const TrsmTask*)(D + st.o_trsm), (int)st.trsm.size(), kPanel, s);
        });
        run(kind, st.tiles.size(), 0.0, 0.0, [&] {
          launch_schur((const SchurTile*)(D + st.o_tiles), (int)st.tiles.size(),
                       (const SchurContrib*)(D + st.o_contribs), s);
        });
      }
    };
    run_potrf(KK_POTRF, plan_int);
    run(KK_TRSM, trsm_int.size(), trsm_flops(trsm_int), trsm_bytes(trsm_int),
        [&] { launch_trsm((const TrsmTask*)(D + o_ti), (int)trsm_int.size(), max_m_int, s); });
    {
      double fl = 0.0, by = 0.0;
      schur_work(tiles, contribs, &fl, &by);
      run(KK_SCHUR, tiles.size(), fl, by, [&] {
        launch_schur((const SchurTile*)(D + o_tiles), (int)tiles.size(),
                     (const SchurContrib*)(D + o_contr), s);
      });
    }
    if (S.sparsify) {
      run(KK_SCALE_COPY, zcopy.size(), 0.0, copy_bytes(zcopy),
          [&] { launch_copy((const CopyTask*)(D + o_zc), (int)zcopy.size(), s); });
      run_potrf(KK_SCALE_POTRF, plan_z);
      run(KK_SCALE_TRSM, ltrsm.size(), trsm_flops(ltrsm), trsm_bytes(ltrsm),
          [&] { launch_trsm((const TrsmTask*)(D + o_lt), (int)ltrsm.size(), max_m_if, s); });
      run(KK_SCALE_TRSM, rtrsm.size(), trsm_flops(rtrsm), trsm_bytes(rtrsm),
          [&] { launch_trsm((const TrsmTask*)(D + o_rt), (int)rtrsm.size(), max_m_if, s); });
      run(KK_SCALE_COPY, mirror.size(), 0.0, copy_bytes(mirror),
          [&] { launch_copy((const CopyTask*)(D + o_mi), (int)mirror.size(), s); });
      run(KK_SCALE_COPY, ident.size(), 0.0, potrf_bytes(ident) / 2,
          [&] { launch_set_identity((const PotrfTask*)(D + o_id), (int)ident.size(), s); });
      for (size_t c = 0; c < qr_tasks.size(); ++c) {
        run(KK_RRQR, qr_tasks[c].size(), 0.0, 0.0, [&] {
          if (qr_csize[c] == 0)
            launch_rrqr((const RRQRTask*)(D + o_qr[c]), (int)qr_tasks[c].size(),
                        (const RRQRSeg*)(D + o_seg), (int*)(D + o_cur), (int*)(D + o_rank),
                        (int*)(D + o_nref), (int*)(D + o_flag), h->eps, h->scheme, qr_max_m[c],
                        qr_max_cols[c], qr_max_segs[c], s);
          else
            launch_rrqr_cluster((const RRQRTask*)(D + o_qr[c]), (int)qr_tasks[c].size(),
                                (const RRQRSeg*)(D + o_seg), (int*)(D + o_cur), (int*)(D + o_rank),
                                (int*)(D + o_nref), (int*)(D + o_flag), h->eps, h->scheme,
                                qr_csize[c], qr_smem[c], s);
        });
      }
    }
    CK(cudaGetLastError());
    h->launches += nl;
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
    auto explicit_inverse = [&](const double* L, int m, double** out) -> int {
      void* ip = nullptr;
      RET(h->farena.alloc(std::max<size_t>((size_t)m * m * 8, 16), &ip));
      *out = (double*)ip;
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
        double* Linv = nullptr;
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
        double* Zinv = nullptr;
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
            RET(h->farena.alloc((size_t)m * m * 8, &qp));
            a.Qt = (double*)qp;
            for (int c0 = 0; c0 < m; c0 += 32) {
              FormQtTask ft;
              ft.V = Ly.V[p];
              ft.tau = Ly.tau[p];
              ft.Qt = (double*)a.Qt + (size_t)c0 * m;
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
            RET(h->farena.alloc((size_t)nE * ncols * 8, &ep));
            double* Edst = (double*)ep;
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
    RET(h->tables.ensure(blob.h.size() + 16));
    char* D = h->tables.p;
    CK(cudaMemcpyAsync(D, blob.h.data(), blob.h.size(), cudaMemcpyHostToDevice, s));
    if (!pending_e.empty()) {
      h->prof.run(KK_ECOPY, s, 0.0, copy_bytes(pending_e), [&] {
        launch_copy((const CopyTask*)(D + o_e), (int)pending_e.size(), s);
      });
      h->launches += 1;
    }
    if (!pending_inv.empty()) {
      h->prof.run(KK_TRTRI, s, trtri_flops(pending_inv), trsm_bytes(pending_inv), [&] {
        launch_trsm((const TrsmTask*)(D + o_inv), (int)pending_inv.size(), pending_inv_m, s);
      });
      h->launches += 1;
    }
    if (!pending_qt.empty()) {
      h->prof.run(KK_FORMQ, s, formqt_flops(pending_qt), 0.0, [&] {
        launch_form_qt((const FormQtTask*)(D + o_fq), (int)pending_qt.size(), pending_qt_m, s);
      });
      h->launches += 1;
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
  h->d_api = (ApInterior*)pa;
  h->d_aps = (ApScale*)ps;
  h->d_apq = (ApQE*)pq;
  h->phases = phases;
  h->nnz_factor = nnzf;
  h->factored = true;
  h->factor_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return SPAND_OK;
}

int apply_impl(spand_s* h, const double* r, double* z, cudaStream_t s) {
  if (!h->factored) return fail(SPAND_ESTATE, "spand_apply before a successful spand_factor");
  Prof& P = h->prof;
  const int n = h->n;
  if (r != z) P.run(KK_VEC, s, 0.0, 16.0 * n, [&] { launch_copy_vec(n, r, z, s); });
  auto one = [&](const Phase& ph, bool fwd) {
    const int nt = ph.end - ph.begin;
    const int kind = ph.kind == PH_INTERIOR ? KK_AP_INTERIOR : ph.kind == PH_SCALE ? KK_AP_SCALE : KK_AP_QE;
    P.run(kind, s, ph.flops, ph.bytes, [&] {
      if (ph.kind == PH_INTERIOR)
        launch_ap_interior(h->d_api + ph.begin, nt, ph.K, ph.max_m, ph.max_cols, z, fwd, s);
      else if (ph.kind == PH_SCALE)
        launch_ap_scale(h->d_aps + ph.begin, nt, ph.K, ph.max_m, z, fwd, s);
      else launch_ap_qe(h->d_apq + ph.begin, nt, ph.K, ph.max_m, ph.max_cols, z, fwd, s);
    });
  };
  for (const Phase& ph : h->phases) one(ph, true);
  for (auto it = h->phases.rbegin(); it != h->phases.rend(); ++it) one(*it, false);
  CK(cudaGetLastError());
  return SPAND_OK;
}

int ensure_pcg(spand_s* h) {
  if (h->d_r) return SPAND_OK;
  const size_t n = (size_t)h->n;
  CK(cudaMalloc(&h->d_r, n * 8));
  CK(cudaMalloc(&h->d_z, n * 8));
  CK(cudaMalloc(&h->d_p, n * 8));
  CK(cudaMalloc(&h->d_q, n * 8));
  CK(cudaMalloc(&h->d_scal, 16 * 8));
  CK(cudaMalloc(&h->d_partial, (size_t)dot_partials(h->n) * 8));
  CK(cudaMallocHost(&h->h_scal, 16 * 8));
  return SPAND_OK;
}

// scal slots: 0 rz, 1 pq, 2 rz_new, 3 rr, 4 bb
int pcg_impl(spand_s* h, const double* b, double* x, double tol, int32_t* iters, double* relres,
             cudaStream_t s) {
  if (!h->factored) return fail(SPAND_ESTATE, "spand_pcg before a successful spand_factor");
  RET(ensure_pcg(h));
  auto t0 = std::chrono::steady_clock::now();
  const int n = h->n;
  double* sc = h->d_scal;
  Prof& P = h->prof;
  const double nnz = (double)h->nnz;
  auto dot = [&](const double* a, const double* c, int slot) {
    P.run(KK_DOT, s, 2.0 * n, 16.0 * n, [&] { launch_dot(n, a, c, h->d_partial, sc + slot, s); });
  };
  auto spmv = [&](const double* xin, double* yout) {
    P.run(KK_SPMV, s, 2.0 * nnz, 12.0 * nnz + 4.0 * (n + 1) + 16.0 * n,
          [&] { launch_spmv(n, h->d_rowptr, h->d_colind, h->d_val, xin, yout, s); });
  };
  auto read = [&](int slot, double* out) -> int {
    CK(cudaMemcpyAsync(h->h_scal + slot, sc + slot, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (P.on) P.resolve();
    *out = h->h_scal[slot];
    return SPAND_OK;
  };
  P.run(KK_VEC, s, 0.0, 24.0 * n, [&] { launch_pcg_init(n, b, x, h->d_r, s); });
  dot(b, b, 4);
  double bb = 0.0;
  RET(read(4, &bb));
  const double bnorm = std::sqrt(bb);
  int it = 0, restarts = 0;
  double rel = 0.0;
  int rc = SPAND_OK;
  if (bnorm == 0.0) {
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return SPAND_OK;
  }
  double rr = bb;
  while (true) {
    RET(apply_impl(h, h->d_r, h->d_z, s));
    P.run(KK_VEC, s, 0.0, 16.0 * n, [&] { launch_copy_vec(n, h->d_z, h->d_p, s); });
    dot(h->d_r, h->d_z, 0);
    while (it < h->maxit && std::sqrt(rr) / bnorm >= tol) {
      spmv(h->d_p, h->d_q);
      dot(h->d_p, h->d_q, 1);
      P.run(KK_VEC, s, 4.0 * n, 48.0 * n, [&] { launch_pcg_step_x(n, sc, h->d_p, h->d_q, x, h->d_r, s); });
      ++it;
      if (it % h->true_every == 0) {
        spmv(x, h->d_q);
        P.run(KK_VEC, s, 1.0 * n, 24.0 * n, [&] { launch_residual(n, b, h->d_q, h->d_r, s); });
      }
      dot(h->d_r, h->d_r, 3);
      RET(read(3, &rr));
      if (std::sqrt(rr) / bnorm < tol) break;
      RET(apply_impl(h, h->d_r, h->d_z, s));
      dot(h->d_r, h->d_z, 2);
      P.run(KK_VEC, s, 2.0 * n, 24.0 * n, [&] { launch_pcg_step_p(n, sc, h->d_z, h->d_p, s); });
      launch_pcg_scalars(sc, 0, s);
    }
    // true residual
    spmv(x, h->d_q);
    P.run(KK_VEC, s, 1.0 * n, 24.0 * n, [&] { launch_residual(n, b, h->d_q, h->d_r, s); });
    dot(h->d_r, h->d_r, 3);
    RET(read(3, &rr));
    rel = std::sqrt(rr) / bnorm;
    if (rel < tol || it >= h->maxit || restarts >= h->max_restarts) break;
    ++restarts;
  }
  CK(cudaGetLastError());
  if (rel >= tol && it >= h->maxit) rc = fail(SPAND_ENOCONV, "PCG reached maxit");
  if (iters) *iters = it;
  if (relres) *relres = rel;
  h->pcg_iters = it;
  h->pcg_relres = rel;
  h->pcg_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return rc;
}

int validate_csr(const spand_csr* A, std::string& err) {
  if (!A || !A->rowptr || !A->colind || !A->val) return (err = "null CSR array", SPAND_EINVAL);
  const int n = A->n;
  if (n < 1) return (err = "n must be >= 1", SPAND_EINVAL);
  if (A->rowptr[0] != 0 || A->rowptr[n] != A->nnz) return (err = "rowptr inconsistent with nnz", SPAND_EINVAL);
  std::vector<int32_t> cnt(n, 0);
  for (int i = 0; i < n; ++i) {
    if (A->rowptr[i + 1] < A->rowptr[i]) return (err = "rowptr not monotone", SPAND_EINVAL);
    bool diag = false;
    for (int64_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) {
      const int j = A->colind[e];
      if (j < 0 || j >= n) return (err = "column index out of range", SPAND_EINVAL);
      if (e > A->rowptr[i] && A->colind[e - 1] >= j) return (err = "columns not strictly ascending", SPAND_EINVAL);
      if (j == i) diag = true;
      ++cnt[j];
    }
    if (!diag) return (err = "missing diagonal entry in row " + std::to_string(i), SPAND_EINVAL);
  }
  // pattern symmetry: every (i, j) has (j, i)
  for (int i = 0; i < n; ++i) {
    if (cnt[i] != A->rowptr[i + 1] - A->rowptr[i]) return (err = "pattern is not symmetric", SPAND_EINVAL);
  }
  for (int i = 0; i < n; ++i)
    for (int64_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) {
      const int j = A->colind[e];
      const int32_t* b = A->colind + A->rowptr[j];
      const int32_t* en = A->colind + A->rowptr[j + 1];
      if (!std::binary_search(b, en, i)) return (err = "pattern is not symmetric", SPAND_EINVAL);
    }
  return SPAND_OK;
}

void free_handle(spand_s* h) {
  if (!h) return;
  h->farena.release();
  h->scratch[0].release();
  h->scratch[1].release();
  h->tables.release();
  cudaFree(h->d_rowptr);
  cudaFree(h->d_colind);
  cudaFree(h->d_val);
  cudaFree(h->d_pack);
  cudaFree(h->d_err);
  cudaFree(h->d_r);
  cudaFree(h->d_z);
  cudaFree(h->d_p);
  cudaFree(h->d_q);
  cudaFree(h->d_b);
  cudaFree(h->d_x);
  cudaFree(h->d_scal);
  cudaFree(h->d_partial);
  if (h->h_scal) cudaFreeHost(h->h_scal);
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  h->prof.release();
  delete h;
}

int analyze_impl(const spand_csr* A, const double* coords, int dim, int nlevels, double eps,
                 int scheme, const spand_opts* opts, spand_t* out) {
  if (!out) return fail(SPAND_EINVAL, "out is NULL");
  *out = nullptr;
  std::string err;
  if (validate_csr(A, err) != SPAND_OK) return fail(SPAND_EINVAL, err);
  if (!coords) return fail(SPAND_EINVAL, "coords is NULL");
  if (dim < 1 || dim > 3) return fail(SPAND_EINVAL, "dim must be 1, 2 or 3");
  if (!(eps >= 0.0 && eps <= 1.0)) return fail(SPAND_EINVAL, "eps must lie in [0, 1]");
  if (nlevels < 1 || nlevels > 30) return fail(SPAND_EINVAL, "nlevels must be in [1, 30]");
  if (scheme < 0 || scheme > 2) return fail(SPAND_EINVAL, "unknown scheme");
  std::unique_ptr<spand_s, void (*)(spand_s*)> h(new spand_s(), free_handle);
  h->n = A->n;
  h->nnz = A->nnz;
  h->dim = dim;
  h->nlevels = nlevels;
  h->eps = eps;
  h->scheme = scheme;
  {
    const double leaf = A->n / std::ldexp(1.0, nlevels - 1);
    int sk = 4 - (int)std::nearbyint(std::log2(leaf / 25.0));
    sk = std::min(std::max(sk, 0), std::max(nlevels - 2, 0));
    h->skip = sk;
  }
  if (opts) {
    if (opts->skip >= 0) h->skip = opts->skip;
    if (opts->maxit > 0) h->maxit = opts->maxit;
    if (opts->true_res_every > 0) h->true_every = opts->true_res_every;
    if (opts->max_restarts >= 0) h->max_restarts = opts->max_restarts;
    if (opts->rrqr_kernel < 0 || opts->rrqr_kernel > 1) return fail(SPAND_EINVAL, "rrqr_kernel must be 0 or 1");
    h->rrqr_path = opts->rrqr_kernel;
  }
  int rc = build_tree(coords, A->n, dim, nlevels, h->tree, err);
  if (rc != SPAND_OK) return fail(rc, err);
  rc = build_stages(h->tree, A->rowptr, A->colind, h->skip, h->st, err);
  if (rc != SPAND_OK) return fail(rc, err);
  // stage-0 layout (sizes are the cluster sizes) -> destination of every nonzero
  const StageSym& S0 = h->st[0];
  const int n = A->n;
  std::vector<int> cl(n), pos(n);
  for (int c = 0; c < S0.ncl; ++c)
    for (size_t i = 0; i < S0.members0[c].size(); ++i) {
      cl[S0.members0[c][i]] = c;
      pos[S0.members0[c][i]] = (int)i;
    }
  std::vector<int64_t> roff(S0.ncl);
  std::vector<std::vector<int>> segcol(S0.ncl);
  int64_t fsz = 0, ssz = 0;
  for (int c = 0; c < S0.ncl; ++c) {
    const auto& rs = S0.rowsegs[c];
    segcol[c].resize(rs.size());
    int acc = 0;
    for (size_t i = 0; i < rs.size(); ++i) {
      segcol[c][i] = acc;
      acc += (int)S0.members0[rs[i]].size();
    }
    const int64_t el = (int64_t)S0.members0[c].size() * acc;
    const int64_t padded = ((el * 8 + 15) & ~int64_t(15)) / 8;
    if (S0.interior[c]) {
      roff[c] = fsz;
      fsz += padded;
    } else {
      roff[c] = ssz;
      ssz += padded;
    }
  }
  h->pack_split = fsz;
  h->h_pack.assign(A->nnz, -1);
  for (int i = 0; i < n; ++i)
    for (int64_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) {
      const int j = A->colind[e];
      const int a = cl[i], b = cl[j];
      const auto& rs = S0.rowsegs[a];
      auto it = std::lower_bound(rs.begin(), rs.end(), b);
      if (it == rs.end() || *it != b) continue;  // interface row, interior column: kept in the interior's row
      const int64_t col = segcol[a][it - rs.begin()] + pos[j];
      const int64_t idx = roff[a] + pos[i] + col * (int64_t)S0.members0[a].size();
      h->h_pack[e] = S0.interior[a] ? idx : fsz + idx;
    }
  h->h_rowptr.assign(A->rowptr, A->rowptr + n + 1);
  h->h_colind.assign(A->colind, A->colind + A->nnz);
  h->h_val.assign(A->val, A->val + A->nnz);
  *out = h.release();
  return SPAND_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI.
// ---------------------------------------------------------------------------
extern "C" {

int spand_analyze(const spand_csr* A, const double* coords, int dim, int nlevels, double eps,
                  int scheme, const spand_opts* opts, spand_t* out) {
  try {
    return analyze_impl(A, coords, dim, nlevels, eps, scheme, opts, out);
  } catch (const std::bad_alloc&) {
    return fail(SPAND_ENOMEM, "host allocation failed");
  }
}

int spand_factor(spand_t h, void* stream) {
  if (!h) return fail(SPAND_EINVAL, "null handle");
  try {
    int rc = factor_impl(h, (cudaStream_t)stream);
    if (rc != SPAND_OK) h->factored = false;
    return rc;
  } catch (const std::bad_alloc&) {
    h->factored = false;
    return fail(SPAND_ENOMEM, "host allocation failed");
  }
}

int spand_apply(spand_t h, const double* r, double* z, void* stream) {
  if (!h || !r || !z) return fail(SPAND_EINVAL, "null argument");
  return apply_impl(h, r, z, (cudaStream_t)stream);
}

int spand_pcg(spand_t h, const double* b, double* x, double tol, int32_t* iters, double* relres,
              void* stream) {
  if (!h || !b || !x) return fail(SPAND_EINVAL, "null argument");
  if (!(tol > 0.0)) return fail(SPAND_EINVAL, "tol must be positive");
  return pcg_impl(h, b, x, tol, iters, relres, (cudaStream_t)stream);
}

int spand_pcg_host(spand_t h, const double* b_host, double* x_host, double tol, int32_t* iters,
                   double* relres, void* stream) {
  if (!h || !b_host || !x_host) return fail(SPAND_EINVAL, "null argument");
  if (!(tol > 0.0)) return fail(SPAND_EINVAL, "tol must be positive");
  cudaStream_t s = (cudaStream_t)stream;
  if (!h->d_b) {
    CK(cudaMalloc(&h->d_b, (size_t)h->n * 8));
    CK(cudaMalloc(&h->d_x, (size_t)h->n * 8));
  }
  CK(cudaMemcpyAsync(h->d_b, b_host, (size_t)h->n * 8, cudaMemcpyHostToDevice, s));
  int rc = pcg_impl(h, h->d_b, h->d_x, tol, iters, relres, s);
  if (rc != SPAND_OK && rc != SPAND_ENOCONV) return rc;
  CK(cudaMemcpyAsync(x_host, h->d_x, (size_t)h->n * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return rc;
}

int spand_matvec(spand_t h, const double* x, double* y, void* stream) {
  if (!h || !x || !y) return fail(SPAND_EINVAL, "null argument");
  RET(ensure_device(h));
  launch_spmv(h->n, h->d_rowptr, h->d_colind, h->d_val, x, y, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return SPAND_OK;
}

int spand_info(spand_t h, spand_stats* s) {
  if (!h || !s) return fail(SPAND_EINVAL, "null argument");
  memset(s, 0, sizeof(*s));
  s->n = h->n;
  s->nnz_a = h->nnz;
  s->nnz_factor = h->nnz_factor;
  s->mu = h->nnz ? (double)h->nnz_factor / (double)h->nnz : 0.0;
  s->nlevels = h->nlevels;
  s->skip = h->skip;
  s->scheme = h->scheme;
  s->eps = h->eps;
  s->nstages = h->nlevels;
  int tot = 0, ns = 0;
  for (int k = 0; k < h->nlevels; ++k) {
    tot += h->st[k].ncl;
    if (h->st[k].sparsify) ns += (int)h->st[k].ifaces.size();
  }
  s->nclusters_total = tot;
  s->ninterfaces_sparsified = ns;
  s->factor_ms = h->factor_ms;
  s->pcg_ms = h->pcg_ms;
  s->pcg_iters = h->pcg_iters;
  s->pcg_relres = h->pcg_relres;
  s->kernel_launches = h->launches;
  s->device_bytes = (int64_t)(h->farena.held() + h->scratch[0].cap + h->scratch[1].cap +
                              h->tables.cap) +
                    (int64_t)h->n * 8 * 6 + h->nnz * 20;
  return SPAND_OK;
}

int spand_ranks(spand_t h, int32_t* out, int64_t cap, int64_t* count) {
  if (!h || !count) return fail(SPAND_EINVAL, "null argument");
  if (!h->factored) return fail(SPAND_ESTATE, "spand_ranks before a successful spand_factor");
  int64_t tot = 0;
  for (int k = 0; k < h->nlevels; ++k) tot += h->st[k].ncl;
  *count = tot;
  if (!out || cap < tot) return fail(SPAND_EINVAL, "output too small");
  int64_t o = 0;
  for (int k = 0; k < h->nlevels; ++k) {
    const StageSym& S = h->st[k];
    for (int c = 0; c < S.ncl; ++c) {
      const bool sp = S.sparsify && !S.interior[c];
      out[3 * o] = h->sizes[k][c];
      out[3 * o + 1] = sp ? h->ranks[k][c] : -1;
      out[3 * o + 2] = sp ? h->flags[k][c] : 0;
      ++o;
    }
  }
  return SPAND_OK;
}

int spand_cluster_map(spand_t h, int stage, int32_t* out) {
  if (!h || !out) return fail(SPAND_EINVAL, "null argument");
  if (stage < 0 || stage >= h->nlevels) return fail(SPAND_EINVAL, "stage out of range");
  std::vector<int> cl;
  cluster_map(h->tree, stage, cl, nullptr);
  for (int v = 0; v < h->n; ++v) out[v] = cl[v];
  return SPAND_OK;
}

int spand_num_clusters(spand_t h, int stage, int32_t* nclusters) {
  if (!h || !nclusters) return fail(SPAND_EINVAL, "null argument");
  if (stage < 0 || stage >= h->nlevels) return fail(SPAND_EINVAL, "stage out of range");
  *nclusters = h->st[stage].ncl;
  return SPAND_OK;
}

int spand_set_profiling(spand_t h, int on) {
  if (!h) return fail(SPAND_EINVAL, "null handle");
  h->prof.resolve();
  h->prof.clear();
  h->prof.on = on != 0;
  return SPAND_OK;
}

int spand_kernel_stats(spand_t h, spand_kernel_stat* out, int cap, int* count) {
  if (!h || !count) return fail(SPAND_EINVAL, "null argument");
  *count = KK_COUNT;
  if (!out || cap < KK_COUNT) return fail(SPAND_EINVAL, "output too small");
  for (int k = 0; k < KK_COUNT; ++k) out[k] = h->prof.stat[k];
  return SPAND_OK;
}

void spand_destroy(spand_t h) { free_handle(h); }

const char* spand_strerror(int code) {
  switch (code) {
    case SPAND_OK: return "success";
    case SPAND_EINVAL: return "invalid argument";
    case SPAND_ENOTSPD: return "matrix is not symmetric positive definite";
    case SPAND_ENOMEM: return "out of memory";
    case SPAND_ECUDA: return "CUDA error";
    case SPAND_ENOCONV: return "PCG did not converge within maxit";
    case SPAND_ESTATE: return "call out of order";
    default: return "unknown error";
  }
}

const char* spand_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// PCG that allocates nothing.
//
// spand_pcg allocates its four work vectors (and pinned host memory for the
// scalars) on first use.  Some callers cannot allow that: a host program whose
// device memory is entirely reserved by another allocator (for instance a
// framework's caching allocator that owns the whole GPU), or a real-time loop
// that must not allocate once it is running.  spand_pcg_noalloc runs the same
// PCG with its work vectors in one statically sized device array that is part
// of the loaded library, so it calls no cudaMalloc, cudaFree or other
// allocating routine.  Limits and sharing rules are stated in include/spand.h.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kNoAllocMaxN = 262144;   // largest n the static workspace holds
constexpr int64_t kNoAllocScalars = 1024;  // dot partials (fewer than 1024) + scalars
// r, z, p, q (n doubles each) followed by the partials and the scalars.  Every
// GPU that loads the library holds this array (about 8 MiB) until exit.
static __device__ __align__(256) double g_pcg_noalloc_ws[4 * kNoAllocMaxN + kNoAllocScalars];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[256] = {};  // device address of the array, per device ordinal

// Device address of the workspace on the current device.  Resolved once per
// device (with that device current) by the first call made on it.
int noalloc_workspace(double** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return fail(SPAND_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_pcg_noalloc_ws));
    g_noalloc_ptr[dev] = (double*)p;
  }
  *out = g_noalloc_ptr[dev];
  return SPAND_OK;
}

int pcg_noalloc_impl(spand_s* h, const double* b, double* x, double tol, int32_t* iters,
                     double* relres, cudaStream_t s) {
  if ((int64_t)h->n > kNoAllocMaxN)
    return fail(SPAND_EINVAL, "spand_pcg_noalloc: n = " + std::to_string(h->n) +
                                  " exceeds the static workspace limit of " +
                                  std::to_string(kNoAllocMaxN));
  if (!h->factored) return fail(SPAND_ESTATE, "spand_pcg_noalloc before a successful spand_factor");
  double* ws = nullptr;
  RET(noalloc_workspace(&ws));
  const int n = h->n;
  double* r = ws;
  double* z = ws + kNoAllocMaxN;
  double* p = ws + 2 * kNoAllocMaxN;
  double* q = ws + 3 * kNoAllocMaxN;
  double* partial = ws + 4 * kNoAllocMaxN;
  double* sc = partial + (kNoAllocScalars - 16);
  if (dot_partials(n) > kNoAllocScalars - 16) return fail(SPAND_EINVAL, "internal: too many dot partials");
  // profiling would create CUDA events; keep it off for this call
  const bool prof_on = h->prof.on;
  h->prof.on = false;
  // scalars start from zero (the array keeps whatever the previous call left)
  CK(cudaMemsetAsync(sc, 0, 16 * sizeof(double), s));
  auto dot = [&](const double* a, const double* c, int slot) {
    launch_dot(n, a, c, partial, sc + slot, s);
  };
  auto read = [&](int slot, double* out) -> int {
    double v = 0.0;
    CK(cudaMemcpyAsync(&v, sc + slot, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *out = v;
    return SPAND_OK;
  };
  auto body = [&]() -> int {
    launch_pcg_init(n, b, x, r, s);
    dot(b, b, 4);
    double bb = 0.0;
    RET(read(4, &bb));
    const double bnorm = std::sqrt(bb);
    if (bnorm == 0.0) {
      if (iters) *iters = 0;
      if (relres) *relres = 0.0;
      return SPAND_OK;
    }
    int it = 0, restarts = 0;
    double rr = bb, rel = 0.0;
    while (true) {
      RET(apply_impl(h, r, z, s));
      launch_copy_vec(n, z, p, s);
      dot(r, z, 0);
      while (it < h->maxit && std::sqrt(rr) / bnorm >= tol) {
        launch_spmv(n, h->d_rowptr, h->d_colind, h->d_val, p, q, s);
        dot(p, q, 1);
        launch_pcg_step_x(n, sc, p, q, x, r, s);
        ++it;
        if (it % h->true_every == 0) {
          launch_spmv(n, h->d_rowptr, h->d_colind, h->d_val, x, q, s);
          launch_residual(n, b, q, r, s);
        }
        dot(r, r, 3);
        RET(read(3, &rr));
        if (std::sqrt(rr) / bnorm < tol) break;
        RET(apply_impl(h, r, z, s));
        dot(r, z, 2);
        launch_pcg_step_p(n, sc, z, p, s);
        launch_pcg_scalars(sc, 0, s);
      }
      launch_spmv(n, h->d_rowptr, h->d_colind, h->d_val, x, q, s);
      launch_residual(n, b, q, r, s);
      dot(r, r, 3);
      RET(read(3, &rr));
      rel = std::sqrt(rr) / bnorm;
      if (rel < tol || it >= h->maxit || restarts >= h->max_restarts) break;
      ++restarts;
    }
    CK(cudaGetLastError());
    if (iters) *iters = it;
    if (relres) *relres = rel;
    if (rel >= tol && it >= h->maxit) return fail(SPAND_ENOCONV, "PCG reached maxit");
    return SPAND_OK;
  };
  const int rc = body();
  h->prof.on = prof_on;
  return rc;
}

}  // namespace

extern "C" int spand_pcg_noalloc(spand_t h, const double* b, double* x, double tol, int32_t* iters,
                                 double* relres, void* stream) {
  if (!h || !b || !x) return fail(SPAND_EINVAL, "null argument");
  if (!(tol > 0.0)) return fail(SPAND_EINVAL, "tol must be positive");
  return pcg_noalloc_impl(h, b, x, tol, iters, relres, (cudaStream_t)stream);
}
