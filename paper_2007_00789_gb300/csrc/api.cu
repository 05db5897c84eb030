// The C ABI of include/spand.h: handle life cycle, the host-only symbolic
// analysis, dispatch of the factorization and apply to the FP64 or FP32
// orchestration, and PCG (always FP64) on top of the preconditioner.
#include <memory>
#include <mutex>

#include "spand_handle.h"

namespace spand {

static thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

}  // namespace spand

using namespace spand;

// First device use of a handle: upload A and the stage-0 pack map.
int spand::ensure_device(spand_s* h) {
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
  if (h->prescale) {
    CK(cudaMalloc(&h->d_fval, nnz * 8));
    CK(cudaMalloc(&h->d_scale, n * 8));
    CK(cudaMemcpy(h->d_fval, h->h_fval.data(), (size_t)h->nnz * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_scale, h->h_scale.data(), n * 8, cudaMemcpyHostToDevice));
  } else {
    h->d_fval = h->d_val;
  }
  return SPAND_OK;
}

namespace {

int factor_impl(spand_s* h, cudaStream_t s) {
  return h->precision == 0 ? f64::factor(h, s) : f32::factor(h, s);
}

// z = M r on FP64 vectors; an FP32 preconditioner is applied to an FP32 copy.
// With diagonal prescaling z = S M~ S r, S = D^{-1/2}.
int apply_any(spand_s* h, const double* r, double* z, cudaStream_t s) {
  if (!h->factored) return fail(SPAND_ESTATE, "spand_apply before a successful spand_factor");
  if (h->precision == 0) {
    if (!h->prescale) return f64::apply(h, r, z, s);
    launch_scale(h->n, h->d_scale, r, z, s);
    RET(f64::apply(h, z, z, s));
    launch_scale(h->n, h->d_scale, z, z, s);
    return SPAND_OK;
  }
  if (!h->d_rf) CK(cudaMalloc(&h->d_rf, (size_t)h->n * sizeof(float)));
  if (h->prescale) launch_d2f_scaled(h->n, h->d_scale, r, h->d_rf, s);
  else launch_d2f(h->n, r, h->d_rf, s);
  RET(f32::apply(h, h->d_rf, h->d_rf, s));
  if (h->prescale) launch_f2d_scaled(h->n, h->d_scale, h->d_rf, z, s);
  else launch_f2d(h->n, h->d_rf, z, s);
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
// The abort word of the persistent apply (a grid barrier that ran out of
// polls): reported as SPAND_ETIMEOUT by the next PCG, and cleared.
int sweep_status(spand_s* h, cudaStream_t s) {
  if (!h->sweep_valid || !h->sweep_ws) return SPAND_OK;
  int ab = 0;
  CK(cudaMemcpyAsync(&ab, h->sweep_ws + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (!ab) return SPAND_OK;
  CK(cudaMemsetAsync(h->sweep_ws + 1, 0, sizeof(int), s));
  return fail(SPAND_ETIMEOUT, "a grid barrier of the preconditioner sweep timed out");
}

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
    RET(apply_any(h, h->d_r, h->d_z, s));
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
      RET(apply_any(h, h->d_r, h->d_z, s));
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
  RET(sweep_status(h, s));
  if (iters) *iters = it;
  if (relres) *relres = rel;
  h->pcg_iters = it;
  h->pcg_relres = rel;
  h->pcg_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return rc;
}

// The first defect of row i's entries: 0 none, 1 a column out of range, 2
// columns not strictly ascending, 3 no diagonal entry.
int row_defect(const spand_csr* A, int i) {
  bool diag = false;
  for (int64_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) {
    const int j = A->colind[e];
    if (j < 0 || j >= A->n) return 1;
    if (e > A->rowptr[i] && A->colind[e - 1] >= j) return 2;
    if (j == i) diag = true;
  }
  return diag ? 0 : 3;
}

// Checks the CSR and reports its first defect in row order, as a sweep over
// the rows would meet it; the rows are checked in parallel.
int validate_csr(const spand_csr* A, std::string& err) {
  if (!A || !A->rowptr || !A->colind || !A->val) return (err = "null CSR array", SPAND_EINVAL);
  const int n = A->n;
  if (n < 1) return (err = "n must be >= 1", SPAND_EINVAL);
  if (A->rowptr[0] != 0 || A->rowptr[n] != A->nnz) return (err = "rowptr inconsistent with nnz", SPAND_EINVAL);
  // the first row whose extent is not within [rowptr[i], nnz] (its entries are not read)
  int bad_ptr = n;
  for (int i = 0; i < n; ++i)
    if (A->rowptr[i + 1] < A->rowptr[i] || A->rowptr[i + 1] > A->nnz) {
      bad_ptr = i;
      break;
    }
  std::atomic<int> bad_row(bad_ptr);
  parallel_for(bad_ptr, [&](int i, int) {
    if (row_defect(A, i)) {
      int cur = bad_row.load();
      while (i < cur && !bad_row.compare_exchange_weak(cur, i)) {
      }
    }
  }, 4096);
  const int r = bad_row.load();
  if (r < bad_ptr) {
    const int d = row_defect(A, r);
    err = d == 1 ? std::string("column index out of range")
        : d == 2 ? std::string("columns not strictly ascending")
                 : "missing diagonal entry in row " + std::to_string(r);
    return SPAND_EINVAL;
  }
  if (bad_ptr < n) return (err = "rowptr not monotone", SPAND_EINVAL);
  // pattern symmetry: every (i, j) has (j, i) (columns are ascending and in range now)
  std::atomic<bool> asym(false);
  parallel_for(n, [&](int i, int) {
    for (int64_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) {
      const int j = A->colind[e];
      const int32_t* b = A->colind + A->rowptr[j];
      const int32_t* en = A->colind + A->rowptr[j + 1];
      if (!std::binary_search(b, en, i)) {
        asym.store(true, std::memory_order_relaxed);
        return;
      }
    }
  }, 4096);
  if (asym.load()) return (err = "pattern is not symmetric", SPAND_EINVAL);
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
  if (h->d_fval != h->d_val) cudaFree(h->d_fval);
  cudaFree(h->d_scale);
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
  cudaFree(h->d_rf);
  spand::destroy_engine(h->eng);
  h->eng = nullptr;
  h->free_graphs();
  h->prof.release();
  delete h;
}

int analyze_impl(const spand_csr* A, const double* coords, int dim, int nlevels, double eps,
                 int scheme, const spand_opts* opts, spand_t* out) {
  if (!out) return fail(SPAND_EINVAL, "out is NULL");
  *out = nullptr;
  std::string err;
  if (validate_csr(A, err) != SPAND_OK) return fail(SPAND_EINVAL, err);
  const bool algebraic = !coords || dim == 0 || (opts && opts->partition == 1);
  if (opts && (opts->partition < 0 || opts->partition > 1))
    return fail(SPAND_EINVAL, "partition must be 0 or 1");
  if (!algebraic && (dim < 1 || dim > 3)) return fail(SPAND_EINVAL, "dim must be 1, 2 or 3");
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
    if (opts->rrqr_kernel < 0 || opts->rrqr_kernel > 5)
      return fail(SPAND_EINVAL, "rrqr_kernel must be 0 .. 5");
    h->rrqr_path = opts->rrqr_kernel;
    if (opts->precision < 0 || opts->precision > 1) return fail(SPAND_EINVAL, "precision must be 0 or 1");
    h->precision = opts->precision;
    if (opts->plain_launches < 0 || opts->plain_launches > 1)
      return fail(SPAND_EINVAL, "plain_launches must be 0 or 1");
    h->no_graph = opts->plain_launches == 1;
    if (opts->rrqr_threads != 0 && opts->rrqr_threads != 256 && opts->rrqr_threads != 512)
      return fail(SPAND_EINVAL, "rrqr_threads must be 0, 256 or 512");
    h->rrqr_threads = opts->rrqr_threads;
  }
  if (opts && (opts->prescale < 0 || opts->prescale > 1)) return fail(SPAND_EINVAL, "prescale must be 0 or 1");
  h->prescale = opts && opts->prescale == 1;
  if (opts && (opts->schur_simt < 0 || opts->schur_simt > 1)) return fail(SPAND_EINVAL, "schur_simt must be 0 or 1");
  h->schur_simt = opts && opts->schur_simt == 1;
  if (opts && (opts->apply_kernels < 0 || opts->apply_kernels > 2))
    return fail(SPAND_EINVAL, "apply_kernels must be 0, 1 or 2");
  h->apply_mode = opts ? opts->apply_kernels : 0;
  if (algebraic) h->dim = 0;
  // SPAND_DEBUG_TIME=1: host time of the analysis' parts (stderr, milliseconds)
  const char* dbg = getenv("SPAND_DEBUG_TIME");
  const bool timing = dbg && dbg[0] == '1';
  auto t_prev = std::chrono::steady_clock::now();
  auto lap = [&](const char* what) {
    if (!timing) return;
    const auto now = std::chrono::steady_clock::now();
    fprintf(stderr, "spand time: analyze %s %.2f ms\n", what,
            std::chrono::duration<double, std::milli>(now - t_prev).count());
    t_prev = now;
  };
  int rc = algebraic ? build_tree_graph(A->rowptr, A->colind, A->n, nlevels, h->tree, err)
                     : build_tree(coords, A->n, dim, nlevels, h->tree, err);
  if (rc != SPAND_OK) return fail(rc, err);
  lap("tree");
  rc = build_stages(h->tree, A->rowptr, A->colind, h->skip, h->st, err);
  if (rc != SPAND_OK) return fail(rc, err);
  lap("stages");
  // stage-0 layout (sizes are the cluster sizes) -> destination of every nonzero
  const StageSym& S0 = h->st[0];
  const int n = A->n;
  std::vector<int> cl(n), pos(n);
  parallel_for(S0.ncl, [&](int c, int) {
    for (size_t i = 0; i < S0.members0[c].size(); ++i) {
      cl[S0.members0[c][i]] = c;
      pos[S0.members0[c][i]] = (int)i;
    }
  }, 256);
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
    const int64_t padded = (el + 3) & ~int64_t(3);  // row regions start on 4-element boundaries
    if (S0.interior[c]) {
      roff[c] = fsz;
      fsz += padded;
    } else {
      roff[c] = ssz;
      ssz += padded;
    }
  }
  h->pack_split = fsz;
  h->h_pack.resize(A->nnz);  // every entry written below
  constexpr int kRows = 4096;  // rows per parallel chunk (the entries are independent)
  parallel_for((n + kRows - 1) / kRows, [&](int ch, int) {
    for (int i = ch * kRows; i < std::min(n, (ch + 1) * kRows); ++i)
      for (int64_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) {
        const int j = A->colind[e];
        const int a = cl[i], b = cl[j];
        const auto& rs = S0.rowsegs[a];
        auto it = std::lower_bound(rs.begin(), rs.end(), b);
        if (it == rs.end() || *it != b) {  // interface row, interior column: kept in the interior's row
          h->h_pack[e] = -1;
          continue;
        }
        const int64_t col = segcol[a][it - rs.begin()] + pos[j];
        const int64_t idx = roff[a] + pos[i] + col * (int64_t)S0.members0[a].size();
        h->h_pack[e] = S0.interior[a] ? idx : fsz + idx;
      }
  });
  lap("pack map");
  h->h_rowptr.resize(n + 1);
  parallel_copy(h->h_rowptr.data(), A->rowptr, n + 1);
  h->h_colind.resize(A->nnz);
  parallel_copy(h->h_colind.data(), A->colind, A->nnz);
  h->h_val.resize(A->nnz);
  parallel_copy(h->h_val.data(), A->val, A->nnz);
  if (h->prescale) {
    // S = D^{-1/2}, D = diag(A); the factorization sees S A S (rows in
    // parallel; the first non-positive pivot in row order is reported)
    h->h_scale.resize(n);
    std::atomic<int> bad(n);
    parallel_for(n, [&](int i, int) {
      const int32_t* c = A->colind + A->rowptr[i];
      const int64_t e = A->rowptr[i] + (std::lower_bound(c, A->colind + A->rowptr[i + 1], i) - c);
      if (!(A->val[e] > 0.0)) {  // the diagonal is present (checked above)
        int cur = bad.load();
        while (i < cur && !bad.compare_exchange_weak(cur, i)) {
        }
        h->h_scale[i] = 0.0;
        return;
      }
      h->h_scale[i] = 1.0 / std::sqrt(A->val[e]);
    }, 4096);
    if (bad.load() < n)
      return fail(SPAND_ENOTSPD, "non-positive diagonal entry in row " + std::to_string(bad.load()));
    h->h_fval.resize(A->nnz);
    parallel_for(n, [&](int i, int) {
      for (int64_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e)
        h->h_fval[e] = h->h_scale[i] * A->val[e] * h->h_scale[A->colind[e]];
    }, 4096);
  }
  lap("copies");
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

int spand_tune(spand_t h, void* stream, int32_t* choice) {
  if (!h) return fail(SPAND_EINVAL, "null handle");
  cudaStream_t s = (cudaStream_t)stream;
  const bool prof_was = h->prof.on;
  int saved_thr[6], saved_grow[6];
  std::copy(h->tune_thr, h->tune_thr + 6, saved_thr);
  std::copy(h->tune_grow, h->tune_grow + 6, saved_grow);
  double best_ms[6];
  int best_thr[6] = {0, 0, 0, 0, 0, 0}, best_grow[6] = {0, 0, 0, 0, 0, 0};
  for (int b = 0; b < 6; ++b) best_ms[b] = 1e300;
  auto restore = [&]() {
    h->tuning = false;
    std::copy(saved_thr, saved_thr + 6, h->tune_thr);
    std::copy(saved_grow, saved_grow + 6, h->tune_grow);
    h->prof.resolve();
    h->prof.clear();
    h->prof.on = prof_was;
  };
  try {
    // every candidate shape for every bucket at once: while tuning, the buckets'
    // RRQR launches are separate, so each bucket's time is read from its own launches
    h->tuning = true;
    for (int thr : {256, 512})
      for (int grow : {1, 2}) {
        for (int b = 1; b <= 5; ++b) {
          h->tune_thr[b] = thr;
          h->tune_grow[b] = grow;
        }
        h->drop_graphs();
        h->prof.resolve();
        h->prof.clear();
        h->prof.on = true;  // per-launch events, plain launches
        const int rc = factor_impl(h, s);
        h->prof.resolve();
        if (rc != SPAND_OK) {
          restore();
          h->factored = false;
          return rc;
        }
        for (const auto& kv : h->prof.rrqr_tag_ms) {
          const int b = kv.first;
          if (b >= 1 && b <= 5 && kv.second < best_ms[b]) {
            best_ms[b] = kv.second;
            best_thr[b] = thr;
            best_grow[b] = grow;
          }
        }
      }
    h->tuning = false;
    h->prof.clear();
    h->prof.on = prof_was;
    for (int b = 1; b <= 5; ++b) {
      h->tune_thr[b] = best_thr[b];
      h->tune_grow[b] = best_grow[b];
    }
    h->drop_graphs();
    if (h->apply_mode == 0) h->sweep_pref = 0;  // build the persistent sweep, to time it
    const int rc = factor_impl(h, s);  // the tuned factorization (graphs captured)
    if (rc != SPAND_OK) {
      h->factored = false;
      return rc;
    }
  } catch (const std::bad_alloc&) {
    restore();
    h->factored = false;
    return fail(SPAND_ENOMEM, "host allocation failed");
  }
  // the single-vector apply: one persistent launch or one launch per phase,
  // whichever is faster on this problem (timed on the handle's own vectors)
  int apply_choice = h->sweep_valid ? 0 : 1;
  if (h->apply_mode == 0 && h->sweep_valid) {
    RET(ensure_pcg(h));
    double* r = h->d_r;
    double* z = h->d_z;
    CK(cudaMemsetAsync(r, 0, (size_t)h->n * sizeof(double), s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float ms[2] = {0.f, 0.f};
    int rc = SPAND_OK;
    for (int v = 0; v < 2 && rc == SPAND_OK; ++v) {
      h->sweep_valid = (v == 0);
      for (int w = 0; w < 2 && rc == SPAND_OK; ++w) rc = apply_any(h, r, z, s);  // warm-up, graph capture
      if (rc != SPAND_OK) break;
      cudaEventRecord(e0, s);
      for (int w = 0; w < 5 && rc == SPAND_OK; ++w) rc = apply_any(h, r, z, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(SPAND_ECUDA, "timing the apply forms");
      cudaEventElapsedTime(&ms[v], e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    RET(rc);
    apply_choice = ms[0] <= ms[1] ? 0 : 1;
    h->sweep_valid = apply_choice == 0;
    h->sweep_pref = apply_choice;  // later factorizations build the sweep only if it won
  }
  if (choice) {
    for (int b = 1; b <= 5; ++b) {
      choice[2 * (b - 1)] = best_thr[b];
      choice[2 * (b - 1) + 1] = best_grow[b];
    }
    choice[10] = apply_choice;
    choice[11] = 0;
  }
  return SPAND_OK;
}

int spand_apply(spand_t h, const double* r, double* z, void* stream) {
  if (!h || !r || !z) return fail(SPAND_EINVAL, "null argument");
  return apply_any(h, r, z, (cudaStream_t)stream);
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
  // the stage-0 clusters of the vertices, then each stage's interiors dropped
  // and its interfaces taken to their parents: the structure the
  // factorization walks
  std::vector<int> cl;
  stage0_cluster_map(h->tree, cl);
  for (int k = 0; k < stage; ++k) {
    const StageSym& S = h->st[k];
    for (int& c : cl)
      if (c >= 0) c = S.interior[c] ? -1 : S.parent[c];
  }
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
  h->prof.resolve();
  for (int k = 0; k < KK_COUNT; ++k) out[k] = h->prof.stat[k];
  return SPAND_OK;
}

int spand_test_set_qr_wait(spand_t h, int64_t limit, int32_t unreachable) {
  if (!h) return fail(SPAND_EINVAL, "null handle");
  h->qr_wait_limit = limit > 0 ? (long long)limit : spand_s::kQrWaitDefault;
  h->qr_wait_extra = unreachable ? 1 : 0;
  h->drop_graphs();  // the captured task tables hold the previous values
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
    case SPAND_ETIMEOUT: return "a bounded device-side wait timed out";
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
  if (h->precision != 0)
    return fail(SPAND_EINVAL, "spand_pcg_noalloc supports the FP64 preconditioner only");
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
  // profiling would create CUDA events and a graph capture allocates: plain launches only
  const bool prof_on = h->prof.on;
  const bool no_graph = h->no_graph;
  h->prof.on = false;
  h->no_graph = true;
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
      RET(apply_any(h, r, z, s));
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
        RET(apply_any(h, r, z, s));
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
    RET(sweep_status(h, s));
    return SPAND_OK;
  };
  const int rc = body();
  h->prof.on = prof_on;
  h->no_graph = no_graph;
  return rc;
}

}  // namespace

extern "C" int spand_pcg_noalloc(spand_t h, const double* b, double* x, double tol, int32_t* iters,
                                 double* relres, void* stream) {
  if (!h || !b || !x) return fail(SPAND_EINVAL, "null argument");
  if (!(tol > 0.0)) return fail(SPAND_EINVAL, "tol must be positive");
  return pcg_noalloc_impl(h, b, x, tol, iters, relres, (cudaStream_t)stream);
}
