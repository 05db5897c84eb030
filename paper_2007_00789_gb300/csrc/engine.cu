// Multi-segment PCG and the batch C ABI.
//
// The PCG of §4 (Hestenes-Stiefel, x0 = 0, stop on the recursive residual
// ||r||/||b|| < tol, true residual b - A x every true_res_every iterations and
// at the end, up to max_restarts restarts when the true residual misses tol)
// is run for many segments at once.  A segment is one right-hand side of one
// factored problem; its vectors are ranges of concatenated device arrays.
// Every kernel takes the list of chunks of the segments that need that step,
// so segments at different points of their iteration share each launch, and
// the preconditioner applies of all segments that need one are merged into
// one launch per (stage, kind, colour, cluster size).
//
// Per segment the host drives a small state machine, one tick at a time
// (one host synchronisation per tick):
//   NEW    -> x = 0, r = b, bb = <b, b>
//   NEEDZ  -> z = M r, rz_new = <r, z>, p = z (+ beta p), rz = rz_new
//   ITER   -> q = A p, alpha = rz / <p, q>, x += alpha p, r -= alpha q,
//             (every true_res_every iterations r = b - A x), rr = <r, r>
//   VERIFY -> r = b - A x, rr = <r, r>: done, or restart (NEEDZ with p = z)
// The arithmetic of each segment is that of the single-problem PCG; only the
// order of the dot-product sums differs (fixed per segment, independent of
// the other segments, so a segment's iterates are the same alone and in a
// batch).
#include "spand_handle.h"

namespace spand {

namespace {

enum SegPhase { SP_NEW = 0, SP_NEEDZ, SP_ITER, SP_VERIFY, SP_DONE };

struct Seg {
  spand_s* h = nullptr;
  int64_t off = 0;
  int n = 0;
  int phase = SP_NEW;
  int mode = 1;  // NEEDZ: 1 = (re)start the direction p = z, 0 = continue
  int it = 0, restarts = 0;
  double tol = 0.0, bnorm = 0.0, rel = 0.0;
  int status = SPAND_OK;
};

struct List {
  std::vector<VChunk> ch;
  std::vector<VSegRef> refs;
  size_t o_ch = 0, o_refs = 0;
  int nch() const { return (int)ch.size(); }
  int nref() const { return (int)refs.size(); }
};

}  // namespace

struct Engine {
  std::vector<Seg> segs;
  std::vector<VSeg> vsegs;
  int64_t N = 0;
  int precision = 0;
  size_t max_chunks = 0;
  DevBuf vb, vx, vr, vz, vp, vq, vzf, vsc, vpart, vseg, vlists;
  double* h_sc = nullptr;
  size_t h_sc_cap = 0;
  MultiApply ma;
  int64_t ticks = 0;

  ~Engine() {
    ma.release();
    for (DevBuf* d : {&vb, &vx, &vr, &vz, &vp, &vq, &vzf, &vsc, &vpart, &vseg, &vlists}) d->release();
    if (h_sc) cudaFreeHost(h_sc);
  }

  // Lays out one segment per (handle, right-hand side) and copies the right-hand sides in.
  int setup(spand_s* const* hs, const int* nrhs, int count, const double* const* b, double tol,
            cudaStream_t s) {
    segs.clear();
    vsegs.clear();
    N = 0;
    max_chunks = 0;
    int k = 0;
    for (int i = 0; i < count; ++i) {
      for (int j = 0; j < nrhs[i]; ++j, ++k) {
        Seg g;
        g.h = hs[i];
        g.off = N;
        g.n = hs[i]->n;
        g.tol = tol;
        segs.push_back(g);
        VSeg v;
        v.rowptr = hs[i]->d_rowptr;
        v.colind = hs[i]->d_colind;
        v.val = hs[i]->d_val;
        v.off = N;
        v.n = hs[i]->n;
        v.pad = 0;
        vsegs.push_back(v);
        // segments start on 32-entry boundaries (aligned vector accesses)
        N += ((int64_t)hs[i]->n + 31) & ~int64_t(31);
        max_chunks += (hs[i]->n + kSegChunk - 1) / kSegChunk;
      }
    }
    const size_t nv = std::max<size_t>((size_t)N, 32) * sizeof(double);
    for (DevBuf* d : {&vb, &vx, &vr, &vz, &vp, &vq}) RET(d->ensure(nv));
    if (precision == 1) RET(vzf.ensure(nv / 2));
    RET(vsc.ensure(std::max<size_t>(segs.size(), 1) * kSegScal * sizeof(double)));
    RET(vpart.ensure(std::max<size_t>(max_chunks, 1) * sizeof(double)));
    RET(vseg.ensure(std::max<size_t>(vsegs.size(), 1) * sizeof(VSeg)));
    RET(vlists.ensure(std::max<size_t>(4 * max_chunks * sizeof(VChunk), 4096)));
    const size_t nsc = segs.size() * kSegScal;
    if (nsc > h_sc_cap) {
      if (h_sc) cudaFreeHost(h_sc);
      h_sc = nullptr;
      h_sc_cap = 0;
      CK(cudaMallocHost(&h_sc, nsc * sizeof(double)));
      h_sc_cap = nsc;
    }
    CK(cudaMemcpyAsync(vseg.p, vsegs.data(), vsegs.size() * sizeof(VSeg), cudaMemcpyHostToDevice, s));
    for (size_t i = 0; i < segs.size(); ++i)
      CK(cudaMemcpyAsync(B() + segs[i].off, b[i], (size_t)segs[i].n * sizeof(double),
                         cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));  // the segment table must outlive its copy
    return SPAND_OK;
  }

  double* B() { return (double*)vb.p; }
  double* X() { return (double*)vx.p; }
  double* R() { return (double*)vr.p; }
  double* Z() { return (double*)vz.p; }
  double* Pv() { return (double*)vp.p; }
  double* Q() { return (double*)vq.p; }
  double* SC() { return (double*)vsc.p; }

  void add(List& L, int si, int mode) {
    const Seg& g = segs[si];
    VSegRef ref;
    ref.seg = si;
    ref.chunk0 = (int)L.ch.size();
    ref.pad = 0;
    for (int64_t c = 0; c < g.n; c += kSegChunk) {
      VChunk k;
      k.begin = g.off + c;
      k.end = g.off + std::min<int64_t>(g.n, c + kSegChunk);
      k.seg = si;
      k.mode = mode;
      L.ch.push_back(k);
    }
    ref.nchunks = (int)L.ch.size() - ref.chunk0;
    L.refs.push_back(ref);
  }

  int upload(std::vector<List*> lists, cudaStream_t s) {
    Blob blob;
    for (List* L : lists) {
      L->o_ch = blob.add(L->ch);
      L->o_refs = blob.add(L->refs);
    }
    RET(vlists.ensure(blob.h.size() + 16));
    CK(cudaMemcpyAsync(vlists.p, blob.h.data(), blob.h.size(), cudaMemcpyHostToDevice, s));
    return SPAND_OK;
  }
  const VChunk* chunks(const List& L) { return (const VChunk*)(vlists.p + L.o_ch); }
  const VSegRef* refs(const List& L) { return (const VSegRef*)(vlists.p + L.o_refs); }

  int read_scalars(cudaStream_t s) {
    CK(cudaMemcpyAsync(h_sc, vsc.p, segs.size() * kSegScal * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return SPAND_OK;
  }

  int apply(const List& L, Prof& P, cudaStream_t s) {
    std::vector<ApSeg> as;
    as.reserve(L.refs.size());
    for (const auto& r : L.refs) as.push_back({segs[r.seg].h, segs[r.seg].off});
    const bool graph = !P.on;
    if (precision == 0) {
      P.run(KK_VEC, s, 0.0, 16.0 * chunk_entries(L),
            [&] { launch_seg_copy(chunks(L), L.nch(), R(), Z(), s); });
      RET(f64::apply_multi(as.data(), (int)as.size(), Z(), ma, P, graph, s));
    } else {
      float* zf = (float*)vzf.p;
      P.run(KK_VEC, s, 0.0, 12.0 * chunk_entries(L),
            [&] { launch_seg_d2f(chunks(L), L.nch(), R(), zf, s); });
      RET(f32::apply_multi(as.data(), (int)as.size(), zf, ma, P, graph, s));
      P.run(KK_VEC, s, 0.0, 12.0 * chunk_entries(L),
            [&] { launch_seg_f2d(chunks(L), L.nch(), zf, Z(), s); });
    }
    return SPAND_OK;
  }

  static double chunk_entries(const List& L) {
    double e = 0.0;
    for (const auto& c : L.ch) e += (double)(c.end - c.begin);
    return e;
  }
  double nnz_of(const List& L) {
    double e = 0.0;
    for (const auto& r : L.refs) e += (double)segs[r.seg].h->nnz;
    return e;
  }

  // One tick of every unfinished segment; returns the number still running.
  int tick(Prof& P, cudaStream_t s, int* running) {
    ++ticks;
    // ---- new segments: x = 0, r = b, bb
    {
      List NW;
      for (size_t i = 0; i < segs.size(); ++i)
        if (segs[i].phase == SP_NEW) add(NW, (int)i, 0);
      if (!NW.refs.empty()) {
        RET(upload({&NW}, s));
        const double e = chunk_entries(NW);
        P.run(KK_VEC, s, 0.0, 24.0 * e, [&] { launch_seg_init(chunks(NW), NW.nch(), B(), X(), R(), s); });
        P.run(KK_DOT, s, 2.0 * e, 8.0 * e, [&] {
          launch_seg_dot(chunks(NW), NW.nch(), refs(NW), NW.nref(), B(), B(), (double*)vpart.p, SC(), 4, s);
        });
        RET(read_scalars(s));
        if (P.on) P.resolve();
        for (const auto& r : NW.refs) {
          Seg& g = segs[r.seg];
          const double bb = h_sc[kSegScal * r.seg + 4];
          g.bnorm = std::sqrt(bb);
          if (g.bnorm == 0.0) {
            g.phase = SP_DONE;
            g.rel = 0.0;
            continue;
          }
          g.phase = (g.it < g.h->maxit && 1.0 >= g.tol) ? SP_NEEDZ : SP_VERIFY;
          g.mode = 1;
        }
      }
    }
    List NZ, IT, RP, VF;
    for (size_t i = 0; i < segs.size(); ++i) {
      const Seg& g = segs[i];
      if (g.phase == SP_NEEDZ) add(NZ, (int)i, g.mode);
      if (g.phase == SP_NEEDZ || g.phase == SP_ITER) {
        add(IT, (int)i, 0);
        if ((g.it + 1) % g.h->true_every == 0) add(RP, (int)i, 0);
      }
      if (g.phase == SP_VERIFY) add(VF, (int)i, 0);
    }
    if (IT.refs.empty() && VF.refs.empty()) {
      *running = 0;
      return SPAND_OK;
    }
    RET(upload({&NZ, &IT, &RP, &VF}, s));
    double* part = (double*)vpart.p;
    // (1) z = M r, rz_new = <r, z>, p update, rz = rz_new
    if (!NZ.refs.empty()) {
      RET(apply(NZ, P, s));
      const double e = chunk_entries(NZ);
      P.run(KK_DOT, s, 2.0 * e, 16.0 * e, [&] {
        launch_seg_dot(chunks(NZ), NZ.nch(), refs(NZ), NZ.nref(), R(), Z(), part, SC(), 2, s);
      });
      P.run(KK_VEC, s, 2.0 * e, 24.0 * e, [&] {
        launch_seg_step_p(chunks(NZ), NZ.nch(), refs(NZ), NZ.nref(), SC(), Z(), Pv(), s);
      });
    }
    // (2) one CG step
    if (!IT.refs.empty()) {
      const double e = chunk_entries(IT), nz = nnz_of(IT);
      P.run(KK_SPMV, s, 2.0 * nz, 12.0 * nz + 16.0 * e, [&] {
        launch_seg_spmv(chunks(IT), IT.nch(), (const VSeg*)vseg.p, Pv(), Q(), s);
      });
      P.run(KK_DOT, s, 2.0 * e, 16.0 * e, [&] {
        launch_seg_dot(chunks(IT), IT.nch(), refs(IT), IT.nref(), Pv(), Q(), part, SC(), 1, s);
      });
      P.run(KK_VEC, s, 4.0 * e, 48.0 * e, [&] {
        launch_seg_step_x(chunks(IT), IT.nch(), SC(), Pv(), Q(), X(), R(), s);
      });
      if (!RP.refs.empty()) {
        const double er = chunk_entries(RP), nr = nnz_of(RP);
        P.run(KK_SPMV, s, 2.0 * nr, 12.0 * nr + 16.0 * er, [&] {
          launch_seg_spmv(chunks(RP), RP.nch(), (const VSeg*)vseg.p, X(), Q(), s);
        });
        P.run(KK_VEC, s, er, 24.0 * er,
              [&] { launch_seg_residual(chunks(RP), RP.nch(), B(), Q(), R(), s); });
      }
      P.run(KK_DOT, s, 2.0 * e, 8.0 * e, [&] {
        launch_seg_dot(chunks(IT), IT.nch(), refs(IT), IT.nref(), R(), R(), part, SC(), 3, s);
      });
    }
    // (3) true residual of the segments whose recursive residual met tol
    if (!VF.refs.empty()) {
      const double e = chunk_entries(VF), nz = nnz_of(VF);
      P.run(KK_SPMV, s, 2.0 * nz, 12.0 * nz + 16.0 * e, [&] {
        launch_seg_spmv(chunks(VF), VF.nch(), (const VSeg*)vseg.p, X(), Q(), s);
      });
      P.run(KK_VEC, s, e, 24.0 * e, [&] { launch_seg_residual(chunks(VF), VF.nch(), B(), Q(), R(), s); });
      P.run(KK_DOT, s, 2.0 * e, 8.0 * e, [&] {
        launch_seg_dot(chunks(VF), VF.nch(), refs(VF), VF.nref(), R(), R(), part, SC(), 3, s);
      });
    }
    CK(cudaGetLastError());
    RET(read_scalars(s));
    if (P.on) P.resolve();
    int run = 0;
    for (const auto& r : IT.refs) {
      Seg& g = segs[r.seg];
      ++g.it;
      g.rel = std::sqrt(h_sc[kSegScal * r.seg + 3]) / g.bnorm;
      if (g.rel < g.tol || g.it >= g.h->maxit) {
        g.phase = SP_VERIFY;
      } else {
        g.phase = SP_NEEDZ;
        g.mode = 0;
      }
    }
    for (const auto& r : VF.refs) {
      Seg& g = segs[r.seg];
      g.rel = std::sqrt(h_sc[kSegScal * r.seg + 3]) / g.bnorm;
      if (g.rel < g.tol || g.it >= g.h->maxit || g.restarts >= g.h->max_restarts) {
        g.phase = SP_DONE;
        g.status = (g.rel < g.tol) ? SPAND_OK : SPAND_ENOCONV;
      } else {
        ++g.restarts;
        g.phase = SP_NEEDZ;
        g.mode = 1;
      }
    }
    for (const auto& g : segs) run += g.phase != SP_DONE;
    *running = run;
    return SPAND_OK;
  }

  int run(Prof& P, cudaStream_t s) {
    ticks = 0;
    int running = 1;
    while (running) RET(tick(P, s, &running));
    return SPAND_OK;
  }
};

}  // namespace spand

struct spand_batch_s {
  std::vector<spand_s*> hs;
  spand::FactorGroup fg;
  spand::Prof prof;
  spand::Engine eng;
  int precision = 0;
  double factor_ms = 0.0, pcg_ms = 0.0;
  int64_t ticks = 0;
  ~spand_batch_s() {
    fg.release();
    prof.release();
  }
};

using namespace spand;

extern "C" {

int spand_batch_create(const spand_t* handles, int32_t count, spand_batch_t* out) {
  if (!handles || !out || count < 1) return fail(SPAND_EINVAL, "null argument or empty batch");
  *out = nullptr;
  std::vector<spand_s*> hs(handles, handles + count);
  for (int i = 0; i < count; ++i) {
    if (!hs[i]) return fail(SPAND_EINVAL, "null handle in batch");
    if (hs[i]->precision != hs[0]->precision)
      return fail(SPAND_EINVAL, "batch handles must share one precision");
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return fail(SPAND_EINVAL, "handle listed twice in batch");
  }
  spand_batch_s* b = new (std::nothrow) spand_batch_s();
  if (!b) return fail(SPAND_ENOMEM, "host allocation failed");
  b->hs = hs;
  b->precision = hs[0]->precision;
  b->eng.precision = b->precision;
  *out = b;
  return SPAND_OK;
}

int spand_batch_factor(spand_batch_t b, void* stream) {
  if (!b) return fail(SPAND_EINVAL, "null batch");
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  const int rc = b->precision == 0
                     ? f64::factor_group(b->hs.data(), (int)b->hs.size(), b->fg, b->prof, s)
                     : f32::factor_group(b->hs.data(), (int)b->hs.size(), b->fg, b->prof, s);
  b->factor_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return rc;
}

int spand_batch_pcg(spand_batch_t b, const double* const* bvec, double* const* xvec, double tol,
                    int32_t* iters, double* relres, void* stream) {
  if (!b || !bvec || !xvec) return fail(SPAND_EINVAL, "null argument");
  if (!(tol > 0.0)) return fail(SPAND_EINVAL, "tol must be positive");
  const int count = (int)b->hs.size();
  for (int i = 0; i < count; ++i) {
    if (!b->hs[i]->factored) return fail(SPAND_ESTATE, "spand_batch_pcg before a successful factorization");
    if (!bvec[i] || !xvec[i]) return fail(SPAND_EINVAL, "null vector in batch");
  }
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int> ones(count, 1);
  Engine& E = b->eng;
  RET(E.setup(b->hs.data(), ones.data(), count, bvec, tol, s));
  RET(E.run(b->prof, s));
  int rc = SPAND_OK;
  for (int i = 0; i < count; ++i) {
    const auto& g = E.segs[i];
    CK(cudaMemcpyAsync(xvec[i], E.X() + g.off, (size_t)g.n * sizeof(double),
                       cudaMemcpyDeviceToDevice, s));
    if (iters) iters[i] = g.it;
    if (relres) relres[i] = g.rel;
    if (g.status != SPAND_OK && rc == SPAND_OK) rc = g.status;
  }
  CK(cudaStreamSynchronize(s));
  b->ticks = E.ticks;
  b->pcg_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (rc == SPAND_ENOCONV) return fail(SPAND_ENOCONV, "PCG reached maxit for a problem of the batch");
  return rc;
}

int spand_batch_info(spand_batch_t b, double* factor_ms, double* pcg_ms, int64_t* launches,
                     int64_t* ticks) {
  if (!b) return fail(SPAND_EINVAL, "null batch");
  if (factor_ms) *factor_ms = b->factor_ms;
  if (pcg_ms) *pcg_ms = b->pcg_ms;
  if (launches) *launches = b->hs.empty() ? 0 : b->hs[0]->launches;
  if (ticks) *ticks = b->ticks;
  return SPAND_OK;
}

int spand_batch_set_profiling(spand_batch_t b, int on) {
  if (!b) return fail(SPAND_EINVAL, "null batch");
  b->prof.resolve();
  b->prof.clear();
  b->prof.on = on != 0;
  return SPAND_OK;
}

int spand_batch_kernel_stats(spand_batch_t b, spand_kernel_stat* out, int cap, int* count) {
  if (!b || !count) return fail(SPAND_EINVAL, "null argument");
  *count = KK_COUNT;
  if (!out || cap < KK_COUNT) return fail(SPAND_EINVAL, "output too small");
  for (int k = 0; k < KK_COUNT; ++k) out[k] = b->prof.stat[k];
  return SPAND_OK;
}

void spand_batch_destroy(spand_batch_t b) { delete b; }

}  // extern "C"
