// Multi-segment PCG, the batch C ABI and the solve server.
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
// the other segments, so a segment's iterates do not depend on what else is
// in flight).  Segments can join and leave between ticks: that is what the
// server's continuous batching uses.
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "spand_handle.h"

namespace spand {

namespace {

enum SegPhase { SP_NEW = 0, SP_NEEDZ, SP_ITER, SP_VERIFY, SP_DONE };

struct Seg {
  bool live = false;
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
  std::vector<Seg> segs;  // by segment id
  std::vector<int> free_ids;
  std::vector<VSeg> vsegs;
  bool vseg_dirty = false;
  int64_t cap = 0;  // entries of every concatenated vector
  int precision = 0;
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

  int live_count() const {
    int c = 0;
    for (const auto& g : segs) c += g.live;
    return c;
  }

  // Vectors of `entries` entries and room for `nsegs` segments.  Contents are
  // not kept: only called while no segment is live.
  int reserve(int64_t entries, int nsegs) {
    if (live_count() != 0) return fail(SPAND_ESTATE, "internal: engine resized while solving");
    entries = std::max<int64_t>(entries, 32);
    const size_t nv = (size_t)entries * sizeof(double);
    for (DevBuf* d : {&vb, &vx, &vr, &vz, &vp, &vq}) RET(d->ensure(nv));
    if (precision == 1) RET(vzf.ensure(nv / 2));
    cap = entries;
    nsegs = std::max(nsegs, 1);
    RET(vsc.ensure((size_t)nsegs * kSegScal * sizeof(double)));
    RET(vpart.ensure(((size_t)entries / kSegChunk + nsegs + 1) * sizeof(double)));
    RET(vseg.ensure((size_t)nsegs * sizeof(VSeg)));
    const size_t nsc = (size_t)nsegs * kSegScal;
    if (nsc > h_sc_cap) {
      if (h_sc) cudaFreeHost(h_sc);
      h_sc = nullptr;
      h_sc_cap = 0;
      CK(cudaMallocHost(&h_sc, nsc * sizeof(double)));
      h_sc_cap = nsc;
    }
    return SPAND_OK;
  }
  int capacity_segs() const { return (int)(vseg.cap / sizeof(VSeg)); }

  // A new segment for problem h at entries [off, off + n); b: n doubles
  // (device or host, as kind says), copied in on stream s.
  int add(spand_s* h, int64_t off, double tol, const double* b, cudaMemcpyKind kind,
          cudaStream_t s, int* id) {
    if (off < 0 || off + h->n > cap) return fail(SPAND_EINVAL, "internal: segment outside the vectors");
    int sid;
    if (!free_ids.empty()) {
      sid = free_ids.back();
      free_ids.pop_back();
    } else {
      sid = (int)segs.size();
      if (sid >= capacity_segs()) return fail(SPAND_ENOMEM, "internal: no segment slot left");
      segs.emplace_back();
      vsegs.emplace_back();
    }
    Seg g;
    g.live = true;
    g.h = h;
    g.off = off;
    g.n = h->n;
    g.tol = tol;
    segs[sid] = g;
    VSeg v;
    v.rowptr = h->d_rowptr;
    v.colind = h->d_colind;
    v.val = h->d_val;
    v.scale = h->prescale ? h->d_scale : nullptr;
    v.off = off;
    v.n = h->n;
    v.pad = 0;
    vsegs[sid] = v;
    vseg_dirty = true;
    CK(cudaMemcpyAsync(B() + off, b, (size_t)h->n * sizeof(double), kind, s));
    *id = sid;
    return SPAND_OK;
  }
  void remove(int sid) {
    segs[sid].live = false;
    segs[sid].h = nullptr;
    free_ids.push_back(sid);
  }

  double* B() { return (double*)vb.p; }
  double* X() { return (double*)vx.p; }
  double* R() { return (double*)vr.p; }
  double* Z() { return (double*)vz.p; }
  double* Pv() { return (double*)vp.p; }
  double* Q() { return (double*)vq.p; }
  double* SC() { return (double*)vsc.p; }

  void add_to(List& L, int si, int mode) {
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
    if (vseg_dirty && !vsegs.empty()) {
      CK(cudaMemcpyAsync(vseg.p, vsegs.data(), vsegs.size() * sizeof(VSeg), cudaMemcpyHostToDevice, s));
      vseg_dirty = false;
    }
    return SPAND_OK;
  }
  const VChunk* chunks(const List& L) { return (const VChunk*)(vlists.p + L.o_ch); }
  const VSegRef* refs(const List& L) { return (const VSegRef*)(vlists.p + L.o_refs); }

  // also the point where the host tables of this tick may be reused
  int read_scalars(cudaStream_t s) {
    CK(cudaMemcpyAsync(h_sc, vsc.p, segs.size() * kSegScal * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return SPAND_OK;
  }

  static double entries(const List& L) {
    double e = 0.0;
    for (const auto& c : L.ch) e += (double)(c.end - c.begin);
    return e;
  }
  double nnz_of(const List& L) {
    double e = 0.0;
    for (const auto& r : L.refs) e += (double)segs[r.seg].h->nnz;
    return e;
  }

  int apply(const List& L, Prof& P, cudaStream_t s) {
    std::vector<ApSeg> as;
    as.reserve(L.refs.size());
    for (const auto& r : L.refs) as.push_back({segs[r.seg].h, segs[r.seg].off});
    const bool graph = !P.on;
    const VSeg* vs = (const VSeg*)vseg.p;
    bool scaled = false;
    for (const auto& r : L.refs) scaled = scaled || segs[r.seg].h->prescale;
    if (precision == 0) {
      P.run(KK_VEC, s, 0.0, 16.0 * entries(L),
            [&] { launch_seg_copy(chunks(L), L.nch(), vs, R(), Z(), s); });
      RET(f64::apply_multi(as.data(), (int)as.size(), Z(), ma, P, graph, s));
      if (scaled)
        P.run(KK_VEC, s, 0.0, 16.0 * entries(L),
              [&] { launch_seg_rescale(chunks(L), L.nch(), vs, Z(), s); });
    } else {
      float* zf = (float*)vzf.p;
      P.run(KK_VEC, s, 0.0, 12.0 * entries(L),
            [&] { launch_seg_d2f(chunks(L), L.nch(), vs, R(), zf, s); });
      RET(f32::apply_multi(as.data(), (int)as.size(), zf, ma, P, graph, s));
      P.run(KK_VEC, s, 0.0, 12.0 * entries(L),
            [&] { launch_seg_f2d(chunks(L), L.nch(), vs, zf, Z(), s); });
    }
    return SPAND_OK;
  }

  // One tick of every live, unfinished segment; *running: how many remain.
  int tick(Prof& P, cudaStream_t s, int* running) {
    ++ticks;
    double* part = (double*)vpart.p;
    // ---- new segments: x = 0, r = b, bb
    {
      List NW;
      for (size_t i = 0; i < segs.size(); ++i)
        if (segs[i].live && segs[i].phase == SP_NEW) add_to(NW, (int)i, 0);
      if (!NW.refs.empty()) {
        RET(upload({&NW}, s));
        const double e = entries(NW);
        P.run(KK_VEC, s, 0.0, 24.0 * e, [&] { launch_seg_init(chunks(NW), NW.nch(), B(), X(), R(), s); });
        P.run(KK_DOT, s, 2.0 * e, 8.0 * e, [&] {
          launch_seg_dot(chunks(NW), NW.nch(), refs(NW), NW.nref(), B(), B(), part, SC(), 4, s);
        });
        RET(read_scalars(s));
        if (P.on) P.resolve();
        for (const auto& r : NW.refs) {
          Seg& g = segs[r.seg];
          g.bnorm = std::sqrt(h_sc[kSegScal * r.seg + 4]);
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
      if (!g.live) continue;
      if (g.phase == SP_NEEDZ) add_to(NZ, (int)i, g.mode);
      if (g.phase == SP_NEEDZ || g.phase == SP_ITER) {
        add_to(IT, (int)i, 0);
        if ((g.it + 1) % g.h->true_every == 0) add_to(RP, (int)i, 0);
      }
      if (g.phase == SP_VERIFY) add_to(VF, (int)i, 0);
    }
    if (IT.refs.empty() && VF.refs.empty()) {
      *running = 0;
      return SPAND_OK;
    }
    RET(upload({&NZ, &IT, &RP, &VF}, s));
    // (1) z = M r, rz_new = <r, z>, p update, rz = rz_new
    if (!NZ.refs.empty()) {
      RET(apply(NZ, P, s));
      const double e = entries(NZ);
      P.run(KK_DOT, s, 2.0 * e, 16.0 * e, [&] {
        launch_seg_dot(chunks(NZ), NZ.nch(), refs(NZ), NZ.nref(), R(), Z(), part, SC(), 2, s);
      });
      P.run(KK_VEC, s, 2.0 * e, 24.0 * e, [&] {
        launch_seg_step_p(chunks(NZ), NZ.nch(), refs(NZ), NZ.nref(), SC(), Z(), Pv(), s);
      });
    }
    // (2) one CG step
    if (!IT.refs.empty()) {
      const double e = entries(IT), nz = nnz_of(IT);
      P.run(KK_SPMV, s, 2.0 * nz, 12.0 * nz + 16.0 * e, [&] {
        launch_seg_spmv(chunks(IT), IT.nch(), (const VSeg*)vseg.p, Pv(), Q(), s);
      });
      P.run(KK_DOT, s, 2.0 * e, 16.0 * e, [&] {
        launch_seg_dot(chunks(IT), IT.nch(), refs(IT), IT.nref(), Pv(), Q(), part, SC(), 1, s);
      });
      P.run(KK_VEC, s, 4.0 * e, 48.0 * e,
            [&] { launch_seg_step_x(chunks(IT), IT.nch(), SC(), Pv(), Q(), X(), R(), s); });
      if (!RP.refs.empty()) {
        const double er = entries(RP), nr = nnz_of(RP);
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
      const double e = entries(VF), nz = nnz_of(VF);
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
    int run = 0;
    for (const auto& g : segs) run += g.live && g.phase != SP_DONE;
    *running = run;
    return SPAND_OK;
  }

  int run_all(Prof& P, cudaStream_t s) {
    int running = 1;
    while (running) RET(tick(P, s, &running));
    return SPAND_OK;
  }
};

// ---------------------------------------------------------------------------
// Solve server: resident factored problems, requests of several right-hand
// sides, continuous batching.  Two host threads: the factor thread factors
// newly admitted problems on its own stream while the solve thread runs the
// engine's ticks on another, so a factorization overlaps the PCG of the
// requests already in flight.  Requests join the engine between ticks as
// segment slots and vector space free up, and leave it as soon as all their
// right-hand sides are done.
// ---------------------------------------------------------------------------
struct Server {
  struct Mat {
    spand_s* h = nullptr;
    bool pinned = false;
    int state = 0;  // 0 waiting for admission, 1 factoring, 2 ready, 3 failed
    int status = SPAND_OK;
    size_t bytes = 0;  // device bytes held by its factorization
    int users = 0;     // queued or running requests
    int64_t last_use = 0;
    std::chrono::steady_clock::time_point t_ready;  // when its factorization last completed
  };
  struct Req {
    int64_t id = 0;
    int mid = 0, nrhs = 0;
    const double* b = nullptr;  // host, n x nrhs column-major
    double* x = nullptr;        // host, written on completion
    int64_t off = -1;           // entries [off, off + nrhs * stride) of the engine vectors
    int64_t stride = 0;
    std::vector<int> seg;
    int done = 0;               // 0 queued, 1 running, 2 finished
    int status = SPAND_OK;
    std::vector<int32_t> iters;
    std::vector<double> relres;
    // submission, admission to the solve engine, completion; the wait for the
    // problem's factorization ends at max(t_submit, the problem's t_ready)
    std::chrono::steady_clock::time_point t_submit, t_ready, t_admit, t_done;
  };

  spand_server_opts opts{};
  std::deque<Mat> mats;  // a deque: references stay valid while problems are added
  std::map<int64_t, Req> reqs;
  std::deque<int64_t> queue;  // submitted, not yet admitted
  std::map<int64_t, int64_t> free_ranges;  // offset -> length of free vector space
  int64_t next_id = 1;
  size_t resident = 0;
  double mu_estimate = 60.0;  // factor entries per nonzero of A, refined after each factorization
  Engine eng;
  Prof prof;  // never enabled: the server's ticks run as graphs
  cudaStream_t s_solve = nullptr, s_factor = nullptr;
  std::mutex mu;
  std::condition_variable cv_solve, cv_factor, cv_done;
  bool stop = false;
  std::thread th_solve, th_factor;
  int error = SPAND_OK;
  std::string error_msg;
  std::vector<double> lat_ms;
  // per completed request: waiting for the factorization, queued with the
  // problem ready (slots, vector space), and solving (admission to completion)
  std::vector<double> wait_factor_ms, wait_queue_ms, solve_ms;
  int64_t solves = 0;
  std::chrono::steady_clock::time_point t_first, t_last;
  bool any = false;
  int64_t tick_count = 0;
  int max_inflight = 0;

  size_t est_bytes(const Mat& m) const {
    const size_t el = m.h->precision == 1 ? 4 : 8;
    return (size_t)(mu_estimate * (double)m.h->nnz * (double)el * 1.25);
  }

  // ---- factor thread
  void factor_loop() {
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      cv_factor.wait(lk, [&] {
        if (stop) return true;
        for (auto& m : mats)
          if (m.state == 0 && m.users > 0) return true;
        return false;
      });
      if (stop) return;
      int pick = -1;
      for (size_t i = 0; i < mats.size(); ++i)
        if (mats[i].state == 0 && mats[i].users > 0) {
          pick = (int)i;
          break;
        }
      if (pick < 0) continue;
      Mat& m = mats[pick];
      // admission by footprint: evict idle, unpinned problems (least recently used first)
      const size_t need = est_bytes(m);
      while (resident + need > opts.hbm_budget) {
        int victim = -1;
        for (size_t i = 0; i < mats.size(); ++i) {
          const Mat& v = mats[i];
          if (v.state == 2 && !v.pinned && v.users == 0 &&
              (victim < 0 || v.last_use < mats[victim].last_use))
            victim = (int)i;
        }
        if (victim < 0) break;
        Mat& v = mats[victim];
        v.h->drop_graphs();
        v.h->farena.release();
        v.h->scratch[0].release();
        v.h->scratch[1].release();
        v.h->factored = false;
        resident -= std::min(resident, v.bytes);
        v.bytes = 0;
        v.state = 0;
      }
      bool running = false;
      for (const auto& kv : reqs) running = running || kv.second.done == 1;
      if (resident + need > opts.hbm_budget && running) {
        // nothing idle to evict: wait until a running request finishes (with
        // nothing running, admit over budget rather than wait forever)
        cv_factor.wait(lk);
        continue;
      }
      m.state = 1;
      spand_s* h = m.h;
      lk.unlock();
      const int rc = h->precision == 0 ? f64::factor(h, s_factor) : f32::factor(h, s_factor);
      const std::string msg = rc == SPAND_OK ? std::string() : std::string(spand_last_error());
      lk.lock();
      if (rc == SPAND_OK) {
        m.bytes = h->farena.held() + h->scratch[0].cap + h->scratch[1].cap;
        resident += m.bytes;
        const size_t el = h->precision == 1 ? 4 : 8;
        mu_estimate = (double)m.bytes / ((double)h->nnz * el);  // the latest problem's ratio
        m.state = 2;
        m.t_ready = std::chrono::steady_clock::now();
      } else {
        m.state = 3;
        m.status = rc;
        error_msg = msg;
      }
      cv_solve.notify_all();
    }
  }

  // ---- solve thread
  bool alloc_range(int64_t len, int64_t* off) {
    for (auto it = free_ranges.begin(); it != free_ranges.end(); ++it) {
      if (it->second >= len) {
        *off = it->first;
        const int64_t rest = it->second - len;
        const int64_t o = it->first + len;
        free_ranges.erase(it);
        if (rest > 0) free_ranges[o] = rest;
        return true;
      }
    }
    return false;
  }
  void free_range(int64_t off, int64_t len) {
    auto it = free_ranges.emplace(off, len).first;
    auto nx = std::next(it);
    if (nx != free_ranges.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_ranges.erase(nx);
    }
    if (it != free_ranges.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_ranges.erase(it);
      }
    }
  }

  // Admits queued requests (FIFO among those whose problem is ready); the
  // caller holds the lock.  Returns an error code of the copies.
  int admit() {
    int free_slots = opts.max_segments - eng.live_count();
    for (auto qi = queue.begin(); qi != queue.end();) {
      Req& q = reqs[*qi];
      Mat& m = mats[q.mid];
      if (m.state == 3) {  // its factorization failed
        q.done = 2;
        q.status = m.status;
        q.t_done = std::chrono::steady_clock::now();
        m.users -= 1;
        qi = queue.erase(qi);
        cv_done.notify_all();
        continue;
      }
      if (m.state != 2 || q.nrhs > free_slots) {
        ++qi;
        continue;
      }
      int64_t off = 0;
      if (!alloc_range(q.stride * q.nrhs, &off)) {
        ++qi;
        continue;
      }
      q.off = off;
      q.seg.assign(q.nrhs, -1);
      for (int j = 0; j < q.nrhs; ++j)
        RET(eng.add(m.h, off + j * q.stride, opts.tol, q.b + (size_t)j * m.h->n,
                    cudaMemcpyHostToDevice, s_solve, &q.seg[j]));
      q.done = 1;
      q.t_admit = std::chrono::steady_clock::now();
      q.t_ready = std::max(q.t_submit, m.t_ready);
      free_slots -= q.nrhs;
      m.last_use = tick_count;
      qi = queue.erase(qi);
    }
    return SPAND_OK;
  }

  // Retires finished requests: copies x out, frees their segments and space.
  int retire() {
    for (auto& kv : reqs) {
      Req& q = kv.second;
      if (q.done != 1) continue;
      bool fin = true;
      for (int sid : q.seg) fin = fin && eng.segs[sid].phase == SP_DONE;
      if (!fin) continue;
      Mat& m = mats[q.mid];
      q.iters.resize(q.nrhs);
      q.relres.resize(q.nrhs);
      for (int j = 0; j < q.nrhs; ++j) {
        const Seg& g = eng.segs[q.seg[j]];
        CK(cudaMemcpyAsync(q.x + (size_t)j * m.h->n, eng.X() + g.off, (size_t)g.n * sizeof(double),
                           cudaMemcpyDeviceToHost, s_solve));
        q.iters[j] = g.it;
        q.relres[j] = g.rel;
        if (g.status != SPAND_OK && q.status == SPAND_OK) q.status = g.status;
      }
      CK(cudaStreamSynchronize(s_solve));
      for (int sid : q.seg) eng.remove(sid);
      free_range(q.off, q.stride * q.nrhs);
      q.done = 2;
      q.t_done = std::chrono::steady_clock::now();
      lat_ms.push_back(std::chrono::duration<double, std::milli>(q.t_done - q.t_submit).count());
      wait_factor_ms.push_back(std::chrono::duration<double, std::milli>(q.t_ready - q.t_submit).count());
      wait_queue_ms.push_back(std::chrono::duration<double, std::milli>(q.t_admit - q.t_ready).count());
      solve_ms.push_back(std::chrono::duration<double, std::milli>(q.t_done - q.t_admit).count());
      solves += q.nrhs;
      t_last = q.t_done;
      m.users -= 1;
      m.last_use = tick_count;
      cv_done.notify_all();
      cv_factor.notify_all();
    }
    return SPAND_OK;
  }

  void solve_loop() {
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      int rc = admit();
      if (rc == SPAND_OK && eng.live_count() > 0) {
        max_inflight = std::max(max_inflight, eng.live_count());
        ++tick_count;
        int running = 0;
        lk.unlock();  // ticks run without the lock: submitters are not blocked
        rc = eng.tick(prof, s_solve, &running);
        lk.lock();
        if (rc == SPAND_OK) rc = retire();
      }
      if (rc != SPAND_OK) {
        error = rc;
        error_msg = spand_last_error();
        stop = true;
        cv_done.notify_all();
        cv_factor.notify_all();
        return;
      }
      if (stop) return;
      if (eng.live_count() == 0) {
        cv_solve.wait(lk, [&] {
          if (stop) return true;
          for (int64_t id : queue) {
            const Mat& m = mats[reqs[id].mid];
            if (m.state >= 2) return true;
          }
          return false;
        });
        if (stop) return;
      }
    }
  }

  int start() {
    CK(cudaStreamCreateWithFlags(&s_solve, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&s_factor, cudaStreamNonBlocking));
    RET(eng.reserve(opts.max_entries, opts.max_segments));
    free_ranges.clear();
    free_ranges[0] = eng.cap;
    th_factor = std::thread([this] { factor_loop(); });
    th_solve = std::thread([this] { solve_loop(); });
    return SPAND_OK;
  }

  void shutdown() {
    {
      std::lock_guard<std::mutex> lk(mu);
      stop = true;
    }
    cv_solve.notify_all();
    cv_factor.notify_all();
    cv_done.notify_all();
    if (th_solve.joinable()) th_solve.join();
    if (th_factor.joinable()) th_factor.join();
    if (s_solve) cudaStreamSynchronize(s_solve);
    if (s_factor) cudaStreamSynchronize(s_factor);
  }

  ~Server() {
    shutdown();
    if (s_solve) cudaStreamDestroy(s_solve);
    if (s_factor) cudaStreamDestroy(s_factor);
  }
};

void destroy_engine(Engine* e) { delete e; }

int handle_engine(spand_s* h, Engine** out) {
  if (!h->eng) {
    h->eng = new (std::nothrow) Engine();
    if (!h->eng) return fail(SPAND_ENOMEM, "host allocation failed");
    h->eng->precision = h->precision;
  }
  *out = h->eng;
  return SPAND_OK;
}

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

struct spand_server_s {
  spand::Server srv;
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
  Engine& E = b->eng;
  std::vector<int64_t> offs(count);
  int64_t N = 0;
  for (int i = 0; i < count; ++i) {
    offs[i] = N;
    N += ((int64_t)b->hs[i]->n + 31) & ~int64_t(31);  // segments start on 32-entry boundaries
  }
  RET(E.reserve(N, count));
  std::vector<int> ids(count);
  for (int i = 0; i < count; ++i)
    RET(E.add(b->hs[i], offs[i], tol, bvec[i], cudaMemcpyDeviceToDevice, s, &ids[i]));
  E.ticks = 0;
  int rc = E.run_all(b->prof, s);
  for (int i = 0; rc == SPAND_OK && i < count; ++i) {
    const auto& g = E.segs[ids[i]];
    const cudaError_t ce = cudaMemcpyAsync(xvec[i], E.X() + g.off, (size_t)g.n * sizeof(double),
                                           cudaMemcpyDeviceToDevice, s);
    if (ce != cudaSuccess) rc = fail(SPAND_ECUDA, cudaGetErrorString(ce));
    if (iters) iters[i] = g.it;
    if (relres) relres[i] = g.rel;
    if (g.status != SPAND_OK && rc == SPAND_OK) rc = g.status;
  }
  for (int i = 0; i < count; ++i) E.remove(ids[i]);
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
  b->prof.resolve();
  for (int k = 0; k < KK_COUNT; ++k) out[k] = b->prof.stat[k];
  return SPAND_OK;
}

void spand_batch_destroy(spand_batch_t b) { delete b; }

// ---- several right-hand sides of one problem

int spand_apply_many(spand_t h, const double* r, double* z, int32_t nrhs, int64_t ld, void* stream) {
  if (!h || !r || !z) return fail(SPAND_EINVAL, "null argument");
  if (nrhs < 1 || ld < h->n) return fail(SPAND_EINVAL, "nrhs must be >= 1 and ld >= n");
  if (!h->factored) return fail(SPAND_ESTATE, "spand_apply_many before a successful spand_factor");
  cudaStream_t s = (cudaStream_t)stream;
  Engine* E = nullptr;
  RET(handle_engine(h, &E));
  std::vector<ApSeg> as(nrhs);
  for (int j = 0; j < nrhs; ++j) as[j] = {h, (int64_t)j * ld};
  const bool graph = !h->prof.on && !h->no_graph;
  const double* sc = h->prescale ? h->d_scale : nullptr;  // z = S M~ S r when prescaled
  if (h->precision == 0) {
    if (sc) {
      for (int j = 0; j < nrhs; ++j) launch_scale(h->n, sc, r + (size_t)j * ld, z + (size_t)j * ld, s);
    } else if (r != z) {
      CK(cudaMemcpy2DAsync(z, (size_t)ld * 8, r, (size_t)ld * 8, (size_t)h->n * 8, nrhs,
                           cudaMemcpyDeviceToDevice, s));
    }
    RET(f64::apply_multi(as.data(), nrhs, z, E->ma, h->prof, graph, s));
    if (sc)
      for (int j = 0; j < nrhs; ++j) launch_scale(h->n, sc, z + (size_t)j * ld, z + (size_t)j * ld, s);
    CK(cudaGetLastError());
    return SPAND_OK;
  }
  // FP32 preconditioner: an FP32 copy of the columns (the padding rows are not touched)
  RET(E->vzf.ensure((size_t)nrhs * ld * sizeof(float)));
  float* zf = (float*)E->vzf.p;
  for (int j = 0; j < nrhs; ++j) {
    if (sc) launch_d2f_scaled(h->n, sc, r + (size_t)j * ld, zf + (size_t)j * ld, s);
    else launch_d2f(h->n, r + (size_t)j * ld, zf + (size_t)j * ld, s);
  }
  RET(f32::apply_multi(as.data(), nrhs, zf, E->ma, h->prof, graph, s));
  for (int j = 0; j < nrhs; ++j) {
    if (sc) launch_f2d_scaled(h->n, sc, zf + (size_t)j * ld, z + (size_t)j * ld, s);
    else launch_f2d(h->n, zf + (size_t)j * ld, z + (size_t)j * ld, s);
  }
  CK(cudaGetLastError());
  return SPAND_OK;
}

int spand_pcg_many(spand_t h, const double* b, double* x, int32_t nrhs, int64_t ld, double tol,
                   int32_t* iters, double* relres, void* stream) {
  if (!h || !b || !x) return fail(SPAND_EINVAL, "null argument");
  if (nrhs < 1 || ld < h->n) return fail(SPAND_EINVAL, "nrhs must be >= 1 and ld >= n");
  if (!(tol > 0.0)) return fail(SPAND_EINVAL, "tol must be positive");
  if (!h->factored) return fail(SPAND_ESTATE, "spand_pcg_many before a successful spand_factor");
  cudaStream_t s = (cudaStream_t)stream;
  Engine* E = nullptr;
  RET(handle_engine(h, &E));
  const int64_t stride = ((int64_t)h->n + 31) & ~int64_t(31);
  RET(E->reserve(stride * nrhs, nrhs));
  std::vector<int> ids(nrhs);
  for (int j = 0; j < nrhs; ++j)
    RET(E->add(h, (int64_t)j * stride, tol, b + (size_t)j * ld, cudaMemcpyDeviceToDevice, s, &ids[j]));
  E->ticks = 0;
  int rc = E->run_all(h->prof, s);
  for (int j = 0; rc == SPAND_OK && j < nrhs; ++j) {
    const auto& g = E->segs[ids[j]];
    const cudaError_t ce = cudaMemcpyAsync(x + (size_t)j * ld, E->X() + g.off,
                                           (size_t)g.n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (ce != cudaSuccess) rc = fail(SPAND_ECUDA, cudaGetErrorString(ce));
    if (iters) iters[j] = g.it;
    if (relres) relres[j] = g.rel;
    if (g.status != SPAND_OK && rc == SPAND_OK) rc = g.status;
  }
  for (int j = 0; j < nrhs; ++j) E->remove(ids[j]);
  CK(cudaStreamSynchronize(s));
  if (rc == SPAND_ENOCONV) return fail(SPAND_ENOCONV, "PCG reached maxit for a right-hand side");
  return rc;
}

// ---- server

int spand_server_create(const spand_server_opts* o, spand_server_t* out) {
  if (!out) return fail(SPAND_EINVAL, "null argument");
  *out = nullptr;
  spand_server_opts op{};
  if (o) op = *o;
  if (op.precision < 0 || op.precision > 1) return fail(SPAND_EINVAL, "precision must be 0 or 1");
  if (op.tol < 0.0 || op.tol >= 1.0) return fail(SPAND_EINVAL, "tol must be in [0, 1)");
  if (op.tol == 0.0) op.tol = 1e-10;
  if (op.max_segments <= 0) op.max_segments = 256;
  if (op.max_entries <= 0) op.max_entries = int64_t(32) << 20;
  if (op.hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    op.hbm_budget = (size_t)(0.6 * (double)fr);
  }
  spand_server_s* s = new (std::nothrow) spand_server_s();
  if (!s) return fail(SPAND_ENOMEM, "host allocation failed");
  s->srv.opts = op;
  s->srv.eng.precision = op.precision;
  const int rc = s->srv.start();
  if (rc != SPAND_OK) {
    delete s;
    return rc;
  }
  *out = s;
  return SPAND_OK;
}

int spand_server_add(spand_server_t s, spand_t h, int32_t pinned, int32_t* mid) {
  if (!s || !h || !mid) return fail(SPAND_EINVAL, "null argument");
  Server& S = s->srv;
  if (h->precision != S.opts.precision) return fail(SPAND_EINVAL, "handle precision differs from the server's");
  RET(ensure_device(h));
  std::lock_guard<std::mutex> lk(S.mu);
  for (const auto& m : S.mats)
    if (m.h == h) return fail(SPAND_EINVAL, "handle already added");
  Server::Mat m;
  m.h = h;
  m.pinned = pinned != 0;
  m.state = 0;
  S.mats.push_back(m);
  *mid = (int32_t)S.mats.size() - 1;
  if (m.pinned) {
    S.mats.back().users += 1;  // factored at once; the extra user keeps it resident
    S.cv_factor.notify_all();
  }
  return SPAND_OK;
}

int spand_server_submit(spand_server_t s, int32_t mid, int32_t nrhs, const double* b, double* x,
                        int64_t* rid) {
  if (!s || !b || !x || !rid) return fail(SPAND_EINVAL, "null argument");
  Server& S = s->srv;
  std::lock_guard<std::mutex> lk(S.mu);
  if (S.error != SPAND_OK) return fail(S.error, "server stopped: " + S.error_msg);
  if (mid < 0 || mid >= (int)S.mats.size()) return fail(SPAND_EINVAL, "unknown matrix id");
  Server::Mat& m = S.mats[mid];
  if (nrhs < 1 || nrhs > S.opts.max_segments) return fail(SPAND_EINVAL, "nrhs out of range");
  const int64_t stride = ((int64_t)m.h->n + 31) & ~int64_t(31);
  if (stride * nrhs > S.eng.cap) return fail(SPAND_EINVAL, "request larger than the server's vectors");
  Server::Req q;
  q.id = S.next_id++;
  q.mid = mid;
  q.nrhs = nrhs;
  q.b = b;
  q.x = x;
  q.stride = stride;
  q.t_submit = std::chrono::steady_clock::now();
  if (!S.any) {
    S.any = true;
    S.t_first = q.t_submit;
  }
  m.users += 1;
  S.reqs[q.id] = q;
  S.queue.push_back(q.id);
  *rid = q.id;
  if (m.state == 0) S.cv_factor.notify_all();
  S.cv_solve.notify_all();
  return SPAND_OK;
}

int spand_server_wait(spand_server_t s, int64_t rid, int32_t* iters, double* relres,
                      double* latency_ms) {
  if (!s) return fail(SPAND_EINVAL, "null argument");
  Server& S = s->srv;
  std::unique_lock<std::mutex> lk(S.mu);
  auto it = S.reqs.find(rid);
  if (it == S.reqs.end()) return fail(SPAND_EINVAL, "unknown request id");
  S.cv_done.wait(lk, [&] { return it->second.done == 2 || S.error != SPAND_OK; });
  if (it->second.done != 2) return fail(S.error, "server stopped: " + S.error_msg);
  Server::Req q = it->second;
  S.reqs.erase(it);
  lk.unlock();
  for (int j = 0; j < q.nrhs; ++j) {
    if (iters) iters[j] = j < (int)q.iters.size() ? q.iters[j] : 0;
    if (relres) relres[j] = j < (int)q.relres.size() ? q.relres[j] : 0.0;
  }
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(q.t_done - q.t_submit).count();
  if (q.status != SPAND_OK) return fail(q.status, "request failed");
  return SPAND_OK;
}

int spand_server_get_stats(spand_server_t s, spand_server_stats* st) {
  if (!s || !st) return fail(SPAND_EINVAL, "null argument");
  Server& S = s->srv;
  std::lock_guard<std::mutex> lk(S.mu);
  memset(st, 0, sizeof(*st));
  auto pct = [](std::vector<double> l, double p) {
    if (l.empty()) return 0.0;
    std::sort(l.begin(), l.end());
    const size_t i = std::min(l.size() - 1, (size_t)std::ceil(p * (double)l.size()) - (p > 0 ? 1 : 0));
    return l[i];
  };
  st->requests = (int64_t)S.lat_ms.size();
  st->solves = S.solves;
  st->p50_ms = pct(S.lat_ms, 0.50);
  st->p99_ms = pct(S.lat_ms, 0.99);
  st->max_ms = pct(S.lat_ms, 1.0);
  st->factor_wait_p50_ms = pct(S.wait_factor_ms, 0.50);
  st->factor_wait_p99_ms = pct(S.wait_factor_ms, 0.99);
  st->queue_p50_ms = pct(S.wait_queue_ms, 0.50);
  st->queue_p99_ms = pct(S.wait_queue_ms, 0.99);
  st->solve_p50_ms = pct(S.solve_ms, 0.50);
  st->solve_p99_ms = pct(S.solve_ms, 0.99);
  // the slowest request's parts
  size_t w = 0;
  for (size_t i = 1; i < S.lat_ms.size(); ++i)
    if (S.lat_ms[i] > S.lat_ms[w]) w = i;
  if (!S.lat_ms.empty()) {
    st->max_split_ms[0] = S.wait_factor_ms[w];
    st->max_split_ms[1] = S.wait_queue_ms[w];
    st->max_split_ms[2] = S.solve_ms[w];
  }
  st->elapsed_s = S.any ? std::chrono::duration<double>(S.t_last - S.t_first).count() : 0.0;
  st->solves_per_s = st->elapsed_s > 0 ? (double)S.solves / st->elapsed_s : 0.0;
  st->ticks = S.tick_count;
  st->max_inflight = S.max_inflight;
  st->resident_bytes = (int64_t)S.resident;
  int nres = 0;
  for (const auto& m : S.mats) nres += m.state == 2;
  st->resident_problems = nres;
  return SPAND_OK;
}

void spand_server_destroy(spand_server_t s) { delete s; }

}  // extern "C"
