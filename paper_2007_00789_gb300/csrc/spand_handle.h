// Internal: the handle of the C ABI and the host-side helpers shared by the
// FP64 and FP32 orchestration (factor_core.cu, compiled once per precision)
// and the ABI layer (api.cu).
#pragma once

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "spand_internal.h"

namespace spand {

int fail(int code, const std::string& msg);  // records spand_last_error(), returns code

#define CK(call)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return ::spand::fail(e_ == cudaErrorMemoryAllocation ? SPAND_ENOMEM : SPAND_ECUDA, \
                           std::string(#call) + ": " + cudaGetErrorString(e_));     \
  } while (0)

#define RET(call)                    \
  do {                               \
    int rc_ = (call);                \
    if (rc_ != SPAND_OK) return rc_; \
  } while (0)


// Bump allocator over device chunks; pointers stay valid until release().
struct DevArena {
  struct Chunk {
    char* p;
    size_t cap, used;
  };
  std::vector<Chunk> chunks;
  size_t cur = 0;
  size_t min_chunk = size_t(64) << 20;

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
  int gen = 0;  // bumped whenever p changes (graphs that captured the old p are stale)
  int ensure(size_t bytes) {
    if (bytes <= cap) return SPAND_OK;
    ++gen;
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
  KK_VEC, KK_RRQR_GRID, KK_SCHUR_TC, KK_AP_SWEEP, KK_COUNT
};
static const char* const kKindName[KK_COUNT] = {
    "pack", "merge", "potrf", "trsm", "schur", "scale_potrf", "scale_trsm", "scale_copy",
    "rrqr", "e_copy", "trtri", "form_qt", "apply_interior", "apply_scale", "apply_qe", "spmv",
    "dot", "vector", "rrqr_grid", "schur_tc", "apply_sweep"};

struct Prof {
  bool on = false;
  int tag = -1;  // caller-set label of the next launches (e.g. the apply's stage), for the dump
  struct Pend {
    int kind;
    cudaEvent_t a, b;
    double flops, bytes;
    int tag;
  };
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<Pend> pend;
  spand_kernel_stat stat[KK_COUNT];
  std::map<int, double> rrqr_tag_ms;  // cluster-RRQR launch time by tag (the autotuner's key)
  Prof() { clear(); }
  void clear() {
    rrqr_tag_ms.clear();
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
    Pend p{kind, ev(), ev(), flops, bytes, tag};
    cudaEventRecord(p.a, s);
    launch();
    cudaEventRecord(p.b, s);
    pend.push_back(p);
  }
  void add_flops(int kind, double flops) {
    if (on) stat[kind].flops += flops;
  }
  // call after the stream has been synchronised; SPAND_DEBUG_PROF=1 in the
  // environment also prints every launch (kind, tag, ms, flops, bytes) to stderr
  void resolve() {
    static const bool dump = [] {
      const char* e = getenv("SPAND_DEBUG_PROF");
      return e && e[0] == '1';
    }();
    for (auto& p : pend) {
      float ms = 0.f;
      cudaEventSynchronize(p.b);
      cudaEventElapsedTime(&ms, p.a, p.b);
      if (dump)
        fprintf(stderr, "spand launch: %s tag %d ms %.4f flops %.4g bytes %.4g\n", kKindName[p.kind],
                p.tag, ms, p.flops, p.bytes);
      stat[p.kind].launches += 1;
      stat[p.kind].total_ms += ms;
      if (p.kind == KK_RRQR) rrqr_tag_ms[p.tag % 100] += ms;  // by base bucket
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

constexpr int kQrClusterSmem = 224 * 1024;  // shared-memory slice per CTA of the on-chip RRQR
constexpr int kNumSMs = 152;                 // GB300

enum PhaseKind { PH_INTERIOR = 0, PH_SCALE = 1, PH_QE = 2 };
struct Phase {
  int kind, begin, end, max_m;
  double flops, bytes;  // algorithmic, forward sweep (the backward one is the same)
  int max_cols = 0;     // widest neighbour gather
  int K = 1;            // CTAs per operator (thread-block cluster)
  int stage = 0, colour = 0;  // position in the sweep: (stage, kind, colour) orders the phases
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
  // by cluster size, and within one cluster size the largest operators first
  // (CTAs are handed out in order as SMs free up: the launch ends on small ones)
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (Ks[a] != Ks[b]) return Ks[a] < Ks[b];
    return fl[a] > fl[b];
  });
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

// CUDA-graph replay of the refactorization of one problem or of a batch of
// problems factored together: one graph per stage (plus one for the work after
// the last stage).  The graphs stay valid while every stage reproduces the
// ranks they were built with and no problem of the group has been factored
// another way since (its arena layout may then differ).
struct FactorGroup {
  struct StageGraph {
    char* d_blob = nullptr;  // the stage's task tables (kept: the graph reads them)
    size_t cap = 0;
    cudaGraph_t graph = nullptr;  // the captured stage (kept for the chain below)
    cudaGraphExec_t exec = nullptr;
    // counters of the stage: problem index, offset and cluster count per problem
    std::vector<int> who, ncl;
    std::vector<size_t> ioff;
    size_t nints = 0;
    std::vector<int> expect;  // per problem: ranks then reflector counts at capture
  };
  std::vector<StageGraph> sg;
  // The whole refactorization as one graph: stage k+1 is the body of a
  // conditional node that a check kernel after stage k enables only when the
  // stage's ranks and reflector counts equal the ones the graphs were built
  // with and no error word is set; the host reads one status block at the end.
  cudaGraphExec_t chain = nullptr;
  DevBuf chain_buf;             // status (4 ints), check tables, expected ranks, flags
  size_t chain_flags = 0;       // int offset of the flags in chain_buf
  size_t chain_ints = 0;        // ints of chain_buf read back after a launch
  std::vector<std::vector<size_t>> chain_foff;  // per stage, per problem: flags offset
  bool chain_failed = false;    // building it failed once: replay stage by stage
  bool valid = false;
  int prec = -1;
  std::vector<uint64_t> layouts;  // layout_id of every problem when the graphs were built
  DevBuf ints;                     // live counters of the running stage (device)
  DevBuf tables;                   // task tables when not capturing
  int* h_ints = nullptr;           // pinned readback of the counters
  size_t h_cap = 0;
  cudaStream_t cap_stream = nullptr;
  // the previous stage's apply operators (explicit inverses, Q^T, E-tilde
  // copies) are formed on a side branch beside the stage's own launches
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  void drop() {
    for (auto& g : sg) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.graph) cudaGraphDestroy(g.graph);
      g.exec = nullptr;
      g.graph = nullptr;
    }
    if (chain) cudaGraphExecDestroy(chain);
    chain = nullptr;
    chain_foff.clear();
    valid = false;
  }
  void release() {
    drop();
    for (auto& g : sg)
      if (g.d_blob) cudaFree(g.d_blob);
    sg.clear();
    ints.release();
    tables.release();
    chain_buf.release();
    if (h_ints) cudaFreeHost(h_ints);
    h_ints = nullptr;
    h_cap = 0;
    if (cap_stream) cudaStreamDestroy(cap_stream);
    cap_stream = nullptr;
    if (side) cudaStreamDestroy(side);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    side = nullptr;
    ev_fork = ev_join = nullptr;
  }
};

// A merged preconditioner apply over several problems whose vectors sit in
// one concatenated vector: problem i's operators act on z + zoff_i.  The
// phases of all problems with the same (stage, kind, colour, cluster size)
// become one launch; each problem's own phase order is kept.  The plan (and a
// CUDA graph of it) is cached for the last set of problems and offsets.
struct ApSeg {
  spand_s* h;
  int64_t zoff;
};
struct Engine;                  // multi-segment PCG (engine.cu)
void destroy_engine(Engine* e);
struct MultiApply {
  std::vector<std::pair<const spand_s*, int64_t>> key;
  std::vector<uint64_t> layouts;
  struct Launch {
    int kind, K, max_m, max_cols, max_nvec, nitems, ntasks;
    int stage, colour;  // launches of equal (stage, kind, colour) are independent
    size_t item0;
    double flops, bytes;
  };
  std::vector<Launch> launches;  // forward order
  DevBuf items;
  cudaGraphExec_t exec = nullptr;
  const void* gz = nullptr;
  cudaStream_t cap_stream = nullptr;
  // side streams of the captured graph: the independent launches of one
  // logical phase (its cluster-size groups) become parallel graph nodes
  static constexpr int kSide = 4;
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork = nullptr, join[kSide] = {};
  void drop() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    gz = nullptr;
    key.clear();
    layouts.clear();
    launches.clear();
  }
  void release() {
    drop();
    items.release();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    cap_stream = nullptr;
    for (int i = 0; i < kSide; ++i) {
      if (side[i]) cudaStreamDestroy(side[i]);
      if (join[i]) cudaEventDestroy(join[i]);
      side[i] = nullptr;
      join[i] = nullptr;
    }
    if (fork) cudaEventDestroy(fork);
    fork = nullptr;
  }
};

}  // namespace spand

struct spand_s {
  int n = 0, dim = 0, nlevels = 0, scheme = 0, skip = 0;
  int64_t nnz = 0;
  double eps = 0.0;
  int maxit = 500, true_every = 50, max_restarts = 2;
  spand::Tree tree;
  std::vector<spand::StageSym> st;
  spand::host_vec<int32_t> h_rowptr, h_colind;
  spand::host_vec<double> h_val;
  // device copy of A
  int32_t* d_rowptr = nullptr;
  int32_t* d_colind = nullptr;
  double* d_val = nullptr;
  int64_t* d_pack = nullptr;     // stage-0 destination of every nonzero
  // diagonal prescaling: the factorization is of D^{-1/2} A D^{-1/2} (values
  // d_fval) and the apply is D^{-1/2} M~ D^{-1/2}; without it d_fval = d_val
  bool prescale = false;
  spand::host_vec<double> h_scale, h_fval;
  double* d_scale = nullptr;
  double* d_fval = nullptr;
  int64_t pack_split = 0;        // interior part / interface part of the stage-0 layout
  spand::host_vec<int64_t> h_pack;
  // memory
  spand::DevArena farena;
  spand::DevBuf scratch[2];
  spand::DevBuf tables;
  int* d_err = nullptr;
  int* h_pinned = nullptr;       // rank/nref/err readback
  size_t h_pinned_cap = 0;
  // factor results
  bool factored = false;
  std::vector<std::vector<int>> sizes, ranks, nrefs, flags;
  std::vector<spand::Phase> phases;
  void* d_api = nullptr;  // apply descriptors of the handle's precision
  void* d_aps = nullptr;
  void* d_apq = nullptr;
  int precision = 0;      // 0: FP64 factor and apply; 1: FP32 factor and apply (PCG stays FP64)
  float* d_rf = nullptr;  // FP32 copy of the vector an FP32 apply works on
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
  spand::Prof prof;
  // 0: choose per interface; 1: always the global-memory kernel; 2: clusters <= 8;
  // 3: always the streamed multi-CTA kernel; 4: always the on-chip multi-CTA kernel where it fits;
  // 5: as 0 with the multi-CTA tasks streamed
  int rrqr_path = 0;
  int rrqr_threads = 0;  // CTA size of the cluster RRQR (256, 512); 0 = automatic
  bool schur_simt = false;  // FP32: keep every Schur tile on the SIMT path (no tensor cores)
  // spand_tune's choices per base bucket b0 = 1..5 (the smallest thread-block
  // cluster, 2^(b0-1) CTAs, whose shared memory holds an interface's block):
  // CTA size of the cluster RRQR (0 = 256) and growth factor of the cluster size
  int tune_thr[6] = {0, 0, 0, 0, 0, 0};
  int tune_grow[6] = {0, 0, 0, 0, 0, 0};
  bool tuning = false;  // inside spand_tune: RRQR launches split by base bucket
  // the persistent single-vector apply (k_ap_sweep): its program, scratch
  // vector and barrier words (factor arena), launch shape and work
  int apply_mode = 0;   // spand_opts.apply_kernels: 0 automatic, 1 per phase, 2 persistent
  int sweep_pref = -1;  // spand_tune's timed choice: 0 persistent, 1 per phase, -1 none yet
  bool sweep_valid = false;
  // untuned automatic choice: the persistent sweep for FP32 factors from this
  // many unknowns up (below it a sub-phase holds too few items to pay for its
  // grid barrier; FP64 keeps the per-phase launches)
  static constexpr int64_t kSweepMinN = 1 << 21;
  void *sweep_phases = nullptr, *sweep_items = nullptr, *sweep_y = nullptr;
  int* sweep_ws = nullptr;
  long long* sweep_trace = nullptr;  // SPAND_DEBUG_SWEEP=1: clock per sub-phase
  std::vector<int> sweep_trace_kinds, sweep_trace_items;
  int sweep_nph = 0, sweep_ctas = 0, sweep_smem = 0;
  double sweep_flops = 0.0, sweep_bytes = 0.0;
  static constexpr long long kSweepWait = 1LL << 25;  // polls per barrier, a second or so
  int cluster_state[2][5] = {{-1, -1, -1, -1, -1}, {-1, -1, -1, -1, -1}};  // per precision
  spand::Engine* eng = nullptr;  // multi-RHS apply and PCG of this problem (created on first use)
  spand::FactorGroup fg;      // stage graphs of this problem factored on its own
  uint64_t layout_id = 0;     // new value at every full factorization (arena layout changes)
  cudaStream_t cap_stream = nullptr;  // capture needs a stream other than the legacy one
  spand::MultiApply self_ma;  // the apply plan (and graph) of this problem alone
  bool no_graph = false;  // plain launches only (set by the allocation-free PCG)
  // bounded wait of the multi-CTA RRQR: polls per barrier before it gives up, and
  // the testing hook that makes the first barrier unreachable (spand_test_set_qr_wait)
  static constexpr long long kQrWaitDefault = 1LL << 24;  // about a second
  long long qr_wait_limit = kQrWaitDefault;
  int qr_wait_extra = 0;
  void drop_graphs() {
    fg.drop();
    self_ma.drop();
  }
  void free_graphs() {
    drop_graphs();
    fg.release();
    self_ma.release();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    cap_stream = nullptr;
  }
};

namespace spand {
int ensure_device(spand_s* h);  // first device use: upload A and the stage-0 pack map
namespace f64 {
int factor(spand_s* h, cudaStream_t s);
// Factors count problems of this precision together: every kernel step of a
// stage is one launch over the tasks of all problems.
int factor_group(spand_s* const* hs, int count, FactorGroup& G, Prof& P, cudaStream_t s);
int apply(spand_s* h, const double* r, double* z, cudaStream_t s);
int apply_multi(const ApSeg* segs, int nseg, double* z, MultiApply& M, Prof& P, bool graph,
                cudaStream_t s);
}  // namespace f64
namespace f32 {
int factor(spand_s* h, cudaStream_t s);
int factor_group(spand_s* const* hs, int count, FactorGroup& G, Prof& P, cudaStream_t s);
int apply(spand_s* h, const float* r, float* z, cudaStream_t s);
int apply_multi(const ApSeg* segs, int nseg, float* z, MultiApply& M, Prof& P, bool graph,
                cudaStream_t s);
}  // namespace f32
}  // namespace spand
