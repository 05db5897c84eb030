/*
 * spand.h -- C ABI of a single-GPU (sm_103a) Sparsified Nested Dissection
 * preconditioner with first- and second-order sparsification, and the PCG
 * solver that uses it.
 *
 * Method: Klockiewicz, Cambier, Humble, Tchelepi, Darve, "Second Order
 * Accurate Hierarchical Approximate Factorization of Sparse SPD Matrices",
 * arXiv 2007.00789.  Section references below are to that paper.
 *
 * Conventions shared by every entry point
 *   - Return value: SPAND_OK (0) on success, a negative SPAND_E* code on
 *     failure.  spand_strerror() turns a code into text; spand_last_error()
 *     gives a message about the most recent failure in the calling thread.
 *   - Floating point is IEEE binary64 everywhere.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the current device (e.g. torch.Tensor.data_ptr()).
 *   - stream: a cudaStream_t cast to void* (NULL = the legacy default
 *     stream).  Every device-side effect is ordered on that stream; calls
 *     that return results to the host (ranks, iteration counts) synchronise
 *     it before returning.
 *   - A handle is not thread safe: use one handle from one thread at a time.
 */
#ifndef SPAND_H
#define SPAND_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPAND_OK 0
#define SPAND_EINVAL (-1)   /* bad argument: CSR, coordinates, eps, levels, scheme, sizes */
#define SPAND_ENOTSPD (-2)  /* a Cholesky pivot was not positive (A is not SPD) */
#define SPAND_ENOMEM (-3)   /* a device or host allocation failed */
#define SPAND_ECUDA (-4)    /* a CUDA runtime call failed */
#define SPAND_ENOCONV (-5)  /* PCG reached maxit; x holds the last iterate */
#define SPAND_ESTATE (-6)   /* call out of order (e.g. apply before factor) */
#define SPAND_ETIMEOUT (-7) /* a bounded device-side wait ran out (the CTAs of a multi-CTA RRQR
                               lost each other); the handle is left unfactored, the device
                               stays usable, and the call may be retried */

/* Sparsification schemes (Algorithm 1 / §2). */
#define SPAND_FIRST_ORDER 0            /* eq. trailing-1: E dropped */
#define SPAND_SECOND_ORDER_FULL 1      /* eq. trailing-2: E kept, only E^T E dropped */
#define SPAND_SECOND_ORDER_SUPERFINE 2 /* eq. trailing-3: only E_2 kept (QR run to eps^2) */

typedef struct spand_s* spand_t;

/* Sparse SPD matrix A (§1, "A x = b, A sparse SPD").  Full symmetric
 * pattern: both triangles present, column indices ascending within each row,
 * 0-based int32 indices.  All three arrays are host pointers; analyze copies
 * what it needs, the caller keeps ownership. */
typedef struct {
  int32_t n;
  int64_t nnz;
  const int32_t* rowptr; /* n+1 entries, rowptr[0] = 0, rowptr[n] = nnz */
  const int32_t* colind; /* nnz entries */
  const double* val;     /* nnz entries */
} spand_csr;

/* Optional knobs; pass NULL for the defaults shown. */
typedef struct {
  int32_t skip;           /* stages without scaling/sparsification; <0 = default
                             clamp(4 - round(log2((n / 2^(ell-1)) / 25)), 0, ell-2),
                             i.e. 4 at the paper's ell = round(log2(n/25)) (§4) */
  int32_t maxit;          /* PCG iteration cap; <=0 = 500 */
  int32_t true_res_every; /* replace the recursive residual by b - A x every this
                             many iterations; <=0 = 50 */
  int32_t max_restarts;   /* PCG restarts when the true residual misses tol; <0 = 2 */
  int32_t rrqr_kernel;    /* 0 = keep each interface block on chip (one CTA, or a thread-block
                             cluster of up to 16 CTAs) where it fits, else spread it over several
                             CTAs of a cooperative launch (at most one per SM) that keep their
                             slices in shared memory where they fit, else stream them from
                             global memory;
                             1 = always stream from global memory with one CTA per interface;
                             2 = as 0 with clusters of at most 8 CTAs (the portable cluster
                             size); 3 = always the multi-CTA streamed kernel; 4 = always the
                             multi-CTA on-chip kernel where the block fits (else streamed);
                             5 = as 0, but blocks too wide for a cluster always streamed.
                             Same results up to the order of some FP sums. */
  int32_t precision;      /* 0 = FP64 factorization and apply (the default);
                             1 = FP32 factorization and apply, with the RRQR rank decisions
                             (nu_0 and every step within 1e-4 of the threshold) taken on norms
                             recomputed in FP64; PCG, its dot products and residuals stay FP64 */
  int32_t plain_launches; /* 0 = replay refactorizations and applies from CUDA graphs (the
                             default); 1 = plain kernel launches only.  Same kernels, same
                             results; meant for profilers that cannot replay graph nodes. */
  int32_t rrqr_threads;   /* threads per CTA of the on-chip RRQR: 256 or 512; 0 = the
                             library's choice.  Changes only the order of some FP sums. */
  int32_t partition;      /* 0 = geometric nested dissection of the coordinates (algebraic when
                             coords is NULL or dim is 0); 1 = algebraic nested dissection of the
                             graph of A: breadth-first bisection, interfaces keyed by the
                             subdomains their vertices reach (for general SPD input) */
  int32_t prescale;       /* 1 = factor D^{-1/2} A D^{-1/2} (D = diag(A)) and precondition with
                             D^{-1/2} M~ D^{-1/2}; SPAND_ENOTSPD at analyze if a diagonal entry is
                             not positive; 0 = no prescaling (the default) */
  int32_t schur_simt;     /* precision = 1 only: 0 = the Schur updates of large blocks (both
                             sides >= 64, contribution depth >= 96) run on the tensor cores in
                             TF32 with a head/tail split of each operand (about FP32 accuracy),
                             the others on the FP32 pipe (the default); 1 = all on the FP32
                             pipe.  FP64 factorizations never use the tensor cores. */
  int32_t apply_kernels;  /* form of the single-vector apply (spand_apply, spand_pcg): 0 =
                             automatic (the default: spand_tune's timed choice once it has
                             run, before that the persistent form for FP32 factors with
                             n >= 2^21, else the per-phase launches); 1 = one
                             launch per phase, as the multi-vector forms; 2 = one persistent
                             cooperative launch that walks every phase of the sweep. */
} spand_opts;

/* Summary of a factorization (§4 notation). */
typedef struct {
  int32_t n;
  int64_t nnz_a;           /* nnz(A) */
  int64_t nnz_factor;      /* stored entries of L_s, W_s, Z_p, Householder V/tau, E-tilde */
  double mu;               /* nnz_factor / nnz_a */
  int32_t nlevels;         /* ell */
  int32_t skip;
  int32_t scheme;
  double eps;
  int32_t nstages;         /* = nlevels */
  int32_t nclusters_total; /* sum over stages of the clusters alive at the stage start */
  int32_t ninterfaces_sparsified;
  double factor_ms;        /* wall time of the last spand_factor (host clock, synchronised) */
  double pcg_ms;           /* wall time of the last spand_pcg */
  int32_t pcg_iters;       /* iterations of the last spand_pcg */
  double pcg_relres;       /* true relative residual at the end of the last spand_pcg */
  int64_t kernel_launches; /* kernels launched by the last spand_factor */
  int64_t device_bytes;    /* device memory held by the handle */
} spand_stats;

/* Symbolic analysis (the multilevel spaND partitioning of §3, built
 * geometrically from grid coordinates).  Host-only: A is copied into the
 * handle and uploaded to the device by the first call that needs it
 * (spand_factor or spand_matvec), so analyze works without a GPU.  Runs on up
 * to 16 host threads, which the library keeps (idle) between calls; analyses
 * may run concurrently on different handles.
 *   A       -- the matrix (host arrays, see spand_csr).
 *   coords  -- host, n x dim row-major coordinates of the unknowns (grid
 *              coordinates; only their order along each axis matters).
 *   dim     -- 1..3.
 *   nlevels -- ell >= 1: nested dissection to depth ell-1, ell stages.
 *   eps     -- RRQR tolerance in [0, 1] (Algorithm 1); 0 gives an exact block
 *              Cholesky factorization (§3.2).
 *   scheme  -- SPAND_FIRST_ORDER / _SECOND_ORDER_FULL / _SECOND_ORDER_SUPERFINE.
 *   out     -- receives the new handle (owned by the caller; spand_destroy).
 * Errors: SPAND_EINVAL for a malformed CSR (unsorted or out-of-range columns,
 * asymmetric pattern, missing diagonal), n < 1, dim out of range, eps outside
 * [0, 1], nlevels < 1, an empty nested-dissection box, or scheme out of
 * range.  No device memory is kept on failure. */
int spand_analyze(const spand_csr* A, const double* coords, int dim, int nlevels,
                  double eps, int scheme, const spand_opts* opts, spand_t* out);

/* Numerical factorization, Algorithm 2: per level, eliminate interiors
 * (block Cholesky), scale interfaces (eq. prescale), sparsify interfaces
 * (Algorithm 1 + the chosen scheme), merge and recurse; the top separator is
 * factored by dense Cholesky.  May be called again (refactor) on the same
 * handle.  Synchronises the stream once per level to learn the ranks.
 * Errors: SPAND_ENOTSPD (the handle stays valid but unfactored),
 * SPAND_ENOMEM, SPAND_ECUDA, SPAND_ETIMEOUT (the barrier wait of a multi-CTA
 * RRQR ran out; the handle stays valid but unfactored). */
int spand_factor(spand_t h, void* stream);

/* Autotuner of the RRQR launch shapes (a launch-configuration search; the
 * paper has no counterpart).  Interface blocks fall into size buckets 1..5,
 * keyed by the smallest thread-block cluster (1, 2, 4, 8 or 16 CTAs) whose
 * shared memory holds the block.  spand_tune factors the problem once per
 * candidate shape -- 256 or 512 threads per CTA, times the cluster size of the
 * default rule or twice it -- timing every RRQR launch with CUDA events on the
 * stream, keeps the fastest shape of every bucket, and factors once more with
 * it (graphs captured), leaving the handle factored as spand_factor does.  The
 * handle keeps the choices for later factorizations (also inside a batch).
 * Then, unless spand_opts.apply_kernels fixes the form, it times the two forms
 * of the single-vector apply (one persistent launch, or one launch per phase)
 * and keeps the faster.  The choices change only the order of some floating-point sums.
 *   choice -- host, may be NULL: 12 int32: the chosen CTA size and cluster
 *             growth of buckets 1..5 (0 where no interface fell in a bucket),
 *             then the apply form (0 persistent, 1 per phase) and a zero.
 * Costs five factorizations and a few applies.  Errors: those of
 * spand_factor. */
int spand_tune(spand_t h, void* stream, int32_t* choice);

/* Testing hook for the one bounded device-side wait of the factorization:
 * the barrier between the CTAs of a multi-CTA RRQR (Algorithm 1 on interface
 * blocks too wide for a thread-block cluster; rrqr_kernel = 3 forces it for
 * every interface).  limit: polls of the barrier counter before a wait gives
 * up (<= 0 restores the default, about a second); unreachable != 0 raises the
 * first barrier's target by one, so that it is never met and every wait of
 * the task runs out after `limit` polls.  The next spand_factor then returns
 * SPAND_ETIMEOUT and leaves the handle unfactored; no kernel is left
 * running.  Takes effect at the next spand_factor (the handle's captured
 * graphs are dropped).  Not meant for production use. */
int spand_test_set_qr_wait(spand_t h, int64_t limit, int32_t unreachable);

/* z = M r with M = L^{-T} L^{-1} (Algorithm 2 caption).  r and z are device
 * arrays of n doubles; they may alias.  Requires a successful spand_factor,
 * else SPAND_ESTATE. */
int spand_apply(spand_t h, const double* r, double* z, void* stream);

/* Preconditioned CG on A x = b with M as preconditioner, x0 = 0, stopping
 * when ||r_k||_2 / ||b||_2 < tol (§4).  b and x are device arrays of n
 * doubles (x is overwritten).  iters and relres (host, may be NULL) receive
 * the iteration count and the true relative residual ||b - A x|| / ||b||.
 * Returns SPAND_ENOCONV if maxit is reached. */
int spand_pcg(spand_t h, const double* b, double* x, double tol, int32_t* iters,
              double* relres, void* stream);

/* Same as spand_pcg with HOST arrays b and x: the host->device copy of b
 * and the device->host copy of x are part of the call. */
int spand_pcg_host(spand_t h, const double* b_host, double* x_host, double tol,
                   int32_t* iters, double* relres, void* stream);

/* Same as spand_pcg, but allocates nothing, for callers that cannot allocate
 * device memory while they solve: a program whose GPU memory is entirely
 * reserved by another allocator, or a loop that must not allocate once it
 * runs.  (The paper has no counterpart; this is a deployment variant.)
 * The four work vectors live in one device array that is part of the
 * library image (about 8 MiB, held by every GPU that loads the library
 * until the process exits), so the call needs no cudaMalloc / cudaFree and
 * no pinned host memory.
 *   - Limit: n <= 262144; larger systems return SPAND_EINVAL before any
 *     device work.  The handle must have been factored (SPAND_ESTATE).
 *   - The first call on a device looks up the array's device address for
 *     that device (cudaGetSymbolAddress) and keeps it for the rest of the
 *     process; make that first call before any stream capture on that
 *     device.  The address belongs to the device's primary context: do not
 *     call this after cudaDeviceReset (or from a non-primary driver context)
 *     in the same process, since the kept address would then name memory of
 *     a context that no longer exists.
 *   - Every call, from any handle, uses the same array, which keeps the
 *     previous call's contents (x is set to 0 and the scalars are cleared at
 *     the start, so stale data does not leak into a result).  Calls that
 *     overlap on the GPU (different streams or threads) race on it and give
 *     wrong results: serialise them.
 *   - Profiling (spand_set_profiling) is suspended for the call.
 *   - Handles analysed with precision = 1 are refused with SPAND_EINVAL.
 * Arguments and results are those of spand_pcg. */
int spand_pcg_noalloc(spand_t h, const double* b, double* x, double tol, int32_t* iters,
                      double* relres, void* stream);

/* Several right-hand sides at once (the block form of spand_apply and
 * spand_pcg): column j of r, z, b, x starts at element j * ld (device arrays,
 * ld >= n).  spand_apply_many computes z_j = M r_j for every column with one
 * launch per apply phase over all columns (r == z allowed); spand_pcg_many
 * runs the PCG of spand_pcg for every column, all columns advancing together
 * (iters, relres: host arrays of nrhs entries, NULL allowed).  Results per
 * column equal those of the single-column calls up to the order of the
 * dot-product sums and the apply's atomic accumulation.  Errors as spand_apply
 * and spand_pcg; SPAND_EINVAL for nrhs < 1 or ld < n. */
int spand_apply_many(spand_t h, const double* r, double* z, int32_t nrhs, int64_t ld, void* stream);
int spand_pcg_many(spand_t h, const double* b, double* x, int32_t nrhs, int64_t ld, double tol,
                   int32_t* iters, double* relres, void* stream);

/* y = A x with the uploaded A (device arrays of n doubles). */
int spand_matvec(spand_t h, const double* x, double* y, void* stream);

/* Factorization summary; s is a host struct filled by the call. */
int spand_info(spand_t h, spand_stats* s);

/* Ranks decided by Algorithm 1, for parity checks.  For every stage k in
 * 0..ell-1 and every cluster alive at the start of stage k (in cluster-id
 * order), out[] receives three int32: the cluster's size at the start of the
 * stage, its coarse rank (-1 when the stage does not sparsify or the cluster
 * is an interior) and near-tie flags of its pivoted QR (bit 0: at some step
 * the two largest candidate column norms were within 1e-12 relative; bit 1:
 * a step's norm was within 1e-10 relative of the eps threshold; there, a
 * differently rounded correct implementation may choose another pivot or
 * rank).  *count receives the number of clusters; if cap (in clusters) is too
 * small nothing is written and SPAND_EINVAL is returned with *count set.
 * Host pointers.  Requires a successful spand_factor (else SPAND_ESTATE). */
int spand_ranks(spand_t h, int32_t* out, int64_t cap, int64_t* count);

/* Cluster id of every vertex at stage k (-1 for vertices already
 * eliminated); out is a host array of n int32.  Available after analyze.
 * The ids follow the analysis' own stage structure: each vertex's stage-0
 * cluster, carried through the merges of the stages before k. */
int spand_cluster_map(spand_t h, int stage, int32_t* out);

/* Number of stages (ell) and of clusters alive at the start of stage k. */
int spand_num_clusters(spand_t h, int stage, int32_t* nclusters);

/* Per-kernel timing, for roofline measurements.  When enabled, every launch
 * group of spand_factor / spand_apply / spand_pcg is bracketed by CUDA events
 * on the caller's stream; the elapsed times are accumulated per kernel kind
 * together with the kind's algorithmic work (FLOPs and bytes counted on the
 * host from the task sizes, e.g. m^3/3 per Cholesky, 6 (m-t)(N-t) per QR step).
 * Enabling or disabling clears the accumulated statistics; reading them waits
 * for the recorded launches to finish (an event synchronisation). */
typedef struct {
  char name[32];
  int64_t launches;
  double total_ms;
  double flops;
  double bytes;
} spand_kernel_stat;

int spand_set_profiling(spand_t h, int on);
/* out: host array of cap entries; *count receives the number of kernel kinds.
 * Launches still in flight are waited for and counted. */
int spand_kernel_stats(spand_t h, spand_kernel_stat* out, int cap, int* count);

/* ---------------------------------------------------------------------------
 * Batches of independent problems.
 *
 * A batch groups analysed handles of one precision.  spand_batch_factor runs
 * the numerical factorization of all of them together: stage k of every
 * problem (k counted from the leaves) goes into the same launches, one launch
 * per kernel step, so many small and uneven problems fill the GPU as one large
 * one does (Algorithm 2 is applied to each problem exactly as by
 * spand_factor; the results are the same as factoring each handle on its
 * own).  Refactorizations with unchanged ranks replay CUDA graphs of the whole
 * batch, as spand_factor does for one handle.
 *
 * spand_batch_pcg solves A_i x_i = b_i for every problem i with the PCG of §4
 * (x0 = 0, per-problem tol, maxit, true-residual and restart rules), all
 * problems advancing together; each step of all problems is one launch, and
 * the preconditioner applies are merged across problems.
 *
 * Ownership: the batch references the handles, which the caller keeps alive
 * (and does not destroy) until spand_batch_destroy.  Factoring a member
 * handle on its own in between is allowed; the batch then rebuilds its graphs.
 * Errors: SPAND_EINVAL (null, empty, mixed precisions, a handle listed twice),
 * the errors of spand_factor (SPAND_ENOTSPD names the problem index), and of
 * spand_pcg (SPAND_ENOCONV if any problem reached maxit; the others are
 * still solved).  Stream-ordered; the calls synchronise the stream.
 * --------------------------------------------------------------------------- */
typedef struct spand_batch_s* spand_batch_t;

/* handles: host array of count analysed handles. */
int spand_batch_create(const spand_t* handles, int32_t count, spand_batch_t* out);
int spand_batch_factor(spand_batch_t b, void* stream);
/* b, x: host arrays of count DEVICE pointers (n_i doubles each); iters, relres:
 * host arrays of count entries (NULL allowed); relres is the true residual. */
int spand_batch_pcg(spand_batch_t b, const double* const* bvec, double* const* xvec, double tol,
                    int32_t* iters, double* relres, void* stream);
/* Wall time of the last factor and PCG calls, kernel launches of the last
 * factorization, and host synchronisations (ticks) of the last PCG. */
int spand_batch_info(spand_batch_t b, double* factor_ms, double* pcg_ms, int64_t* launches,
                     int64_t* ticks);
int spand_batch_set_profiling(spand_batch_t b, int on);
int spand_batch_kernel_stats(spand_batch_t b, spand_kernel_stat* out, int cap, int* count);
void spand_batch_destroy(spand_batch_t b);

/* ---------------------------------------------------------------------------
 * Solve server (continuous batching).
 *
 * The server keeps factored problems resident in device memory and answers
 * requests of 1 or more right-hand sides with the PCG of §4.  Two internal
 * host threads: one factors problems as their first request arrives (on its
 * own stream, admitting a problem when its estimated factor footprint fits
 * hbm_budget, evicting idle unpinned problems least recently used first),
 * the other advances every admitted right-hand side of every problem by one
 * PCG step per tick (one launch per step over all of them, merged applies).
 * Requests join between ticks as segment slots and vector space free up and
 * leave as soon as their right-hand sides are done, so a factorization, new
 * requests and requests already in flight overlap on the GPU.  A right-hand
 * side's iterates do not depend on the other requests in flight (fixed
 * per-right-hand-side reduction order); only the apply's atomic accumulation
 * order can change the last bits.
 *
 * Handles are caller-owned, analysed with the server's precision, and must
 * outlive the server; while added they must not be used directly.  Host
 * buffers of a request (b: n x nrhs column-major, x: the same) must stay
 * valid until spand_server_wait returns for it.  The calls are thread-safe.
 * --------------------------------------------------------------------------- */
typedef struct spand_server_s* spand_server_t;
typedef struct {
  size_t hbm_budget;      /* device bytes for resident factors; 0 = 60% of the free memory */
  int64_t max_entries;    /* entries of the PCG work vectors over all admitted right-hand sides
                             (each right-hand side takes n rounded up to 32); 0 = 32 Mi */
  int32_t max_segments;   /* right-hand sides in flight at most; 0 = 256 */
  int32_t precision;      /* factorization and apply precision of every problem (0 FP64, 1 FP32) */
  double tol;             /* PCG tolerance on ||r|| / ||b||; 0 = 1e-10 */
} spand_server_opts;
typedef struct {
  int64_t requests;       /* completed requests */
  int64_t solves;         /* completed right-hand sides */
  double p50_ms, p99_ms, max_ms;  /* request latency, submission to completion */
  double elapsed_s;       /* first submission to last completion */
  double solves_per_s;
  int64_t ticks;          /* PCG ticks run */
  int32_t max_inflight;   /* most right-hand sides in flight at once */
  int32_t resident_problems;
  int64_t resident_bytes;
  /* latency split of the completed requests: waiting for the problem's
   * factorization (submission to the problem being ready), queued with the
   * problem ready (for segment slots and vector space), and solving (admission
   * to completion; includes the copies of b and x); p50 and p99 of each, and
   * the three parts of the slowest request */
  double factor_wait_p50_ms, factor_wait_p99_ms;
  double queue_p50_ms, queue_p99_ms;
  double solve_p50_ms, solve_p99_ms;
  double max_split_ms[3];
} spand_server_stats;

int spand_server_create(const spand_server_opts* opts, spand_server_t* out);
/* Registers an analysed handle; pinned != 0 factors it at once and never
 * evicts it.  *mid receives the problem id used by spand_server_submit. */
int spand_server_add(spand_server_t s, spand_t h, int32_t pinned, int32_t* mid);
/* Queues a request of nrhs right-hand sides; *rid identifies it. */
int spand_server_submit(spand_server_t s, int32_t mid, int32_t nrhs, const double* b, double* x,
                        int64_t* rid);
/* Blocks until the request is done; iters, relres: host arrays of nrhs entries
 * (NULL allowed), relres the true relative residual; *latency_ms the time from
 * submission to completion.  Returns the request's status (SPAND_ENOCONV if a
 * right-hand side reached maxit, the factorization's error if it failed). */
int spand_server_wait(spand_server_t s, int64_t rid, int32_t* iters, double* relres,
                      double* latency_ms);
int spand_server_get_stats(spand_server_t s, spand_server_stats* st);
/* Stops the threads (requests still queued are abandoned) and frees the
 * server's memory; the handles stay with the caller. */
void spand_server_destroy(spand_server_t s);

/* ---------------------------------------------------------------------------
 * Measurement aid (the paper has no counterpart).
 *
 * The factorization kernels are bound by the fused multiply-add pipe of their
 * precision, and no measured FP64 rate of the GPU is published to divide by.
 * spand_measure_fma_peak times independent FMA chains in every thread of a
 * grid of 8 CTAs of 256 threads per SM on the current device (best of five
 * launches after a warm-up, CUDA events on a stream of its own) and returns the
 * achieved rate in TFLOP/s (2 flops per FMA) in *tflops and the best launch
 * time in *ms (may be NULL).  precision: 0 = FP64, 1 = FP32.  Synchronises
 * the device's work on its own stream only; allocates no device memory.
 * Errors: SPAND_EINVAL (bad precision, null tflops), SPAND_ECUDA.
 * --------------------------------------------------------------------------- */
int spand_measure_fma_peak(int precision, double* tflops, double* ms);

/* Frees every device and host resource of the handle.  NULL is ignored. */
void spand_destroy(spand_t h);

const char* spand_strerror(int code);
const char* spand_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SPAND_H */
