"""Benchmark: spaND factor + PCG to a relative residual of 1e-12 on one GB300.

A step is one pass of the whole hot path over the resident problem: the
numerical factorization (Algorithm 2 with the chosen scheme) followed by PCG
with the spaND preconditioner from x0 = 0 to ||r||/||b|| < 1e-12.  The default
workload is the 3D high-contrast diffusion problem on a 128^3 grid
(n = 2097152, 7-point finite volumes, per-cell coefficient 10^U(-3,3) from
seed 0 with harmonic face averages, 15 nested-dissection levels, eps = 1e-2,
full second-order scheme, RHS N(0, 1) from seed 1), factored in FP64; the
FP32 factorization of the same problem (PCG in FP64) is timed beside it.  The
symbolic analysis (host) and the upload of A happen before the timed region;
the factor's working set (panel rows of several GB) is far larger than the
129 MB L2, so no L2 flush is needed between steps.

Printed: one JSON line (rank 0).  ``value`` is the device-timed seconds per
step (CUDA events on the launch stream, max over ranks), ``e2e`` the same
solve through the host-buffer C-ABI path (analyze + factor + PCG with the
H2D copy of A and b and the D2H copy of x inside the timed region),
``roofline`` the dominant kernel's algorithmic FP64 rate against the FP64
peak, ``cpu_baseline`` the CPU oracle on a bounded sample: one full
factor + PCG of the same kind of problem on a 64^3 grid (the oracle needs
hours at 128^3), single-threaded like the paper's code.

``--impl reference`` times the same CPU oracle sample instead (the reference
arm; there is no other implementation of the paper to run).

Multi-GPU: independent problems, one replica per rank (weak scaling, no data
exchange; the method's own multi-GPU partitioning is not built).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "factor+PCG time to rel. residual 1e-12, CG its; served solves/s, p99 latency"
# Nominal ALU peaks (context): GB300 FP64 1.25 TFLOP/s (152 SMs x 2070 MHz x
# 2 FP64 FMA/clk/SM); FP32 152 SMs x 2070 MHz x 128 FMA/clk/SM.  The roofline
# divides by the FMA rate measured live on the same GPU (measured_peak).
FP64_NOMINAL_TFLOPS = 1.25
FP32_NOMINAL_TFLOPS = 152 * 2.07e9 * 128 * 2 / 1e12
_PEAKS = {}


def measured_peak(precision):
    """(TFLOP/s, source) of the FMA pipe of this precision, measured once per run
    on the current GPU (FMA chains in every thread of 8 CTAs per SM, best of 5)."""
    if precision not in _PEAKS:
        from paper_2007_00789_gb300 import spand
        try:
            tf, ms = spand.measure_fma_peak(precision)
            _PEAKS[precision] = (tf, f"measured in this run: spand_measure_fma_peak({precision}),"
                                     f" FMA chains on every SM, best launch {ms:.2f} ms")
        except Exception as exc:  # keep the line: fall back to the nominal figure, said so
            nom = FP64_NOMINAL_TFLOPS if precision == 0 else FP32_NOMINAL_TFLOPS
            _PEAKS[precision] = (nom, f"nominal (measurement failed: {exc})"[:200])
    return _PEAKS[precision]

# DRAM bytes (read + write) of the dominant kernel per factorization, from an
# ncu capture of every launch of that kernel in one factorization of this
# bench's workload (profiles/dram_k_rrqr_cluster_diffusion3d_128_fp64.txt):
# (workload, precision, kernel kind) -> bytes per step; the line reports them
# per launch (divided by the step's launches of the kernel, which the tuned
# shapes change, the bytes not).  Only valid for the kernel version that was
# captured; absent entries report null.
TRAFFIC_PER_STEP = {("diffusion3d_128", 0, "rrqr"): 15.123e9}

WORKLOADS = {
    # name: (factory, ell, rhs, rhs seed)
    "poisson3d_64": ("laplacian_3d(64)", 12, "rhs_normal", 0),
    "poisson2d_64": ("laplacian_2d(64)", 6, "rhs_uniform", 0),
    "diffusion3d_64": ("diffusion_3d(64, seed=0)", 12, "rhs_normal", 0),
    "poisson3d_32": ("laplacian_3d(32)", 9, "rhs_normal", 0),
    # smaller cases of the 128^3 family (same coefficient law, 128-vertex leaves), for profiling
    "diffusion3d_48": ("diffusion_3d(48, seed=0)", 11, "rhs_normal", 1),
    "diffusion3d_96": ("diffusion_3d(96, seed=0)", 14, "rhs_normal", 1),
    # 3D high-contrast diffusion, a = 10^U(-3,3) per cell (seed 0), b ~ N(0,1) from seed 1
    "diffusion3d_128": ("diffusion_3d(128, seed=0)", 15, "rhs_normal", 1),
}


def make_problem(name):
    import spand_inputs as si
    expr, ell, rhs, seed = WORKLOADS[name]
    prob = eval("si." + expr, {"si": si})
    b = getattr(si, rhs)(prob.n, seed=seed)
    return prob, ell, b


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={q}",
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        import statistics
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[0]))
                mx.append(float(s[1]))
                for i, nm in enumerate(names):
                    if s[3 + i].lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# The CPU oracle's sample for each GPU workload: the same problem family at a
# size the oracle finishes in about a minute on one core (the 128^3 solve takes
# it hours).  Every other workload is its own sample.
ORACLE_SAMPLE = {"diffusion3d_128": "diffusion3d_64"}


def oracle_sample(name="diffusion3d_64", scheme=1, eps=1e-2):
    """Time the CPU oracle (factor + PCG) on one problem, single-threaded BLAS."""
    code = (
        "import time,sys,json; sys.path.insert(0, %r)\n"
        "import bench, oracle.spand as OS\n"
        "prob, ell, b = bench.make_problem(%r)\n"
        "A = prob.to_scipy(); t0 = time.perf_counter()\n"
        "F, res = OS.solve(A, prob.coords, b, ell, %r, %d)\n"
        "t = time.perf_counter() - t0\n"
        "print(json.dumps({'s': t, 'iters': res.iters, 'relres': res.relres, 'n': prob.n}))\n"
    ) % (ROOT, name, eps, scheme)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def oracle_batch(indices, eps=1e-2, scheme=1, tol=1e-12):
    """The CPU oracle's throughput on problems of the batch64 workload: one
    single-threaded process per problem, as many at a time as the host has
    cores (and 4 GB of memory each).  Returns (solves/s, processes at a time,
    wall seconds, the slowest solve's seconds)."""
    import concurrent.futures as cf

    code = (
        "import time,sys,json; sys.path.insert(0, %r)\n"
        "import spand_inputs as si, oracle.spand as OS\n"
        "prob, ell, b = si.batch_problem(int(sys.argv[1]))\n"
        "A = prob.to_scipy(); t0 = time.perf_counter()\n"
        "F, res = OS.solve(A, prob.coords, b, ell, %r, %d, tol=%r)\n"
        "print(json.dumps({'s': time.perf_counter() - t0, 'iters': res.iters}))\n"
    ) % (ROOT, eps, scheme, tol)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")

    def one(i):
        out = subprocess.run([sys.executable, "-c", code, str(i)], capture_output=True, text=True,
                             env=env, timeout=1800)
        if out.returncode != 0:
            raise RuntimeError(out.stderr[-2000:])
        return json.loads(out.stdout.strip().splitlines()[-1])

    try:
        mem_gb = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES") / 2 ** 30
    except (ValueError, OSError, AttributeError):
        mem_gb = 16.0
    par = max(1, min(len(indices), os.cpu_count() or 1, int(mem_gb // 4)))
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(par) as ex:
        res = list(ex.map(one, indices))
    wall = time.perf_counter() - t0
    return len(indices) / wall, par, wall, max(o["s"] for o in res)


def sample_text(name, o):
    return (f"oracle factor+PCG to 1e-12, measured unscaled on the full {name} problem"
            f" (n={o['n']}, {o['iters']} CG iterations), one core; a lower bound for the"
            " workload's own size where that is larger")


def run_reference(args, rank):
    """The reference arm: the CPU oracle on the workload's sample problem.

    W warm-up and K timed steps, each one full oracle solve of the sample
    (about a minute at 64^3, single-threaded BLAS), run as separate processes,
    as many at a time as the host has cores, so that the arm ends within a few
    minutes; the value is the mean per-solve time of the K timed steps."""
    if rank != 0:
        return
    import concurrent.futures as cf

    sample = ORACLE_SAMPLE.get(args.workload, args.workload)
    jobs = args.warmup + args.steps
    # one process per core, and at most one per 4 GB of the host's memory (an
    # oracle solve at 64^3 peaks near 1.1 GB)
    try:
        mem_gb = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES") / 2 ** 30
    except (ValueError, OSError, AttributeError):
        mem_gb = 16.0
    par = max(1, min(jobs, os.cpu_count() or 1, int(mem_gb // 4)))
    with cf.ThreadPoolExecutor(par) as ex:
        res = list(ex.map(lambda _: oracle_sample(sample, args.scheme, args.eps), range(jobs)))
    timed = res[args.warmup:]
    per = sum(o["s"] for o in timed) / len(timed)
    last = timed[-1]
    line = {
        "impl": "reference", "metric": METRIC, "value": per, "unit": "s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": per, "unit": "s", "cores": par, "kind": "oracle",
                         "sample": sample_text(sample, last) + f"; {jobs} solves as separate"
                                   f" single-threaded processes, {par} at a time, mean of the last"
                                   f" {args.steps} ({min(o['s'] for o in timed):.1f}..."
                                   f"{max(o['s'] for o in timed):.1f} s)"},
        "e2e": {"value": per, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def max_over_ranks(value, dist):
    """The largest value over the ranks of the process group (the job's time is
    its slowest rank's); the value itself without one.  NCCL reduces a device
    tensor, gloo a host one."""
    if dist is None:
        return value
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_config(args):
    """The config object both arms print for a single-problem workload."""
    return {"workload": args.workload, "scheme": args.scheme, "eps": args.eps, "tol": 1e-12,
            "precision": "fp64 factor+apply, fp64 pcg" if args.precision == 0
                         else "fp32 factor+apply, fp64 pcg",
            "l2": "inputs larger than L2 (no flush)"}


def run_batch(args, rank, world, local, dist, emit=True):
    """64 independent problems (2D 128^2..512^2 and 3D 24^3..48^3 FV diffusion,
    a = 10^U(-2,2)): one step = batch factorization + batch PCG of all of them.
    Prints the JSON line (emit) or returns it."""
    import numpy as np
    import torch

    import spand_inputs as si
    from paper_2007_00789_gb300 import spand

    import concurrent.futures as cf

    tol = 1e-12
    work = si.batch_workload(64)
    stream = torch.cuda.current_stream()

    def analyze_all(plain):
        # the host analyses are independent: one thread per problem (the C call releases the GIL)
        with cf.ThreadPoolExecutor(16) as ex:
            return list(ex.map(lambda w: spand.Spand.from_problem(
                w[0], w[1], args.eps, args.scheme, precision=args.precision,
                rrqr_kernel=args.rrqr_kernel, plain_launches=plain,
                rrqr_threads=args.rrqr_threads, apply_kernels=args.apply_kernels), work))

    hs = analyze_all(args.plain_launches)
    batch = spand.SpandBatch(hs)
    bs = [torch.from_numpy(b).cuda() for _, _, b in work]
    xs = [torch.zeros_like(b) for b in bs]
    its = rels = None
    for _ in range(args.warmup):
        batch.factor(stream)
        its, rels = batch.pcg(bs, xs, tol, stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    fac_ms = []
    with ClockSampler(local) as clk:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            batch.factor(stream)
            fac_ms.append(batch.info()["factor_ms"])
            its, rels = batch.pcg(bs, xs, tol, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    info = batch.info()
    batch.set_profiling(True)
    for _ in range(args.steps):
        batch.factor(stream)
        batch.pcg(bs, xs, tol, stream)
    torch.cuda.synchronize()
    kstats = batch.kernel_stats()
    batch.set_profiling(False)
    ms = max_over_ranks(ms, dist)
    true_rel = max(float(np.linalg.norm(b - p.to_scipy() @ x.cpu().numpy()) / np.linalg.norm(b))
                   for (p, _, b), x in zip(work, xs))
    # end to end: analyze + batch factor + batch PCG with the H2D copies of every
    # problem's matrix and right-hand side and the D2H copies of the solutions
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        he = analyze_all(False)
        be = spand.SpandBatch(he)
        be.factor(stream)
        pin = [torch.from_numpy(b).pin_memory() for _, _, b in work]
        bd = [t.cuda(non_blocking=True) for t in pin]
        xd = [torch.zeros_like(b) for b in bd]
        be.pcg(bd, xd, tol, stream)
        xh = [x.cpu() for x in xd]
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        be.close()
        for h in he:
            h.close()
        h2d = sum(4 * (p.n + 1) + 12 * p.nnz + 8 * p.n for p, _, _ in work)
        d2h = sum(8 * p.n for p, _, _ in work)
        e2e = {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "includes": "host analysis of all 64 problems (16 threads)"}
    dom = max(kstats, key=lambda k: k["total_ms"])
    achieved = dom["flops"] / (dom["total_ms"] * 1e-3) / 1e12 if dom["total_ms"] > 0 else 0.0
    peak, peak_src = measured_peak(args.precision)
    roof = {"bound": "alu", "kernel": dom["name"], "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
            "peak_source": peak_src,
            "avg_launch_ms": dom["total_ms"] / max(dom["launches"], 1),
            "launches_per_step": dom["launches"] / args.steps}
    n_total = sum(p.n for p, _, _ in work)
    line = {
        "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if args.precision == 0 else "f32 factor/apply + f64 pcg",
        "data": "synthetic",
        "config": {"workload": "batch64", "problems": len(work), "n_total": n_total,
                   "nnz_total": sum(p.nnz for p, _, _ in work), "eps": args.eps,
                   "scheme": args.scheme, "tol": tol, "nlevels": "round(log2(n/25)) per problem",
                   "cg_iters_max": int(max(its)), "cg_iters_mean": float(np.mean(its)),
                   "relres_max": float(max(rels)), "true_relres_max_host": true_rel,
                   "factor_ms": float(np.median(fac_ms)), "pcg_ticks": info["ticks"],
                   "solves_per_s": len(work) / (ms / 1e3),
                   "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{world}",
                   "cuda_graphs": not args.plain_launches},
        "clocks": clk.summary(),
        "e2e": e2e,
        "gpu_launches": int(sum(k["launches"] for k in kstats) // args.steps),
        "roofline": roof,
        "kernels": {k["name"]: {"ms_per_step": k["total_ms"] / args.steps,
                                "launches_per_step": k["launches"] / args.steps,
                                "gflop_per_step": k["flops"] / args.steps / 1e9}
                    for k in kstats if k["launches"]},
    }
    batch.close()
    for h in hs:
        h.close()
    if not emit:
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def one_at_a_time(precision, eps, scheme, steps=1, warmup=1):
    """The batch64 problems factored and solved one after another (FP64 or FP32),
    each through its own handle: the plain single-problem baseline of the batched
    form.  Returns (seconds per pass over all 64 problems, max CG its, max relres)."""
    import concurrent.futures as cf

    import torch

    import spand_inputs as si
    from paper_2007_00789_gb300 import spand

    tol = 1e-12
    work = si.batch_workload(64)
    stream = torch.cuda.current_stream()
    with cf.ThreadPoolExecutor(16) as ex:
        hs = list(ex.map(lambda w: spand.Spand.from_problem(w[0], w[1], eps, scheme,
                                                            precision=precision), work))
    bs = [torch.from_numpy(b).cuda() for _, _, b in work]
    xs = [torch.zeros_like(b) for b in bs]
    its, rels = [], []

    def one_pass():
        its.clear()
        rels.clear()
        for h, b, x in zip(hs, bs, xs):
            h.factor(stream)
            it, rel = h.pcg(b, x, tol, stream)
            its.append(it)
            rels.append(rel)

    for _ in range(warmup):
        one_pass()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        one_pass()
    e1.record(stream)
    torch.cuda.synchronize()
    for h in hs:
        h.close()
    return e0.elapsed_time(e1) / steps / 1e3, max(its), max(rels)


def serve_trace(precision, eps, scheme, rate, local, requests=120, new_problems=12):
    """Run one serving trace: a resident 96^3 diffusion problem plus new problems of
    n = 16k..500k, requests of 1..32 right-hand sides arriving as a Poisson process
    of the given rate, PCG to 1e-10.  Returns the measurements (a dict)."""
    import concurrent.futures as cf

    import numpy as np

    import spand_inputs as si
    from paper_2007_00789_gb300 import spand

    tol = 1e-10
    probs, trace = si.serve_workload(requests=requests, rate=rate, new_problems=new_problems)
    max_n = max(p.n for p, _ in probs)
    srv = spand.SpandServer(precision=precision, tol=tol, max_segments=512,
                            max_entries=6 * 32 * ((max_n + 31) // 32 * 32))
    # analysis (host) of every problem happens before the trace starts
    with cf.ThreadPoolExecutor(16) as ex:
        hs = list(ex.map(lambda pe: spand.Spand.from_problem(pe[0], pe[1], eps, scheme,
                                                             precision=precision), probs))
    mids = [srv.add(h, pinned=(i == 0)) for i, h in enumerate(hs)]
    # warm-up: the resident problem is factored and one request solved
    rng0 = np.random.default_rng(1)
    srv.wait(srv.submit(mids[0], rng0.standard_normal((1, probs[0][0].n))))
    rhs = {k: np.random.default_rng(sd).standard_normal((nr, probs[pi][0].n))
           for k, (_, pi, nr, sd) in enumerate(trace)}
    results = [None] * len(trace)
    start = time.perf_counter()

    def waiter(k, rid):
        results[k] = srv.wait(rid)

    with ClockSampler(local) as clk, cf.ThreadPoolExecutor(64) as pool:
        futs = []
        for k, (t, pi, nr, _) in enumerate(trace):
            dt = start + t - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            futs.append(pool.submit(waiter, k, srv.submit(mids[pi], rhs[k])))
        for fu in futs:
            fu.result()
    wall = time.perf_counter() - start
    st = srv.stats()
    worst = 0.0
    for k, (_, pi, nr, _) in enumerate(trace):
        x = results[k][0]
        A = probs[pi][0].to_scipy()
        b = rhs[k]
        worst = max(worst, max(np.linalg.norm(b[j] - A @ x[j]) / np.linalg.norm(b[j])
                               for j in range(nr)))
    lat = np.array([results[k][3] for k in range(len(trace))])
    solves = sum(nr for _, _, nr, _ in trace)
    iters = np.concatenate([results[k][1] for k in range(len(trace))])
    h2d = sum(8 * nr * probs[pi][0].n for _, pi, nr, _ in trace)
    srv.close()
    for h in hs:
        h.close()
    return {"solves_per_s": solves / wall, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()), "wall_s": wall,
            "requests": len(trace), "solves": solves, "new_problems": len(probs) - 1,
            "arrival_rate_per_s": rate, "tol": tol, "cg_iters_max": int(iters.max()),
            "cg_iters_mean": float(iters.mean()), "true_relres_max_host": worst,
            "server": {k: st[k] for k in ("ticks", "max_inflight", "resident_problems",
                                          "resident_bytes", "solves_per_s")},
            "latency_split": {
                "factor_wait_ms": {"p50": st["factor_wait_p50_ms"], "p99": st["factor_wait_p99_ms"]},
                "queue_ms": {"p50": st["queue_p50_ms"], "p99": st["queue_p99_ms"]},
                "solve_ms": {"p50": st["solve_p50_ms"], "p99": st["solve_p99_ms"]},
                "slowest_request_ms": dict(zip(("factor_wait", "queue", "solve"),
                                               st["max_split_ms"])),
                "note": "server clock: submission -> problem factored -> admitted -> done"},
            "h2d_bytes": h2d, "clocks": clk.summary()}


def run_serve(args, rank, world, local, dist):
    """The serving workload as its own JSON line (value = served solves/s)."""
    r = serve_trace(args.precision, args.eps, args.scheme, args.serve_rate, local)
    cfg = {"workload": "serve", "resident": "diffusion_3d(96), a=10^U(-3,3)", "nrhs": "1..32",
           "timing": "host wall clock from first submission (requests' b and x in host memory,"
                     " copies and factorizations of new problems included)"}
    cfg.update({k: v for k, v in r.items() if k not in ("clocks", "h2d_bytes")})
    line = {
        "metric": METRIC, "value": r["solves_per_s"], "unit": "solves/s", "n_gpus": world,
        "steps": r["requests"], "warmup": 1, "ms_per_step": r["wall_s"] * 1e3 / r["requests"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == 0 else "f32 factor/apply + f64 pcg",
        "data": "synthetic", "config": cfg, "clocks": r["clocks"],
        "e2e": {"value": r["solves_per_s"], "unit": "solves/s",
                "h2d_bytes_per_step": r["h2d_bytes"] // r["requests"],
                "d2h_bytes_per_step": r["h2d_bytes"] // r["requests"]},
        "gpu_launches": None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="spand", choices=["spand", "reference"])
    ap.add_argument("--workload", default="diffusion3d_128",
                    choices=sorted(WORKLOADS) + ["batch64", "serve"],
                    help="batch64: 64 independent 2D/3D diffusion problems factored and solved"
                         " as one batch (FP32 factor by default)")
    ap.add_argument("--scheme", type=int, default=1)
    ap.add_argument("--eps", type=float, default=1e-2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", type=int, default=None, choices=[0, 1],
                    help="0: FP64 factor+apply; 1: FP32 factor+apply (PCG stays FP64)")
    ap.add_argument("--no-variant", action="store_true",
                    help="skip timing the other precision")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched and served measurements beside the headline line")
    ap.add_argument("--serve-rate", type=float, default=5.0,
                    help="serve workload: request arrivals per second (Poisson process)")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip spand_tune (the RRQR launch-shape autotuner) before the timed region")
    ap.add_argument("--plain-launches", action="store_true",
                    help="no CUDA graphs: every kernel launched on its own (for profilers)")
    ap.add_argument("--rrqr-threads", type=int, default=0, choices=[0, 256, 512],
                    help="threads per CTA of the on-chip RRQR (0: the library's choice)")
    ap.add_argument("--apply-kernels", type=int, default=0, choices=[0, 1, 2],
                    help="single-vector apply: 0 the library's choice (tuned, else by size),"
                         " 1 one launch per phase, 2 one persistent launch")
    ap.add_argument("--rrqr-kernel", type=int, default=0, choices=[0, 1, 2, 3, 4, 5],
                    help="0: on-chip RRQR in clusters of up to 16 CTAs, wider blocks over several"
                         " CTAs with their slices in shared memory where they fit; 1: global-memory"
                         " RRQR; 2: clusters of up to 8 CTAs; 3: always the streamed multi-CTA"
                         " kernel; 4: always the on-chip multi-CTA kernel; 5: as 0 with the"
                         " multi-CTA blocks streamed")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.precision is None:
        args.precision = 1 if args.workload in ("batch64", "serve") else 0

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if args.workload in ("batch64", "serve"):
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm covers the"
                              " single-problem workloads only"}), flush=True)
            return
        run_reference(args, rank)
        return

    import numpy as np
    import torch

    from paper_2007_00789_gb300 import spand

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload == "batch64":
        run_batch(args, rank, world, local, dist)
        return
    if args.workload == "serve":
        run_serve(args, rank, world, local, dist)
        return

    prob, ell, b = make_problem(args.workload)
    tol = 1e-12
    stream = torch.cuda.current_stream()
    h = spand.Spand.from_problem(prob, ell, args.eps, args.scheme, precision=args.precision,
                                 rrqr_kernel=args.rrqr_kernel, plain_launches=args.plain_launches,
                                 rrqr_threads=args.rrqr_threads,
                                 apply_kernels=args.apply_kernels)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    measured_peak(args.precision)  # the roofline's denominator, measured before the timed region
    # the RRQR launch shapes, tuned once per problem before the timed region
    # (five factorizations; the handle keeps the choice)
    tuned = None if args.no_tune else h.tune(stream)
    iters = rel = None
    for _ in range(args.warmup):
        h.factor(stream)
        iters, rel = h.pcg(bd, xd, tol, stream)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---- timed region: K steps of factor + PCG, events on the launch stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            h.factor(stream)
            iters, rel = h.pcg(bd, xd, tol, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = e0.elapsed_time(e1) / args.steps
    # ---- roofline pass: the same K steps again with per-launch CUDA events
    #      recorded by the library on the launch stream (plain launches, no graphs)
    h.set_profiling(True)
    for _ in range(args.steps):
        h.factor(stream)
        h.pcg(bd, xd, tol, stream)
    torch.cuda.synchronize()
    kstats = h.kernel_stats()
    h.set_profiling(False)
    ms = max_over_ranks(ms, dist)
    info = h.info()

    # ---- end to end through the host-buffer path (analyze + factor + PCG, host A/b/x)
    e2e = None
    if not args.no_e2e:
        times = []
        # the right-hand side and the solution in pinned host memory (prepared
        # before the timed region); A is copied from the handle's host arrays
        b_pin = torch.from_numpy(b).pin_memory()
        x_pin = torch.empty(prob.n, dtype=torch.float64, pin_memory=True)
        splits = []
        for i in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            he = spand.Spand.from_problem(prob, ell, args.eps, args.scheme, precision=args.precision,
                                          rrqr_kernel=args.rrqr_kernel,
                                          plain_launches=args.plain_launches,
                                          rrqr_threads=args.rrqr_threads,
                                          apply_kernels=args.apply_kernels)
            t1 = time.perf_counter()
            he.factor(stream)  # returns after the factorization's last stage has finished
            t2 = time.perf_counter()
            x_host, it_e, rel_e = he.pcg_host(b_pin.numpy(), tol, stream, out=x_pin.numpy())
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            times.append(t3 - t0)
            splits.append({"analyze": t1 - t0, "factor": t2 - t1, "pcg_host": t3 - t2})
            he.close()
        h2d = 4 * (prob.n + 1) + 12 * prob.nnz + 8 * prob.nnz + 8 * prob.n
        d2h = 8 * prob.n + 12 * sum(1 for _ in range(ell))
        best = min(range(1, len(times)) or range(len(times)), key=lambda j: times[j])
        e2e = {"value": times[best], "unit": "s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h,
               "split_s": {k: round(v, 4) for k, v in splits[best].items()}}

    # ---- the other precision, same workload and timing rules (reported beside the line)
    variant = None
    if not args.no_variant:
        other = 1 - args.precision
        hv = spand.Spand.from_problem(prob, ell, args.eps, args.scheme, precision=other,
                                      rrqr_kernel=args.rrqr_kernel,
                                      plain_launches=args.plain_launches,
                                      rrqr_threads=args.rrqr_threads,
                                      apply_kernels=args.apply_kernels)
        xv = torch.zeros_like(bd)
        for _ in range(args.warmup):
            hv.factor(stream)
            itv, relv = hv.pcg(bd, xv, tol, stream)
        torch.cuda.synchronize()
        v0 = torch.cuda.Event(enable_timing=True)
        v1 = torch.cuda.Event(enable_timing=True)
        v0.record(stream)
        for _ in range(args.steps):
            hv.factor(stream)
            itv, relv = hv.pcg(bd, xv, tol, stream)
        v1.record(stream)
        torch.cuda.synchronize()
        true_rel = float(np.linalg.norm(b - prob.to_scipy() @ xv.cpu().numpy()) / np.linalg.norm(b))
        variant = {"precision": "fp32 factor+apply, fp64 PCG" if other == 1 else "fp64",
                   "value": v0.elapsed_time(v1) / args.steps / 1e3, "unit": "s",
                   "cg_iters": itv, "relres": relv, "true_relres_host": true_rel}
        hv.close()

    # ---- roofline of the dominant kernel (FP64 ALU bound)
    dom = max(kstats, key=lambda k: k["total_ms"])
    dom_launch_ms = dom["total_ms"] / max(dom["launches"], 1)
    achieved = dom["flops"] / (dom["total_ms"] * 1e-3) / 1e12 if dom["total_ms"] > 0 else 0.0
    peak, peak_src = measured_peak(args.precision)
    roof = {"bound": "alu", "kernel": dom["name"], "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": (TRAFFIC_PER_STEP[(args.workload, args.precision, dom["name"])]
                        / (dom["launches"] / args.steps)
                        if (args.workload, args.precision, dom["name"]) in TRAFFIC_PER_STEP
                        and dom["launches"] else None),
            "algorithmic_bytes_per_launch": dom["bytes"] / max(dom["launches"], 1),
            "peak_source": peak_src, "peak_nominal": FP64_NOMINAL_TFLOPS if args.precision == 0
                                                     else FP32_NOMINAL_TFLOPS,
            "avg_launch_ms": dom_launch_ms, "launches_per_step": dom["launches"] / args.steps,
            "measured": "per-launch CUDA events in a second pass of the same K steps (plain launches)"}
    launches = sum(k["launches"] for k in kstats) // args.steps
    line = {
        "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == 0 else "f32 factor/apply + f64 pcg",
        "data": "synthetic",
        "config": workload_config(args),
        "details": {"n": prob.n, "nnz": prob.nnz, "nlevels": ell, "cg_iters": iters,
                    "relres": rel, "mu": info["mu"], "skip": info["skip"],
                    "parallelism": f"replicas x{world}", "cuda_graphs": not args.plain_launches,
                    "rrqr_kernel": args.rrqr_kernel, "rrqr_threads": args.rrqr_threads,
                    "apply_kernels": args.apply_kernels,
                    "tuned": {str(k): v for k, v in tuned.items()} if tuned else None},
        "clocks": clk.summary(),
        "variant": variant,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "roofline": roof,
        "kernels": {k["name"]: {"ms_per_step": k["total_ms"] / args.steps,
                                "launches_per_step": k["launches"] / args.steps,
                                "gflop_per_step": k["flops"] / args.steps / 1e9}
                    for k in kstats if k["launches"]},
    }
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        try:
            sample = ORACLE_SAMPLE.get(args.workload, args.workload)
            o = oracle_sample(sample, args.scheme, args.eps)
            line["cpu_baseline"] = {"value": o["s"], "unit": "s", "cores": 1, "kind": "oracle",
                                    "sample": sample_text(sample, o)}
        except Exception as exc:  # the baseline must not sink the GPU line
            line["cpu_baseline"] = {"value": None, "unit": "s", "cores": 1, "kind": "oracle",
                                    "sample": f"failed: {exc}"[:300]}
    # the metric's other parts, measured beside the headline: batched problems and
    # served solves (rank 0 at N=1; a failure here is reported, not fatal)
    h.close()
    if rank == 0 and world == 1 and not args.no_extras:
        import copy
        bw = ("batch64: 64 FV diffusion problems, 2D 128^2..512^2 and 3D 24^3..48^3,"
              " a=10^U(-2,2), PCG (FP64) to 1e-12")
        line["batched"] = {"workload": bw}
        for prec, tag in ((1, "fp32_factor"), (0, "fp64")):
            try:
                ab = copy.copy(args)
                ab.precision, ab.steps, ab.warmup, ab.no_e2e = prec, 2, 3, True
                bl = run_batch(ab, rank, world, local, None, emit=False)
                line["batched"][tag] = {
                    "s_per_step": bl["value"],
                    **{k: bl["config"][k] for k in ("problems", "n_total", "solves_per_s",
                                                    "cg_iters_max", "relres_max",
                                                    "true_relres_max_host", "factor_ms")}}
            except Exception as exc:
                line["batched"][tag] = {"error": str(exc)[:300]}
        try:
            t1, itmax, relmax = one_at_a_time(0, args.eps, args.scheme)
            line["batched"]["fp64_one_at_a_time"] = {
                "s_per_step": t1, "solves_per_s": 64 / t1, "cg_iters_max": int(itmax),
                "relres_max": relmax,
                "how": "each problem factored and solved through its own handle, one after another"}
        except Exception as exc:
            line["batched"]["fp64_one_at_a_time"] = {"error": str(exc)[:300]}
        if not args.no_cpu_baseline:
            try:  # every fourth problem: eight 2D and eight 3D, all sizes of the batch
                idx = list(range(0, 64, 4)) + list(range(1, 64, 4))
                sps, par, wall, slow = oracle_batch(idx, args.eps, args.scheme)
                line["batched"]["cpu_baseline"] = {
                    "value": sps, "unit": "solves/s", "cores": par, "kind": "oracle",
                    "sample": f"oracle factor+PCG (FP64) to 1e-12 on {len(idx)} of the 64 problems"
                              f" (every fourth 2D and every fourth 3D one), one single-threaded"
                              f" process per problem, {par} at a time: {wall:.1f} s wall,"
                              f" slowest solve {slow:.1f} s"}
            except Exception as exc:
                line["batched"]["cpu_baseline"] = {"value": None, "unit": "solves/s",
                                                   "kind": "oracle", "sample": f"failed: {exc}"[:300]}
        line["served"] = {"workload": "resident 96^3 diffusion + 6 new 3D problems, 60 requests of"
                                      " 1..32 RHS arriving at 5/s, PCG (FP64) to 1e-10"}
        for prec, tag in ((1, "fp32_factor"), (0, "fp64")):
            try:
                sv = serve_trace(prec, args.eps, args.scheme, 5.0, local, requests=60,
                                 new_problems=6)
                line["served"][tag] = {k: sv[k] for k in (
                    "solves_per_s", "p50_ms", "p99_ms", "max_ms", "requests", "solves",
                    "cg_iters_max", "true_relres_max_host", "wall_s", "latency_split")
                    if k in sv}
            except Exception as exc:
                line["served"][tag] = {"error": str(exc)[:300]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
