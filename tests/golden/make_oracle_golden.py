"""Write full-size reference values from the CPU oracle.

Calls only the oracle (and the seeded input generators).  The full-size grids
take minutes (64^3) to hours (128^3) per factorization in the oracle, too slow
for the test suite, so the values the GPU tests compare against at full size
are stored:

* PCG iteration counts to 1e-12 and the true relative residual at exit;
* the sum of the coarse ranks, the factor size nnz(L), the number of RRQR
  steps flagged as near ties, and a SHA-256 of every (size, rank) pair in
  cluster order so that ranks can be compared exactly;
* the coarse rank sum of every stage (to locate a difference);
* (128^3 only) the preconditioner applied to one seeded vector r: M r at 4096
  seeded positions, ||M r||_2, and <u, M r> for a second seeded vector u.
  M r is linear in every stored factor entry, so these check the factor as a
  whole without storing a 2M-entry vector.

Run:
  OPENBLAS_NUM_THREADS=1 python tests/golden/make_oracle_golden.py 64
  OPENBLAS_NUM_THREADS=2 python tests/golden/make_oracle_golden.py 128 --scheme 1
(one process per scheme at 128^3; each merges its entry into oracle_128.json
under a file lock).
"""
import argparse
import fcntl
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import spand_inputs as si  # noqa: E402
from oracle import spand as OS  # noqa: E402

# M r probe of the 128^3 entries: r ~ N(0,1) from this seed, u ~ N(0,1) from the
# next, and MR_SAMPLES positions drawn without replacement from default_rng(MR_SEED + 2)
MR_SEED = 2
MR_SAMPLES = 4096


def rank_pairs(F):
    out = []
    for k, keys in enumerate(F.stage_keys):
        for key in keys:
            out.append((F.stage_sizes[k][key], F.stage_ranks[k].get(key, -1)))
    return np.array(out, dtype=np.int32)


def mr_probe(n):
    """The seeded vectors and positions of the M r probe (shared with the GPU test)."""
    r = si.rhs_normal(n, seed=MR_SEED)
    u = si.rhs_normal(n, seed=MR_SEED + 1)
    idx = np.sort(np.random.default_rng(MR_SEED + 2).choice(n, MR_SAMPLES, replace=False))
    return r, u, idx


def entry(name, prob, ell, b, scheme, probe):
    A = prob.to_scipy()
    t0 = time.perf_counter()
    F = OS.factor(A, prob.coords, ell, 1e-2, scheme)
    t1 = time.perf_counter()
    res = OS.pcg(lambda v: A @ v, lambda v: OS.apply(F, v), b, 1e-12)
    t2 = time.perf_counter()
    pairs = rank_pairs(F)
    ties = sum(1 for fl in F.stage_flags for v in fl.values() if v)
    e = {
        "n": prob.n, "nlevels": ell, "eps": 1e-2, "scheme": scheme, "tol": 1e-12,
        "cg_iters": res.iters, "relres": res.relres,
        "rank_sum": int(pairs[pairs[:, 1] >= 0, 1].sum()),
        "nnz_factor": int(F.nnz_factor()), "near_ties": ties,
        "rank_sha256": hashlib.sha256(pairs.tobytes()).hexdigest(),
        "stage_rank_sums": [int(sum(rk.values())) for rk in F.stage_ranks],
        "oracle_factor_s": t1 - t0, "oracle_pcg_s": t2 - t1,
    }
    if probe:
        r, u, idx = mr_probe(prob.n)
        z = OS.apply(F, r)
        e["mr"] = {"seed": MR_SEED, "samples": MR_SAMPLES, "idx": idx.tolist(),
                   "val": z[idx].tolist(), "norm2": float(np.linalg.norm(z)),
                   "u_dot": float(u @ z), "max_abs": float(np.abs(z).max())}
    return e


def merge(path, key, value):
    with open(path + ".lock", "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        data = json.load(open(path)) if os.path.exists(path) else {}
        data[key] = value
        with open(path, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        fcntl.flock(lk, fcntl.LOCK_UN)
    os.remove(path + ".lock")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("size", type=int, choices=[64, 128])
    ap.add_argument("--scheme", type=int, action="append")
    args = ap.parse_args()
    gdir = os.path.join(ROOT, "tests", "golden")
    if args.size == 64:
        cases = [
            ("poisson3d_64", si.laplacian_3d(64), 12, si.rhs_normal(64 ** 3, seed=0), [0, 1, 2]),
            ("diffusion3d_64", si.diffusion_3d(64, seed=0), 12, si.rhs_normal(64 ** 3, seed=0), [1]),
        ]
        path = os.path.join(gdir, "oracle_64.json")
        probe = False
    else:
        # 3D high-contrast diffusion: a = 10^U(-3,3) per cell from seed 0, b ~ N(0,1) from seed 1
        cases = [("diffusion3d_128", si.diffusion_3d(128, seed=0), 15,
                  si.rhs_normal(128 ** 3, seed=1), args.scheme or [0, 1, 2])]
        path = os.path.join(gdir, "oracle_128.json")
        probe = True
    for name, prob, ell, b, schemes in cases:
        for scheme in schemes:
            if args.scheme and scheme not in args.scheme:
                continue
            e = entry(name, prob, ell, b, scheme, probe)
            print(name, scheme, {k: v for k, v in e.items() if k != "mr"}, flush=True)
            merge(path, f"{name}_scheme{scheme}", e)


if __name__ == "__main__":
    main()
