"""Write tests/golden/oracle_64.json: full-size reference values from the CPU oracle.

Calls only the oracle (and the seeded input generators).  The 64^3 grids take
one to three minutes per factorization in the oracle, too slow for the test
suite, so the values the GPU tests compare against at full size are stored:
PCG iteration counts, the sum of the coarse ranks, the factor size nnz(L),
and, for the random-coefficient problem (no pivot ties), a SHA-256 of every
(size, rank) pair in cluster order so that ranks can be compared exactly.

Run:  OPENBLAS_NUM_THREADS=1 python tests/golden/make_oracle_golden.py
"""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import spand_inputs as si  # noqa: E402
from oracle import spand as OS  # noqa: E402


def rank_pairs(F):
    out = []
    for k, keys in enumerate(F.stage_keys):
        for key in keys:
            out.append((F.stage_sizes[k][key], F.stage_ranks[k].get(key, -1)))
    return np.array(out, dtype=np.int32)


def main():
    out = {}
    cases = [
        ("poisson3d_64", si.laplacian_3d(64), 12, si.rhs_normal, [0, 1, 2]),
        ("diffusion3d_64", si.diffusion_3d(64, seed=0), 12, si.rhs_normal, [1]),
    ]
    for name, prob, ell, rhs, schemes in cases:
        A = prob.to_scipy()
        b = rhs(prob.n, seed=0)
        for scheme in schemes:
            F, res = OS.solve(A, prob.coords, b, ell, 1e-2, scheme)
            pairs = rank_pairs(F)
            ties = sum(1 for fl in F.stage_flags for v in fl.values() if v)
            entry = {
                "n": prob.n, "nlevels": ell, "eps": 1e-2, "scheme": scheme, "tol": 1e-12,
                "cg_iters": res.iters, "relres": res.relres,
                "rank_sum": int(pairs[pairs[:, 1] >= 0, 1].sum()),
                "nnz_factor": int(F.nnz_factor()), "near_ties": ties,
                "rank_sha256": hashlib.sha256(pairs.tobytes()).hexdigest(),
            }
            out[f"{name}_scheme{scheme}"] = entry
            print(name, scheme, entry, flush=True)
    with open(os.path.join(ROOT, "tests", "golden", "oracle_64.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
