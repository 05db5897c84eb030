"""The RRQR launch-shape autotuner (spand_tune).

It times every candidate shape (CTA size, cluster growth) per size bucket of
interface blocks and refactors with the fastest.  The shapes change only the
order of some floating-point sums, so the tuned factorization must give the
ranks of the default one exactly (random coefficients: no near ties), the
same preconditioner to 1e-10 (FP64) and the same CG iterations, and a replayed
refactorization must keep them.
"""
import numpy as np
import pytest

import spand_inputs as si

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_tuned_shapes_reproduce_the_factorization(precision):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_00789_gb300 import spand as S
    prob = si.diffusion_3d(40, seed=3)
    ell = 10
    ref = S.Spand.from_problem(prob, ell, 1e-2, 1, precision=precision)
    ref.factor()
    h = S.Spand.from_problem(prob, ell, 1e-2, 1, precision=precision)
    choice = h.tune()
    print("tuned shapes per bucket:", choice)
    assert choice, "no interface fell in any cluster bucket"
    assert choice.pop("apply") in ("persistent", "per_phase")
    for thr, grow in choice.values():
        assert thr in (256, 512) and grow in (1, 2)
    r = np.random.default_rng(2).standard_normal(prob.n)
    rd = torch.from_numpy(r).cuda()
    za, zb = torch.empty_like(rd), torch.empty_like(rd)
    b = torch.from_numpy(si.rhs_normal(prob.n, seed=4)).cuda()
    tol_apply = 1e-10 if precision == 0 else 1e-4
    for _ in range(2):  # the tuned factorization, then its graph replay
        assert np.array_equal(h.ranks()[:, :2], ref.ranks()[:, :2])
        ref.apply(rd, za)
        h.apply(rd, zb)
        torch.cuda.synchronize()
        err = float((za - zb).abs().max() / za.abs().max())
        assert err <= tol_apply, err
        xa, xb = torch.zeros_like(b), torch.zeros_like(b)
        ita, _ = ref.pcg(b, xa, 1e-12)
        itb, relb = h.pcg(b, xb, 1e-12)
        assert abs(ita - itb) <= 1 and relb <= 1e-12
        h.factor()
    ref.close()
    h.close()
