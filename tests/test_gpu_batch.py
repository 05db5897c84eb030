"""Batched factorization and PCG of independent problems (spand_batch_*).

A batch runs stage k of every problem in the same launches and advances the
PCG of all problems together.  Against the same problems factored and solved
one at a time through spand_factor / spand_pcg:

* ranks and reflector counts per cluster are identical (the factorization
  kernels are deterministic and see the same blocks);
* the preconditioner of a batch-factored handle equals the one-at-a-time
  preconditioner to 1e-12 relative (the apply accumulates neighbour updates
  with atomics, so the last bits may differ between any two runs);
* batch PCG takes the same iteration counts (within one, since the dot
  products are summed in another fixed order) and reaches the true relative
  residual tol for every problem;
* a problem's iterates do not depend on the other problems of the batch.
"""
import numpy as np
import pytest

import spand_inputs as si

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _mix(precision=0):
    """Uneven 2D and 3D problems with different depths and coefficients."""
    from paper_2007_00789_gb300 import spand as S
    probs = [
        (si.diffusion_grid((40, 33), seed=3, lo=-2, hi=2), 5, 1),
        (si.laplacian_3d(16), 7, 1),
        (si.diffusion_3d(20, seed=4, lo=-2, hi=2), 8, 2),
        (si.diffusion_grid((64, 64), seed=5, lo=-2, hi=2), 6, 0),
        (si.diffusion_3d(12, seed=6, lo=-2, hi=2), 6, 1),
    ]
    hs = [S.Spand.from_problem(p, ell, 1e-2, scheme, precision=precision) for p, ell, scheme in probs]
    return [p for p, _, _ in probs], hs


def _rhs(probs):
    return [si.rhs_normal(p.n, seed=10 + i) for i, p in enumerate(probs)]


def test_batch_factor_matches_single():
    torch = _torch()
    from paper_2007_00789_gb300 import spand as S
    probs, hb = _mix()
    _, h1 = _mix()
    batch = S.SpandBatch(hb)
    batch.factor()
    for h in h1:
        h.factor()
    rng = np.random.default_rng(0)
    for p, a, b in zip(probs, hb, h1):
        ra, rb = a.ranks(), b.ranks()
        assert np.array_equal(ra, rb)
        assert a.info()["nnz_factor"] == b.info()["nnz_factor"]
        r = torch.from_numpy(rng.standard_normal(p.n)).cuda()
        za, zb = torch.empty_like(r), torch.empty_like(r)
        a.apply(r, za)
        b.apply(r, zb)
        torch.cuda.synchronize()
        err = float((za - zb).abs().max() / zb.abs().max())
        assert err <= 1e-12, err
    batch.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_pcg_matches_single(precision):
    torch = _torch()
    from paper_2007_00789_gb300 import spand as S
    probs, hb = _mix(precision)
    _, h1 = _mix(precision)
    batch = S.SpandBatch(hb)
    batch.factor()
    rhs = _rhs(probs)
    bs = [torch.from_numpy(b).cuda() for b in rhs]
    xs = [torch.zeros_like(b) for b in bs]
    its, rels = batch.pcg(bs, xs, 1e-12)
    for i, (p, h) in enumerate(zip(probs, h1)):
        h.factor()
        x1 = torch.zeros_like(bs[i])
        it1, rel1 = h.pcg(bs[i], x1, 1e-12)
        x = xs[i].cpu().numpy()
        true_rel = np.linalg.norm(rhs[i] - p.to_scipy() @ x) / np.linalg.norm(rhs[i])
        print(f"problem {i}: n={p.n} batch iters {its[i]} single {it1}, true relres {true_rel:.2e}")
        assert rels[i] <= 1e-12 and true_rel <= 1e-12
        assert abs(int(its[i]) - it1) <= 1, (its[i], it1)
    info = batch.info()
    assert info["ticks"] >= max(its)
    batch.close()


def test_batch_result_independent_of_mix():
    """A problem solved in a batch of one and inside the mix: same iterates."""
    torch = _torch()
    from paper_2007_00789_gb300 import spand as S
    probs, hb = _mix()
    batch = S.SpandBatch(hb)
    batch.factor()
    rhs = _rhs(probs)
    bs = [torch.from_numpy(b).cuda() for b in rhs]
    xs = [torch.zeros_like(b) for b in bs]
    its, _ = batch.pcg(bs, xs, 1e-12)
    for i in (0, 2):
        alone = S.SpandBatch([hb[i]])
        x1 = torch.zeros_like(bs[i])
        it1, _ = alone.pcg([bs[i]], [x1], 1e-12)
        assert it1[0] == its[i]
        d = float((x1 - xs[i]).abs().max() / xs[i].abs().max())
        assert d <= 1e-10, d
        alone.close()
    batch.close()


def test_batch_refactor_replays():
    torch = _torch()
    from paper_2007_00789_gb300 import spand as S
    probs, hb = _mix()
    batch = S.SpandBatch(hb)
    batch.factor()
    first = [h.ranks() for h in hb]
    rhs = _rhs(probs)
    bs = [torch.from_numpy(b).cuda() for b in rhs]
    xs = [torch.zeros_like(b) for b in bs]
    its0, _ = batch.pcg(bs, xs, 1e-12)
    for _ in range(2):
        batch.factor()  # unchanged ranks: replayed from the batch's graphs
        for h, r0 in zip(hb, first):
            assert np.array_equal(h.ranks(), r0)
        its, rels = batch.pcg(bs, xs, 1e-12)
        assert np.array_equal(its, its0) and (rels <= 1e-12).all()
    # a member factored on its own in between: the batch rebuilds
    hb[1].factor()
    batch.factor()
    its, rels = batch.pcg(bs, xs, 1e-12)
    assert np.array_equal(its, its0) and (rels <= 1e-12).all()
    batch.close()


def test_batch_not_spd_names_problem():
    _torch()
    from paper_2007_00789_gb300 import spand as S
    good = si.laplacian_2d(16)
    val = good.val.copy()
    val[np.nonzero(good.colind == 0)[0][0]] = -4.0  # diagonal of row 0: not SPD
    hs = [S.Spand.from_problem(good, 4, 1e-2, 1),
          S.Spand(good.rowptr, good.colind, val, good.coords, 4, 1e-2, 1)]
    batch = S.SpandBatch(hs)
    with pytest.raises(S.SpandError) as ei:
        batch.factor()
    assert ei.value.code == S.SPAND_ENOTSPD
    assert "problem 1" in str(ei.value)
    batch.close()


@pytest.mark.parametrize("precision,nrhs", [(0, 5), (1, 5), (1, 21)])
def test_many_rhs_match_single(precision, nrhs):
    """spand_apply_many / spand_pcg_many (padded leading dimension) against the
    single-column calls; 21 columns run five passes of 4 vectors plus one."""
    torch = _torch()
    from paper_2007_00789_gb300 import spand as S
    p = si.diffusion_3d(20, seed=9, lo=-2, hi=2)
    h = S.Spand.from_problem(p, 8, 1e-2, 1, precision=precision)
    h.factor()
    ld = p.n + 5
    rng = np.random.default_rng(4)
    R = torch.zeros((nrhs, ld), dtype=torch.float64, device="cuda")
    R[:, :p.n] = torch.from_numpy(rng.standard_normal((nrhs, p.n))).cuda()
    Z = torch.zeros_like(R)
    h.apply_many(R, Z)
    its, rels = h.pcg_many(R, torch.zeros_like(R), 1e-12)
    X = torch.zeros_like(R)
    its, rels = h.pcg_many(R, X, 1e-12)
    torch.cuda.synchronize()
    A = p.to_scipy()
    for j in range(nrhs):
        r = R[j, :p.n].contiguous()
        z1 = torch.empty_like(r)
        h.apply(r, z1)
        x1 = torch.zeros_like(r)
        it1, _ = h.pcg(r, x1, 1e-12)
        torch.cuda.synchronize()
        err = float((Z[j, :p.n] - z1).abs().max() / z1.abs().max())
        assert err <= (1e-12 if precision == 0 else 1e-5), err
        assert abs(int(its[j]) - it1) <= 1
        x = X[j, :p.n].cpu().numpy()
        b = r.cpu().numpy()
        assert rels[j] <= 1e-12 and np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1e-12
    assert float(Z[:, p.n:].abs().max()) == 0.0  # padding untouched
    h.close()
