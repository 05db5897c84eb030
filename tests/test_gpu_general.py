"""General SPD input on the GPU: algebraic partition and diagonal prescaling.

Against the CPU oracle run with the same options (FP64):
* without coordinates (vertices relabelled at random, so nothing of the grid
  is left but the graph of A) the ranks are identical cluster by cluster,
  M r agrees to 1e-10 relative, nnz(L) is equal, and PCG takes the oracle's
  iteration count within one to a true relative residual <= 1e-12;
* with diagonal prescaling on a badly scaled matrix T A T (T = 10^U(-3,3))
  the same holds (the attainable true residual of such a matrix is limited by
  rounding in b - A x: the bar is then ten times what the oracle attains), and
  the prescaled GPU factorization of T A T has exactly the ranks of the
  prescaled factorization of A;
* the FP32 factorization, batches and the multi-RHS PCG accept both options.
"""
import numpy as np
import pytest

import spand_inputs as si
from oracle import spand as OS

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _relabel(prob, seed):
    perm = np.random.default_rng(seed).permutation(prob.n)
    A = prob.to_scipy()[perm][:, perm].tocsr()
    A.sort_indices()
    return A


def _scaled(prob, seed, decades=3):
    import scipy.sparse as sp
    t = 10.0 ** np.random.default_rng(seed).uniform(-decades, decades, prob.n)
    B = (sp.diags(t) @ prob.to_scipy() @ sp.diags(t)).tocsr()
    B.sort_indices()
    return B


def _oracle_ranks(F):
    out = []
    for k, keys in enumerate(F.stage_keys):
        for key in keys:
            out.append((F.stage_sizes[k][key], F.stage_ranks[k].get(key, -1)))
    return np.array(out, dtype=np.int64)


def _apply(h, r):
    torch = _torch()
    rd = torch.from_numpy(r).cuda()
    zd = torch.empty_like(rd)
    h.apply(rd, zd)
    torch.cuda.synchronize()
    return zd.cpu().numpy()


def _pcg(h, A, b, tol=1e-12):
    torch = _torch()
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    it, rel = h.pcg(bd, x, tol)
    xh = x.cpu().numpy()
    return it, rel, np.linalg.norm(b - A @ xh) / np.linalg.norm(b)


CASES = [
    # name, matrix, coords, ell, scheme, prescale
    ("graph_diff3d_16", lambda: _relabel(si.diffusion_3d(16, seed=2), 0), None, 7, 1, False),
    ("graph_diff2d_40x33", lambda: _relabel(si.diffusion_grid((40, 33), seed=3), 1), None, 6, 2, False),
    ("graph_scaled_diff3d_12", lambda: _scaled(si.diffusion_3d(12, seed=4), 2), None, 6, 1, True),
    ("geom_scaled_diff3d_16", lambda: _scaled(si.diffusion_3d(16, seed=5), 3), "grid", 7, 1, True),
]


@pytest.mark.parametrize("name,make,coords,ell,scheme,prescale", CASES, ids=[c[0] for c in CASES])
def test_general_input_parity(name, make, coords, ell, scheme, prescale):
    _torch()
    from paper_2007_00789_gb300 import spand as S
    A = make()
    n = A.shape[0]
    side = round(n ** (1 / 3)) if "3d" in name else None
    xyz = si.diffusion_3d(side, seed=0).coords if coords == "grid" else None
    F = OS.factor(A, xyz, ell, 1e-2, scheme, prescale=prescale)
    h = S.Spand(A.indptr, A.indices, A.data, xyz, ell, 1e-2, scheme, prescale=prescale)
    h.factor()
    got = h.ranks()
    want = _oracle_ranks(F)
    assert np.array_equal(got[:, :2], want), "ranks differ"
    assert not got[:, 2].any(), "unexpected near tie"
    assert h.info()["nnz_factor"] == F.nnz_factor()
    rng = np.random.default_rng(7)
    for _ in range(2):
        r = rng.standard_normal(n)
        zo = OS.apply(F, r)
        err = np.abs(_apply(h, r) - zo).max() / np.abs(zo).max()
        assert err <= 1e-10, err
    b = si.rhs_normal(n, seed=1)
    res = OS.pcg(lambda v: A @ v, lambda v: OS.apply(F, v), b, 1e-12)
    it, rel, true_rel = _pcg(h, A, b)
    # a badly scaled matrix limits the attainable true residual (rounding in
    # b - A x): the bar is 1e-12 or ten times what the oracle attains
    floor = max(1e-12, 10.0 * res.relres)
    print(f"{name}: iters gpu {it} oracle {res.iters}, true relres {true_rel:.2e} "
          f"(oracle {res.relres:.2e})")
    assert abs(it - res.iters) <= 1 and rel <= floor and true_rel <= floor
    h.close()


def test_prescaled_ranks_ignore_diagonal_scaling():
    _torch()
    from paper_2007_00789_gb300 import spand as S
    prob = si.diffusion_3d(16, seed=8)
    A = prob.to_scipy()
    B = _scaled(prob, 9)
    ha = S.Spand(A.indptr, A.indices, A.data, prob.coords, 7, 1e-2, 1, prescale=True)
    hb = S.Spand(B.indptr, B.indices, B.data, prob.coords, 7, 1e-2, 1, prescale=True)
    hn = S.Spand(B.indptr, B.indices, B.data, prob.coords, 7, 1e-2, 1)
    for h in (ha, hb, hn):
        h.factor()
    assert np.array_equal(ha.ranks()[:, :2], hb.ranks()[:, :2])
    b = si.rhs_normal(prob.n, seed=2)
    it_b, _, rb = _pcg(hb, B, b)
    it_n, _, rn = _pcg(hn, B, b)
    print(f"scaled matrix: iters with prescaling {it_b} (true relres {rb:.1e}),"
          f" without {it_n} ({rn:.1e})")
    assert it_b <= it_n
    for h in (ha, hb, hn):
        h.close()


def test_general_input_fp32_batch_and_many():
    torch = _torch()
    from paper_2007_00789_gb300 import spand as S
    A1 = _relabel(si.diffusion_3d(14, seed=3), 4)
    A2 = _scaled(si.diffusion_grid((50, 41), seed=5), 5, decades=1)
    hs = [S.Spand(A1.indptr, A1.indices, A1.data, None, 6, 1e-2, 1, precision=1),
          S.Spand(A2.indptr, A2.indices, A2.data, None, 6, 1e-2, 1, precision=1, prescale=True)]
    batch = S.SpandBatch(hs)
    batch.factor()
    bs = [torch.from_numpy(si.rhs_normal(A.shape[0], seed=i)).cuda() for i, A in enumerate((A1, A2))]
    xs = [torch.zeros_like(b) for b in bs]
    tol = 1e-10  # attainable on the rescaled second problem (its floor is about 1e-11)
    its, rels = batch.pcg(bs, xs, tol)
    for A, b, x in zip((A1, A2), bs, xs):
        bh, xh = b.cpu().numpy(), x.cpu().numpy()
        assert np.linalg.norm(bh - A @ xh) / np.linalg.norm(bh) <= tol
    # several right-hand sides of the prescaled problem
    B = torch.from_numpy(np.random.default_rng(0).standard_normal((3, A2.shape[0]))).cuda()
    X = torch.zeros_like(B)
    it3, rel3 = hs[1].pcg_many(B, X, tol)
    assert (rel3 <= tol).all()
    batch.close()
    for h in hs:
        h.close()
