"""Pins for the oracle's spaND (Algorithm 2), its apply and its PCG (§3-§4).

* eps = 0 makes spaND an exact block Cholesky with nested-dissection ordering
  (§3.2), so M must equal A^{-1} (dense brute force) and PCG must stop after
  one iteration;
* M is symmetric and L^{-1} A L^{-T} is SPD (the middle matrix stays SPD by the
  implicit Schur compensation, §2.2); for the full second-order scheme the
  dropped term -E^T E is negative semi-definite, so L L^T >= A and every
  eigenvalue of L^{-1} A L^{-T} lies in (0, 1];
* the error ||I - M A|| shrinks like eps for the first-order scheme and like
  eps^2 for the second-order schemes;
* the coarse ranks do not depend on the scheme (the middle matrix is the same
  in eqs. trailing-1/2/3);
* the Dirichlet Laplacian eigenpairs of §4.1.1 pin the input stencil, and the
  second-order forward error on them is below the first-order one;
* PCG iteration counts are about halved (§4.1.2);
* general SPD input: with the algebraic partition, eps = 0 is still exact;
  diagonal prescaling makes the factorization invariant to a diagonal
  rescaling T A T and changes nothing on a constant diagonal.
"""
import numpy as np
import pytest

import spand_inputs as si
from oracle import spand as S

CASES = [
    ("2d16", lambda: si.laplacian_2d(16), 4),
    ("3d8", lambda: si.laplacian_3d(8), 5),
    ("diff3d8", lambda: si.diffusion_3d(8, seed=3), 5),
    ("diff2d_10x13", lambda: si.diffusion_grid((10, 13), seed=4), 4),
]


def _dense_m(F, n):
    return np.stack([S.apply(F, e) for e in np.eye(n)], axis=1)


@pytest.mark.parametrize("name,make,ell", CASES)
@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_eps_zero_is_exact_cholesky(name, make, ell, scheme):
    prob = make()
    A = prob.to_scipy()
    Ainv = np.linalg.inv(A.toarray())
    for skip in (0, 1):
        F = S.factor(A, prob.coords, ell, 0.0, scheme, skip=skip)
        M = _dense_m(F, prob.n)
        assert np.abs(M - Ainv).max() <= 1e-12 * np.abs(Ainv).max()
    b = si.rhs_uniform(prob.n, seed=0)
    res = S.pcg(lambda v: A @ v, lambda v: S.apply(F, v), b, 1e-12)
    assert res.iters == 1 and res.relres < 1e-12


@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_symmetric_and_spd(scheme):
    prob = si.diffusion_grid((20, 20), seed=7, lo=-2, hi=2)
    A = prob.to_scipy()
    F = S.factor(A, prob.coords, 5, 0.1, scheme, skip=1)
    assert sum(sum(r.values()) for r in F.stage_ranks) > 0
    Linv = np.stack([S.apply_linv(F, e) for e in np.eye(prob.n)], axis=1)
    LinvT = np.stack([S.apply_lt_inv(F, e) for e in np.eye(prob.n)], axis=1)
    assert np.allclose(LinvT, Linv.T, atol=1e-13 * np.abs(Linv).max())
    P = Linv @ A.toarray() @ Linv.T
    lam = np.linalg.eigvalsh(0.5 * (P + P.T))
    assert lam.min() > 0
    if scheme == S.SECOND_ORDER_FULL:
        assert lam.max() <= 1.0 + 1e-10
    M = _dense_m(F, prob.n)
    assert np.abs(M - M.T).max() <= 1e-13 * np.abs(M).max()


def test_error_order_in_eps():
    prob = si.laplacian_2d(32)
    A = prob.to_scipy()
    Ad = A.toarray()
    err = {}
    for eps in (1e-1, 1e-2, 1e-3):
        for scheme in (0, 1, 2):
            F = S.factor(A, prob.coords, 5, eps, scheme, skip=1)
            err[eps, scheme] = np.linalg.norm(np.eye(prob.n) - _dense_m(F, prob.n) @ Ad, 2)
    for lo, hi in ((1e-2, 1e-1), (1e-3, 1e-2)):
        fo = err[hi, 0] / err[lo, 0]
        so = err[hi, 1] / err[lo, 1]
        sf = err[hi, 2] / err[lo, 2]
        assert 5 < fo < 20, fo
        assert 40 < so < 400, so
        assert 40 < sf < 400, sf
    for eps in (1e-1, 1e-2, 1e-3):
        assert err[eps, 1] < err[eps, 0] and err[eps, 2] < err[eps, 0]


def test_ranks_do_not_depend_on_scheme():
    prob = si.diffusion_3d(12, seed=5)
    A = prob.to_scipy()
    F = [S.factor(A, prob.coords, 6, 1e-2, s, skip=1) for s in (0, 1, 2)]
    assert F[0].stage_ranks == F[1].stage_ranks == F[2].stage_ranks
    assert F[0].nnz_factor() < F[2].nnz_factor() <= F[1].nnz_factor()


def test_poisson_eigenpairs_and_forward_error():
    d = 32
    prob = si.laplacian_2d(d)
    A = prob.to_scipy()
    x, y = prob.coords[:, 0] + 1, prob.coords[:, 1] + 1
    F1 = S.factor(A, prob.coords, 5, 0.1, 0, skip=1)
    F2 = S.factor(A, prob.coords, 5, 0.1, 1, skip=1)
    for p in (1, 2, 4, 8, 16, 24, 31):
        v = np.sin(p * x * np.pi / (d + 1)) * np.sin(p * y * np.pi / (d + 1))
        v /= np.linalg.norm(v)
        lam = 8.0 * np.sin(p * np.pi / (2 * (d + 1))) ** 2
        assert np.allclose(A @ v, lam * v, atol=1e-12)
        e1 = np.linalg.norm(v - S.apply(F1, A @ v))
        e2 = np.linalg.norm(v - S.apply(F2, A @ v))
        assert e2 < e1


def test_pcg_iterations_about_halved():
    prob = si.laplacian_2d(64)
    A = prob.to_scipy()
    b = si.rhs_uniform(prob.n, seed=0)
    it = {}
    for scheme in (0, 1, 2):
        F, res = S.solve(A, prob.coords, b, 6, 1e-2, scheme)
        assert res.relres < 1e-12
        it[scheme] = res.iters
    assert 0.4 <= it[1] / it[0] <= 0.65
    assert 0.4 <= it[2] / it[0] <= 0.65


def test_bad_inputs():
    prob = si.laplacian_2d(8)
    A = prob.to_scipy()
    with pytest.raises(ValueError):
        S.factor(A, prob.coords, 3, 1.5)
    with pytest.raises(ValueError):
        S.factor(A, prob.coords, 3, 0.1, scheme=3)
    bad = A.tolil()
    bad[5, 5] = -4.0
    with pytest.raises(S.NotSPDError):
        S.factor(bad.tocsr(), prob.coords, 3, 0.1)


# ---- general SPD input: algebraic partition and diagonal prescaling ----

def _relabel(prob, seed):
    perm = np.random.default_rng(seed).permutation(prob.n)
    A = prob.to_scipy()[perm][:, perm].tocsr()
    A.sort_indices()
    return A


def test_algebraic_partition_exact_at_eps0():
    """With eps = 0 the factorization is exact for any partition: M = A^{-1}, one PCG step."""
    A = _relabel(si.diffusion_grid((11, 9), seed=4), 0)
    F = S.factor(A, None, 4, 0.0, S.SECOND_ORDER_FULL)
    Ad = A.toarray()
    M = np.column_stack([S.apply(F, e) for e in np.eye(A.shape[0])])
    assert np.abs(M @ Ad - np.eye(A.shape[0])).max() < 1e-10
    b = si.rhs_normal(A.shape[0], seed=1)
    res = S.pcg(lambda v: A @ v, lambda v: S.apply(F, v), b, 1e-12)
    assert res.iters == 1


def test_prescaling_removes_diagonal_scaling():
    """Prescaled factorizations of A and of T A T (T diagonal, positive) coincide:
    both factor the same matrix D^{-1/2} A D^{-1/2}, so ranks are identical and
    M_{TAT} = T^{-1} M_A T^{-1}."""
    import scipy.sparse as sp
    prob = si.diffusion_3d(8, seed=5)
    A = prob.to_scipy()
    t = 10.0 ** np.random.default_rng(2).uniform(-3, 3, prob.n)
    T = sp.diags(t)
    B = (T @ A @ T).tocsr()
    FA = S.factor(A, prob.coords, 5, 1e-2, S.SECOND_ORDER_FULL, prescale=True)
    FB = S.factor(B, prob.coords, 5, 1e-2, S.SECOND_ORDER_FULL, prescale=True)
    assert FA.stage_ranks == FB.stage_ranks
    r = si.rhs_normal(prob.n, seed=3)
    za = S.apply(FA, r / t) / t
    zb = S.apply(FB, r)
    assert np.abs(za - zb).max() <= 1e-10 * np.abs(zb).max()


def test_prescaling_constant_diagonal_is_neutral():
    """With a constant diagonal (the Poisson matrix) prescaling changes nothing but rounding."""
    prob = si.laplacian_2d(16)
    A = prob.to_scipy()
    F0 = S.factor(A, prob.coords, 5, 1e-2, S.SECOND_ORDER_FULL)
    F1 = S.factor(A, prob.coords, 5, 1e-2, S.SECOND_ORDER_FULL, prescale=True)
    assert F0.stage_ranks == F1.stage_ranks
    r = si.rhs_normal(prob.n, seed=0)
    z0, z1 = S.apply(F0, r), S.apply(F1, r)
    assert np.abs(z0 - z1).max() <= 1e-12 * np.abs(z0).max()
