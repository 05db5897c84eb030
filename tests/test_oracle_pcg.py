"""Pins for the oracle's PCG: Theorem 1 (§2.3.4) and plain CG facts.

Theorem 1: for A1 = [[I, C], [C^T, I]] and A2 = diag(I, I - C^T C) with
||C|| < 1 and C^T b1 = 0, CG from x0 = 0 gives r^(1)_{2k} = r^(2)_k.  This
holds for the residual vectors of any correct CG recurrence and fails for a
wrong step length, a wrong conjugation coefficient or a missing update.
"""
import numpy as np
import pytest

from oracle.spand import pcg


def _theorem_system(n1, n2, seed):
    rng = np.random.default_rng(seed)
    C = rng.standard_normal((n1, n2))
    C *= 0.9 / np.linalg.norm(C, 2)
    # b1 in the null space of C^T
    U, s, Vt = np.linalg.svd(C)
    null = U[:, n2:]
    b1 = null @ rng.standard_normal(n1 - n2)
    b2 = rng.standard_normal(n2)
    A1 = np.block([[np.eye(n1), C], [C.T, np.eye(n2)]])
    A2 = np.block([[np.eye(n1), np.zeros((n1, n2))], [np.zeros((n2, n1)), np.eye(n2) - C.T @ C]])
    return A1, A2, np.r_[b1, b2], C, b1


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_theorem_1_residuals(seed):
    A1, A2, b, C, b1 = _theorem_system(14, 6, seed)
    assert np.abs(C.T @ b1).max() < 1e-12
    ident = lambda v: v  # noqa: E731
    r1 = pcg(lambda v: A1 @ v, ident, b, 1e-14, maxit=40, true_every=10**9,
             max_restarts=0, keep_residuals=True).residuals
    r2 = pcg(lambda v: A2 @ v, ident, b, 1e-14, maxit=40, true_every=10**9,
             max_restarts=0, keep_residuals=True).residuals
    bn = np.linalg.norm(b)
    checked = 0
    for k in range(len(r2)):
        if 2 * k >= len(r1) or np.linalg.norm(r2[k]) < 1e-8 * bn:
            break
        assert np.allclose(r1[2 * k], r2[k], atol=1e-10 * bn), k
        checked += 1
    assert checked >= 4


def test_exact_preconditioner_one_iteration():
    rng = np.random.default_rng(3)
    G = rng.standard_normal((30, 30))
    A = G @ G.T + 30 * np.eye(30)
    Ainv = np.linalg.inv(A)
    b = rng.standard_normal(30)
    res = pcg(lambda v: A @ v, lambda v: Ainv @ v, b, 1e-12)
    assert res.iters == 1 and res.relres < 1e-12


def test_cg_finite_termination_and_zero_rhs():
    rng = np.random.default_rng(4)
    d = np.array([1.0, 2.0, 5.0, 9.0])
    Q, _ = np.linalg.qr(rng.standard_normal((4, 4)))
    A = Q @ np.diag(d) @ Q.T
    b = rng.standard_normal(4)
    res = pcg(lambda v: A @ v, lambda v: v, b, 1e-12)
    assert res.iters <= 5 and res.relres < 1e-12  # 4 distinct eigenvalues (+1 for rounding)
    assert np.allclose(A @ res.x, b)
    z = pcg(lambda v: A @ v, lambda v: v, np.zeros(4), 1e-12)
    assert z.iters == 0 and np.all(z.x == 0)
