"""Pins for the oracle's Algorithm 1 (early-stopping column-pivoted QR, §3.1).

Checked against orthogonality and reconstruction, the stop rule's own bound,
a library cross-check (scipy's pivoted QR rank on well-separated spectra),
the degenerate cases, and the superfine invariants (Q_c unchanged, r2 >= r).
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.rrqr import (FIRST_ORDER, SECOND_ORDER_FULL, SECOND_ORDER_SUPERFINE,
                         apply_q, apply_qt, explicit_q, fine_block, rrqr)


def _matrix_with_spectrum(m, n, sigma, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, m)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    S = np.zeros((m, n))
    k = min(m, n, len(sigma))
    S[np.arange(k), np.arange(k)] = sigma[:k]
    return U @ S @ V.T


@pytest.mark.parametrize("m,n", [(12, 40), (30, 30), (40, 9), (1, 5), (7, 1)])
def test_reconstruction_and_orthogonality(m, n):
    rng = np.random.default_rng(m * 100 + n)
    A = rng.standard_normal((m, n))
    res = rrqr(A, 0.0, SECOND_ORDER_FULL)
    assert res.r == min(m, n) == res.nref
    Q = explicit_q(res.V, res.tau)
    assert np.allclose(Q.T @ Q, np.eye(m), atol=1e-13)
    assert np.allclose(Q @ res.R, A, atol=1e-12)
    # R Pi is upper trapezoidal: pivot column t has zeros below row t
    for t, j in enumerate(res.piv):
        assert np.all(res.R[t + 1:, j] == 0.0)
    # Q^T z and Q z by reflectors agree with the explicit matrix
    z = rng.standard_normal(m)
    assert np.allclose(apply_qt(res.V, res.tau, z), Q.T @ z, atol=1e-13)
    assert np.allclose(apply_q(res.V, res.tau, z), Q @ z, atol=1e-13)


@pytest.mark.parametrize("eps", [1e-1, 1e-2, 1e-3])
def test_stop_rule_bound_and_fine_block(eps):
    sigma = 10.0 ** (-0.5 * np.arange(20))
    A = _matrix_with_spectrum(20, 50, sigma, seed=1)
    res = rrqr(A, eps, SECOND_ORDER_FULL)
    nu0 = np.max(np.linalg.norm(A, axis=0))
    E = fine_block(res, SECOND_ORDER_FULL)
    assert E.shape == (20 - res.r, 50)
    # every trailing column is below eps * nu_0 when the QR stops (§3.1 stop rule)
    assert np.max(np.linalg.norm(E, axis=0)) < eps * nu0
    assert np.linalg.norm(E, 2) <= np.sqrt(50 - res.r) * eps * nu0
    # E = Q_f^T A and Q_c^T A are the two row blocks of Q^T A (Algorithm 1 outputs)
    Q = explicit_q(res.V, res.tau)
    assert np.allclose(E, Q[:, res.r:].T @ A, atol=1e-13)
    assert np.allclose(res.R[:res.r], Q[:, :res.r].T @ A, atol=1e-13)
    assert fine_block(res, FIRST_ORDER).shape[0] == 0


@pytest.mark.parametrize("seed", range(4))
def test_rank_matches_library_pivoted_qr(seed):
    # well separated spectrum: 6 values near 1, then a 1e4 gap around the threshold
    sigma = np.r_[np.linspace(1.0, 0.5, 6), 1e-5 * np.linspace(1.0, 0.5, 10)]
    A = _matrix_with_spectrum(16, 40, sigma, seed)
    res = rrqr(A, 1e-3, SECOND_ORDER_FULL)
    _, R, _ = sla.qr(A, pivoting=True)
    d = np.abs(np.diag(R))
    assert res.r == int(np.sum(d >= 1e-3 * d[0])) == 6


def test_degenerate_cases():
    assert rrqr(np.zeros((5, 7)), 0.1).r == 0
    assert rrqr(np.zeros((5, 0)), 0.1).r == 0
    assert rrqr(np.zeros((0, 4)), 0.1).r == 0
    res = rrqr(np.ones((3, 4)), 1.0)
    assert res.r == 1  # eps = 1: only the first step passes nu >= nu_0
    A = np.random.default_rng(0).standard_normal((6, 8))
    assert rrqr(A, 0.0).r == 6


def test_tie_goes_to_lowest_index():
    A = np.zeros((3, 4))
    A[:, 1] = [1.0, 2.0, 2.0]  # norm 3
    A[:, 3] = [2.0, 2.0, 1.0]  # norm 3 as well
    A[:, 0] = [0.5, 0.0, 0.0]
    res = rrqr(A, 0.0)
    assert res.piv[0] == 1
    # reflector sign convention: beta = -sign(alpha) ||x|| with sign(0) = +1
    assert res.R[0, 1] == pytest.approx(-3.0)
    res = rrqr(np.array([[0.0], [3.0], [4.0]]), 0.0)
    assert res.R[0, 0] == pytest.approx(-5.0)


def test_superfine_extends_first_order():
    sigma = 10.0 ** (-0.5 * np.arange(16))
    A = _matrix_with_spectrum(16, 30, sigma, seed=3)
    eps = 1e-2
    fo = rrqr(A, eps, FIRST_ORDER)
    sf = rrqr(A, eps, SECOND_ORDER_SUPERFINE)
    assert sf.r == fo.r and fo.nref == fo.r
    assert sf.nref >= sf.r
    nu0 = np.max(np.linalg.norm(A, axis=0))
    # coarse rows Q_c^T A and Q_c itself are unchanged (§2.2.1)
    assert np.array_equal(sf.R[:sf.r], fo.R[:fo.r])
    Qf, Qs = explicit_q(fo.V, fo.tau), explicit_q(sf.V, sf.tau)
    assert np.allclose(Qf[:, :fo.r], Qs[:, :sf.r], atol=1e-14)
    E2 = fine_block(sf, SECOND_ORDER_SUPERFINE)
    E1 = sf.R[sf.nref:]
    assert E2.shape[0] == sf.nref - sf.r
    assert np.max(np.linalg.norm(E1, axis=0)) < eps * eps * nu0
    assert np.allclose(E2, Qs[:, sf.r:sf.nref].T @ A, atol=1e-13)
