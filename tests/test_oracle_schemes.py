"""Two-level pins of the three sparsification schemes (§2.1-2.3).

The toy matrix of eq. (A), ``A = [[I, A12, 0], [A21, A22, A23], [0, A32, A33]]``,
is sparsified once with the oracle's Algorithm 1.  The two-level factors of
eqs. (l1), (l2), (l3) built from its outputs must satisfy the paper's exact
identities: ||A - L1 L1^T|| = ||E||, ||A - L2 L2^T|| = ||E||^2, the condition
numbers of Propositions 1 and 2, and the block pattern of Proposition 3.  A
dropped term, a wrong sign or a transposed E in Algorithm 1 breaks one of them.
"""
import numpy as np
import pytest

from oracle.rrqr import (FIRST_ORDER, SECOND_ORDER_FULL, SECOND_ORDER_SUPERFINE,
                         explicit_q, fine_block, rrqr)

M1, M2, M3 = 10, 12, 8


def _toy(seed=0):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((M1, M1)))
    V, _ = np.linalg.qr(rng.standard_normal((M2, M2)))
    sig = 0.6 * 10.0 ** (-0.4 * np.arange(M1))
    A12 = U @ np.diag(sig) @ V[:, :M1].T
    G = rng.standard_normal((M2, M2))
    A22 = 3.0 * np.eye(M2) + 0.1 * (G + G.T)
    A23 = 0.3 * rng.standard_normal((M2, M3))
    H = rng.standard_normal((M3, M3))
    A33 = 3.0 * np.eye(M3) + 0.1 * (H + H.T)
    A = np.zeros((M1 + M2 + M3,) * 2)
    A[:M1, :M1] = np.eye(M1)
    A[:M1, M1:M1 + M2] = A12
    A[M1:M1 + M2, :M1] = A12.T
    A[M1:M1 + M2, M1:M1 + M2] = A22
    A[M1:M1 + M2, M1 + M2:] = A23
    A[M1 + M2:, M1:M1 + M2] = A23.T
    A[M1 + M2:, M1 + M2:] = A33
    assert np.linalg.eigvalsh(A).min() > 0
    return A, A12


def _two_level(A, A12, eps, scheme):
    res = rrqr(A12, eps, scheme)
    r, nref = res.r, res.nref
    Q = explicit_q(res.V, res.tau)
    Qc = Q[:, :r]
    nf = M1 - r
    # middle matrix A-hat over (c, 2, 3), eq. trailing-1
    nh = r + M2 + M3
    Ah = np.zeros((nh, nh))
    Ah[:r, :r] = np.eye(r)
    Ah[:r, r:r + M2] = Qc.T @ A12
    Ah[r:r + M2, :r] = (Qc.T @ A12).T
    Ah[r:, r:] = A[M1:, M1:]
    Lh = np.linalg.cholesky(Ah)
    # V maps (f, c, 2, 3) coordinates to the original ordering; Q_f = Q[:, r:]
    Vb = np.zeros((M1 + M2 + M3,) * 2)
    Vb[:M1, :nf] = Q[:, r:]
    Vb[:M1, nf:M1] = Qc
    Vb[M1:, M1:] = np.eye(M2 + M3)
    return res, Q, Lh, Vb, nf


def _hat(E_rows, r):
    """E-hat = (0 E 0) over the (c, 2, 3) columns."""
    Eh = np.zeros((E_rows.shape[0], r + M2 + M3))
    Eh[:, r:r + M2] = E_rows
    return Eh


def _blk(*mats):
    n = sum(m.shape[0] for m in mats)
    out = np.zeros((n, n))
    o = 0
    for m in mats:
        out[o:o + m.shape[0], o:o + m.shape[0]] = m
        o += m.shape[0]
    return out


@pytest.mark.parametrize("eps", [3e-1, 1e-1, 3e-2, 1e-2])
def test_first_and_second_order_errors(eps):
    A, A12 = _toy()
    res, Q, Lh, Vb, nf = _two_level(A, A12, eps, SECOND_ORDER_FULL)
    E = fine_block(res, SECOND_ORDER_FULL)
    assert E.shape[0] == nf > 0
    Eh = _hat(E, res.r)
    L1 = Vb @ _blk(np.eye(nf), Lh)
    low = np.eye(nf + Lh.shape[0])
    low[nf:, :nf] = Eh.T
    L2 = Vb @ low @ _blk(np.eye(nf), Lh)
    nE = np.linalg.norm(E, 2)
    # eq. for E_1: A - L1 L1^T = V [[0, Eh], [Eh^T, 0]] V^T, so its 2-norm is ||E||
    assert np.linalg.norm(A - L1 @ L1.T, 2) == pytest.approx(nE, rel=1e-10)
    # eq. for E_2: A - L2 L2^T = -V (0 + Eh^T Eh) V^T, so its 2-norm is ||E||^2
    assert np.linalg.norm(A - L2 @ L2.T, 2) == pytest.approx(nE ** 2, rel=1e-8)

    # Propositions 1 and 2 with t = ||Lh^{-1} Eh^T||_2 computed on its own
    t = np.linalg.norm(np.linalg.solve(Lh, Eh.T), 2)
    assert t < 1.0
    P1 = np.linalg.solve(L1, np.linalg.solve(L1, A).T)
    P2 = np.linalg.solve(L2, np.linalg.solve(L2, A).T)
    assert np.linalg.cond(P1) == pytest.approx((1 + t) / (1 - t), rel=1e-8)
    assert np.linalg.cond(P2) == pytest.approx(1.0 / (1 - t * t), rel=1e-8)
    C = np.linalg.solve(Lh, Eh.T)
    want2 = _blk(np.eye(nf), np.eye(Lh.shape[0]) - C @ C.T)
    assert np.allclose(P2, want2, atol=1e-12)
    # the convergence-rate bound of the second-order scheme is the square of the first
    R1 = (np.sqrt((1 + t) / (1 - t)) - 1) / (np.sqrt((1 + t) / (1 - t)) + 1)
    R2 = (np.sqrt(1 / (1 - t * t)) - 1) / (np.sqrt(1 / (1 - t * t)) + 1)
    assert R2 == pytest.approx(R1 ** 2, rel=1e-12)


@pytest.mark.parametrize("eps", [1e-1, 3e-2])
def test_superfine_proposition_3(eps):
    A, A12 = _toy(1)
    res, Q, Lh, Vb, nf = _two_level(A, A12, eps, SECOND_ORDER_SUPERFINE)
    r, r2 = res.r, res.nref
    nf2, nf1 = r2 - r, M1 - r2
    assert nf1 > 0 and nf2 > 0
    E2 = fine_block(res, SECOND_ORDER_SUPERFINE)
    E1 = res.R[r2:]
    # V for the (f1, f2, c, 2, 3) ordering of eq. trailing-3
    V3 = np.zeros_like(Vb)
    V3[:M1, :nf1] = Q[:, r2:]
    V3[:M1, nf1:nf1 + nf2] = Q[:, r:r2]
    V3[:M1, M1 - r:M1] = Q[:, :r]
    V3[M1:, M1:] = np.eye(M2 + M3)
    nh = Lh.shape[0]
    low = np.eye(M1 - r + nh)
    low[nf1 + nf2:, nf1:nf1 + nf2] = _hat(E2, r).T
    L3 = V3 @ low @ _blk(np.eye(nf1 + nf2), Lh)
    P3 = np.linalg.solve(L3, np.linalg.solve(L3, A).T)
    E1h, E2h = _hat(E1, r), _hat(E2, r)
    Li = np.linalg.inv(Lh)
    want = np.eye(M1 - r + nh)
    o = nf1 + nf2
    want[:nf1, o:] += E1h @ Li.T
    want[o:, :nf1] += Li @ E1h.T
    want[o:, o:] -= Li @ E2h.T @ E2h @ Li.T
    assert np.allclose(P3, want, atol=1e-12)
    # with f1 = f this is the first-order scheme, with f2 = f the full second-order one
    fo = rrqr(A12, eps, FIRST_ORDER)
    assert fo.r == r
