"""Algorithm 1 of the paper: early-stopping column-pivoted QR of A_pw.

Test infrastructure only (see ``oracle/__init__``).

Given the scaled off-diagonal block ``A_pw`` (m x N) of an interface p,
column-pivoted Householder QR ``A_pw Pi = Q R`` is run until the rank rule of
§3.1 stops it.  Conventions (the paper uses LAPACK's dlaqps and states none of
them, so these are the readings this project fixes):

* step t (0-based) pivots on the non-pivoted column with the largest squared
  2-norm of its rows t..m-1, recomputed exactly at every step (no downdating);
  ties go to the lowest column index;
* with nu_t^2 that largest squared norm, step t is taken only while
  ``nu_t^2 >= (eps*eps) * nu_0^2``; the number of steps taken is the rank r
  (so r >= 1 whenever A_pw != 0 and eps <= 1, r = min(m, N) at eps = 0, and
  r = 0 when N = 0 or A_pw = 0).  The superfine scheme keeps going while
  ``nu_t^2 >= (eps*eps)*(eps*eps) * nu_0^2`` to get r2 >= r (§3.1: the
  decomposition is stopped at eps^2 instead of eps);
* reflector: x = R[t:, j], alpha = x[0], beta = -sign(alpha) ||x|| with
  sign(0) = +1, tau = (beta - alpha) / beta, v = x / (alpha - beta), v[0] = 1;
  a zero x gives tau = 0 (H = I);
* a step is flagged as a near tie when the two largest candidate norms
  differ by at most 1e-12 relative (bit 0 of ``flags``), or when nu_t^2 lies
  within 1e-10 relative of a stopping threshold (bit 1).  There, rounding
  differences between two correct implementations may pick another pivot or
  rank, so parity is judged on the preconditioner's quality instead;
* columns are never physically swapped: the result R is ``Q^T A_pw`` in the
  original column order, i.e. ``R Pi`` of the paper.  Its first r rows are
  ``Q_c^T A_pw = (R_cc R_cf) Pi^T`` and rows r..m-1 are
  ``E = Q_f^T A_pw = (0 R_ff) Pi^T`` (§3.1).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

FIRST_ORDER = 0
SECOND_ORDER_FULL = 1
SECOND_ORDER_SUPERFINE = 2


@dataclass
class RRQRResult:
    r: int  # coarse rank (columns of Q_c)
    nref: int  # reflectors applied: r, or r2 for the superfine scheme
    V: np.ndarray  # m x nref, column t holds v_t in rows t..m-1 (v_t[t] = 1), zero above
    tau: np.ndarray  # nref
    R: np.ndarray  # m x N, Q^T A_pw in original column order
    piv: np.ndarray  # nref pivot columns, in step order
    flags: int = 0  # bit 0: pivot near tie, bit 1: threshold near tie


def rrqr(A: np.ndarray, eps: float, scheme: int = SECOND_ORDER_FULL) -> RRQRResult:
    """Early-stopping column-pivoted Householder QR (Algorithm 1)."""
    R = np.array(A, dtype=np.float64, copy=True)
    m, N = R.shape
    pivoted = np.zeros(N, dtype=bool)
    thr1 = eps * eps
    thr2 = thr1 * thr1
    Vcols, taus, pivs = [], [], []
    r = None
    nu0sq = 0.0
    flags = 0
    for t in range(min(m, N)):
        cand = np.nonzero(~pivoted)[0]
        normsq = np.sum(R[t:, cand] ** 2, axis=0)
        j_local = int(np.argmax(normsq))  # first maximum -> lowest column index
        j = int(cand[j_local])
        nusq = float(normsq[j_local])
        if normsq.size > 1 and nusq > 0.0:
            second = float(np.max(np.delete(normsq, j_local)))
            if nusq - second <= 1e-12 * nusq:
                flags |= 1
        if t == 0:
            nu0sq = nusq
            if nu0sq == 0.0:
                r = 0
                break
        for thr in ((thr1, thr2) if scheme == SECOND_ORDER_SUPERFINE else (thr1,)):
            if abs(nusq - thr * nu0sq) <= 1e-10 * thr * nu0sq:
                flags |= 2
        if r is None and nusq < thr1 * nu0sq:
            r = t
            if scheme != SECOND_ORDER_SUPERFINE:
                break
        if scheme == SECOND_ORDER_SUPERFINE and nusq < thr2 * nu0sq:
            break
        x = R[t:, j].copy()
        alpha = x[0]
        normx = np.sqrt(nusq)
        v = np.zeros(m)
        if normx == 0.0:
            tau = 0.0
            beta = alpha
            v[t] = 1.0
        else:
            beta = -normx if alpha >= 0.0 else normx
            tau = (beta - alpha) / beta
            v[t:] = x / (alpha - beta)
            v[t] = 1.0
        rest = cand[cand != j]
        if rest.size:
            w = v[t:] @ R[t:, rest]
            R[t:, rest] -= tau * np.outer(v[t:], w)
        R[t, j] = beta
        R[t + 1:, j] = 0.0
        pivoted[j] = True
        Vcols.append(v)
        taus.append(tau)
        pivs.append(j)
    nref = len(taus)
    if r is None:
        r = nref
    V = np.stack(Vcols, axis=1) if nref else np.zeros((m, 0))
    return RRQRResult(r=r, nref=nref, V=V, tau=np.array(taus, dtype=np.float64), R=R,
                      piv=np.array(pivs, dtype=np.int64), flags=flags)


def apply_qt(V: np.ndarray, tau: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Q^T z with Q = H_0 H_1 ... H_{nref-1} (H_0 applied first)."""
    z = np.array(z, dtype=np.float64, copy=True)
    for t in range(tau.size):
        v = V[t:, t]
        z[t:] -= tau[t] * v * (v @ z[t:])
    return z


def apply_q(V: np.ndarray, tau: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Q z (the last reflector applied first)."""
    z = np.array(z, dtype=np.float64, copy=True)
    for t in reversed(range(tau.size)):
        v = V[t:, t]
        z[t:] -= tau[t] * v * (v @ z[t:])
    return z


def explicit_q(V: np.ndarray, tau: np.ndarray) -> np.ndarray:
    """The m x m orthogonal Q = H_0 ... H_{nref-1}."""
    m = V.shape[0]
    Q = np.eye(m)
    for i in range(m):
        Q[:, i] = apply_q(V, tau, Q[:, i])
    return Q


def fine_block(res: RRQRResult, scheme: int) -> np.ndarray:
    """The E-tilde kept in the outer factor by each scheme (Algorithm 1).

    First order: nothing.  Full second order: E = rows r..m-1 of Q^T A_pw.
    Superfine: E_2 = rows r..r2-1 (the rows r2..m-1, E_1, are dropped).
    """
    if scheme == FIRST_ORDER:
        return res.R[res.r:res.r, :]
    if scheme == SECOND_ORDER_FULL:
        return res.R[res.r:, :]
    return res.R[res.r:res.nref, :]
