"""Algorithm 2 of the paper (spaND), its preconditioner apply, and PCG.

Test infrastructure only (see ``oracle/__init__``).

The live matrix is kept as a dictionary of dense blocks ``B[(c, d)]`` over the
clusters of the current stage (both orientations, ``B[(d, c)] = B[(c, d)].T``).
Stage ``k = 0 .. ell-1`` runs, in this order (Algorithm 2, §3):

1. *Eliminate interiors* (the clusters of level k, mutually non-adjacent), in
   cluster-id order: ``A_ss = L_s L_s^T``; ``W_s^T = L_s^{-1} A_sw``;
   ``A_ww -= W_s W_s^T`` (block Gaussian elimination, §1).  The elimination
   operator is ``G_s = [[I, 0], [-W_s, I]] diag(L_s^{-1}, I)`` with
   ``W_s = A_ws L_s^{-T}``, which gives ``G_s A G_s^T = diag(I, A_ww - A_ws
   A_ss^{-1} A_sw)`` (the printed G_s lacks the L_s^{-1} factor in its (2,1)
   block; this is the reading that satisfies the displayed identity).
2. If ``skip <= k < ell-1``, *scale interfaces* (eq. prescale, §2.2, with the
   double-sided scaling of §2.3.2): for every interface ``A_pp = Z_p Z_p^T``,
   then every pair ``A_pq <- Z_p^{-1} A_pq Z_q^{-T}`` and ``A_pp <- I``.
3. Same condition: *sparsify interfaces* one at a time in (colour, id) order,
   the colours being a greedy colouring of the interface adjacency, so that
   interfaces of one colour never touch each other's blocks.  For interface p
   with live neighbours w (all live clusters sharing a block with p, in id
   order, already-sparsified ones contributing their coarse variables only):
   Algorithm 1 on ``A_pw`` gives Q, r and ``Q^T A_pw``; p's rows and columns
   become the r coarse rows ``Q_c^T A_pw`` and ``A_cc = I``; the fine
   variables leave the live set.  The outer factor keeps ``E_p`` with
   ``E-tilde = 0`` (first order, eq. trailing-1), ``E`` (full second order,
   eq. trailing-2) or ``E_2`` (superfine, eq. trailing-3).
4. The surviving interfaces are merged into the clusters of stage k+1
   (recursion on the not-yet-eliminated interfaces).

The last stage eliminates the top separator as its only interior (dense
Cholesky).  ``L^{-1}`` is the product of all operators in processing order,
so ``apply`` runs them forward and then their transposes in reverse:
``M r = L^{-T} L^{-1} r``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.linalg import solve_triangular

from . import partition
from .rrqr import (FIRST_ORDER, SECOND_ORDER_FULL, SECOND_ORDER_SUPERFINE,
                   apply_q, apply_qt, fine_block, rrqr)

__all__ = ["FIRST_ORDER", "SECOND_ORDER_FULL", "SECOND_ORDER_SUPERFINE",
           "Factor", "factor", "apply", "pcg", "NotSPDError"]


class NotSPDError(ValueError):
    """A Cholesky pivot was not positive."""


def _chol(a: np.ndarray, what: str) -> np.ndarray:
    if a.shape[0] == 0:
        return np.zeros((0, 0))
    try:
        return np.linalg.cholesky(a)
    except np.linalg.LinAlgError as exc:
        raise NotSPDError(f"Cholesky failed on {what}") from exc


@dataclass
class OpG:  # interior elimination G_s
    slots: np.ndarray
    L: np.ndarray
    WT: np.ndarray  # m_s x |w| = L_s^{-1} A_sw
    wslots: np.ndarray


@dataclass
class OpD:  # interface scaling D_p
    slots: np.ndarray
    Z: np.ndarray


@dataclass
class OpQ:  # change of basis Q_p^T followed by E_p
    slots: np.ndarray  # the m_p positions before sparsification
    V: np.ndarray
    tau: np.ndarray
    r: int
    Et: np.ndarray  # kept fine rows (E-tilde), rows r..r+Et.shape[0]-1 of Q^T A_pw
    wslots: np.ndarray


@dataclass
class Factor:
    n: int
    nlevels: int
    eps: float
    scheme: int
    skip: int
    ops: list = field(default_factory=list)
    # per stage: {cluster key: size at stage start}, {interface key: rank}, colours
    stage_sizes: list = field(default_factory=list)
    stage_ranks: list = field(default_factory=list)
    stage_colours: list = field(default_factory=list)
    stage_flags: list = field(default_factory=list)  # {interface key: near-tie flags}
    stage_keys: list = field(default_factory=list)
    # diagonal prescaling: the factorization is of S A S with S = D^{-1/2},
    # D = diag(A), and M = S M~ S (None: no prescaling)
    scale: np.ndarray | None = None

    def nnz_factor(self) -> int:
        """Stored entries of the factor operators (L_s, W_s, Z_p, Q_p, E-tilde)."""
        tot = 0
        for op in self.ops:
            if isinstance(op, OpG):
                m = op.L.shape[0]
                tot += m * (m + 1) // 2 + op.WT.size
            elif isinstance(op, OpD):
                m = op.Z.shape[0]
                tot += m * (m + 1) // 2
            else:
                tot += op.V.size + op.tau.size + op.Et.size
        return tot


def _blocks_from_csr(A, clusters: partition.StageClusters):
    """Dense blocks of A between the stage-0 clusters (variables in ascending order)."""
    n = A.shape[0]
    cl = np.empty(n, dtype=np.int64)
    pos = np.empty(n, dtype=np.int64)
    for ci, key in enumerate(clusters.keys):
        mem = clusters.members[key]
        cl[mem] = ci
        pos[mem] = np.arange(mem.size)
    coo = A.tocoo()
    ci, cj = cl[coo.row], cl[coo.col]
    B = {}
    order = np.lexsort((cj, ci))
    ci, cj = ci[order], cj[order]
    rr, cc, vv = pos[coo.row][order], pos[coo.col][order], coo.data[order]
    starts = np.nonzero(np.r_[True, (ci[1:] != ci[:-1]) | (cj[1:] != cj[:-1])])[0]
    ends = np.r_[starts[1:], ci.size]
    keys = clusters.keys
    for s, e in zip(starts, ends):
        a, b = keys[ci[s]], keys[cj[s]]
        blk = np.zeros((clusters.members[a].size, clusters.members[b].size))
        np.add.at(blk, (rr[s:e], cc[s:e]), vv[s:e])
        B[(a, b)] = blk
    return B


def factor(A, coords, nlevels: int, eps: float, scheme: int = SECOND_ORDER_FULL,
           skip: int | None = None, prescale: bool = False) -> Factor:
    """spaND factorization (Algorithm 2) of the sparse SPD matrix A (scipy sparse).

    coords None: the multilevel partition is the algebraic one of A's graph
    (``partition.graph_nested_dissection``).  prescale: factor
    D^{-1/2} A D^{-1/2} with D = diag(A), the diagonal prescaling for
    general SPD input; the preconditioner of A is then D^{-1/2} M~ D^{-1/2}."""
    import scipy.sparse as sp

    import spand_inputs

    A = A.tocsr()
    A.sort_indices()
    n = A.shape[0]
    if not (0.0 <= eps <= 1.0):
        raise ValueError("eps must lie in [0, 1]")
    if scheme not in (FIRST_ORDER, SECOND_ORDER_FULL, SECOND_ORDER_SUPERFINE):
        raise ValueError("unknown scheme")
    if skip is None:
        skip = spand_inputs.default_skip(n, nlevels)
    F = Factor(n=n, nlevels=nlevels, eps=eps, scheme=scheme, skip=skip)
    tree = partition.build_tree(coords, nlevels, A.indptr, A.indices)
    if prescale:
        d = A.diagonal()
        if not (d > 0).all():
            raise NotSPDError("a diagonal entry is not positive")
        F.scale = 1.0 / np.sqrt(d)
        S = sp.diags(F.scale)
        A = (S @ A @ S).tocsr()
        A.sort_indices()

    sc0 = partition.stage_clusters(tree, 0)
    B = _blocks_from_csr(A, sc0)
    keys = list(sc0.keys)
    slots = {key: sc0.members[key].copy() for key in keys}  # vector positions of live vars
    verts = {key: sc0.members[key] for key in keys}  # original vertices of each cluster
    level = dict(sc0.level)
    nbrs = {key: set() for key in keys}
    for (a, b) in B:
        if a != b:
            nbrs[a].add(b)

    for k in range(nlevels):
        F.stage_keys.append(list(keys))
        F.stage_sizes.append({key: slots[key].size for key in keys})
        # 1. eliminate interiors
        interiors = [key for key in keys if level[key] == k]
        iset = set(interiors)
        for s in interiors:
            assert not (nbrs[s] & iset), "interiors of a stage must not be adjacent"
        for s in interiors:
            N = sorted(nbrs[s])
            L = _chol(B[(s, s)], f"interior {s}")
            if N:
                Asw = np.hstack([B[(s, q)] for q in N])
                WT = solve_triangular(L, Asw, lower=True) if L.size else np.zeros((0, Asw.shape[1]))
                S = WT.T @ WT
                offs = np.cumsum([0] + [slots[q].size for q in N])
                for a, q in enumerate(N):
                    for b in range(a + 1):
                        rq = N[b]
                        upd = S[offs[a]:offs[a + 1], offs[b]:offs[b + 1]]
                        if (q, rq) in B:
                            B[(q, rq)] = B[(q, rq)] - upd
                        else:
                            B[(q, rq)] = -upd
                            nbrs[q].add(rq)
                            nbrs[rq].add(q)
                        if rq != q:
                            B[(rq, q)] = B[(q, rq)].T.copy()
                wslots = np.concatenate([slots[q] for q in N])
            else:
                WT = np.zeros((slots[s].size, 0))
                wslots = np.zeros(0, dtype=np.int64)
            F.ops.append(OpG(slots=slots[s].copy(), L=L, WT=WT, wslots=wslots))
            for q in N:
                del B[(s, q)]
                del B[(q, s)]
                nbrs[q].discard(s)
            del B[(s, s)]
            del nbrs[s]
        keys = [key for key in keys if key not in iset]

        ranks = {}
        colours = {}
        flags = {}
        if skip <= k < nlevels - 1 and keys:
            # 2. scale interfaces
            Z = {p: _chol(B[(p, p)], f"interface {p}") for p in keys}
            for p in keys:
                F.ops.append(OpD(slots=slots[p].copy(), Z=Z[p]))
            for p in keys:
                for q in nbrs[p]:
                    if q < p:
                        X = B[(p, q)]
                        if Z[p].size and X.size:
                            X = solve_triangular(Z[p], X, lower=True)
                        if Z[q].size and X.size:
                            X = solve_triangular(Z[q], X.T, lower=True).T
                        B[(p, q)] = X
                        B[(q, p)] = X.T.copy()
                B[(p, p)] = np.eye(slots[p].size)
            # 3. sparsify interfaces in (colour, id) order
            colours = partition.greedy_colouring(keys, nbrs)
            for p in sorted(keys, key=lambda c: (colours[c], c)):
                N = sorted(nbrs[p])
                m = slots[p].size
                if N:
                    Apw = np.hstack([B[(p, q)] for q in N])
                    wslots = np.concatenate([slots[q] for q in N])
                else:
                    Apw = np.zeros((m, 0))
                    wslots = np.zeros(0, dtype=np.int64)
                res = rrqr(Apw, eps, scheme)
                r = res.r
                offs = np.cumsum([0] + [slots[q].size for q in N])
                for a, q in enumerate(N):
                    B[(p, q)] = res.R[:r, offs[a]:offs[a + 1]].copy()
                    B[(q, p)] = B[(p, q)].T.copy()
                B[(p, p)] = np.eye(r)
                F.ops.append(OpQ(slots=slots[p].copy(), V=res.V, tau=res.tau, r=r,
                                 Et=fine_block(res, scheme).copy(), wslots=wslots))
                slots[p] = slots[p][:r]
                ranks[p] = r
                flags[p] = res.flags
        F.stage_ranks.append(ranks)
        F.stage_colours.append(colours)
        F.stage_flags.append(flags)

        if k == nlevels - 1:
            assert not keys, "the last stage must eliminate everything"
            break
        # 4. merge into the clusters of stage k+1
        kv_live, kv_rows = partition.tree_cluster_keys(tree, k + 1)
        row_of = {int(v): i for i, v in enumerate(kv_live)}
        parent = {}
        for p in keys:
            parent[p] = tuple(int(t) for t in kv_rows[row_of[int(verts[p][0])]])
        children = {}
        for p in keys:  # keys are in id order, so children end up sorted
            children.setdefault(parent[p], []).append(p)
        new_keys = sorted(children)
        new_slots, new_verts, new_level, offs = {}, {}, {}, {}
        for P in new_keys:
            ch = children[P]
            new_slots[P] = np.concatenate([slots[c] for c in ch])
            new_verts[P] = np.sort(np.concatenate([verts[c] for c in ch]))
            new_level[P] = level[ch[0]]
            o, acc = {}, 0
            for c in ch:
                o[c] = acc
                acc += slots[c].size
            offs[P] = o
        new_B = {}
        new_nbrs = {P: set() for P in new_keys}
        for (a, b), blk in B.items():
            PA, PB = parent[a], parent[b]
            if (PA, PB) not in new_B:
                new_B[(PA, PB)] = np.zeros((new_slots[PA].size, new_slots[PB].size))
                if PA != PB:
                    new_nbrs[PA].add(PB)
            oa, ob = offs[PA][a], offs[PB][b]
            new_B[(PA, PB)][oa:oa + blk.shape[0], ob:ob + blk.shape[1]] = blk
        for P in new_keys:
            if (P, P) not in new_B:
                new_B[(P, P)] = np.zeros((new_slots[P].size,) * 2)
        B, keys, slots, verts, level, nbrs = new_B, new_keys, new_slots, new_verts, new_level, new_nbrs
    return F


def _forward(F: Factor, z: np.ndarray) -> None:
    """z <- L^{-1} z, operators in processing order."""
    for op in F.ops:
        if isinstance(op, OpG):
            zs = solve_triangular(op.L, z[op.slots], lower=True) if op.L.size else z[op.slots]
            z[op.slots] = zs
            if op.wslots.size:
                z[op.wslots] -= op.WT.T @ zs
        elif isinstance(op, OpD):
            if op.Z.size:
                z[op.slots] = solve_triangular(op.Z, z[op.slots], lower=True)
        else:
            zp = apply_qt(op.V, op.tau, z[op.slots])
            z[op.slots] = zp
            ne = op.Et.shape[0]
            if ne and op.wslots.size:
                z[op.wslots] -= op.Et.T @ zp[op.r:op.r + ne]


def _backward(F: Factor, z: np.ndarray) -> None:
    """z <- L^{-T} z, transposed operators in reverse order."""
    for op in reversed(F.ops):
        if isinstance(op, OpG):
            zs = z[op.slots]
            if op.wslots.size:
                zs = zs - op.WT @ z[op.wslots]
            if op.L.size:
                zs = solve_triangular(op.L, zs, lower=True, trans="T")
            z[op.slots] = zs
        elif isinstance(op, OpD):
            if op.Z.size:
                z[op.slots] = solve_triangular(op.Z, z[op.slots], lower=True, trans="T")
        else:
            zp = z[op.slots].copy()
            ne = op.Et.shape[0]
            if ne and op.wslots.size:
                zp[op.r:op.r + ne] -= op.Et @ z[op.wslots]
            z[op.slots] = apply_q(op.V, op.tau, zp)


def apply(F: Factor, r: np.ndarray) -> np.ndarray:
    """The preconditioner M r = L^{-T} L^{-1} r (Algorithm 2 caption); with
    prescaling S L^{-T} L^{-1} S r."""
    z = np.array(r, dtype=np.float64, copy=True)
    if F.scale is not None:
        z *= F.scale
    _forward(F, z)
    _backward(F, z)
    if F.scale is not None:
        z *= F.scale
    return z


def apply_linv(F: Factor, r: np.ndarray) -> np.ndarray:
    """L^{-1} r alone (used to form the preconditioned operator in tests)."""
    z = np.array(r, dtype=np.float64, copy=True)
    _forward(F, z)
    return z


def apply_lt_inv(F: Factor, r: np.ndarray) -> np.ndarray:
    """L^{-T} r alone."""
    z = np.array(r, dtype=np.float64, copy=True)
    _backward(F, z)
    return z


@dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    relres: float  # true relative residual ||b - A x|| / ||b|| at exit
    history: list  # ||r_k|| / ||b|| of the recursive residual, k = 0..iters
    residuals: list | None = None  # the recursive residual vectors if requested


def pcg(matvec, precond, b: np.ndarray, tol: float, maxit: int = 500,
        true_every: int = 50, max_restarts: int = 2, keep_residuals: bool = False) -> PCGResult:
    """Preconditioned CG (Hestenes-Stiefel) with x0 = 0 (§4).

    Stops when the recursive residual satisfies ||r_k|| / ||b|| < tol.  Every
    ``true_every`` iterations the recursive residual is replaced by the true
    one b - A x.  At exit the true residual is computed; if it is not below
    tol, CG restarts from the current x (at most ``max_restarts`` times).
    ``iters`` counts products with A inside the CG loop.
    """
    b = np.asarray(b, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    x = np.zeros_like(b)
    if bnorm == 0.0:
        return PCGResult(x=x, iters=0, relres=0.0, history=[0.0])
    r = b.copy()
    hist = [1.0]
    resid = [r.copy()] if keep_residuals else None
    it = 0
    restarts = 0
    while True:
        z = precond(r)
        p = z.copy()
        rz = float(r @ z)
        while it < maxit and np.linalg.norm(r) / bnorm >= tol:
            q = matvec(p)
            alpha = rz / float(p @ q)
            x = x + alpha * p
            r = r - alpha * q
            it += 1
            if it % true_every == 0:
                r = b - matvec(x)
            hist.append(float(np.linalg.norm(r)) / bnorm)
            if keep_residuals:
                resid.append(r.copy())
            if hist[-1] < tol:
                break
            z = precond(r)
            rz_new = float(r @ z)
            beta = rz_new / rz
            p = z + beta * p
            rz = rz_new
        rtrue = b - matvec(x)
        relres = float(np.linalg.norm(rtrue)) / bnorm
        if relres < tol or it >= maxit or restarts >= max_restarts:
            return PCGResult(x=x, iters=it, relres=relres, history=hist, residuals=resid)
        restarts += 1
        r = rtrue


def solve(A, coords, b, nlevels: int, eps: float, scheme: int = SECOND_ORDER_FULL,
          skip: int | None = None, tol: float = 1e-12, maxit: int = 500,
          prescale: bool = False):
    """Factor A with spaND and solve A x = b by PCG; returns (Factor, PCGResult)."""
    A = A.tocsr()
    F = factor(A, coords, nlevels, eps, scheme, skip, prescale=prescale)
    res = pcg(lambda v: A @ v, lambda v: apply(F, v), b, tol, maxit)
    return F, res
