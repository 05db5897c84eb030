"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only *generates* problems: sparse SPD matrices on grids (with their
grid coordinates) and right-hand sides.  It contains none of the spaND
arithmetic, so both the CPU oracle and the CUDA path can draw identical inputs
from it without sharing any part of the method.

Problem families (paper §4.1 and the grid problems the method targets):

* ``laplacian_2d(d)`` -- 5-point Dirichlet Laplacian on a d x d grid, diagonal 4
  and off-diagonal -1 (no h^2 factor).  This is the scaling for which the paper
  states the eigenpairs ``lambda_p = 8 sin^2(p pi / (2(d+1)))`` (§4.1.1).
* ``laplacian_3d(d)`` -- 7-point Dirichlet Laplacian, diagonal 6, off -1.
* ``diffusion_3d(d, seed, lo, hi)`` -- 7-point finite-volume diffusion with an
  i.i.d. per-cell coefficient ``a = 10**U(lo, hi)``; a face between two cells
  carries the harmonic mean ``2 a_i a_j / (a_i + a_j)``, a Dirichlet boundary
  face carries the cell's own ``a``.  With ``a == 1`` this is ``laplacian_3d``.
* ``high_contrast_2d(d, rho, seed)`` -- the paper's 2D high-contrast field
  (§4.1): uniform(0,1) cells, Gaussian smoothing with sigma = 2, quantised to
  rho / 1/rho at 0.5, harmonic face means.

Vertex numbering is C-order in the coordinates: ``v = x + nx*(y + ny*z)``.
Every matrix is returned as a full symmetric CSR (both triangles, column
indices sorted within a row, int32 indices, float64 values) together with an
``(n, dim)`` float64 coordinate array.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Problem:
    """A sparse SPD matrix in CSR form plus the grid coordinates of its rows."""

    name: str
    n: int
    rowptr: np.ndarray  # int32, (n+1,)
    colind: np.ndarray  # int32, (nnz,)
    val: np.ndarray  # float64, (nnz,)
    coords: np.ndarray  # float64, (n, dim)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    @property
    def dim(self) -> int:
        return int(self.coords.shape[1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.colind, self.rowptr), shape=(self.n, self.n))


def _grid_coords(shape) -> np.ndarray:
    """Coordinates (x, y[, z]) of every vertex, vertex index = x + nx*(y + ny*z)."""
    axes = [np.arange(s, dtype=np.float64) for s in shape]
    mesh = np.meshgrid(*axes, indexing="ij")  # mesh[k][x, y, z] = coordinate k
    # C-order over (z, y, x) so that x varies fastest.
    cols = [m.transpose(tuple(range(len(shape)))[::-1]).reshape(-1) for m in mesh]
    return np.stack(cols, axis=1)


def _assemble(shape, face_coeff, diag_extra, name) -> Problem:
    """Assemble a finite-volume operator from per-face coefficients.

    ``face_coeff[k]`` is an array over the cells of the grid giving the
    coefficient of the face between cell c and its +e_k neighbour (ignored on
    the last layer); ``diag_extra`` adds the Dirichlet boundary faces.
    """
    dim = len(shape)
    n = int(np.prod(shape))
    idx = np.arange(n).reshape(shape[::-1])  # idx[z, y, x]
    rows, cols, vals = [], [], []
    diag = diag_extra.reshape(-1).copy()
    for k in range(dim):
        ax = dim - 1 - k  # array axis of coordinate k in idx[z, y, x]
        lo = [slice(None)] * dim
        hi = [slice(None)] * dim
        lo[ax] = slice(0, shape[k] - 1)
        hi[ax] = slice(1, shape[k])
        a = face_coeff[k][tuple(lo)].reshape(-1)
        i = idx[tuple(lo)].reshape(-1)
        j = idx[tuple(hi)].reshape(-1)
        rows += [i, j]
        cols += [j, i]
        vals += [-a, -a]
        np.add.at(diag, i, a)
        np.add.at(diag, j, a)
    rows.append(np.arange(n))
    cols.append(np.arange(n))
    vals.append(diag)
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return Problem(
        name=name,
        n=n,
        rowptr=rowptr.astype(np.int32),
        colind=c.astype(np.int32),
        val=v.astype(np.float64),
        coords=_grid_coords(shape),
    )


def _coefficient_problem(shape, a_cell, name) -> Problem:
    """Finite-volume operator with per-cell coefficients and harmonic face means."""
    dim = len(shape)
    a = a_cell.reshape(shape[::-1])
    faces = []
    boundary = np.zeros_like(a)
    for k in range(dim):
        ax = dim - 1 - k
        nxt = np.roll(a, -1, axis=ax)
        faces.append(2.0 * a * nxt / (a + nxt))
        # Dirichlet faces on both ends of axis k use the cell's own coefficient.
        first = [slice(None)] * dim
        last = [slice(None)] * dim
        first[ax] = 0
        last[ax] = shape[k] - 1
        boundary[tuple(first)] += a[tuple(first)]
        boundary[tuple(last)] += a[tuple(last)]
    return _assemble(shape, faces, boundary, name)


def laplacian_2d(d: int) -> Problem:
    """5-point Dirichlet Laplacian on a d x d grid (diag 4, off -1)."""
    return _coefficient_problem((d, d), np.ones(d * d), f"laplacian_2d_{d}")


def laplacian_3d(d: int) -> Problem:
    """7-point Dirichlet Laplacian on a d^3 grid (diag 6, off -1)."""
    return _coefficient_problem((d, d, d), np.ones(d**3), f"laplacian_3d_{d}")


def laplacian_grid(shape) -> Problem:
    """Constant-coefficient Dirichlet Laplacian on a box grid of any shape."""
    shape = tuple(int(s) for s in shape)
    return _coefficient_problem(shape, np.ones(int(np.prod(shape))), "laplacian_" + "x".join(map(str, shape)))


def diffusion_3d(d: int, seed: int = 0, lo: float = -3.0, hi: float = 3.0) -> Problem:
    """7-point FV diffusion on d^3 with a = 10**U(lo, hi) per cell (seeded)."""
    rng = np.random.default_rng(seed)
    a = 10.0 ** rng.uniform(lo, hi, size=d**3)
    return _coefficient_problem((d, d, d), a, f"diffusion_3d_{d}_s{seed}")


def diffusion_grid(shape, seed: int = 0, lo: float = -3.0, hi: float = 3.0) -> Problem:
    """FV diffusion on a box grid of any shape with a = 10**U(lo, hi) per cell."""
    shape = tuple(int(s) for s in shape)
    rng = np.random.default_rng(seed)
    a = 10.0 ** rng.uniform(lo, hi, size=int(np.prod(shape)))
    return _coefficient_problem(shape, a, "diffusion_" + "x".join(map(str, shape)) + f"_s{seed}")


def high_contrast_2d(d: int, rho: float, seed: int = 0) -> Problem:
    """The paper's 2D high-contrast field (§4.1): smoothed uniform field quantised to rho^{+-1}."""
    from scipy.ndimage import gaussian_filter

    rng = np.random.default_rng(seed)
    ahat = rng.uniform(0.0, 1.0, size=(d, d))
    ahat = gaussian_filter(ahat, sigma=2.0, mode="reflect", truncate=4.0)
    a = np.where(ahat >= 0.5, rho, 1.0 / rho)
    return _coefficient_problem((d, d), a.reshape(-1), f"high_contrast_2d_{d}_rho{rho:g}_s{seed}")


def rhs_uniform(n: int, seed: int = 0, nrhs: int = 1) -> np.ndarray:
    """Right-hand side(s) with i.i.d. U[-1, 1] entries; shape (n,) or (nrhs, n)."""
    rng = np.random.default_rng(seed)
    b = rng.uniform(-1.0, 1.0, size=(nrhs, n))
    return b[0] if nrhs == 1 else b


def rhs_normal(n: int, seed: int = 0, nrhs: int = 1) -> np.ndarray:
    """Right-hand side(s) with i.i.d. N(0, 1) entries; shape (n,) or (nrhs, n)."""
    rng = np.random.default_rng(seed)
    b = rng.standard_normal(size=(nrhs, n))
    return b[0] if nrhs == 1 else b


def default_skip(n: int, nlevels: int) -> int:
    """Number of leading levels without scaling/sparsification.

    The paper skips the first four levels when the leaves hold about 25
    unknowns (ell = round(log2(n/25)), §4).  For other leaf sizes the same
    interface size is reached correspondingly earlier or later:
    skip = clamp(4 - round(log2(leaf/25)), 0, ell-2) with leaf = n / 2^(ell-1).
    """
    leaf = n / float(2 ** (nlevels - 1))
    s = 4 - int(np.round(np.log2(leaf / 25.0)))
    return int(min(max(s, 0), max(nlevels - 2, 0)))


# Named workloads: (problem factory, nlevels, eps, rhs factory).
WORKLOADS = {
    "poisson2d_64": dict(problem=lambda: laplacian_2d(64), nlevels=6, eps=1e-2,
                         rhs=lambda n: rhs_uniform(n, seed=0)),
    "poisson3d_64": dict(problem=lambda: laplacian_3d(64), nlevels=12, eps=1e-2,
                         rhs=lambda n: rhs_normal(n, seed=0)),
    "diffusion3d_128": dict(problem=lambda: diffusion_3d(128, seed=0), nlevels=15, eps=1e-2,
                            rhs=lambda n: rhs_normal(n, seed=1)),
}


def paper_nlevels(n: int) -> int:
    """The paper's depth rule for leaves of about 25 unknowns: round(log2(n / 25)) (§4)."""
    return max(2, int(np.round(np.log2(n / 25.0))))


def batch_workload(count: int = 64, lo: float = -2.0, hi: float = 2.0):
    """Independent SPD problems of uneven sizes: even i a 2D 5-point FV grid with
    side 128 .. 512, odd i a 3D 7-point FV grid with side 24 .. 48 (sides spread
    evenly over the problems of each kind), coefficients a = 10**U(lo, hi) per
    cell from seed i, RHS N(0, 1) from seed 1000 + i, depth by the paper's rule.

    Returns a list of (problem, nlevels, rhs)."""
    return [batch_problem(i, count, lo, hi) for i in range(count)]


def batch_problem(i: int, count: int = 64, lo: float = -2.0, hi: float = 2.0):
    """Problem i of batch_workload(count, lo, hi): (problem, nlevels, rhs)."""
    n2 = (count + 1) // 2
    n3 = count // 2
    j = i // 2
    if i % 2 == 0:
        d = 128 + int(round(384 * j / max(n2 - 1, 1)))
        prob = diffusion_grid((d, d), seed=i, lo=lo, hi=hi)
    else:
        d = 24 + int(round(24 * j / max(n3 - 1, 1)))
        prob = diffusion_grid((d, d, d), seed=i, lo=lo, hi=hi)
    return prob, paper_nlevels(prob.n), rhs_normal(prob.n, seed=1000 + i)


def serve_workload(requests: int = 120, rate: float = 20.0, new_problems: int = 12,
                   p_new: float = 0.3, seed: int = 0):
    """A seeded serving trace: a resident 3D FV diffusion problem on 96^3 with
    a = 10**U(-3, 3) (seed 0), new 3D 7-point FV problems of n = 16k .. 500k
    (sides 25 .. 79 spread evenly, a = 10**U(-3, 3) from seeds 1, 2, ...), and
    requests arriving as a Poisson process of the given rate (per second); a
    request targets a new problem with probability p_new (else the resident
    one) and carries 1 .. 32 right-hand sides N(0, 1).

    Returns (problems, trace): problems = [(problem, nlevels)] with the
    resident one first; trace = [(arrival time s, problem index, nrhs, rhs seed)]."""
    rng = np.random.default_rng(seed)
    probs = [(diffusion_3d(96, seed=0), paper_nlevels(96 ** 3))]
    for i in range(new_problems):
        d = 25 + int(round(54 * i / max(new_problems - 1, 1)))
        probs.append((diffusion_3d(d, seed=1 + i), paper_nlevels(d ** 3)))
    t = 0.0
    trace = []
    for k in range(requests):
        t += rng.exponential(1.0 / rate)
        pi = 0 if rng.uniform() >= p_new else 1 + int(rng.integers(new_problems))
        trace.append((t, pi, int(rng.integers(1, 33)), 5000 + k))
    return probs, trace
