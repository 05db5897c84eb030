"""Pins for the oracle's multilevel partition (paper §3, spaND partitioning).

Hand-derived golden clusters on tiny grids plus the structural invariants the
algorithm relies on: every live vertex in exactly one cluster, stage k+1
clusters are unions of stage k clusters, interiors of a stage never touch.
"""
import os

import numpy as np
import pytest

import spand_inputs as si
from oracle import partition as P


def _read_golden(path):
    stages = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("stage"):
            stages.append([])
            continue
        lev, verts = line.split(":")
        stages[-1].append((int(lev), [int(v) for v in verts.split()]))
    return stages


@pytest.mark.parametrize("fname,shape,ell", [
    ("partition_2d_8x8_l3.txt", (8, 8), 3),
    ("partition_3d_4x4x4_l3.txt", (4, 4, 4), 3),
])
def test_golden_partition(golden_dir, fname, shape, ell):
    want = _read_golden(os.path.join(golden_dir, fname))
    prob = si.laplacian_grid(shape)
    tree = P.nested_dissection(prob.coords, ell)
    assert len(want) == ell
    for k in range(ell):
        sc = P.stage_clusters(tree, k)
        got = [(sc.level[key], sc.members[key].tolist()) for key in sc.keys]
        assert got == want[k], f"stage {k}"


@pytest.mark.parametrize("shape,ell", [((32, 32), 5), ((16, 16, 16), 7), ((12, 10, 9), 5)])
def test_partition_invariants(shape, ell):
    prob = si.laplacian_grid(shape)
    tree = P.nested_dissection(prob.coords, ell)
    A = prob.to_scipy().tocoo()
    prev = None
    for k in range(ell):
        sc = P.stage_clusters(tree, k)
        live = np.nonzero(tree.level_of >= k)[0]
        allv = np.concatenate([sc.members[key] for key in sc.keys])
        assert np.array_equal(np.sort(allv), live), "each live vertex in exactly one cluster"
        cl = np.full(prob.n, -1)
        for i, key in enumerate(sc.keys):
            cl[sc.members[key]] = i
        # interiors are whole level-k separators (or leaves) and pairwise non-adjacent in A
        interiors = [i for i, key in enumerate(sc.keys) if sc.level[key] == k]
        for i in interiors:
            node = sc.keys[i][0]
            assert set(sc.members[sc.keys[i]]) == set(np.nonzero(tree.node_of == node)[0])
        isint = np.zeros(len(sc.keys), dtype=bool)
        isint[interiors] = True
        mask = (cl[A.row] >= 0) & (cl[A.col] >= 0)
        ci, cj = cl[A.row[mask]], cl[A.col[mask]]
        assert not np.any(isint[ci] & isint[cj] & (ci != cj))
        if prev is not None:
            # every surviving stage-(k-1) cluster lies inside one stage-k cluster
            for key, mem in prev.members.items():
                if prev.level[key] == k - 1:
                    continue
                ids = set(cl[mem].tolist())
                assert len(ids) == 1 and -1 not in ids
        prev = sc


def test_cut_values_follow_distinct_coordinates():
    # [0, 64) -> 32 at the root; the upper child [33, 64) holds 31 values -> 33 + 15 = 48
    prob = si.laplacian_grid((64, 4))
    tree = P.nested_dissection(prob.coords, 4)
    assert tree.cut_val[0] == 32.0 and tree.cut_dim[0] == 0
    assert tree.cut_dim[1] == 1 and tree.cut_dim[2] == 1
    assert tree.cut_val[5] == 48.0 and tree.cut_val[3] == 16.0


def test_empty_box_rejected():
    prob = si.laplacian_grid((4, 4))
    with pytest.raises(ValueError):
        P.nested_dissection(prob.coords, 5)


def test_greedy_colouring_is_proper():
    prob = si.laplacian_grid((16, 16))
    adj = {}
    A = prob.to_scipy().tocoo()
    for i, j in zip(A.row, A.col):
        if i != j:
            adj.setdefault(int(i), set()).add(int(j))
    col = P.greedy_colouring(list(range(prob.n)), adj)
    assert all(col[i] != col[j] for i in adj for j in adj[i])
    assert col[0] == 0 and col[1] == 1


# ---- algebraic partition (no coordinates) ----

def _path_graph(n):
    rows, cols = [], []
    for i in range(n):
        for j in (i - 1, i, i + 1):
            if 0 <= j < n:
                rows.append(i)
                cols.append(j)
    rowptr = np.searchsorted(np.array(rows), np.arange(n + 1)).astype(np.int32)
    return rowptr, np.array(cols, dtype=np.int32)


def test_golden_graph_partition(golden_dir):
    want = _read_golden(os.path.join(golden_dir, "partition_graph_path7_l3.txt"))
    rowptr, colind = _path_graph(7)
    tree = P.graph_nested_dissection(rowptr, colind, 3)
    assert list(tree.node_of) == [6, 2, 5, 0, 4, 1, 3]
    assert tree.reach[3] == (4, 5) and tree.reach[5] == (3, 4) and tree.reach[1] == (5, 6)
    for k in range(3):
        sc = P.stage_clusters(tree, k)
        got = [(sc.level[key], sorted(int(v) for v in sc.members[key])) for key in sc.keys]
        assert got == [(lv, sorted(vs)) for lv, vs in want[k]], (k, got)


def _permuted(prob, seed):
    """The same matrix with its vertices relabelled at random (coordinates dropped)."""
    import scipy.sparse as sp
    perm = np.random.default_rng(seed).permutation(prob.n)
    A = prob.to_scipy()[perm][:, perm].tocsr()
    A.sort_indices()
    return A


@pytest.mark.parametrize("make,ell,seed", [
    (lambda: si.laplacian_2d(20), 5, 0),
    (lambda: si.laplacian_grid((9, 7, 6)), 5, 1),
    (lambda: si.diffusion_grid((30, 11), seed=2), 6, 2),
])
def test_graph_partition_invariants(make, ell, seed):
    A = _permuted(make(), seed)
    rowptr, colind = A.indptr, A.indices
    tree = P.graph_nested_dissection(rowptr, colind, ell)
    n = A.shape[0]
    assert (tree.node_of >= 0).all() and (tree.level_of >= 0).all()
    # separators separate: no edge joins the two children's subtrees of any node
    dmax = ell - 1

    def under(i, node):
        while P.node_depth(i) > P.node_depth(node):
            i = (i - 1) // 2
        return i == node
    for node in range(2 ** dmax - 1):
        lo, hi = 2 * node + 1, 2 * node + 2
        in_lo = np.array([under(int(x), lo) for x in tree.node_of])
        in_hi = np.array([under(int(x), hi) for x in tree.node_of])
        for v in np.nonzero(in_lo)[0]:
            assert not in_hi[colind[rowptr[v]:rowptr[v + 1]]].any()
    # clusters: each live vertex once; stage k+1 clusters are unions of stage k ones;
    # interiors of a stage are never adjacent
    for k in range(ell):
        sc = P.stage_clusters(tree, k)
        cl = np.full(n, -1)
        for ci, key in enumerate(sc.keys):
            assert (cl[sc.members[key]] == -1).all()
            cl[sc.members[key]] = ci
        assert ((cl >= 0) == (tree.level_of >= k)).all()
        inter = np.array([sc.level[key] == k for key in sc.keys])
        for v in np.nonzero((cl >= 0) & inter[np.maximum(cl, 0)])[0]:
            nb = colind[rowptr[v]:rowptr[v + 1]]
            nb = nb[cl[nb] >= 0]
            assert (~inter[cl[nb]] | (cl[nb] == cl[v])).all()
        if k + 1 < ell:
            nx = P.stage_clusters(tree, k + 1)
            cl1 = np.full(n, -1)
            for ci, key in enumerate(nx.keys):
                cl1[nx.members[key]] = ci
            for key in sc.keys:
                if sc.level[key] > k:
                    assert np.unique(cl1[sc.members[key]]).size == 1
