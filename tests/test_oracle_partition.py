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
