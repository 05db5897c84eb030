"""C-ABI checks that need no GPU.

* libspand.so loads and exports every function declared in include/spand.h;
* the host-only symbolic phase (spand_analyze) reproduces the oracle's
  multilevel partition bit for bit (cluster of every vertex at every stage);
* malformed input is rejected with SPAND_EINVAL.
"""
import os
import re

import numpy as np
import pytest

import spand_inputs as si
from oracle import partition as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    from paper_2007_00789_gb300 import spand as S
    if not os.path.exists(S.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return S


def test_exports_every_declared_symbol():
    S = _lib()
    L = S.load_library()
    header = open(os.path.join(ROOT, "include", "spand.h")).read()
    declared = set(re.findall(r"\b(spand_[a-z_]+)\s*\(", header))
    assert declared, "no declarations found"
    assert declared == set(S.EXPORTS)
    for name in declared:
        assert hasattr(L, name), name
    assert os.path.dirname(os.path.abspath(L._name)) == os.path.join(ROOT, "paper_2007_00789_gb300")


@pytest.mark.parametrize("make,ell", [
    (lambda: si.laplacian_2d(64), 6),
    (lambda: si.laplacian_3d(16), 7),
    (lambda: si.diffusion_grid((12, 10, 9), seed=1), 5),
    (lambda: si.laplacian_grid((9, 7)), 4),
    (lambda: si.laplacian_grid((5,)), 2),
    (lambda: si.laplacian_2d(8), 1),
    # large enough for the analysis' parallel pieces (bisection of the first
    # boxes, the stage-0 map over several vertex ranges)
    (lambda: si.laplacian_3d(52), 10),
    (lambda: si.laplacian_grid((400, 380)), 12),
])
def test_partition_matches_oracle(make, ell):
    S = _lib()
    prob = make()
    h = S.Spand.from_problem(prob, ell, 0.1, 1)
    tree = P.nested_dissection(prob.coords, ell)
    for k in range(ell):
        sc = P.stage_clusters(tree, k)
        want = np.full(prob.n, -1, dtype=np.int64)
        for i, key in enumerate(sc.keys):
            want[sc.members[key]] = i
        assert h.num_clusters(k) == len(sc.keys)
        assert np.array_equal(h.cluster_map(k), want), f"stage {k}"
    h.close()


def test_rejects_bad_input():
    S = _lib()
    prob = si.laplacian_2d(8)
    with pytest.raises(S.SpandError) as e:
        S.Spand.from_problem(prob, 3, 1.5, 1)
    assert e.value.code == S.SPAND_EINVAL
    with pytest.raises(S.SpandError):
        S.Spand.from_problem(prob, 3, 0.1, 7)
    with pytest.raises(S.SpandError):
        S.Spand.from_problem(prob, 0, 0.1, 1)
    with pytest.raises(S.SpandError):  # empty nested-dissection box
        S.Spand.from_problem(prob, 6, 0.1, 1)
    col = prob.colind.copy()
    col[3], col[4] = col[4], col[3]  # unsorted row
    with pytest.raises(S.SpandError):
        S.Spand(prob.rowptr, col, prob.val, prob.coords, 3, 0.1, 1)
    A = prob.to_scipy().tolil()
    A[0, 9] = -0.5  # asymmetric pattern
    A = A.tocsr()
    A.sort_indices()
    with pytest.raises(S.SpandError):
        S.Spand(A.indptr, A.indices, A.data, prob.coords, 3, 0.1, 1)


@pytest.mark.parametrize("make,ell", [
    (lambda: si.laplacian_grid((2,)), 2),
    (lambda: si.laplacian_grid((6, 5)), 6),
    (lambda: si.laplacian_2d(8), 6),
])
def test_too_many_levels_rejected_like_the_oracle(make, ell):
    """More levels than the grid can be cut into leave an empty box in the
    nested dissection: the library refuses the analysis (EINVAL) where the
    oracle refuses the partition."""
    from oracle import spand as OS
    S = _lib()
    prob = make()
    with pytest.raises(ValueError):
        OS.factor(prob.to_scipy(), prob.coords, ell, 1e-2, 1)
    with pytest.raises(S.SpandError) as e:
        S.Spand.from_problem(prob, ell, 1e-2, 1)
    assert e.value.code == S.SPAND_EINVAL
    assert "empty nested-dissection box" in str(e.value)


def test_factor_before_gpu_is_refused_cleanly():
    """Without a GPU the numeric calls return an error code, never crash."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    S = _lib()
    h = S.Spand.from_problem(si.laplacian_2d(8), 3, 0.1, 1)
    with pytest.raises(S.SpandError) as e:
        h.factor(stream=0)
    assert e.value.code in (S.SPAND_ECUDA, S.SPAND_ENOMEM)
    assert h.info()["n"] == 64


def test_batch_arguments_checked_without_gpu():
    """Batch creation is host-only: bad member lists are refused with EINVAL."""
    from paper_2007_00789_gb300 import spand as S
    p = si.laplacian_2d(8)
    a = S.Spand.from_problem(p, 3, 1e-2, 1)
    b = S.Spand.from_problem(p, 3, 1e-2, 1, precision=1)
    with pytest.raises(S.SpandError) as e:
        S.SpandBatch([a, a])
    assert e.value.code == S.SPAND_EINVAL
    with pytest.raises(S.SpandError) as e:
        S.SpandBatch([a, b])
    assert e.value.code == S.SPAND_EINVAL
    batch = S.SpandBatch([a])
    batch.close()
    a.close()
    b.close()


@pytest.mark.parametrize("make,ell,seed", [
    (lambda: si.laplacian_2d(20), 5, 1),
    (lambda: si.laplacian_grid((9, 7, 6)), 5, 2),
    (lambda: si.diffusion_grid((30, 11), seed=2), 6, 3),
    # large enough for the parallel pieces of the analysis (n = 140,608)
    (lambda: si.laplacian_3d(52), 8, 4),
])
def test_algebraic_partition_matches_oracle(make, ell, seed):
    """Without coordinates the library partitions A's graph; cluster maps equal the oracle's."""
    from paper_2007_00789_gb300 import spand as S
    prob = make()
    perm = np.random.default_rng(seed).permutation(prob.n)
    A = prob.to_scipy()[perm][:, perm].tocsr()
    A.sort_indices()
    h = S.Spand(A.indptr, A.indices, A.data, None, ell, 1e-2, 1)
    tree = P.graph_nested_dissection(A.indptr, A.indices, ell)
    for k in range(ell):
        sc = P.stage_clusters(tree, k)
        want = np.full(prob.n, -1)
        for ci, key in enumerate(sc.keys):
            want[sc.members[key]] = ci
        assert np.array_equal(h.cluster_map(k), want), k
    h.close()


def test_prescale_rejects_nonpositive_diagonal():
    from paper_2007_00789_gb300 import spand as S
    p = si.laplacian_2d(8)
    val = p.val.copy()
    val[np.nonzero(p.colind == 0)[0][0]] = 0.0
    with pytest.raises(S.SpandError) as e:
        S.Spand(p.rowptr, p.colind, val, p.coords, 3, 1e-2, 1, prescale=True)
    assert e.value.code == S.SPAND_ENOTSPD


def test_concurrent_analyses_match_sequential():
    """Analyses on several host threads at once (the library's kept worker
    threads serve one loop at a time; the others run on threads of their own)
    give the same partition as one at a time."""
    import threading
    S = _lib()
    probs = [(si.laplacian_3d(40), 9), (si.laplacian_grid((300, 280)), 11),
             (si.diffusion_grid((36, 30, 28), seed=3), 9), (si.laplacian_3d(24), 7)]
    # the algebraic partition as well: no coordinates
    probs.append((si.laplacian_3d(30), 7))

    def maps(prob, ell, algebraic):
        coords = None if algebraic else prob.coords
        h = S.Spand(prob.rowptr, prob.colind, prob.val, coords, ell, 0.1, 1)
        out = [h.cluster_map(k) for k in range(ell)]
        h.close()
        return out

    jobs = [(p, ell, i == len(probs) - 1) for i, (p, ell) in enumerate(probs)]
    want = [maps(*j) for j in jobs]
    got = [None] * len(jobs)
    errors = []

    def run(i):
        try:
            for _ in range(2):
                got[i] = maps(*jobs[i])
        except Exception as e:  # reported below, on the test's thread
            errors.append(e)

    threads = [threading.Thread(target=run, args=(i,)) for i in range(len(jobs))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for w, g in zip(want, got):
        assert len(w) == len(g)
        for a, b in zip(w, g):
            assert np.array_equal(a, b)


def test_csr_defects_reported_in_row_order():
    """The CSR check reports the first defect in row order (rows are checked in
    parallel), and never reads entries past a row pointer beyond nnz."""
    S = _lib()
    prob = si.laplacian_3d(24)  # n = 13824: several parallel chunks of rows
    rp, ci, val = prob.rowptr.copy(), prob.colind.copy(), prob.val.copy()

    def err(rp_, ci_, val_=None):
        with pytest.raises(S.SpandError) as e:
            S.Spand(rp_, ci_, val if val_ is None else val_, prob.coords, 5, 0.1, 1)
        assert e.value.code == S.SPAND_EINVAL
        return str(e.value)

    def without_entry(row, col):
        e = rp[row] + int(np.nonzero(ci[rp[row]:rp[row + 1]] == col)[0][0])
        rp2 = rp.copy()
        rp2[row + 1:] -= 1
        return rp2, np.delete(ci, e), np.delete(val, e)

    # missing diagonal late and early: the early row is named
    r2, c2, v2 = without_entry(9000, 9000)
    assert "missing diagonal entry in row 9000" in err(r2, c2, v2)
    r2, c2, v2 = without_entry(9000, 9000)
    c2[rp[20] + 1], c2[rp[20] + 2] = c2[rp[20] + 2], c2[rp[20] + 1]  # row 20 unsorted
    assert "columns not strictly ascending" in err(r2, c2, v2)
    c3 = ci.copy()
    c3[rp[5000 + 1] - 1] = prob.n  # out of range in row 5000
    assert "column index out of range" in err(rp, c3)
    # a row pointer past nnz, then a decrease: reported, not read
    r4 = rp.copy()
    r4[100] = len(ci) + 1000
    assert "rowptr not monotone" in err(r4, ci)
    # entry defects in rows before a bad row pointer come first
    r5 = r4.copy()
    c5 = ci.copy()
    c5[rp[10]], c5[rp[10] + 1] = c5[rp[10] + 1], c5[rp[10]]
    assert "columns not strictly ascending" in err(r5, c5)
    # an entry without its mirror
    A = prob.to_scipy().tolil()
    A[12000, 3] = -0.5
    A = A.tocsr()
    A.sort_indices()
    with pytest.raises(S.SpandError) as e:
        S.Spand(A.indptr, A.indices, A.data, prob.coords, 5, 0.1, 1)
    assert "pattern is not symmetric" in str(e.value)


def test_analysis_in_a_forked_child():
    """A child forked after the library's host threads exist (which it does not
    inherit) still analyses: it starts host threads of its own."""
    import signal
    import time
    import warnings
    S = _lib()
    prob = si.laplacian_3d(40)  # large enough for parallel loops
    h = S.Spand.from_problem(prob, 9, 0.1, 1)
    want = h.cluster_map(3)
    h.close()
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", DeprecationWarning)  # fork of a threaded process
        pid = os.fork()
    if pid == 0:
        code = 1
        try:
            signal.alarm(60)
            hc = S.Spand.from_problem(prob, 9, 0.1, 1)
            code = 0 if np.array_equal(hc.cluster_map(3), want) else 1
            hc.close()
        finally:
            os._exit(code)
    deadline = time.time() + 90
    while True:
        done, status = os.waitpid(pid, os.WNOHANG)
        if done:
            break
        if time.time() > deadline:
            os.kill(pid, signal.SIGKILL)
            os.waitpid(pid, 0)
            pytest.fail("the forked child's analysis did not finish")
        time.sleep(0.05)
    assert os.WIFEXITED(status) and os.WEXITSTATUS(status) == 0


@pytest.mark.parametrize("comps,ell,seed", [
    ([(8, 8), (8, 8)], 3, 0),             # the first sweep reaches exactly half: empty separator
    ([(5, 4), (9, 7)], 3, 3),
    ([(4, 4), (4, 4), (6, 6)], 3, 4),
    ([(10,), (10,), (10,), (10,)], 3, 5),
    ([(7, 7), (7, 7)], 4, 6),
])
def test_algebraic_partition_of_disconnected_graphs(comps, ell, seed):
    """Graphs of several components (unreached vertices in the breadth-first
    sweeps, medians among them): the library's partition equals the oracle's."""
    import scipy.sparse as sp
    from paper_2007_00789_gb300 import spand as S
    A = sp.block_diag([si.laplacian_grid(c).to_scipy() for c in comps]).tocsr()
    n = A.shape[0]
    perm = np.random.default_rng(seed).permutation(n)
    A = A[perm][:, perm].tocsr()
    A.sort_indices()
    tree = P.graph_nested_dissection(A.indptr, A.indices, ell)
    h = S.Spand(A.indptr, A.indices, A.data, None, ell, 1e-2, 1)
    for k in range(ell):
        sc = P.stage_clusters(tree, k)
        want = np.full(n, -1)
        for ci, key in enumerate(sc.keys):
            want[sc.members[key]] = ci
        assert np.array_equal(h.cluster_map(k), want), k
    h.close()
