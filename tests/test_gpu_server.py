"""Solve server: resident factors, multi-RHS requests, continuous batching.

* every right-hand side reaches the true relative residual tol, and its
  iteration count matches spand_pcg on the same problem within one;
* a request's result is the same alone and mixed with other requests that
  overlap it (same iterations, x within 1e-10 relative: only the apply's
  atomic accumulation order may differ);
* a budget too small for all problems evicts idle ones and refactors them
  when they are asked for again, with the same results;
* a problem whose factorization fails fails only its own requests.
"""
import threading
import time

import numpy as np
import pytest

import spand_inputs as si

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _problems():
    return [
        (si.diffusion_3d(20, seed=1), 8),             # the resident problem
        (si.diffusion_grid((48, 40, 24), seed=2), 9),
        (si.diffusion_grid((90, 70), seed=3), 7),
        (si.diffusion_3d(16, seed=4), 7),
    ]


def _true_rel(p, b, x):
    A = p.to_scipy()
    return max(np.linalg.norm(b[j] - A @ x[j]) / np.linalg.norm(b[j]) for j in range(b.shape[0]))


@pytest.mark.parametrize("precision", [0, 1])
def test_server_results_and_iterations(precision):
    torch = _torch()
    from paper_2007_00789_gb300 import spand as S
    probs = _problems()
    srv = S.SpandServer(precision=precision, tol=TOL, max_entries=1 << 22, max_segments=64)
    hs = [S.Spand.from_problem(p, ell, 1e-2, 1, precision=precision) for p, ell in probs]
    mids = [srv.add(h, pinned=(i == 0)) for i, h in enumerate(hs)]
    rng = np.random.default_rng(0)
    reqs = []
    for k in range(10):
        i = k % len(probs)
        nrhs = 1 + (k * 3) % 5
        b = rng.standard_normal((nrhs, probs[i][0].n))
        reqs.append((i, b, srv.submit(mids[i], b)))
    results = [(i, b) + srv.wait(rid) for i, b, rid in reqs]
    st = srv.stats()
    srv.close()
    assert st["requests"] == len(reqs) and st["solves"] == sum(b.shape[0] for _, b, _ in reqs)
    assert st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    # single-problem PCG on the same problems
    ref = {}
    for i, (p, ell) in enumerate(probs):
        h = S.Spand.from_problem(p, ell, 1e-2, 1, precision=precision)
        h.factor()
        ref[i] = h
    for i, b, x, it, rel, lat in results:
        p = probs[i][0]
        assert (rel <= TOL).all() and _true_rel(p, b, x) <= TOL
        for j in range(b.shape[0]):
            bd = torch.from_numpy(b[j]).cuda()
            xd = torch.zeros_like(bd)
            it1, _ = ref[i].pcg(bd, xd, TOL)
            assert abs(int(it[j]) - it1) <= 1, (i, j, it[j], it1)
    for h in list(ref.values()) + hs:
        h.close()


def test_server_same_alone_and_in_mix():
    _torch()
    from paper_2007_00789_gb300 import spand as S
    probs = _problems()
    srv = S.SpandServer(tol=TOL, max_entries=1 << 22, max_segments=64)
    hs = [S.Spand.from_problem(p, ell, 1e-2, 1) for p, ell in probs]
    mids = [srv.add(h, pinned=(i == 0)) for i, h in enumerate(hs)]
    rng = np.random.default_rng(7)
    bA = rng.standard_normal((3, probs[0][0].n))
    xA, itA, relA, _ = srv.wait(srv.submit(mids[0], bA))  # alone
    # the mix: other requests submitted from another thread while A runs again
    others = [(i, rng.standard_normal((1 + i, probs[i][0].n))) for i in (1, 2, 3, 1, 2)]
    out = []

    def feeder():
        for i, b in others:
            out.append((i, b, srv.submit(mids[i], b)))
            time.sleep(0.002)

    t = threading.Thread(target=feeder)
    t.start()
    rid = srv.submit(mids[0], bA)
    t.join()
    xM, itM, relM, _ = srv.wait(rid)
    for i, b, r in out:
        x, it, rel, _ = srv.wait(r)
        assert (rel <= TOL).all() and _true_rel(probs[i][0], b, x) <= TOL
    st = srv.stats()
    srv.close()
    assert np.array_equal(itA, itM)
    d = np.abs(xA - xM).max() / np.abs(xA).max()
    print("alone vs mix: iterations", itA, "max rel diff", d, "max in flight", st["max_inflight"])
    assert d <= 1e-10
    for h in hs:
        h.close()


def test_server_evicts_under_budget():
    _torch()
    from paper_2007_00789_gb300 import spand as S
    probs = _problems()
    hs = [S.Spand.from_problem(p, ell, 1e-2, 1) for p, ell in probs]
    # a budget that holds the resident factorization and about one other
    srv = S.SpandServer(tol=TOL, hbm_budget=160 << 20, max_entries=1 << 22, max_segments=64)
    mids = [srv.add(h, pinned=(i == 0)) for i, h in enumerate(hs)]
    rng = np.random.default_rng(3)
    first = {}
    for rnd in range(2):
        for i in (1, 2, 3):
            b = np.random.default_rng(100 + i).standard_normal((2, probs[i][0].n))
            x, it, rel, _ = srv.wait(srv.submit(mids[i], b))
            assert (rel <= TOL).all() and _true_rel(probs[i][0], b, x) <= TOL
            if rnd == 0:
                first[i] = (x, it)
            else:
                assert np.array_equal(first[i][1], it)
                assert np.abs(first[i][0] - x).max() <= 1e-10 * np.abs(x).max()
        b = rng.standard_normal((1, probs[0][0].n))
        x, it, rel, _ = srv.wait(srv.submit(mids[0], b))
        assert (rel <= TOL).all()
    st = srv.stats()
    srv.close()
    print("resident bytes", st["resident_bytes"], "problems", st["resident_problems"])
    assert st["resident_problems"] <= 2
    for h in hs:
        h.close()


def test_server_failed_factorization_is_isolated():
    _torch()
    from paper_2007_00789_gb300 import spand as S
    good = si.laplacian_2d(32)
    val = good.val.copy()
    val[np.nonzero(good.colind == 0)[0][0]] = -4.0  # diagonal of row 0: not SPD
    hg = S.Spand.from_problem(good, 5, 1e-2, 1)
    hb = S.Spand(good.rowptr, good.colind, val, good.coords, 5, 1e-2, 1)
    srv = S.SpandServer(tol=TOL, max_entries=1 << 20, max_segments=16)
    mg, mb = srv.add(hg), srv.add(hb)
    b = np.random.default_rng(1).standard_normal((2, good.n))
    rb = srv.submit(mb, b)
    rg = srv.submit(mg, b)
    with pytest.raises(S.SpandError) as e:
        srv.wait(rb)
    assert e.value.code == S.SPAND_ENOTSPD
    x, it, rel, _ = srv.wait(rg)
    assert (rel <= TOL).all()
    srv.close()
    hg.close()
    hb.close()
