"""spand_pcg_noalloc: the PCG entry point that allocates nothing.

It exists for callers that cannot allocate device memory while they solve
(a program whose GPU memory is fully reserved by another allocator, or a
loop that must not allocate once running); its work vectors live in a fixed
device array inside the library.  These tests call it through the C ABI and
check it against spand_pcg on the same factorization, twice in a row (the
second call starts from the array contents the first one left behind), and
check that a system larger than the array is refused before any GPU work.

The file name makes pytest collect it last, so a failure here does not stop
the other GPU tests from running first.
"""
import numpy as np
import pytest

import spand_inputs as si

pytestmark = pytest.mark.gpu

TOL_X = 1e-10  # the tolerance the other GPU parity tests use for M r


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("make,ell,scheme", [
    (lambda: si.laplacian_2d(64), 6, 1),
    (lambda: si.diffusion_3d(24, seed=3), 8, 2),
])
def test_noalloc_matches_pcg_twice(make, ell, scheme):
    torch = _torch()
    from paper_2007_00789_gb300 import spand as S
    prob = make()
    h = S.Spand.from_problem(prob, ell, 1e-2, scheme)
    h.factor()
    b = torch.from_numpy(si.rhs_normal(prob.n, seed=7)).cuda()
    x_ref = torch.zeros_like(b)
    it_ref, rel_ref = h.pcg(b, x_ref, 1e-12)
    assert rel_ref <= 1e-12
    for call in range(2):
        x = torch.full_like(b, float("nan"))  # whatever the caller's buffer holds is overwritten
        it, rel = h.pcg_noalloc(b, x, 1e-12)
        torch.cuda.synchronize()
        assert rel <= 1e-12, (call, rel)
        assert abs(it - it_ref) <= 1, (call, it, it_ref)
        err = float((x - x_ref).abs().max() / x_ref.abs().max())
        assert err <= TOL_X, (call, err)
    h.close()


def test_noalloc_allocates_nothing():
    """On a handle that has only been factored, the no-alloc solve leaves the
    device's free memory unchanged; spand_pcg (which allocates its work
    vectors) runs only afterwards, for the comparison."""
    torch = _torch()
    from paper_2007_00789_gb300 import spand as S
    prob = si.diffusion_3d(20, seed=5)
    ell, scheme = 7, 1
    b = torch.from_numpy(si.rhs_normal(prob.n, seed=8)).cuda()
    # the same problem shape solved once first: CUDA loads the kernels a call
    # launches on their first use, and that load takes device memory of its own
    warm = S.Spand.from_problem(prob, ell, 1e-2, scheme)
    warm.factor()
    xw = torch.zeros_like(b)
    warm.pcg_noalloc(b, xw, 1e-12)
    warm.close()
    h = S.Spand.from_problem(prob, ell, 1e-2, scheme)
    h.factor()
    x = torch.zeros_like(b)
    x_ref = torch.zeros_like(b)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    it, rel = h.pcg_noalloc(b, x, 1e-12)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert rel <= 1e-12
    it_ref, rel_ref = h.pcg(b, x_ref, 1e-12)
    assert abs(it - it_ref) <= 1, (it, it_ref)
    err = float((x - x_ref).abs().max() / x_ref.abs().max())
    assert err <= TOL_X, err
    h.close()


def test_noalloc_rejects_too_large_system():
    torch = _torch()
    from paper_2007_00789_gb300 import spand as S
    prob = si.laplacian_3d(65)  # n = 274625 > 262144, the static array's limit
    h = S.Spand.from_problem(prob, 12, 1e-2, 1)  # analysed only: the size check comes first
    b = torch.ones(prob.n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(S.SpandError) as e:
        h.pcg_noalloc(b, x, 1e-12)
    assert e.value.code == S.SPAND_EINVAL
    assert "262144" in str(e.value)
    h.close()
