"""Failure detection of the factorization's one bounded device-side wait.

The multi-CTA RRQR (Algorithm 1 on interface blocks too wide for a
thread-block cluster) synchronises its CTAs with a barrier in global memory
whose waits give up after a fixed number of polls.  A wait that runs out must
reach the caller as SPAND_ETIMEOUT, leave the handle unfactored and the
device usable, and a later factorization must succeed with the same result.

No GPU fault or hang is caused: the testing hook raises the first barrier's
target by one, so the wait can never be met, and shortens the poll limit; every
CTA of the affected tasks then leaves on its own after that many polls.
"""
import time

import numpy as np
import pytest

import spand_inputs as si

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_qr_barrier_timeout_is_reported_and_recoverable():
    torch = _torch()
    from paper_2007_00789_gb300 import spand as S
    prob = si.diffusion_3d(16, seed=2)
    ell, eps, scheme = 6, 1e-2, 1
    # rrqr_kernel = 3: every interface goes through the multi-CTA kernel
    ref = S.Spand.from_problem(prob, ell, eps, scheme, rrqr_kernel=3)
    ref.factor()
    r = torch.from_numpy(np.random.default_rng(4).standard_normal(prob.n)).cuda()
    z_ref = torch.empty_like(r)
    ref.apply(r, z_ref)

    h = S.Spand.from_problem(prob, ell, eps, scheme, rrqr_kernel=3)
    h.test_set_qr_wait(limit=1 << 12, unreachable=True)
    t0 = time.perf_counter()
    with pytest.raises(S.SpandError) as e:
        h.factor()
    assert e.value.code == S.SPAND_ETIMEOUT, str(e.value)
    assert time.perf_counter() - t0 < 60.0
    # the handle is unfactored, the device still answers
    z = torch.empty_like(r)
    with pytest.raises(S.SpandError) as e2:
        h.apply(r, z)
    assert e2.value.code == S.SPAND_ESTATE
    torch.cuda.synchronize()
    assert float((r * r).sum()) > 0.0

    # default wait restored: the factorization succeeds and equals the reference
    # (ranks exactly; M r up to the apply's atomic accumulation order)
    h.test_set_qr_wait(0, False)
    h.factor()
    assert np.array_equal(h.ranks(), ref.ranks())

    def err():
        h.apply(r, z)
        torch.cuda.synchronize()
        return float((z - z_ref).abs().max() / z_ref.abs().max())

    assert err() <= 1e-12
    # and a refactorization replayed from its graphs still agrees
    h.factor()
    assert err() <= 1e-12
    h.close()
    ref.close()
