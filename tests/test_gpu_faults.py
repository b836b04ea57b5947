"""Failure detection without faulting the GPU.

Every device-side wait in the library (the grid barriers of the cooperative
kernels) has a poll limit; when it runs out the kernel records the failure
and returns.  Here the wait is made to run out on purpose -- a barrier that
expects one CTA more than the grid has -- and the status is checked, then
the same process keeps solving.  Host-side failures (bad arguments) are
covered in test_capi_cpu.py and test_gpu_parity.py.
"""
from __future__ import annotations

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_1510_02237_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)


def test_bounded_wait_gives_up_and_context_survives():
    st, sec = P.parareal_selftest_wait_timeout(torch.cuda.current_stream())
    assert st == P.PR_ETIMEOUT
    assert 0.0 < sec < 5.0
    # the context is still usable: a small solve afterwards works
    p = W.make_problem(64, 32, 8)
    q0 = torch.from_numpy(W.ic_gaussian(64, 32, seed=0).ravel()).cuda()
    with P.Solver(p, stream=torch.cuda.current_stream(), K_max=2) as s:
        out = torch.empty_like(q0)
        rep = P.parareal_solve(s.h, q0, 2, qT=out)
        torch.cuda.synchronize()
        assert rep.K == 2 and np.all(np.isfinite(out.cpu().numpy()))
