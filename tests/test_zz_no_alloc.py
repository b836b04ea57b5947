"""The allocation-free fine sweep against the handle-based one.

parareal_fine_sweep_static() exists for callers that cannot allocate device
memory where they need the fine propagator (inside CUDA graph capture, under
a runtime that owns all device memory, or after start-up on hosts that
forbid later allocation).  It must compute what parareal_fine_sweep()
computes.  This file is collected last so that, if it fails, a run stopping
at the first failure has already run every other test; it also passes when
run alone in a fresh process.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_1510_02237_gb300")

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5   # FP32 fine sweep against the FP64 oracle, as in the parity tests


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("V", [0.0, 0.05], ids=["V0", "V005"])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_static_fine_sweep_matches_handle_twice(prec, V):
    """Two calls in a row (sharing the static scratch) against the handle's
    sweep and against the oracle's F on a few of the states."""
    p = W.make_problem(256, 128, 8, V=V)
    n = 8
    stream = torch.cuda.current_stream()
    X = [torch.from_numpy(np.stack([W.ic_random(p.nx, p.ny, seed=s + i).ravel() for i in range(n)])).cuda()
         for s in (100, 200)]
    with P.Solver(p, stream=stream, fine_prec=prec) as s:
        want = []
        for x in X:
            y = torch.empty_like(x)
            P.parareal_fine_sweep(s.h, x, y, n)
            want.append(y)
        torch.cuda.synchronize()
        want = [w.cpu().numpy() for w in want]
    tol_oracle = TOL64 if prec == 0 else TOL32
    for call in range(2):                      # two calls in a row share the static scratch
        x = X[call]
        y = torch.full_like(x, float("nan"))
        P.parareal_fine_sweep_static(p.nx, p.ny, p.U, p.V, p.c_s, p.nu_f, p.dt_f, p.n_f, prec, x, y, n,
                                     stream=stream)
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        assert np.all(np.isfinite(got))
        # FP64: the same kernel arithmetic; FP32: the handle may run the
        # row-streamed kernel (packed pair arithmetic, other rounding order)
        assert _rel(got, want[call]) < (TOL64 if prec == 0 else TOL32)
        xin = x.cpu().numpy()
        for i in (0, n - 1):
            ref = oracle.fine_prop(p, xin[i])
            assert _rel(got[i], ref) < tol_oracle


def test_static_fine_sweep_rejects_oversize():
    p = W.make_problem(512, 256, 8)            # d = 393216: 6 states exceed 2097152 doubles
    x = torch.zeros(6 * p.d, dtype=torch.float64, device="cuda")
    with pytest.raises(P.PararealError) as ei:
        P.parareal_fine_sweep_static(p.nx, p.ny, p.U, p.V, p.c_s, p.nu_f, p.dt_f, p.n_f, 0, x, x.clone(), 6)
    assert ei.value.status == P.PR_EINVAL
