"""Autotuning of the fine step's launch shape (parareal_autotune).

The candidates (tile shapes of the shared-memory kernel, row ranges per CTA
of the row-streamed kernel) lay out the same per-cell arithmetic
differently on the GPU, so a sweep gives the same bits before and after
tuning; a second handle of the same shape takes the choice from the cache.
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


def _sweep(s, X, n):
    out = torch.empty_like(X)
    P.parareal_fine_sweep(s.h, X, out, n)
    torch.cuda.synchronize()
    return out


CASES = [("fp32x_256x128", "FP32X", 256, 128, 4, "tile"),
         ("fp32_256x128", "FP32", 256, 128, 5, "rows"),
         ("fp32_96x20", "FP32", 96, 20, 3, "tile"),
         ("fp32x_64x32", "FP32X", 64, 32, 8, "tile")]


@pytest.mark.parametrize("name,prec,nx,ny,N,kind", CASES, ids=[c[0] for c in CASES])
def test_autotune_same_bits_and_cache(name, prec, nx, ny, N, kind):
    p = W.make_problem(nx, ny, N)
    fp = getattr(P, "PR_" + prec)
    X = torch.from_numpy(np.stack([W.ic_random(nx, ny, seed=60 + i).ravel() for i in range(N)])).cuda().ravel()
    stream = torch.cuda.current_stream()
    with P.Solver(p, stream=stream, fine_prec=fp) as s:
        before = _sweep(s, X, N)
        t = P.parareal_autotune(s.h)
        assert t["kernel"] == kind
        if not t["cached"]:
            assert t["choice"] in t["candidates"] and len(t["candidates"]) == 4
            assert all(u > 0 for u in t["us_per_step"])
        after = _sweep(s, X, N)
    assert torch.equal(before, after)
    with P.Solver(p, stream=stream, fine_prec=fp) as s2:
        t2 = P.parareal_autotune(s2.h)
        assert t2["cached"] and t2["choice"] == t["choice"]
        assert torch.equal(_sweep(s2, X, N), before)


def test_autotune_fp64_has_nothing_to_tune():
    p = W.make_problem(64, 32, 8)
    with P.Solver(p, stream=torch.cuda.current_stream()) as s:
        t = P.parareal_autotune(s.h)
    assert t["kernel"] == "none" and t["choice"] == -1
