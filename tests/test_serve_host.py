"""Host logic of the request loop (paper_1510_02237_gb300.serve), on the CPU.

The loop's admission decides, per waiting request, whether a solver slot
may be reused or created: at most max_inflight solves in flight, the SMs
that the in-flight solves' grid-synchronised kernels use fit on the GPU,
and the slots' device footprint stays within the memory budget (idle slots
are freed largest first to make room).  These tests drive that logic with
stand-ins for the library's handle, stream and buffer calls, so no GPU and
no device memory are involved; the GPU tests run the real loop.
"""
from __future__ import annotations

import types

import pytest

import workloads as W

P = pytest.importorskip("paper_1510_02237_gb300")
serve = pytest.importorskip("paper_1510_02237_gb300.serve")


class _FakeSolver:
    created = []

    def __init__(self, p, stream=None, **opt):
        self.p, self.opt, self.h, self.closed = p, dict(opt), object(), False
        _FakeSolver.created.append(self)

    def close(self):
        self.closed = True


class _Buf:
    def pin_memory(self):
        return self


def _fake_torch():
    return types.SimpleNamespace(float64="float64", empty=lambda *a, **k: _Buf())


def _footprint(nx, ny, N, **opt):
    return 1000 * nx * ny * N   # bytes, proportional to the state count


@pytest.fixture
def server(monkeypatch):
    _FakeSolver.created = []
    monkeypatch.setattr(serve, "Solver", _FakeSolver)
    monkeypatch.setattr(serve, "parareal_footprint_bytes", _footprint)
    monkeypatch.setattr(serve, "parareal_autotune", lambda h: None)
    monkeypatch.setattr(serve, "new_stream", lambda: object())

    def make(**kw):
        s = serve.Server(sms=kw.pop("sms", 152), **kw)
        s.torch = _fake_torch()
        s.stats = serve.ServeStats()
        return s
    return make


def _inst(nx, ny, N, K=2):
    return types.SimpleNamespace(problem=W.make_problem(nx, ny, N), K=K)


def test_sm_limit_rule():
    # one SM per 2048 state values, at least 4, at most the GPU
    assert serve.default_sm_limit(3 * 64 * 32, 152) == 4
    assert serve.default_sm_limit(3 * 256 * 128, 152) == 48
    assert serve.default_sm_limit(3 * 512 * 256, 152) == 152
    assert serve.batch_sm_limit(3 * 256 * 128, 152) == serve.default_sm_limit(3 * 256 * 128, 152)


def test_solver_options_per_mode(server):
    p = W.make_problem(64, 32, 8)
    assert server(mode="fp64").solver_options(p) == {"sm_limit": 4}
    assert server(mode="fp64_tc").solver_options(p) == {"proj_prec": P.PR_PROJ_SPLIT_BF16, "sm_limit": 4}
    assert server(mode="mixed").solver_options(p) == {
        "fine_prec": P.PR_FP32X, "corr_prec": P.PR_FP32, "proj_prec": P.PR_PROJ_SPLIT_BF16, "sm_limit": 4}
    # the tensor-core products need 3 nx ny to be a multiple of 8
    assert "proj_prec" not in server(mode="fp64_tc").solver_options(W.make_problem(15, 9, 4))
    assert server(mode="fp64", sm_limit=None).solver_options(p) == {}
    with pytest.raises(ValueError):
        server(mode="bf16")


def test_slot_reuse_and_inflight_cap(server):
    s = server(mode="fp64", max_inflight=2)
    a = _inst(64, 32, 8)
    s1 = s._acquire(a, 0)
    assert s1 is not None and s.stats.slots_created == 1
    assert s1.solver.opt["K_max"] == 8 and s1.sms == 4
    assert s._acquire(a, 0) is s1                     # idle slot of the same shape: reused
    s1.busy = True
    s2 = s._acquire(a, 1, s1.sms)
    assert s2 is not None and s2 is not s1 and s.stats.slots_created == 2
    assert s._acquire(a, 2, 8) is None                # in-flight cap
    assert s.bytes == 2 * _footprint(64, 32, 8)


def test_sm_admission(server):
    s = server(mode="fp64", sms=64)
    big = _inst(256, 128, 8)                          # 48 SMs per solve
    first = s._acquire(big, 0)
    assert first.sms == 48
    first.busy = True
    assert s._acquire(big, 1, 48) is None             # 48 + 48 > 64
    small = _inst(64, 32, 8)                          # 4 SMs
    assert s._acquire(small, 1, 48) is not None
    # with nothing in flight the SM check is skipped
    assert s._acquire(_inst(512, 256, 8), 0).sms == 64


def test_budget_and_eviction(server):
    unit = _footprint(64, 32, 8)
    s = server(mode="fp64", budget_bytes=3.5 * unit)
    a, b = _inst(64, 32, 8), _inst(128, 64, 8)       # b takes 4 units
    s1 = s._acquire(a, 0)
    s1.busy = True
    s2 = s._acquire(a, 1, 4)
    assert s.bytes == 2 * unit
    s2.busy = True
    assert s._acquire(b, 2, 8) is None                # does not fit; nothing idle to free
    assert s.bytes == 2 * unit and not s1.solver.closed and not s2.solver.closed
    s1.busy = s2.busy = False
    assert s._acquire(b, 0) is None                   # 4 units never fit in 3.5
    s = server(mode="fp64", budget_bytes=4.5 * unit)
    s1 = s._acquire(a, 0)
    s1.busy = False
    s3 = s._acquire(b, 0)                             # frees the idle slot to make room
    assert s3 is not None and s1.solver.closed
    assert s.bytes == 4 * unit and s.slots[s._key(a)] == []
    s.close()
    assert s.bytes == 0 and s3.solver.closed
