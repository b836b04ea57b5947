"""Batches of independent solves and the continuous-batching server.

The kernels reduce in a fixed order and never across handles, so a solve's
result must not depend on what else runs on the GPU: every result produced
in a batch or under the server equals, bit for bit, the same solve run alone
with the same options.
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


def _alone(inst, **opt):
    p = inst.problem
    with P.Solver(p, stream=torch.cuda.current_stream(), K_max=inst.K, **opt) as s:
        u0 = torch.from_numpy(inst.initial_value().ravel()).cuda()
        out = torch.empty_like(u0)
        P.parareal_solve(s.h, u0, inst.K, qT=out, report=False)
        torch.cuda.synchronize()
        return out.cpu().numpy()


@pytest.mark.parametrize("mode", ["fp64", "mixed", "mixed_persistent", "fp32x_persistent"])
def test_batch_equals_alone(mode):
    """The '_persistent' batches (FP32 tendencies, FP32 or FP64 correction)
    run their fine sweeps as one persistent launch per phase over all
    handles (lockstep capture); the others fork the handles' own solves."""
    insts = W.workload_batch(6, seed=2000)
    pers = {"batch_fine": P.PR_BATCH_PERSISTENT}
    opt = {"fp64": {}, "mixed": {"fine_prec": P.PR_FP32X, "corr_prec": P.PR_FP32},
           "mixed_persistent": {"fine_prec": P.PR_FP32X, "corr_prec": P.PR_FP32, **pers},
           "fp32x_persistent": {"fine_prec": P.PR_FP32X, **pers}}[mode]
    want = [_alone(i, sm_limit=8, **opt) for i in insts]
    streams = [P.new_stream() for _ in insts]
    solvers = [P.Solver(i.problem, stream=st, K_max=i.K, sm_limit=8, **opt) for i, st in zip(insts, streams)]
    u0s = [torch.from_numpy(i.initial_value().ravel()).cuda() for i in insts]
    outs = [torch.full_like(u, float("nan")) for u in u0s]
    torch.cuda.synchronize()
    P.parareal_solve_batch([s.h for s in solvers], u0s, [i.K for i in insts], outs)
    for o, w in zip(outs, want):
        assert np.array_equal(o.cpu().numpy(), w)
    # one CUDA graph over all six, replayed twice
    main = P.new_stream()
    for o in outs:
        o.fill_(float("nan"))
    torch.cuda.synchronize()
    b = P.parareal_batch_create([s.h for s in solvers], u0s, [i.K for i in insts], outs, main)
    for _ in range(2):
        P.parareal_batch_launch(b)
        torch.cuda.synchronize()
        for o, w in zip(outs, want):
            assert np.array_equal(o.cpu().numpy(), w)
    P.parareal_batch_destroy(b)
    for s in solvers:
        s.close()


def test_batch_rejects_null_stream_and_duplicates():
    insts = W.workload_batch(2, seed=3000)
    solvers = [P.Solver(i.problem, stream=None, K_max=i.K) for i in insts]
    u0s = [torch.zeros(i.problem.d, dtype=torch.float64, device="cuda") for i in insts]
    with pytest.raises(P.PararealError) as ei:
        P.parareal_batch_create([s.h for s in solvers], u0s, [i.K for i in insts], u0s, P.new_stream())
    assert ei.value.status == P.PR_EINVAL
    st = P.new_stream()
    s1 = P.Solver(insts[0].problem, stream=st, K_max=insts[0].K)
    with pytest.raises(P.PararealError):
        P.parareal_batch_create([s1.h, s1.h], u0s[:1] * 2, [insts[0].K] * 2, u0s[:1] * 2, P.new_stream())
    for s in solvers + [s1]:
        s.close()


def test_server_results_equal_alone_and_budget_holds():
    from paper_1510_02237_gb300 import serve
    reqs = [(0.002 * k, inst) for k, (_, inst) in enumerate(W.request_stream(1000.0, 40, seed=11))
            if inst.problem.nx <= 128][:12]
    budget = 3.0e9
    srv = serve.Server(budget_bytes=budget, max_inflight=5, mode="mixed")
    results, stats = srv.run(reqs)
    opts = [srv.solver_options(inst.problem) for _, inst in reqs]
    srv.close()
    assert stats.completed == len(reqs) and stats.peak_bytes <= budget
    assert 2 <= stats.peak_inflight <= 5     # requests overlapped on the device, within the limit
    for (t, inst), r, opt in zip(reqs, results, opts):
        assert opt["proj_prec"] == P.PR_PROJ_SPLIT_BF16 and opt["corr_prec"] == P.PR_FP32
        want = _alone(inst, **opt)
        assert np.array_equal(r.qT, want)
        assert r.latency > 0
