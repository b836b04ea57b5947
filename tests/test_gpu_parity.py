"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (written from the arithmetic): FP64 paths agree with the oracle to
<= 1e-12 relative (l2 over the compared states) -- both evaluate the same
formulas in IEEE double, differing only in summation order and fused
multiply-adds; the FP32 fine sweep agrees to <= 1e-5 relative.
Integer results (ranks, drop decisions) must agree exactly.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_1510_02237_gb300")

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    a = np.ravel(a)
    b = np.ravel(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def solver(p, **opt):
    return P.Solver(p, stream=torch.cuda.current_stream(), **opt)


def states(p, n, seed):
    return np.stack([W.ic_random(p.nx, p.ny, seed=seed + i).ravel() for i in range(n)])


GRIDS = [
    ("64x32", dict(nx=64, ny=32, N=8)),
    ("ragged40x24", dict(nx=40, ny=24, N=4)),
    ("tiny8x4", dict(nx=8, ny=4, N=4)),
    ("128x64_V", dict(nx=128, ny=64, N=4, V=0.05)),
    ("96x20_negU", dict(nx=96, ny=20, N=3, U=-0.15)),
]


def _prob(spec):
    spec = dict(spec)
    nx, ny, N = spec.pop("nx"), spec.pop("ny"), spec.pop("N")
    return W.make_problem(nx, ny, N, **spec)


# ------------------------------------------------------------------ propagators

@pytest.mark.parametrize("name,spec", GRIDS, ids=[g[0] for g in GRIDS])
def test_fine_sweep_fp64(name, spec):
    p = _prob(spec)
    X = states(p, p.n_slices, 10)
    with solver(p) as s:
        out = torch.empty(p.n_slices * p.d, dtype=torch.float64, device="cuda")
        P.parareal_fine_sweep(s.h, dev(X), out, p.n_slices)
        got = host(out).reshape(p.n_slices, p.d)
    for i in range(p.n_slices):
        assert rel(got[i], oracle.fine_prop(p, X[i])) < TOL64


@pytest.mark.parametrize("name,spec", GRIDS[:4], ids=[g[0] for g in GRIDS[:4]])
def test_fine_sweep_fp32(name, spec):
    p = _prob(spec)
    X = states(p, p.n_slices, 20)
    with solver(p, fine_prec=P.PR_FP32) as s:
        out = torch.empty(p.n_slices * p.d, dtype=torch.float64, device="cuda")
        P.parareal_fine_sweep(s.h, dev(X), out, p.n_slices)
        got = host(out).reshape(p.n_slices, p.d)
    for i in range(p.n_slices):
        assert rel(got[i], oracle.fine_prop(p, X[i])) < TOL32


@pytest.mark.parametrize("name,spec", GRIDS[:4], ids=[g[0] for g in GRIDS[:4]])
def test_fine_sweep_fp32x(name, spec):
    """FP32 tendencies and stages on an FP64 state: the FP64 update
    q^n + dt L(q**) keeps the per-step rounding at dt |L| times FP32's."""
    p = _prob(spec)
    X = states(p, p.n_slices, 20)
    with solver(p, fine_prec=P.PR_FP32X) as s:
        out = torch.empty(p.n_slices * p.d, dtype=torch.float64, device="cuda")
        P.parareal_fine_sweep(s.h, dev(X), out, p.n_slices)
        got = host(out).reshape(p.n_slices, p.d)
    for i in range(p.n_slices):
        assert rel(got[i], oracle.fine_prop(p, X[i])) < 2e-6


# Grids whose rows are a multiple of 128 cells (V = 0) take the row-streamed
# FP32 kernel: one warp per 128 cells of a row, 1 to 8 warps per row; row
# ranges of the persistent grid cross slice boundaries and, with few rows,
# wrap around the periodic y-direction.
ROW_GRIDS = [
    ("128x64", dict(nx=128, ny=64, N=4)),
    ("256x24", dict(nx=256, ny=24, N=5)),
    ("512x16_negU", dict(nx=512, ny=16, N=3, U=-0.12)),
    ("1024x8", dict(nx=1024, ny=8, N=2)),
    ("128x4", dict(nx=128, ny=4, N=3)),
]


@pytest.mark.parametrize("prec", ["fp32", "fp32x"])
@pytest.mark.parametrize("name,spec", ROW_GRIDS, ids=[g[0] for g in ROW_GRIDS])
def test_fine_sweep_rows(name, spec, prec):
    p = _prob(spec)
    X = states(p, p.n_slices, 40)
    fp, tol = (P.PR_FP32, TOL32) if prec == "fp32" else (P.PR_FP32X, 2e-6)
    with solver(p, fine_prec=fp) as s:
        out = torch.empty(p.n_slices * p.d, dtype=torch.float64, device="cuda")
        P.parareal_fine_sweep(s.h, dev(X), out, p.n_slices)
        got = host(out).reshape(p.n_slices, p.d)
    for i in range(p.n_slices):
        assert rel(got[i], oracle.fine_prop(p, X[i])) < tol


def test_fine_sweep_rows_subset():
    """A sweep over fewer states than the handle's slices (n < N) and a
    single RK-3 step per slice through the row-streamed kernel."""
    p = W.Problem(nx=256, ny=12, n_slices=6, n_f=1, n_g=1, dt_f=1.0 / 600, dt_g=1.0 / 600, T=6.0 / 600)
    X = states(p, 4, 50)
    for prec, tol in [(P.PR_FP32, TOL32), (P.PR_FP32X, 2e-6)]:
        with solver(p, fine_prec=prec) as s:
            out = torch.zeros(6 * p.d, dtype=torch.float64, device="cuda")
            P.parareal_fine_sweep(s.h, dev(X), out, 4)
            got = host(out).reshape(6, p.d)
        for i in range(4):
            assert rel(got[i], oracle.fine_prop(p, X[i])) < tol
        assert not got[4:].any()


def test_fine_single_step_slices():
    """N_f = 1 (one RK-3 step per slice) uses the direct in->out launch."""
    p = W.Problem(nx=64, ny=32, n_slices=4, n_f=1, n_g=1, dt_f=1.0 / 160, dt_g=1.0 / 160, T=4.0 / 160)
    X = states(p, 4, 3)
    for prec, tol in [(P.PR_FP64, TOL64), (P.PR_FP32, TOL32)]:
        with solver(p, fine_prec=prec) as s:
            out = torch.empty(4 * p.d, dtype=torch.float64, device="cuda")
            P.parareal_fine_sweep(s.h, dev(X), out, 4)
            got = host(out).reshape(4, p.d)
        for i in range(4):
            assert rel(got[i], oracle.fine_prop(p, X[i])) < tol


@pytest.mark.parametrize("order", [1, 3])
@pytest.mark.parametrize("name,spec", GRIDS, ids=[g[0] for g in GRIDS])
def test_coarse_apply(name, spec, order):
    p = dataclasses.replace(_prob(spec), adv_order_c=order)
    X = states(p, p.n_slices, 30)
    with solver(p) as s:
        out = torch.empty(p.n_slices * p.d, dtype=torch.float64, device="cuda")
        P.parareal_coarse_apply(s.h, dev(X), out, p.n_slices)
        got = host(out).reshape(p.n_slices, p.d)
    for i in range(p.n_slices):
        assert rel(got[i], oracle.coarse_prop(p, X[i])) < TOL64


# Batches large enough for the 64 x 32 coarse tiles (at least two per SM on
# a 152-SM GPU), with full and ragged tiles
BIG_COARSE = [
    ("256x128_N32", dict(nx=256, ny=128, N=32)),
    ("ragged200x72_N64", dict(nx=200, ny=72, N=64)),
]


@pytest.mark.parametrize("variant", ["split_o1", "split_o3", "rk3", "rotation"])
@pytest.mark.parametrize("name,spec", BIG_COARSE, ids=[g[0] for g in BIG_COARSE])
def test_coarse_apply_large_batch(name, spec, variant):
    p = _prob(spec)
    if variant == "split_o3":
        p = dataclasses.replace(p, adv_order_c=3)
    elif variant == "rk3":
        p = _rk3_coarse(p)
    elif variant == "rotation":
        p = _rot(spec)
    X = states(p, p.n_slices, 90)
    with solver(p) as s:
        out = torch.empty(p.n_slices * p.d, dtype=torch.float64, device="cuda")
        P.parareal_coarse_apply(s.h, dev(X), out, p.n_slices)
        got = host(out).reshape(p.n_slices, p.d)
    for i in range(p.n_slices):
        assert rel(got[i], oracle.coarse_prop(p, X[i])) < TOL64


def _rk3_coarse(p, order=1):
    """The RK-3 coarse propagator with a coarse step of two fine steps."""
    return dataclasses.replace(p, adv_order_c=order, coarse_scheme=1, dt_g=2 * p.dt_f, n_g=p.n_f // 2)


@pytest.mark.parametrize("order", [1, 3])
@pytest.mark.parametrize("name,spec", GRIDS, ids=[g[0] for g in GRIDS])
def test_coarse_apply_rk3(name, spec, order):
    """Non-split RK-3 coarse propagator (the instability demonstrations, Sec. 3.1)."""
    p = _rk3_coarse(_prob(spec), order)
    X = states(p, p.n_slices, 31)
    with solver(p) as s:
        out = torch.empty(p.n_slices * p.d, dtype=torch.float64, device="cuda")
        P.parareal_coarse_apply(s.h, dev(X), out, p.n_slices)
        got = host(out).reshape(p.n_slices, p.d)
    for i in range(p.n_slices):
        assert rel(got[i], oracle.coarse_prop(p, X[i])) < TOL64


def test_coarse_sweep_is_serial_chain():
    p = W.make_problem(64, 32, 8)
    q0 = W.ic_gaussian(64, 32, seed=0).ravel()
    with solver(p) as s:
        out = torch.empty(p.n_slices * p.d, dtype=torch.float64, device="cuda")
        P.parareal_coarse_sweep(s.h, dev(q0), out)
        got = host(out).reshape(p.n_slices, p.d)
    q = q0
    for i in range(p.n_slices):
        q = oracle.coarse_prop(p, q)
        assert rel(got[i], q) < TOL64


# ------------------------------------------------------------------ subspace

def test_krylov_update_and_project_match_oracle():
    p = W.make_problem(64, 32, 8)
    rng = np.random.default_rng(5)
    X = states(p, 6, 40)
    X[3] = 0.5 * X[0] - 2.0 * X[2]          # dependent on earlier columns -> dropped
    X[5] = X[1]                             # duplicate -> dropped
    FX = np.stack([oracle.fine_prop(p, x) for x in X])
    B = oracle.Basis(p.d, 16)
    want_kept = [B.add(X[j], FX[j])[0] for j in range(6)]
    with solver(p) as s:
        kept = P.krylov_update(s.h, dev(X[:4]), dev(FX[:4]), 4)
        kept += P.krylov_update(s.h, dev(X[4:]), dev(FX[4:]), 2)
        assert kept == [int(k) for k in want_kept] == [1, 1, 1, 0, 1, 0]
        assert P.krylov_rank(s.h) == B.rank == 4
        for trial in range(3):
            q = rng.standard_normal(p.d)
            Pq = torch.empty(p.d, dtype=torch.float64, device="cuda")
            FPq = torch.empty_like(Pq)
            P.krylov_project(s.h, dev(q), Pq, FPq)
            wPq, wFPq = B.project(q)
            assert rel(host(Pq), wPq) < TOL64
            assert rel(host(FPq), wFPq) < 1e-11
            # and F(P q) is F applied to P q (Eq. Genhance)
            assert rel(host(FPq), oracle.fine_prop(p, host(Pq))) < 1e-11


def test_krylov_cap_freezes_basis():
    p = W.make_problem(64, 32, 8)
    X = states(p, 5, 50)
    FX = np.stack([oracle.fine_prop(p, x) for x in X])
    with solver(p, krylov_cap=3) as s:
        kept = P.krylov_update(s.h, dev(X), dev(FX), 5)
        assert kept == [1, 1, 1, 0, 0] and P.krylov_rank(s.h) == 3
        P.krylov_reset(s.h)
        assert P.krylov_rank(s.h) == 0


# ------------------------------------------------------------------ whole solve

def _solve(p, q0, K, **opt):
    opt.setdefault("K_max", max(K, 1))
    with solver(p, **opt) as s:
        qall = torch.empty((p.n_slices + 1) * p.d, dtype=torch.float64, device="cuda")
        rep = P.parareal_solve(s.h, dev(q0), K, q_out=qall)
        return host(qall).reshape(p.n_slices + 1, p.d), rep


@pytest.mark.parametrize("K", [0, 1, 2, 3, 5, 8])
def test_solve_matches_oracle_64x32(K):
    wl = W.workload_small()
    p = wl.problem
    q0 = wl.ics[0][1]().ravel()
    got, rep = _solve(p, q0, K)
    want = oracle.parareal(p, q0, K)
    assert rel(got, want["q"]) < TOL64
    assert list(rep.rank[:K]) == list(want["rank"])
    assert np.allclose(np.array(rep.r[:K]), want["r"], rtol=1e-9, atol=0)


def test_solve_original_parareal_matches_oracle():
    p = W.make_problem(64, 32, 8)
    q0 = W.ic_gaussian(64, 32, seed=0).ravel()
    got, rep = _solve(p, q0, 3, variant=P.PR_ORIGINAL)
    want = oracle.parareal(p, q0, 3, variant="original")
    assert rel(got, want["q"]) < TOL64
    assert np.allclose(np.array(rep.r[:3]), want["r"], rtol=1e-9)


@pytest.mark.parametrize("variant", ["kse", "original"])
def test_solve_rk3_coarse_matches_oracle(variant):
    """Alg. 2 and Alg. 1 with the RK-3 coarse propagator (serial chain and
    coarse images through the same coarse tile)."""
    p = _rk3_coarse(W.make_problem(64, 32, 8))
    q0 = W.ic_gaussian(64, 32, seed=0).ravel()
    got, rep = _solve(p, q0, 3, variant=P.PR_KSE if variant == "kse" else P.PR_ORIGINAL)
    want = oracle.parareal(p, q0, 3, variant=variant)
    assert rel(got, want["q"]) < TOL64
    assert np.allclose(np.array(rep.r[:3]), want["r"], rtol=1e-9)


def test_instability_demo_matches_oracle():
    """Sec. 3.1, Fig. 2 (acoustic-advection, c_s = 1): four parallel steps of 6
    slices, 5 iterations each, RK-3 coarse propagator.  The original Parareal
    grows by orders of magnitude, KSE-Parareal stays with the sequential fine
    solution; the GPU reproduces the oracle in both (the original's growth
    amplifies the rounding-order differences, hence its looser tolerance)."""
    p = W.demo_instability(40, 1.0)
    q0 = W.demo_initial_value(40).ravel()
    M = 4
    fine = q0
    for _ in range(M * p.n_slices):
        fine = oracle.fine_prop(p, fine)
    pt = dataclasses.replace(p, T=M * p.T)
    out = {}
    for variant, tol in (("original", 1e-6), ("kse", 1e-10)):
        want = oracle.parareal_windows(pt, q0, 5, M, variant=variant)["qT"]
        with solver(p, K_max=5, n_windows=M, variant=P.PR_KSE if variant == "kse" else P.PR_ORIGINAL) as s:
            qT = torch.empty(p.d, dtype=torch.float64, device="cuda")
            P.parareal_solve(s.h, dev(q0), 5, qT=qT)
            got = host(qT)
        assert rel(got, want) < tol, variant
        out[variant] = got
    assert np.abs(out["original"]).max() > 10 * np.abs(fine).max()
    assert np.abs(out["kse"]).max() < 1.1 * np.abs(fine).max()
    assert rel(out["kse"], fine) < 0.1


# ------------------------------------------------------------------ solid-body rotation

ROT_GRIDS = [("64x32", dict(nx=64, ny=32, N=4)), ("40x40", dict(nx=40, ny=40, N=3)),
             ("96x20", dict(nx=96, ny=20, N=3)), ("128x64", dict(nx=128, ny=64, N=2))]


def _rot(spec):
    """Rotation U = (pi/4) (y - 1/2, -(x - 1/2)) on top of a small constant U."""
    return dataclasses.replace(_prob(spec), U=0.05, omega=0.25 * np.pi)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32x"])
@pytest.mark.parametrize("name,spec", ROT_GRIDS, ids=[g[0] for g in ROT_GRIDS])
def test_fine_sweep_rotation(name, spec, prec):
    """Variable advection velocity (Eq. adVel): the x-velocity of each row and
    the y-velocity of each column, at the cell's periodic position."""
    p = _rot(spec)
    X = states(p, p.n_slices, 70)
    fp, tol = {"fp64": (P.PR_FP64, TOL64), "fp32": (P.PR_FP32, TOL32), "fp32x": (P.PR_FP32X, 2e-6)}[prec]
    with solver(p, fine_prec=fp) as s:
        out = torch.empty(p.n_slices * p.d, dtype=torch.float64, device="cuda")
        P.parareal_fine_sweep(s.h, dev(X), out, p.n_slices)
        got = host(out).reshape(p.n_slices, p.d)
    for i in range(p.n_slices):
        assert rel(got[i], oracle.fine_prop(p, X[i])) < tol


@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("name,spec", ROT_GRIDS, ids=[g[0] for g in ROT_GRIDS])
def test_coarse_apply_rotation(name, spec, scheme):
    p = _rot(spec)
    if scheme == 1:
        p = _rk3_coarse(p)
    X = states(p, p.n_slices, 71)
    with solver(p) as s:
        out = torch.empty(p.n_slices * p.d, dtype=torch.float64, device="cuda")
        P.parareal_coarse_apply(s.h, dev(X), out, p.n_slices)
        got = host(out).reshape(p.n_slices, p.d)
    for i in range(p.n_slices):
        assert rel(got[i], oracle.coarse_prop(p, X[i])) < TOL64


def test_paper_rotation_workload_matches_oracle():
    """The paper's own workload (solid-body rotation, c_s = 30, Sec. 3.2) for
    three parallel steps of N_p = 6 slices at C_c = 4 with 2 iterations each."""
    p = W.paper_rotation(40, 4.0, 6)
    q0 = W.paper_rotation_initial_value(40).ravel()
    M, K = 3, 2
    want = oracle.parareal_windows(dataclasses.replace(p, T=M * p.T), q0, K, M)
    with solver(p, K_max=K, n_windows=M) as s:
        qT = torch.empty(p.d, dtype=torch.float64, device="cuda")
        rep = P.parareal_solve(s.h, dev(q0), K, qT=qT)
        got = host(qT)
    assert rel(got, want["qT"]) < 1e-10
    assert list(rep.rank[:M * K]) == [int(x) for w in want["windows"] for x in w["rank"]]


@pytest.mark.parametrize("name,spec", GRIDS[1:], ids=[g[0] for g in GRIDS[1:]])
def test_solve_edge_grids(name, spec):
    p = _prob(spec)
    q0 = W.ic_fourier(p.nx, p.ny, seed=3, n_modes=4, kmax=3.0).ravel()
    K = min(2, p.n_slices)
    got, rep = _solve(p, q0, K)
    want = oracle.parareal(p, q0, K)
    assert rel(got, want["q"]) < TOL64
    assert list(rep.rank[:K]) == list(want["rank"])


def test_single_slice_one_iteration_is_fine():
    p = W.make_problem(64, 32, 1)
    q0 = W.ic_gaussian(64, 32, seed=1).ravel()
    got, _ = _solve(p, q0, 1)
    assert rel(got[1], oracle.fine_prop(p, q0)) < TOL64


def test_K_equals_N_is_serial_fine_bitwise():
    """Converged slices are exact: q_N^N equals N serial fine sweeps bit for bit."""
    p = W.make_problem(64, 32, 8)
    q0 = W.ic_gaussian(64, 32, seed=0).ravel()
    got, _ = _solve(p, q0, 8)
    with solver(p) as s:
        q = dev(q0)
        for i in range(p.n_slices):
            nxt = torch.empty_like(q)
            P.parareal_fine_sweep(s.h, q, nxt, 1)
            q = nxt
            assert np.array_equal(host(q), got[i + 1])
    assert rel(got, oracle.serial_fine(p, q0)) < TOL64


def test_solve_is_deterministic():
    p = W.make_problem(64, 32, 8)
    q0 = W.ic_gaussian(64, 32, seed=0).ravel()
    a, _ = _solve(p, q0, 3)
    b, _ = _solve(p, q0, 3)
    assert np.array_equal(a, b)


def test_solve_fp32_fine_accuracy():
    """Mixed precision (FP32 fine sweep): the error against the serial fine
    solution moves by at most 1e-5 relative."""
    wl = W.workload_small()
    p = wl.problem
    q0 = wl.ics[0][1]().ravel()
    qs = oracle.serial_fine(p, q0)
    for K in (1, 3):
        g32, _ = _solve(p, q0, K, fine_prec=P.PR_FP32)
        want = oracle.parareal(p, q0, K)
        e32 = oracle.rel_error(g32[-1], qs[-1])
        e64 = oracle.rel_error(want["q"][-1], qs[-1])
        assert abs(e32 - e64) <= 1e-5
        assert rel(g32, want["q"]) < 1e-5


@pytest.mark.parametrize("fine_prec", [0, 1, 2], ids=["fine64", "fine32", "fine32x"])
def test_solve_mixed_correction_accuracy(fine_prec):
    """FP32 correction by linearity (corr_prec = FP32): G(delta) + D Q^T delta
    with delta = q_i^{k+1} - q_i^k.  Its rounding scales with ||delta||, so the
    iterates stay within 1e-6 (FP64 fine) / 1e-5 (FP32 fine) of the FP64
    oracle and the error against the serial fine solution moves by <= 1e-5."""
    wl = W.workload_small()
    p = wl.problem
    q0 = wl.ics[0][1]().ravel()
    qs = oracle.serial_fine(p, q0)
    tol = 1e-6 if fine_prec == 0 else 1e-5
    for K in (1, 3, 5):
        got, rep = _solve(p, q0, K, fine_prec=fine_prec, corr_prec=1)
        want = oracle.parareal(p, q0, K)
        assert rel(got, want["q"]) < tol
        assert abs(oracle.rel_error(got[-1], qs[-1]) - oracle.rel_error(want["q"][-1], qs[-1])) <= 1e-5
        assert list(rep.rank[:K]) == list(want["rank"])
        assert np.allclose(np.array(rep.r[:K]), want["r"], rtol=1e-5)


def test_solve_mixed_K_equals_N_is_serial_fine_bitwise():
    """Converged slices stay exact in the FP32 delta form (delta = 0)."""
    p = W.make_problem(64, 32, 8)
    q0 = W.ic_gaussian(64, 32, seed=0).ravel()
    got, _ = _solve(p, q0, 8, fine_prec=1, corr_prec=1)
    with solver(p, fine_prec=1) as s:
        q = dev(q0)
        for i in range(p.n_slices):
            nxt = torch.empty_like(q)
            P.parareal_fine_sweep(s.h, q, nxt, 1)
            q = nxt
            assert np.array_equal(host(q), got[i + 1])


def test_early_stop_matches_oracle():
    """Stopping rule of Sec. 2.1: stop once r^k <= r_tol (same iteration count
    and result as the oracle)."""
    wl = W.workload_small()
    p = wl.problem
    q0 = wl.ics[0][1]().ravel()
    full = oracle.parareal(p, q0, 8)
    r_tol = 0.5 * (full["r"][2] + full["r"][3])        # between r^2 and r^3 -> stops after 4
    want = oracle.parareal(p, q0, 8, r_tol=r_tol)
    assert want["K"] == 4
    got, rep = _solve(p, q0, 8, r_tol=r_tol)
    assert rep.K == 4
    assert rel(got, want["q"]) < TOL64


def test_windows_match_oracle():
    """M_p = 3 parallel steps of N = 4 slices (Sec. 2.1), each started from the
    previous step's final value."""
    p = W.make_problem(64, 32, 4, T=0.5)               # one window: 4 slices of 0.125
    q0 = W.ic_gaussian(64, 32, seed=0).ravel()
    want = oracle.parareal_windows(p, q0, 2, 3)
    with solver(p, K_max=2, n_windows=3) as s:
        out = torch.empty(p.d, dtype=torch.float64, device="cuda")
        rep = P.parareal_solve(s.h, dev(q0), 2, qT=out)
        got = host(out)
    assert rep.n_windows == 3 and list(rep.K_window[:3]) == [2, 2, 2] and rep.K == 6
    assert rel(got, want["qT"]) < TOL64
    assert np.allclose(np.array(rep.r[:6]), np.concatenate([w["r"] for w in want["windows"]]), rtol=1e-9)


def test_solve_host_matches_device():
    p = W.make_problem(64, 32, 8)
    q0 = W.ic_gaussian(64, 32, seed=0).ravel()
    a, _ = _solve(p, q0, 2)
    with solver(p, K_max=2) as s:
        out = np.empty(p.d)
        rep = P.parareal_solve_host(s.h, np.ascontiguousarray(q0), 2, out)
    assert np.array_equal(out, a[-1])
    assert rep.K == 2 and rep.ms_total > 0


def test_invalid_calls_fail_cleanly():
    p = W.make_problem(64, 32, 8)
    with solver(p, K_max=2) as s:
        x = torch.zeros(p.d * 9, dtype=torch.float64, device="cuda")
        with pytest.raises(P.PararealError) as ei:
            P.parareal_solve(s.h, x, 3)
        assert ei.value.status == P.PR_EINVAL
        with pytest.raises(P.PararealError):
            P.parareal_fine_sweep(s.h, x, x, 9)
        with pytest.raises(P.PararealError):
            P.krylov_update(s.h, x, x, 0)
        # the handle still works after rejected calls
        P.parareal_solve(s.h, x, 1)


# ------------------------------------------------------------------ full size (256x128, N = 32, K = 6)

def test_full_size_sampled():
    """The benchmark's configuration: sampled outputs checked one by one
    against the oracle, plus properties that hold at any size."""
    wl = W.workload_medium()
    p = wl.problem
    K = wl.K
    q0 = wl.ics[0][1]().ravel()
    with solver(p, K_max=K, krylov_cap=wl.krylov_cap) as s:
        qall = torch.empty((p.n_slices + 1) * p.d, dtype=torch.float64, device="cuda")
        rep = P.parareal_solve(s.h, dev(q0), K, q_out=qall)
        got = host(qall).reshape(p.n_slices + 1, p.d)
        ranks = list(rep.rank[:K])
        assert all(0 < ranks[k] <= W.krylov_bound(p.n_slices, k + 1) for k in range(K)), ranks
        assert all(np.diff(ranks) > 0), ranks
        # converged slices i <= K are the serial fine solution
        qs = q0
        for i in range(1, K + 1):
            qs = oracle.fine_prop(p, qs)
            assert rel(got[i], qs) < TOL64
        # sampled fine and coarse images of final iterates
        for i in (K + 3, p.n_slices - 1):
            out = torch.empty(p.d, dtype=torch.float64, device="cuda")
            P.parareal_fine_sweep(s.h, dev(got[i]), out, 1)
            assert rel(host(out), oracle.fine_prop(p, got[i])) < TOL64
            P.parareal_coarse_apply(s.h, dev(got[i]), out, 1)
            assert rel(host(out), oracle.coarse_prop(p, got[i])) < TOL64
        # projector properties of S^K and F(P q) by linearity
        q = got[p.n_slices]
        Pq = torch.empty(p.d, dtype=torch.float64, device="cuda")
        FPq = torch.empty_like(Pq)
        P.krylov_project(s.h, dev(q), Pq, FPq)
        pq = host(Pq)
        PPq = torch.empty_like(Pq)
        P.krylov_project(s.h, Pq, PPq, None)
        assert rel(host(PPq), pq) < 1e-12
        assert abs(np.dot(q - pq, pq)) < 1e-12 * np.dot(q, q)
        assert rel(host(FPq), oracle.fine_prop(p, pq)) < 1e-11
