"""The subspace update and K(q_i^k) with the projections on the tensor cores
(proj_prec = PR_PROJ_SPLIT_BF16) against the CPU oracle.

The split-digit products are FP64-accurate (per term 2^-55 of the column
scales), so the same bounds as the FP64 path hold: iterates within 1e-11 of
the oracle on the well-conditioned workloads (the FP64 path reaches 1e-12
with its own summation order; the digit remainders add at most a few units
of 1e-15 per projection, amplified by at most 1/min kept ratio ~ 1e2..1e3
here), identical drop decisions and ranks, converged slices bit-exact.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_1510_02237_gb300")

pytestmark = pytest.mark.gpu

SPLIT = dict(proj_prec=1)
TOL = 1e-11


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
    a, b = np.ravel(a), np.ravel(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def solver(p, **opt):
    return P.Solver(p, stream=torch.cuda.current_stream(), **opt)


def _solve(p, q0, K, **opt):
    opt.setdefault("K_max", max(K, 1))
    with solver(p, **opt) as s:
        qall = torch.empty((p.n_slices + 1) * p.d, dtype=torch.float64, device="cuda")
        rep = P.parareal_solve(s.h, dev(q0), K, q_out=qall)
        return host(qall).reshape(p.n_slices + 1, p.d), rep


def test_krylov_update_and_project_split_match_oracle():
    """24 columns (two 16-column sub-blocks), with a dependent column and a
    duplicate straddling the sub-block boundary."""
    p = W.make_problem(64, 32, 24)
    rng = np.random.default_rng(11)
    X = np.stack([W.ic_random(64, 32, seed=100 + i).ravel() for i in range(24)])
    X[17] = 0.25 * X[3] - 3.0 * X[16]       # dependent on columns of both sub-blocks -> dropped
    X[20] = X[5]                            # duplicate -> dropped
    FX = np.stack([oracle.fine_prop(p, x) for x in X])
    B = oracle.Basis(p.d, 64)
    want = [B.add(X[j], FX[j])[0] for j in range(24)]
    with solver(p, **SPLIT) as s:
        kept = P.krylov_update(s.h, dev(X[:20]), dev(FX[:20]), 20)
        kept += P.krylov_update(s.h, dev(X[20:]), dev(FX[20:]), 4)
        assert kept == [int(k) for k in want]
        assert P.krylov_rank(s.h) == B.rank == 22
        for _ in range(3):
            q = rng.standard_normal(p.d)
            Pq = torch.empty(p.d, dtype=torch.float64, device="cuda")
            FPq = torch.empty_like(Pq)
            P.krylov_project(s.h, dev(q), Pq, FPq)
            wPq, wFPq = B.project(q)
            assert rel(host(Pq), wPq) < 1e-12
            assert rel(host(FPq), wFPq) < 1e-11


@pytest.mark.parametrize("K", [1, 3, 8])
def test_solve_split_matches_oracle_64x32(K):
    wl = W.workload_small()
    p = wl.problem
    q0 = wl.ics[0][1]().ravel()
    got, rep = _solve(p, q0, K, **SPLIT)
    want = oracle.parareal(p, q0, K)
    assert rel(got, want["q"]) < TOL
    assert list(rep.rank[:K]) == list(want["rank"])
    assert np.allclose(np.array(rep.r[:K]), want["r"], rtol=1e-9, atol=0)


@pytest.mark.parametrize("nx,ny,N,U,ic", [(40, 24, 4, 0.1, "fourier"), (96, 20, 3, -0.15, "fourier"),
                                           (128, 64, 20, 0.1, "gaussian")])
def test_solve_split_edge_grids(nx, ny, N, U, ic):
    """Ragged grids (d not a multiple of 32 or of 128), negative U, and N = 20
    (new columns spanning two sub-blocks).  The N = 20 case uses the Gaussian
    IC with noise: a few Fourier modes span only a low-dimensional space, so
    20 slices of iterates are nearly dependent and two correct FP64
    evaluations drift apart (the conditioning effect of Eq. Genhance)."""
    p = W.make_problem(nx, ny, N, U=U)
    if ic == "fourier":
        q0 = W.ic_fourier(nx, ny, seed=3, n_modes=4, kmax=3.0).ravel()
    else:
        q0 = W.ic_gaussian(nx, ny, seed=3).ravel()
    K = min(3, N)
    got, rep = _solve(p, q0, K, **SPLIT)
    want = oracle.parareal(p, q0, K)
    assert rel(got, want["q"]) < TOL
    assert list(rep.rank[:K]) == list(want["rank"])


def test_solve_split_K_equals_N_is_serial_fine_bitwise():
    p = W.make_problem(64, 32, 8)
    q0 = W.ic_gaussian(64, 32, seed=0).ravel()
    got, _ = _solve(p, q0, 8, **SPLIT)
    with solver(p) as s:
        q = dev(q0)
        for i in range(p.n_slices):
            nxt = torch.empty_like(q)
            P.parareal_fine_sweep(s.h, q, nxt, 1)
            q = nxt
            assert np.array_equal(host(q), got[i + 1])


def test_solve_split_is_deterministic():
    p = W.make_problem(128, 64, 20)
    q0 = W.ic_gaussian(128, 64, seed=2).ravel()
    a, _ = _solve(p, q0, 4, **SPLIT)
    b, _ = _solve(p, q0, 4, **SPLIT)
    assert np.array_equal(a, b)


def test_mixed_with_split_projection_accuracy():
    """The served mixed-precision form (FP32X fine, FP32 correction, direct
    images) with the split projection: ranks as the oracle's and the error
    against the serial fine solution within 1e-5 of the oracle's."""
    wl = W.workload_small()
    p = wl.problem
    q0 = wl.ics[0][1]().ravel()
    qs = oracle.serial_fine(p, q0)
    for K in (1, 3, 5):
        got, rep = _solve(p, q0, K, fine_prec=P.PR_FP32X, corr_prec=P.PR_FP32, **SPLIT)
        want = oracle.parareal(p, q0, K)
        assert rel(got, want["q"]) < 1e-5
        assert abs(oracle.rel_error(got[-1], qs[-1]) - oracle.rel_error(want["q"][-1], qs[-1])) <= 1e-5
        assert list(rep.rank[:K]) == list(want["rank"])


def test_split_rejects_d_not_multiple_of_8():
    p = W.make_problem(6, 4, 2)     # d = 72 is a multiple of 8; 6 x 6 gives d = 108
    p2 = W.make_problem(6, 6, 2)
    with pytest.raises(P.PararealError):
        solver(p2, **SPLIT)
    with solver(p, **SPLIT):
        pass
