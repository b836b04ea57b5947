"""GPU parity of the serial chain on every tiling it takes: the coarse sweep
(the literal chain, q_{i+1} = G(q_i)) and KSE-Parareal solves (the chain in
delta form with the basis products) against the oracle, on grids whose
widths and heights are not multiples of the 16-column tiles, with first- and
third-order upwind slow tendencies (a 2- and a 3-cell ring around each
tile), the solid-body rotation (Eq. adVel), and SM limits that change the
tile shape (few CTAs: wider and taller tiles).  FP64 throughout: <= 1e-12
relative, ranks exact.
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)


def _rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _problem(nx, ny, N, order, rotation):
    p = W.make_problem(nx, ny, N, adv_order_c=order)
    if rotation:
        p = dataclasses.replace(p, U=0.05, omega=0.25 * np.pi)
    return p


CASES = [
    # (nx, ny, N): ragged in x (200 = 12 x 16 + 8) and y; a grid narrower than a tile
    (200, 72, 6),
    (64, 32, 8),
    (12, 10, 4),
]


@pytest.mark.parametrize("sm_limit", [0, 5, 24])
@pytest.mark.parametrize("rotation", [False, True], ids=["const", "rotation"])
@pytest.mark.parametrize("order", [1, 3])
@pytest.mark.parametrize("nx,ny,N", CASES, ids=[f"{c[0]}x{c[1]}_N{c[2]}" for c in CASES])
def test_coarse_sweep_chain(nx, ny, N, order, rotation, sm_limit):
    p = _problem(nx, ny, N, order, rotation)
    q0 = W.ic_random(nx, ny, seed=5).ravel()
    with P.Solver(p, stream=torch.cuda.current_stream(), sm_limit=sm_limit) as s:
        out = torch.empty(p.n_slices * p.d, dtype=torch.float64, device="cuda")
        P.parareal_coarse_sweep(s.h, torch.from_numpy(q0).cuda(), out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(p.n_slices, p.d)
    q = q0
    for i in range(p.n_slices):
        q = oracle.coarse_prop(p, q)
        assert _rel(got[i], q) < TOL64, (i, _rel(got[i], q))


@pytest.mark.parametrize("nx,ny,N", [(200, 72, 6), (15, 9, 4)], ids=["200x72_N6", "15x9_N4"])
@pytest.mark.parametrize("sm_limit", [0, 6])
@pytest.mark.parametrize("order", [1, 3])
@pytest.mark.parametrize("variant", ["kse", "original"])
def test_solve_chain_ragged(variant, order, sm_limit, nx, ny, N):
    """K = 3 iterations on ragged grids: the delta-form chain with the basis
    products (KSE) and the literal chain with K_old (original); 15 x 9 has
    an odd number of state values (d = 405), so the basis columns start at
    every 8-byte alignment and the tiles are narrower than one warp."""
    p = _problem(nx, ny, N, order, False)
    q0 = W.ic_gaussian(nx, ny, seed=3).ravel()
    K = 3
    with P.Solver(p, stream=torch.cuda.current_stream(), K_max=K, sm_limit=sm_limit,
                  variant=P.PR_KSE if variant == "kse" else P.PR_ORIGINAL) as s:
        qall = torch.empty((p.n_slices + 1) * p.d, dtype=torch.float64, device="cuda")
        rep = P.parareal_solve(s.h, torch.from_numpy(q0).cuda(), K, q_out=qall)
        torch.cuda.synchronize()
        got = qall.cpu().numpy().reshape(p.n_slices + 1, p.d)
    want = oracle.parareal(p, q0, K, variant=variant)
    assert _rel(got, want["q"]) < TOL64
    if variant == "kse":
        assert list(rep.rank[:K]) == list(want["rank"])
    assert np.allclose(np.array(rep.r[:K]), want["r"], rtol=1e-9)
