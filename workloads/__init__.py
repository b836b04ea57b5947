"""Seeded synthetic workloads for the KSE-Parareal acoustic-advection solver.

This module is shared by the CPU oracle, the tests and the benchmark.  It
holds only problem *definitions* (grid, velocities, time-step rule) and
seeded initial conditions; none of the method's arithmetic (stencils,
propagators, Parareal, Krylov update) lives here.

Problem (Sec. 3, Eq. acousticAd): linear 2D acoustic-advection of the
fields (u, w, p) -- the paper's (u, v, pi) -- on a periodic rectangle,
cell-centred values, layout ``[field][y][x]`` with x contiguous.

Time-step rule (Sec. 2.1, Delta t = N_f * delta t, and the CFL numbers of
Eq. cflNumbers): the nominal fine step is
``dt_nom = cfl * min(dx, dy) / (|U| + c_s)``; with slice length
``DT = T / N`` the coarse steps per slice are
``N_g = ceil(DT / (ratio * dt_nom))``, the fine steps ``N_f = ratio * N_g``,
and ``dt_f = DT / N_f``, ``dt_g = ratio * dt_f`` exactly.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np


@dataclass
class Problem:
    """One KSE-Parareal problem instance (all physical / numerical parameters)."""
    nx: int
    ny: int
    U: float = 0.1
    V: float = 0.0
    c_s: float = 1.0
    T: float = 1.0
    n_slices: int = 8
    n_f: int = 20
    n_g: int = 2
    dt_f: float = 1.0 / 160.0
    dt_g: float = 1.0 / 16.0
    nu_f: float = 0.005      # fine divergence damping (Sec. 3.2)
    nu_c: float = 0.1        # coarse divergence damping (Fig. 3 / Tables 1-2)
    n_sound: int = 4         # acoustic substeps per coarse step
    adv_order_f: int = 6     # 6th-order centred advective flux in F
    adv_order_c: int = 1     # 1st-order upwind advective flux in G
    coarse_scheme: int = 0   # G: 0 split forward Euler / forward-backward, 1 RK-3
    omega: float = 0.0       # solid-body rotation rate (Eq. adVel): velocity
                             # (U + omega (y - ly/2), V - omega (x - lx/2))
    lx: float = 1.0
    ly: float = 1.0

    @property
    def ncell(self) -> int:
        return self.nx * self.ny

    @property
    def d(self) -> int:
        return 3 * self.nx * self.ny

    def as_dict(self) -> dict:
        return asdict(self)


def make_problem(nx: int, ny: int, n_slices: int, *, U: float = 0.1, V: float = 0.0,
                 c_s: float = 1.0, T: float = 1.0, cfl: float = 0.5, ratio: int = 10,
                 **kw) -> Problem:
    """Problem with the integer-step time-step rule described in the module docstring."""
    dx, dy = 1.0 / nx, 1.0 / ny
    dt_nom = cfl * min(dx, dy) / (math.hypot(U, V) + c_s)
    DT = T / n_slices
    n_g = max(1, math.ceil(DT / (ratio * dt_nom) - 1e-12))
    n_f = ratio * n_g
    dt_f = DT / n_f
    dt_g = DT / n_g
    return Problem(nx=nx, ny=ny, U=U, V=V, c_s=c_s, T=T, n_slices=n_slices,
                   n_f=n_f, n_g=n_g, dt_f=dt_f, dt_g=dt_g, **kw)


# ---------------------------------------------------------------- grids

def cell_centres(nx: int, ny: int, lx: float = 1.0, ly: float = 1.0):
    """Cell-centre coordinates x_i = (i + 1/2) dx, y_j = (j + 1/2) dy as [ny, nx] arrays."""
    x = (np.arange(nx) + 0.5) * (lx / nx)
    y = (np.arange(ny) + 0.5) * (ly / ny)
    return np.meshgrid(x, y, indexing="xy")  # X[j, i], Y[j, i]


# ---------------------------------------------------------------- initial conditions
# Every IC returns a float64 array of shape [3, ny, nx] = (u, w, p).

def ic_gaussian(nx: int, ny: int, seed: int = 0, sigma: float = 0.1,
                noise: float = 1e-3) -> np.ndarray:
    """Gaussian pressure bump (sigma at the domain centre) plus i.i.d. N(0, noise^2) on all fields."""
    X, Y = cell_centres(nx, ny)
    q = np.zeros((3, ny, nx))
    q[2] = np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2) / (2.0 * sigma ** 2))
    if noise > 0:
        rng = np.random.default_rng(seed)
        q += noise * rng.standard_normal(q.shape)
    return q


def _half_plane_modes(kmin: float, kmax: float):
    """Integer wavevectors (kx, ky) != 0 with kmin <= |k| <= kmax, one of each +-k pair."""
    out = []
    K = int(math.floor(kmax))
    for kx in range(0, K + 1):
        for ky in range(-K, K + 1):
            if kx == 0 and ky <= 0:
                continue
            r = math.hypot(kx, ky)
            if kmin - 1e-12 <= r <= kmax + 1e-12:
                out.append((kx, ky))
    return out


def ic_fourier(nx: int, ny: int, seed: int = 1, n_modes: int = 8, kmax: float = 8.0) -> np.ndarray:
    """Sum of ``n_modes`` random-phase Fourier modes with |k| <= kmax, drawn independently per field."""
    X, Y = cell_centres(nx, ny)
    rng = np.random.default_rng(seed)
    modes = _half_plane_modes(1.0, kmax)
    q = np.zeros((3, ny, nx))
    for f in range(3):
        pick = rng.choice(len(modes), size=n_modes, replace=False)
        phases = rng.uniform(0.0, 2.0 * math.pi, size=n_modes)
        for m, ph in zip(pick, phases):
            kx, ky = modes[m]
            q[f] += np.cos(2.0 * math.pi * (kx * X + ky * Y) + ph)
    return q


def ic_filtered_noise(nx: int, ny: int, seed: int = 2, kmax: float = 16.0) -> np.ndarray:
    """White noise low-pass filtered to |k| <= kmax (FFT), scaled to unit RMS per field."""
    rng = np.random.default_rng(seed)
    q = rng.standard_normal((3, ny, nx))
    kx = np.fft.fftfreq(nx, d=1.0 / nx)
    ky = np.fft.fftfreq(ny, d=1.0 / ny)
    KX, KY = np.meshgrid(kx, ky, indexing="xy")
    mask = np.hypot(KX, KY) <= kmax + 1e-12
    for f in range(3):
        h = np.fft.fft2(q[f])
        h[~mask] = 0.0
        g = np.real(np.fft.ifft2(h))
        q[f] = g / np.sqrt(np.mean(g ** 2))
    return q


def ic_power_law(nx: int, ny: int, seed: int = 0, kmax: float = 16.0, power: float = 2.0) -> np.ndarray:
    """All modes 1 <= |k| <= kmax with amplitude |k|^-power and random phase, independently per field."""
    X, Y = cell_centres(nx, ny)
    rng = np.random.default_rng(seed)
    modes = _half_plane_modes(1.0, kmax)
    q = np.zeros((3, ny, nx))
    for f in range(3):
        phases = rng.uniform(0.0, 2.0 * math.pi, size=len(modes))
        for (kx, ky), ph in zip(modes, phases):
            q[f] += math.hypot(kx, ky) ** (-power) * np.cos(2.0 * math.pi * (kx * X + ky * Y) + ph)
    return q


def ic_cosine_bell(nx: int, ny: int, x0: float = 0.5, y0: float = 0.5) -> np.ndarray:
    """Cosine bell on u (Eq. advectionIni with Eq. defR), w = p = 0."""
    X, Y = cell_centres(nx, ny)
    r = np.minimum(1.0, 4.0 * np.sqrt((X - x0) ** 2 / 0.25 + (Y - y0) ** 2 / 0.25))
    q = np.zeros((3, ny, nx))
    q[0] = 0.5 * (np.cos(math.pi * r) + 1.0)
    return q


def ic_random(nx: int, ny: int, seed: int = 0) -> np.ndarray:
    """i.i.d. N(0,1) on every cell and field (used for edge cases and linearity checks)."""
    return np.random.default_rng(seed).standard_normal((3, ny, nx))


# ---------------------------------------------------------------- named workloads

@dataclass
class Workload:
    name: str
    problem: Problem
    K: int
    ics: list = field(default_factory=list)   # list of (label, callable -> ndarray)
    krylov_cap: int = 0                        # 0 => no cap beyond the natural bound
    fine_prec: str = "f64"
    proj_prec: str = "f64"


def workload_small() -> Workload:
    """64x32 grid, N = 8 slices, K up to 8, Gaussian bump + N(0, 1e-3^2) noise (seed 0), FP64."""
    p = make_problem(64, 32, 8)
    return Workload("fp64_64x32_N8", p, K=8, ics=[("gaussian+noise", lambda: ic_gaussian(64, 32, seed=0))])


def workload_medium() -> Workload:
    """256x128 grid, N = 32 slices, K = 6, Krylov cap 192, three seeded ICs, FP64."""
    p = make_problem(256, 128, 32)
    nx, ny = 256, 128
    return Workload("fp64_256x128_N32_K6", p, K=6, krylov_cap=192, ics=[
        ("gaussian+noise", lambda: ic_gaussian(nx, ny, seed=0)),
        ("fourier8", lambda: ic_fourier(nx, ny, seed=1)),
        ("filtered_noise16", lambda: ic_filtered_noise(nx, ny, seed=2)),
    ])


def workload_large() -> Workload:
    """512x256 grid, N = 64 slices, K = 5, power-law Fourier IC (seed 0); FP32 fine / FP64 Krylov."""
    p = make_problem(512, 256, 64)
    return Workload("mixed_512x256_N64_K5", p, K=5, fine_prec="f32",
                    ics=[("powerlaw16", lambda: ic_power_law(512, 256, seed=0))])


def demo_instability(nx: int = 40, c_s: float = 1.0, n_slices: int = 6) -> Problem:
    """The instability demonstration of Sec. 3.1 (Figs. 1, 2): nx x nx cells on
    the unit square, U = (1, 1), RK-3 coarse propagator with first-order upwind
    fluxes and C_c = U dt_g / dx = 0.6, RK-3 fine propagator with sixth-order
    fluxes and C_f = 0.1 (six fine steps per coarse step), one coarse step per
    time slice, N_p = 6 slices per parallel step, no divergence damping;
    c_s = 0 is the pure-advection case.  T is the length of one parallel step."""
    dt_g = 0.6 / nx
    return Problem(nx=nx, ny=nx, U=1.0, V=1.0, c_s=c_s, T=n_slices * dt_g, n_slices=n_slices, n_f=6, n_g=1,
                   dt_f=dt_g / 6, dt_g=dt_g, nu_f=0.0, nu_c=0.0, adv_order_c=1, coarse_scheme=1)


def demo_initial_value(nx: int = 40) -> np.ndarray:
    """Cosine bell in u centred at (0.5, 0.5) (Sec. 3.1); w = p = 0."""
    q0 = np.zeros((3, nx, nx))
    q0[0] = ic_cosine_bell(nx, nx)[0]
    return q0


def paper_rotation(nx: int = 40, C_c: float = 2.0, N_p: int = 6, C_f: float = 0.2) -> Problem:
    """The paper's acoustic-advection workload (Sec. 3.2, Eq. adVel; Tables
    1-2, Figs. 3-10): solid-body rotation U = pi (y - 1/2, -(x - 1/2)) on the
    unit square with nx x nx cells, c_s = 30, fine RK-3 with sixth-order
    advective fluxes at C_f = c_s dt / dx = 0.2 (Eq. cflNumbers) and
    nu_f = 0.005, coarse partially split forward Euler with first-order upwind
    fluxes at C_c = c_s Delta t / dx, N_sound = 4 and nu_c = 0.1.  A time slice
    is one coarse step ("coarse interval") and a parallel step has N_p of them;
    T is the length of one parallel step, so [0, 2] takes 2 / T of them."""
    dx = 1.0 / nx
    dt_g = C_c * dx / 30.0
    n_f = int(round(C_c / C_f))
    return Problem(nx=nx, ny=nx, U=0.0, V=0.0, c_s=30.0, T=N_p * dt_g, n_slices=N_p, n_f=n_f, n_g=1,
                   dt_f=dt_g / n_f, dt_g=dt_g, nu_f=0.005, nu_c=0.1, n_sound=4, adv_order_f=6, adv_order_c=1,
                   omega=math.pi)


def paper_rotation_initial_value(nx: int = 40) -> np.ndarray:
    """Cosine bell in u centred at (0.5, 0.65) (Sec. 3.2); w = p = 0."""
    q0 = np.zeros((3, nx, nx))
    q0[0] = ic_cosine_bell(nx, nx, 0.5, 0.65)[0]
    return q0


def krylov_bound(n_slices: int, K: int) -> int:
    """Natural bound on dim S^k after K iterations: sum_{k<K} (N - k) new columns."""
    return sum(n_slices - k for k in range(K))


# ---------------------------------------------------------------- batches and request streams

@dataclass
class Instance:
    """One independent solve of a batch or a request stream."""
    problem: Problem
    K: int
    ic: str              # "gaussian" or "fourier"
    seed: int

    def initial_value(self) -> np.ndarray:
        nx, ny = self.problem.nx, self.problem.ny
        if self.ic == "gaussian":
            return ic_gaussian(nx, ny, seed=self.seed)
        return ic_fourier(nx, ny, seed=self.seed, n_modes=8, kmax=8.0)


def workload_batch(n: int = 64, seed: int = 1000):
    """n independent instances: grid uniform in {64x32, 128x64, 256x128},
    N uniform in {8, 16, 32}, K uniform in 1..N/2, U uniform in [0.05, 0.2],
    c_s = 1; instance i uses seed 1000+i, Gaussian IC for even i, Fourier
    modes for odd i."""
    rng = np.random.default_rng(seed)
    grids = [(64, 32), (128, 64), (256, 128)]
    out = []
    for i in range(n):
        nx, ny = grids[rng.integers(0, 3)]
        N = int(rng.choice([8, 16, 32]))
        K = int(rng.integers(1, N // 2 + 1))
        U = float(rng.uniform(0.05, 0.2))
        p = make_problem(nx, ny, N, U=U)
        out.append(Instance(p, K, "gaussian" if i % 2 == 0 else "fourier", seed + i))
    return out


def request_stream(rate: float, n: int, seed: int = 7):
    """Poisson request stream: exponential inter-arrival times of mean 1/rate
    seconds; each request draws a grid uniform in {64x32, 128x64, 256x128,
    512x256}, N uniform in {8, 16, 32, 64}, K uniform in 1..5 (K <= N), U = 0.1,
    c_s = 1, and a seeded Gaussian or Fourier IC.  Returns (arrival_s, Instance)."""
    rng = np.random.default_rng(seed)
    grids = [(64, 32), (128, 64), (256, 128), (512, 256)]
    t = 0.0
    out = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate))
        nx, ny = grids[rng.integers(0, 4)]
        N = int(rng.choice([8, 16, 32, 64]))
        K = int(min(N, rng.integers(1, 6)))
        p = make_problem(nx, ny, N)
        out.append((t, Instance(p, K, "gaussian" if rng.integers(0, 2) == 0 else "fourier", seed * 100000 + i)))
    return out
