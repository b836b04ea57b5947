"""CPU oracle for KSE-Parareal on the linear 2D acoustic-advection system.

TEST INFRASTRUCTURE ONLY: a plain, slow, serial FP64 implementation written
from the paper (Ruprecht & Krause, arXiv 1510.02237).  Only the tests, the
smoke check and the benchmark's CPU-baseline leg may import it.  It shares no
code with the CUDA path; the only common module is ``workloads`` (problem
parameters and seeded initial conditions, no method arithmetic).

Functions and the passages they follow:
  fine_rhs / fine_steps / fine_prop   -- Sec. 3 flux form, RK-3 fine propagator F
  coarse_steps / coarse_prop          -- Sec. 3.2 partially split forward Euler with
                                         forward-backward acoustic substeps, G
  Basis                               -- Sec. 2.2 subspace S^k, its orthonormal basis
                                         (Householder QR, Eq. subspaceUpdate) and the
                                         fine images used in Eq. Genhance
  parareal                            -- Alg. 2 (KSE-Parareal) and Alg. 1 (original)
  serial_fine                         -- the sequential fine solution q_seq
  rel_error                           -- Eq. errorDef
  set_threads                         -- OpenMP threads of Alg. 2's parallel predictor
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from ._build import build as _build_lib

_lib = None


class _Problem(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("lx", C.c_double), ("ly", C.c_double),
                ("U", C.c_double), ("V", C.c_double), ("cs", C.c_double),
                ("nu_f", C.c_double), ("nu_c", C.c_double), ("n_sound", C.c_int),
                ("dt_f", C.c_double), ("dt_g", C.c_double), ("n_f", C.c_int), ("n_g", C.c_int),
                ("n_slices", C.c_int), ("adv_order_f", C.c_int), ("adv_order_c", C.c_int),
                ("coarse_scheme", C.c_int), ("omega", C.c_double)]


_P = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


def lib():
    global _lib
    if _lib is None:
        path = _build_lib()
        L = C.CDLL(path)
        pp = C.POINTER(_Problem)
        for name in ("orc_fine_rhs",):
            getattr(L, name).argtypes = [pp, _P, _P]
        L.orc_fine_steps.argtypes = [pp, _P, _P, C.c_int]
        L.orc_fine_prop.argtypes = [pp, _P, _P]
        L.orc_coarse_steps.argtypes = [pp, _P, _P, C.c_int]
        L.orc_coarse_prop.argtypes = [pp, _P, _P]
        L.orc_basis_create.argtypes = [C.c_long, C.c_int]
        L.orc_basis_create.restype = C.c_void_p
        L.orc_basis_free.argtypes = [C.c_void_p]
        L.orc_basis_rank.argtypes = [C.c_void_p]
        L.orc_basis_rank.restype = C.c_int
        L.orc_basis_add.argtypes = [C.c_void_p, _P, _P, C.c_double, _P]
        L.orc_basis_add.restype = C.c_int
        L.orc_basis_get_q.argtypes = [C.c_void_p, _P]
        L.orc_basis_get_fq.argtypes = [C.c_void_p, _P]
        L.orc_basis_project.argtypes = [C.c_void_p, _P, _P, _P]
        L.orc_parareal.argtypes = [pp, _P, C.c_int, C.c_int, C.c_double, C.c_int, C.c_double, _P, _P, _I, _I, _P]
        L.orc_parareal.restype = C.c_int
        L.orc_serial_fine.argtypes = [pp, _P, _P]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_set_threads.restype = C.c_int
        _lib = L
    return _lib


def _problem(p, **over) -> _Problem:
    """Marshal a ``workloads.Problem`` (or any object with the same attributes)."""
    g = lambda k, dflt=None: over.get(k, getattr(p, k, dflt))
    return _Problem(int(g("nx")), int(g("ny")), float(g("lx", 1.0)), float(g("ly", 1.0)),
                    float(g("U")), float(g("V", 0.0)), float(g("c_s")),
                    float(g("nu_f")), float(g("nu_c")), int(g("n_sound")),
                    float(g("dt_f")), float(g("dt_g")), int(g("n_f")), int(g("n_g")),
                    int(g("n_slices")), int(g("adv_order_f", 6)), int(g("adv_order_c", 1)),
                    int(g("coarse_scheme", 0)), float(g("omega", 0.0)))


def _arr(x, d=None):
    a = np.ascontiguousarray(x, dtype=np.float64)
    if d is not None:
        assert a.size == d, (a.size, d)
    return a


def _ptr(a):
    return a.ctypes.data_as(_P)


def fine_rhs(p, q, **over):
    pb = _problem(p, **over)
    q = _arr(q, 3 * pb.nx * pb.ny)
    out = np.empty_like(q)
    lib().orc_fine_rhs(C.byref(pb), _ptr(q), _ptr(out))
    return out


def fine_steps(p, q, nsteps, **over):
    pb = _problem(p, **over)
    q = _arr(q, 3 * pb.nx * pb.ny)
    out = np.empty_like(q)
    lib().orc_fine_steps(C.byref(pb), _ptr(q), _ptr(out), int(nsteps))
    return out


def fine_prop(p, q, **over):
    pb = _problem(p, **over)
    return fine_steps(p, q, pb.n_f, **over)


def coarse_steps(p, q, nsteps, **over):
    pb = _problem(p, **over)
    q = _arr(q, 3 * pb.nx * pb.ny)
    out = np.empty_like(q)
    lib().orc_coarse_steps(C.byref(pb), _ptr(q), _ptr(out), int(nsteps))
    return out


def coarse_prop(p, q, **over):
    pb = _problem(p, **over)
    return coarse_steps(p, q, pb.n_g, **over)


class Basis:
    """Orthonormal basis of S^k with the fine images of its vectors (Sec. 2.2)."""

    def __init__(self, d: int, cap: int):
        self.d = int(d)
        self._h = lib().orc_basis_create(self.d, int(cap))

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_basis_free(self._h)
            self._h = None

    @property
    def rank(self) -> int:
        return lib().orc_basis_rank(self._h)

    def add(self, a, fa, eta: float = 1e-10):
        a = _arr(a, self.d)
        fa = _arr(fa, self.d)
        r = C.c_double(0.0)
        kept = lib().orc_basis_add(self._h, _ptr(a), _ptr(fa), float(eta), C.byref(r))
        return bool(kept), r.value

    def Q(self):
        out = np.empty((self.rank, self.d))
        lib().orc_basis_get_q(self._h, _ptr(out))
        return out.T

    def FQ(self):
        out = np.empty((self.rank, self.d))
        lib().orc_basis_get_fq(self._h, _ptr(out))
        return out.T

    def project(self, q):
        q = _arr(q, self.d)
        Pq, FPq = np.empty_like(q), np.empty_like(q)
        lib().orc_basis_project(self._h, _ptr(q), _ptr(Pq), _ptr(FPq))
        return Pq, FPq


def parareal(p, q0, K: int, *, variant: str = "kse", eta: float = 1e-10, cap: int = 0, r_tol: float = 0.0,
             **over):
    """Run Alg. 2 (``variant='kse'``) or Alg. 1 (``'original'``) for K iterations
    (fewer if r_tol > 0 and r^k <= r_tol first, Sec. 2.1).

    Returns dict(q=(N+1, d) iterates q_n^K, r=(K,) error estimates r^k,
    rank=(K,) dim S^k, kept=(K, N) column kept flags, ratio=(K, N) |R_jj|/||a_j||,
    K=iterations performed).
    """
    pb = _problem(p, **over)
    N, d = pb.n_slices, 3 * pb.nx * pb.ny
    q0 = _arr(q0, d)
    if cap <= 0:
        cap = max(1, N * max(K, 1))
    q_all = np.empty((N + 1, d))
    r = np.zeros(max(K, 1))
    rank = np.zeros(max(K, 1), dtype=np.int32)
    kept = np.zeros((max(K, 1), N), dtype=np.int32)
    ratio = np.zeros((max(K, 1), N))
    rc = lib().orc_parareal(C.byref(pb), _ptr(q0), int(K), 0 if variant == "kse" else 1, float(eta),
                            int(cap), float(r_tol), _ptr(q_all), _ptr(r), rank.ctypes.data_as(_I),
                            kept.ctypes.data_as(_I), _ptr(ratio))
    if rc < 0:
        raise MemoryError("oracle parareal: allocation failed")
    Kd = rc
    return dict(q=q_all, r=r[:Kd], rank=rank[:Kd], kept=kept[:Kd], ratio=ratio[:Kd], K=Kd)


def parareal_windows(p, q0, K: int, n_windows: int, **kw):
    """[0, T] as n_windows consecutive parallel steps of N slices each (Sec. 2.1:
    M_p parallel steps of N_c = N_p coarse intervals), each solved by
    ``parareal`` from the previous step's final value; the problem's T is the
    end time of the whole run.  Returns the final value, and per window the
    iterations performed and the r^k history."""
    import dataclasses
    pw = dataclasses.replace(p, T=p.T / n_windows) if dataclasses.is_dataclass(p) else p
    q = _arr(q0)
    wins = []
    for _ in range(n_windows):
        r = parareal(pw, q, K, **kw)
        wins.append(r)
        q = r["q"][-1].copy()
    return dict(qT=q, windows=wins)


def set_threads(n: int) -> int:
    """Host threads of the parallel predictor (OpenMP over slices, Sec. 2.1);
    1 runs it serially.  Results do not depend on it.  Returns the previous value."""
    return int(lib().orc_set_threads(int(n)))


def serial_fine(p, q0, **over):
    """q_n = F^n(q0), n = 0..N: the sequential fine solution."""
    pb = _problem(p, **over)
    d = 3 * pb.nx * pb.ny
    q0 = _arr(q0, d)
    out = np.empty((pb.n_slices + 1, d))
    lib().orc_serial_fine(C.byref(pb), _ptr(q0), _ptr(out))
    return out


def rel_error(q_par, q_seq) -> float:
    """Relative l2 error over all three fields (Eq. errorDef)."""
    q_par = np.asarray(q_par, dtype=np.float64).ravel()
    q_seq = np.asarray(q_seq, dtype=np.float64).ravel()
    return float(np.linalg.norm(q_par - q_seq) / np.linalg.norm(q_seq))
