"""Python binding of the GB300 KSE-Parareal library (``libparareal.so``).

Thin ctypes marshalling over the C ABI declared in ``include/parareal.h``;
every step of the computation runs in the library's CUDA kernels.  PyTorch
is used only for device memory (tensors passed by pointer) and streams.
Importing this module loads the in-tree library and raises if it has not
been built -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libparareal.so")

PR_OK, PR_EINVAL, PR_ENOMEM, PR_ECUDA, PR_ETIMEOUT, PR_ESTATE, PR_ECANCELLED = 0, -1, -2, -3, -4, -5, -6
PR_FP64, PR_FP32, PR_FP32X = 0, 1, 2
PR_KSE, PR_ORIGINAL = 0, 1
PR_IMAGES_LINEARITY, PR_IMAGES_DIRECT = 0, 1
PR_PROJ_FP64, PR_PROJ_SPLIT_BF16 = 0, 1
PR_COARSE_SPLIT_FE, PR_COARSE_RK3 = 0, 1
PR_BATCH_STREAMS, PR_BATCH_PERSISTENT = 0, 1
PR_MAX_ITERS = 128
_STATUS = {0: "PR_OK", -1: "PR_EINVAL", -2: "PR_ENOMEM", -3: "PR_ECUDA", -4: "PR_ETIMEOUT",
           -5: "PR_ESTATE", -6: "PR_ECANCELLED"}


class pr_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("lx", C.c_double), ("ly", C.c_double)]


class pr_options(C.Structure):
    _fields_ = [("T", C.c_double), ("nu_f", C.c_double), ("nu_c", C.c_double), ("n_sound", C.c_int32),
                ("adv_order_f", C.c_int32), ("adv_order_c", C.c_int32), ("V", C.c_double),
                ("K_max", C.c_int32), ("krylov_cap", C.c_int32), ("drop_tol", C.c_double),
                ("fine_prec", C.c_int32), ("variant", C.c_int32), ("corr_prec", C.c_int32),
                ("r_tol", C.c_double), ("n_windows", C.c_int32), ("images", C.c_int32),
                ("sm_limit", C.c_int32), ("stream", C.c_void_p), ("proj_prec", C.c_int32),
                ("coarse_scheme", C.c_int32), ("omega", C.c_double), ("batch_fine", C.c_int32)]


class pr_report(C.Structure):
    _fields_ = [("K", C.c_int32), ("rank", C.c_int32 * PR_MAX_ITERS), ("r", C.c_double * PR_MAX_ITERS),
                ("ms_total", C.c_float), ("n_windows", C.c_int32), ("K_window", C.c_int32 * PR_MAX_ITERS),
                ("min_ratio", C.c_double * PR_MAX_ITERS)]


class pr_timing(C.Structure):
    _fields_ = [("n_solves", C.c_int32), ("ms_init", C.c_double), ("ms_fine", C.c_double),
                ("ms_coarse", C.c_double), ("ms_krylov", C.c_double), ("ms_gs_block", C.c_double),
                ("ms_gs_intra", C.c_double), ("ms_kold", C.c_double), ("ms_chain", C.c_double),
                ("ms_total", C.c_double), ("fine_cell_steps", C.c_double), ("fine_launches", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pr_tuning(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("choice", C.c_int32), ("cached", C.c_int32), ("n_candidates", C.c_int32),
                ("candidates", C.c_int32 * 8), ("us_per_step", C.c_float * 8)]

    def as_dict(self):
        n = self.n_candidates
        return {"kernel": ["none", "tile", "rows"][self.kernel], "choice": self.choice, "cached": bool(self.cached),
                "candidates": list(self.candidates[:n]), "us_per_step": [float(x) for x in self.us_per_step[:n]]}


class PararealError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


EXPORTS = ["parareal_default_options", "parareal_create", "parareal_destroy", "parareal_last_error",
           "parareal_footprint_bytes", "parareal_solve", "parareal_solve_host", "parareal_fine_sweep",
           "parareal_coarse_sweep", "parareal_coarse_apply", "krylov_reset", "krylov_update", "krylov_rank",
           "krylov_project", "parareal_timing_enable", "parareal_timing_read", "parareal_kernel_launches",
           "parareal_alu_probe", "parareal_fine_sweep_static", "parareal_selftest_wait_timeout",
           "parareal_solve_batch", "parareal_batch_create", "parareal_batch_launch", "parareal_batch_destroy",
           "parareal_split_gemm_tn", "parareal_split_gemm_nn", "parareal_autotune", "parareal_status"]

_lib = None


def lib():
    """Load ``libparareal.so`` (raises if missing: build it with ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} not built; run python -c 'import __graft_entry__ as g; g.build()'")
    L = C.CDLL(LIB_PATH)
    P = C.c_void_p
    st = C.c_int
    L.parareal_default_options.argtypes = [C.POINTER(pr_options)]
    L.parareal_default_options.restype = st
    L.parareal_create.argtypes = [C.POINTER(pr_grid), C.c_double, C.c_double, C.c_double, C.c_double,
                                  C.c_int32, C.POINTER(pr_options), C.POINTER(P)]
    L.parareal_create.restype = st
    L.parareal_destroy.argtypes = [P]
    L.parareal_destroy.restype = st
    L.parareal_last_error.argtypes = [P]
    L.parareal_last_error.restype = C.c_char_p
    L.parareal_footprint_bytes.argtypes = [C.POINTER(pr_grid), C.c_int32, C.POINTER(pr_options)]
    L.parareal_footprint_bytes.restype = C.c_size_t
    L.parareal_solve.argtypes = [P, P, C.c_int32, P, P, C.POINTER(pr_report)]
    L.parareal_solve.restype = st
    L.parareal_solve_host.argtypes = [P, P, C.c_int32, P, C.POINTER(pr_report)]
    L.parareal_solve_host.restype = st
    L.parareal_fine_sweep.argtypes = [P, P, P, C.c_int32]
    L.parareal_fine_sweep.restype = st
    L.parareal_coarse_sweep.argtypes = [P, P, P]
    L.parareal_coarse_sweep.restype = st
    L.parareal_coarse_apply.argtypes = [P, P, P, C.c_int32]
    L.parareal_coarse_apply.restype = st
    L.krylov_reset.argtypes = [P]
    L.krylov_reset.restype = st
    L.krylov_update.argtypes = [P, P, P, C.c_int32, C.POINTER(C.c_int32)]
    L.krylov_update.restype = st
    L.krylov_rank.argtypes = [P, C.POINTER(C.c_int32)]
    L.krylov_rank.restype = st
    L.krylov_project.argtypes = [P, P, P, P]
    L.krylov_project.restype = st
    L.parareal_timing_enable.argtypes = [P, C.c_int32]
    L.parareal_timing_enable.restype = st
    L.parareal_timing_read.argtypes = [P, C.POINTER(pr_timing), C.c_int32]
    L.parareal_timing_read.restype = st
    L.parareal_autotune.argtypes = [P, C.POINTER(pr_tuning)]
    L.parareal_autotune.restype = st
    L.parareal_status.argtypes = [P]
    L.parareal_status.restype = st
    L.parareal_kernel_launches.argtypes = []
    L.parareal_kernel_launches.restype = C.c_uint64
    L.parareal_alu_probe.argtypes = [C.c_int32, C.c_int32, C.POINTER(C.c_double)]
    L.parareal_alu_probe.restype = st
    L.parareal_fine_sweep_static.argtypes = [C.POINTER(pr_grid), C.c_double, C.c_double, C.c_double, C.c_double,
                                             C.c_double, C.c_int32, C.c_int32, P, P, C.c_int32, P]
    L.parareal_fine_sweep_static.restype = st
    L.parareal_selftest_wait_timeout.argtypes = [P, C.POINTER(C.c_double)]
    L.parareal_selftest_wait_timeout.restype = st
    PP = C.POINTER(C.c_void_p)
    L.parareal_solve_batch.argtypes = [PP, C.c_int32, PP, C.POINTER(C.c_int32), PP]
    L.parareal_solve_batch.restype = st
    L.parareal_batch_create.argtypes = [PP, C.c_int32, PP, C.POINTER(C.c_int32), PP, P, C.POINTER(P)]
    L.parareal_batch_create.restype = st
    L.parareal_batch_launch.argtypes = [P]
    L.parareal_batch_launch.restype = st
    L.parareal_batch_destroy.argtypes = [P]
    L.parareal_batch_destroy.restype = st
    i64, i32 = C.c_int64, C.c_int32
    for name in ("parareal_split_gemm_tn", "parareal_split_gemm_nn"):
        f = getattr(L, name)
        f.argtypes = [P, i64, i32, P, i64, i32, i64, P, i64, P]
        f.restype = st
    _lib = L
    return L


def _ptr(t):
    """Device (or host) address of a tensor / array, or None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return C.c_void_p(t.data_ptr())
    if hasattr(t, "ctypes"):
        return C.c_void_p(t.ctypes.data)
    return C.c_void_p(int(t))


def _check(h, status):
    if status != PR_OK:
        msg = lib().parareal_last_error(h)
        raise PararealError(status, msg.decode() if msg else "")


def parareal_default_options(**over) -> pr_options:
    o = pr_options()
    lib().parareal_default_options(C.byref(o))
    for k, v in over.items():
        setattr(o, k, v)
    return o


def parareal_footprint_bytes(nx, ny, N, **opt) -> int:
    return int(lib().parareal_footprint_bytes(C.byref(pr_grid(nx, ny, 1.0, 1.0)), int(N),
                                              C.byref(parareal_default_options(**opt))))


def parareal_create(nx, ny, U, c_s, dt_f, dt_g, N_slices, *, stream=None, **opt):
    """Returns an opaque handle (int).  ``stream``: a ``torch.cuda.Stream``/raw handle or None."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    o = parareal_default_options(**opt)
    o.stream = C.c_void_p(stream) if stream else None
    h = C.c_void_p()
    _check(None, lib().parareal_create(C.byref(pr_grid(nx, ny, 1.0, 1.0)), float(U), float(c_s), float(dt_f),
                                       float(dt_g), int(N_slices), C.byref(o), C.byref(h)))
    return h


def parareal_destroy(h):
    _check(h, lib().parareal_destroy(h))


def parareal_last_error(h) -> str:
    m = lib().parareal_last_error(h)
    return m.decode() if m else ""


def parareal_solve(h, u0, K, q_out=None, qT=None, report=True):
    rep = pr_report() if report else None
    _check(h, lib().parareal_solve(h, _ptr(u0), int(K), _ptr(q_out), _ptr(qT),
                                   C.byref(rep) if rep is not None else None))
    return rep


def parareal_solve_host(h, u0_host, K, qT_host, report=True):
    rep = pr_report() if report else None
    _check(h, lib().parareal_solve_host(h, _ptr(u0_host), int(K), _ptr(qT_host),
                                        C.byref(rep) if rep is not None else None))
    return rep


def parareal_status(h):
    """Synchronise the handle's stream; raise if a device-side wait gave up."""
    _check(h, lib().parareal_status(h))


def parareal_fine_sweep(h, q_in, q_out, n):
    _check(h, lib().parareal_fine_sweep(h, _ptr(q_in), _ptr(q_out), int(n)))


def parareal_coarse_sweep(h, q0, q_out):
    _check(h, lib().parareal_coarse_sweep(h, _ptr(q0), _ptr(q_out)))


def parareal_coarse_apply(h, q_in, q_out, n):
    _check(h, lib().parareal_coarse_apply(h, _ptr(q_in), _ptr(q_out), int(n)))


def krylov_reset(h):
    _check(h, lib().krylov_reset(h))


def krylov_update(h, V, FV, m, want_kept=True):
    kept = (C.c_int32 * int(m))() if want_kept else None
    _check(h, lib().krylov_update(h, _ptr(V), _ptr(FV), int(m), kept))
    return list(kept) if want_kept else None


def krylov_rank(h) -> int:
    r = C.c_int32()
    _check(h, lib().krylov_rank(h, C.byref(r)))
    return r.value


def krylov_project(h, q, Pq=None, FPq=None):
    _check(h, lib().krylov_project(h, _ptr(q), _ptr(Pq), _ptr(FPq)))


def parareal_timing_enable(h, max_solves):
    _check(h, lib().parareal_timing_enable(h, int(max_solves)))


def parareal_timing_read(h, reset=True) -> dict:
    t = pr_timing()
    _check(h, lib().parareal_timing_read(h, C.byref(t), 1 if reset else 0))
    return t.as_dict()


def parareal_autotune(h) -> dict:
    """Time the fine step's candidate launch shapes on the handle's buffers and
    keep the fastest (cached per shape for the process); returns the choice."""
    t = pr_tuning()
    _check(h, lib().parareal_autotune(h, C.byref(t)))
    return t.as_dict()


def parareal_kernel_launches() -> int:
    return int(lib().parareal_kernel_launches())


def parareal_alu_probe(prec=PR_FP64, iters=4096) -> float:
    v = C.c_double()
    _check(None, lib().parareal_alu_probe(int(prec), int(iters), C.byref(v)))
    return v.value


def _ptr_array(xs):
    arr = (C.c_void_p * len(xs))()
    for i, x in enumerate(xs):
        arr[i] = x.value if isinstance(x, C.c_void_p) else (x.data_ptr() if hasattr(x, "data_ptr") else int(x))
    return arr


_cudart = None


def new_stream():
    """A dedicated non-blocking CUDA stream (torch.cuda.Stream() recycles a
    pool of 32), wrapped as a torch.cuda.ExternalStream."""
    global _cudart
    import torch
    if _cudart is None:
        lib()
        _cudart = C.CDLL("libcudart.so.13")
        _cudart.cudaStreamCreateWithFlags.argtypes = [C.POINTER(C.c_void_p), C.c_uint]
    s = C.c_void_p()
    if _cudart.cudaStreamCreateWithFlags(C.byref(s), 1) != 0:
        raise PararealError(PR_ECUDA, "cudaStreamCreateWithFlags failed")
    return torch.cuda.ExternalStream(s.value)


def parareal_solve_batch(hs, u0s, Ks, qTs):
    n = len(hs)
    _check(None, lib().parareal_solve_batch(_ptr_array(hs), n, _ptr_array(u0s), (C.c_int32 * n)(*Ks),
                                            _ptr_array(qTs)))


def parareal_batch_create(hs, u0s, Ks, qTs, stream):
    if hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    n = len(hs)
    b = C.c_void_p()
    _check(None, lib().parareal_batch_create(_ptr_array(hs), n, _ptr_array(u0s), (C.c_int32 * n)(*Ks),
                                             _ptr_array(qTs), C.c_void_p(stream), C.byref(b)))
    return b


def parareal_batch_launch(b):
    _check(None, lib().parareal_batch_launch(b))


def parareal_batch_destroy(b):
    _check(None, lib().parareal_batch_destroy(b))


def parareal_selftest_wait_timeout(stream=None):
    """Returns (status, seconds) of the bounded-wait self-test (expected PR_ETIMEOUT)."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    sec = C.c_double()
    st = lib().parareal_selftest_wait_timeout(C.c_void_p(stream) if stream else None, C.byref(sec))
    return st, sec.value


def parareal_fine_sweep_static(nx, ny, U, V, c_s, nu_f, dt_f, n_steps, fine_prec, q_in, q_out, n, stream=None):
    """Allocation-free fine sweep (no handle); see include/parareal.h for its limits."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(None, lib().parareal_fine_sweep_static(C.byref(pr_grid(nx, ny, 1.0, 1.0)), float(U), float(V),
                                                  float(c_s), float(nu_f), float(dt_f), int(n_steps),
                                                  int(fine_prec), _ptr(q_in), _ptr(q_out), int(n),
                                                  C.c_void_p(stream) if stream else None))


def _ld(t):
    """Leading dimension of a (columns, rows) tensor holding a column-major
    matrix (the stride of a size-1 dimension carries no information)."""
    if t.stride(-1) != 1:
        raise ValueError("columns must be contiguous")
    return t.stride(0) if t.shape[0] > 1 else t.shape[1]


def _split_gemm(name, A, B, out, m, n, k, lda, ldb, ldo, stream):
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(None, getattr(lib(), name)(_ptr(A), int(lda), int(m), _ptr(B), int(ldb), int(n), int(k), _ptr(out),
                                      int(ldo), C.c_void_p(stream) if stream else None))


def parareal_split_gemm_tn(A, B, C_out, stream=None):
    """C_out (m x n) = A^T B on the tensor cores, FP64-accurate.  A: k x m and
    B: k x n column-major FP64 device tensors, i.e. torch tensors of shape
    (m, k) and (n, k); C_out of shape (n, m)."""
    m, k = A.shape
    n = B.shape[0]
    _split_gemm("parareal_split_gemm_tn", A, B, C_out, m, n, k, _ld(A), _ld(B), _ld(C_out), stream)


def parareal_split_gemm_nn(A, B, Y, stream=None):
    """Y (k x n) <- Y - A B on the tensor cores, FP64-accurate.  A: k x m,
    B: m x n, Y: k x n column-major FP64 device tensors, i.e. torch tensors of
    shape (m, k), (n, m) and (n, k)."""
    m, k = A.shape
    n = B.shape[0]
    _split_gemm("parareal_split_gemm_nn", A, B, Y, m, n, k, _ld(A), _ld(B), _ld(Y), stream)


class Solver:
    """Convenience owner of a handle for a ``workloads.Problem``-like object."""

    def __init__(self, p, *, stream=None, **opt):
        opt.setdefault("T", p.T * opt.get("n_windows", 1))
        opt.setdefault("nu_f", p.nu_f)
        opt.setdefault("nu_c", p.nu_c)
        opt.setdefault("n_sound", p.n_sound)
        opt.setdefault("adv_order_f", p.adv_order_f)
        opt.setdefault("adv_order_c", p.adv_order_c)
        opt.setdefault("coarse_scheme", getattr(p, "coarse_scheme", 0))
        opt.setdefault("omega", getattr(p, "omega", 0.0))
        opt.setdefault("V", p.V)
        self.p = p
        self.h = parareal_create(p.nx, p.ny, p.U, p.c_s, p.dt_f, p.dt_g, p.n_slices, stream=stream, **opt)

    def close(self):
        if self.h:
            parareal_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
