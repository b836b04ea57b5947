"""Host-side checks of the C ABI library (no GPU needed, no kernel launched)."""
from __future__ import annotations

import ctypes as C
import os
import re

import pytest

import paper_1510_02237_gb300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "parareal.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:pr_status|size_t|uint64_t|const char\s*\*)\s+([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def test_library_exports_every_declared_symbol():
    names = _declared_symbols()
    assert len(names) >= 14, names
    L = P.lib()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(P.EXPORTS) == names


def test_default_options_are_the_papers():
    o = P.parareal_default_options()
    assert (o.nu_f, o.nu_c, o.n_sound, o.adv_order_f, o.adv_order_c) == (0.005, 0.1, 4, 6, 1)
    assert o.drop_tol == 1e-10 and o.T == 1.0 and o.V == 0.0


def test_footprint_grows_with_basis():
    a = P.parareal_footprint_bytes(256, 128, 32, K_max=6)            # cap = 177
    b = P.parareal_footprint_bytes(256, 128, 32, K_max=6, krylov_cap=192)
    c = P.parareal_footprint_bytes(256, 128, 32, K_max=6, fine_prec=P.PR_FP32)
    assert 0 < c < a and b > a
    d = 3 * 256 * 128
    assert b >= 2 * 192 * d * 8


@pytest.mark.parametrize("kw,msg", [
    (dict(nx=2), "nx and ny"),
    (dict(N=0), "N_slices"),
    (dict(dt_f=1.0 / 150), "dt_f"),
    (dict(dt_g=0.07), "dt_g"),
    (dict(c_s=float("nan")), "finite"),
    (dict(adv_order_f=4), "adv_order_f"),
    (dict(adv_order_c=2), "adv_order_c"),
    (dict(n_sound=9), "n_sound"),
    (dict(fine_prec=7), "fine_prec"),
    (dict(K_max=9), "K_max"),
    (dict(omega=float("nan")), "omega"),
    (dict(coarse_scheme=5), "coarse_scheme"),
    (dict(variant=3), "variant"),
    (dict(corr_prec=9), "corr_prec"),
    (dict(n_windows=0), "n_windows"),
    (dict(images=4), "images"),
    (dict(proj_prec=6), "proj_prec"),
])
def test_create_rejects_invalid_arguments(kw, msg):
    """Validation happens on the host before any CUDA call."""
    args = dict(nx=64, ny=32, U=0.1, c_s=1.0, dt_f=1.0 / 160, dt_g=1.0 / 16, N=8)
    opt = {}
    for k, v in kw.items():
        if k in args:
            args[k] = v
        else:
            opt[k] = v
    with pytest.raises(P.PararealError) as ei:
        P.parareal_create(args["nx"], args["ny"], args["U"], args["c_s"], args["dt_f"], args["dt_g"],
                          args["N"], **opt)
    assert ei.value.status == P.PR_EINVAL
    assert msg in str(ei.value)


def test_null_handle_is_einval():
    assert P.lib().parareal_solve(None, None, 1, None, None, None) == P.PR_EINVAL
    assert P.lib().krylov_rank(None, None) == P.PR_EINVAL
