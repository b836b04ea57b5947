"""Closed-form Fourier symbols of the discrete operators (test pins, numpy only).

These are written from textbook modified-wavenumber analysis of periodic
finite differences, independently of the oracle's stencil code:

* centred differences of order 2/4/6 have the purely imaginary symbols
  i sin(t), i(8 sin t - sin 2t)/6, i(45 sin t - 9 sin 2t + sin 3t)/30;
* the odd (upwind-biased) orders 1/3/5 add |U| times the even-order
  hyper-diffusion 2 sin^2(t/2), (16/12) sin^4(t/2), (64/60) sin^6(t/2);
* the compact grad-div damping has symbol -4 sin^2(t/2)/dx^2 on the
  diagonal and -sin(tx) sin(ty)/(dx dy) off it;
* a linear three-stage RK-3 step is the truncated exponential
  I + hA + (hA)^2/2 + (hA)^3/6.
"""
from __future__ import annotations

import numpy as np


def flux_symbol(order: int, theta: float):
    """(centred part c, dissipative part e) of the flux difference per unit velocity."""
    s1, s2, s3 = np.sin(theta), np.sin(2 * theta), np.sin(3 * theta)
    h2 = np.sin(theta / 2.0) ** 2
    if order in (1, 2):
        c = 1j * s1
    elif order in (3, 4):
        c = 1j * (8 * s1 - s2) / 6.0
    else:
        c = 1j * (45 * s1 - 9 * s2 + s3) / 30.0
    e = {1: 2.0 * h2, 3: 16.0 * h2 ** 2 / 12.0, 5: 64.0 * h2 ** 3 / 60.0}.get(order, 0.0)
    return c, e


def adv_symbol(order, U, V, tx, ty, dx, dy):
    cx, ex = flux_symbol(order, tx)
    cy, ey = flux_symbol(order, ty)
    return -(U * cx + abs(U) * ex) / dx - (V * cy + abs(V) * ey) / dy


def fast_symbol(cs, a1, a2, tx, ty, dx, dy):
    """Acoustic + divergence-damping symbol (3x3) acting on (u, w, p)."""
    sx, sy = np.sin(tx), np.sin(ty)
    hx, hy = np.sin(tx / 2) ** 2, np.sin(ty / 2) ** 2
    cross = -sx * sy / (dx * dy)
    A = np.zeros((3, 3), dtype=complex)
    A[0, 0] = a1 * (-4 * hx / dx ** 2)
    A[0, 1] = a1 * cross
    A[0, 2] = -cs * 1j * sx / dx
    A[1, 0] = a2 * cross
    A[1, 1] = a2 * (-4 * hy / dy ** 2)
    A[1, 2] = -cs * 1j * sy / dy
    A[2, 0] = -cs * 1j * sx / dx
    A[2, 1] = -cs * 1j * sy / dy
    return A


def fine_symbol(p, kx, ky):
    nx, ny = p.nx, p.ny
    dx, dy = p.lx / nx, p.ly / ny
    tx, ty = 2 * np.pi * kx / nx, 2 * np.pi * ky / ny
    a1 = p.nu_f * dx * dx / p.dt_f
    a2 = p.nu_f * dy * dy / p.dt_f
    A = fast_symbol(p.c_s, a1, a2, tx, ty, dx, dy)
    A += adv_symbol(p.adv_order_f, p.U, p.V, tx, ty, dx, dy) * np.eye(3)
    return A


def rk3_matrix(A, h):
    Z = h * A
    I = np.eye(A.shape[0])
    return I + Z + Z @ Z / 2.0 + Z @ Z @ Z / 6.0


def fine_amplification(p, kx, ky, nsteps):
    R = rk3_matrix(fine_symbol(p, kx, ky), p.dt_f)
    return np.linalg.matrix_power(R, nsteps)


def damping_symbol(stencil, tx, ty, dx, dy):
    """2x2 symbol of grad(div u) on (u, w): 'compact' (3-point second
    differences plus the 4-point cross difference), or 'wide' (the centred
    divergence followed by the centred gradient, which misses the 2 dx mode)."""
    sx, sy = np.sin(tx), np.sin(ty)
    cross = -sx * sy / (dx * dy)
    if stencil == "compact":
        hx, hy = np.sin(tx / 2) ** 2, np.sin(ty / 2) ** 2
        return np.array([[-4 * hx / dx ** 2, cross], [cross, -4 * hy / dy ** 2]], dtype=complex)
    return np.array([[-sx ** 2 / dx ** 2, cross], [cross, -sy ** 2 / dy ** 2]], dtype=complex)


def coarse_amplification(p, kx, ky, nsteps, *, order="velocity_first", damping="old", stencil="compact",
                         slow="frozen", n_sound=None):
    """Split forward-Euler / forward-backward coarse step as a product of
    substep matrices on z = (q, q^n) -- the slow tendency is frozen at q^n.

    The keywords select readings of what Sec. 3.2 leaves open (defaults: the
    implemented one): ``order`` -- velocities first, then the pressure from the
    new velocities, or the pressure first; ``damping`` -- grad-div damping from
    the velocities at the start of the substep ('old') or applied to the
    velocities just updated ('new'); ``stencil`` -- see damping_symbol;
    ``slow`` -- 'frozen' adds the frozen slow tendency in every substep
    (partially split), 'advect_first' takes one forward-Euler advective step of
    Delta t and then the acoustic substeps (not partially split)."""
    nx, ny = p.nx, p.ny
    dx, dy = p.lx / nx, p.ly / ny
    tx, ty = 2 * np.pi * kx / nx, 2 * np.pi * ky / ny
    ns = p.n_sound if n_sound is None else n_sound
    tau = p.dt_g / ns
    a1 = p.nu_c * dx * dx / tau
    a2 = p.nu_c * dy * dy / tau
    s = adv_symbol(p.adv_order_c, p.U, p.V, tx, ty, dx, dy)
    F = fast_symbol(p.c_s, 0.0, 0.0, tx, ty, dx, dy)   # acoustics only
    Dm = np.diag([a1, a2]) @ damping_symbol(stencil, tx, ty, dx, dy)
    sf = s if slow == "frozen" else 0.0
    # forward part: (u, w) <- (u, w) + tau (s q^n + F[0:2,:] q [+ damping])
    def vel(with_damping):
        M = np.eye(6, dtype=complex)
        M[0:2, 0:3] += tau * F[0:2, :]
        M[0:2, 3:5] += tau * sf * np.eye(2)
        if with_damping:
            M[0:2, 0:2] += tau * Dm
        return M
    # backward part: p <- p + tau (s p^n + F[2, :] q_new)
    Mb = np.eye(6, dtype=complex)
    Mb[2, 0:3] += tau * F[2, :]
    Mb[2, 5] += tau * sf
    Md = np.eye(6, dtype=complex)
    Md[0:2, 0:2] += tau * Dm
    Mv = vel(True) if damping == "old" else Md @ vel(False)
    sub = Mb @ Mv if order == "velocity_first" else Mv @ Mb
    Msub = np.linalg.matrix_power(sub, ns)
    # start from z = (q, q): big step map is Msub[0:3,0:3] + Msub[0:3,3:6]
    if slow == "frozen":
        step = Msub[0:3, 0:3] + Msub[0:3, 3:6]
    else:
        step = Msub[0:3, 0:3] @ ((1.0 + p.dt_g * s) * np.eye(3))
    return np.linalg.matrix_power(step, nsteps)


def coarse_rk3_amplification(p, kx, ky, nsteps):
    """Non-split RK-3 coarse step of length dt_g: the truncated exponential of
    dt_g times (upwind advection of order adv_order_c + acoustics + damping
    with alpha = nu_c dx^2 / dt_g)."""
    nx, ny = p.nx, p.ny
    dx, dy = p.lx / nx, p.ly / ny
    tx, ty = 2 * np.pi * kx / nx, 2 * np.pi * ky / ny
    a1 = p.nu_c * dx * dx / p.dt_g
    a2 = p.nu_c * dy * dy / p.dt_g
    A = fast_symbol(p.c_s, a1, a2, tx, ty, dx, dy)
    A += adv_symbol(p.adv_order_c, p.U, p.V, tx, ty, dx, dy) * np.eye(3)
    return np.linalg.matrix_power(rk3_matrix(A, p.dt_g), nsteps)


def plane_wave(nx, ny, kx, ky, qhat):
    """Real field Re(qhat_f exp(i(tx*i + ty*j))) on cell indices, shape (3, ny, nx)."""
    i = np.arange(nx)
    j = np.arange(ny)
    ph = np.exp(1j * (2 * np.pi * kx / nx * i[None, :] + 2 * np.pi * ky / ny * j[:, None]))
    return np.real(np.asarray(qhat)[:, None, None] * ph[None, :, :])
