// coarse_tile.cuh -- one partially split forward-Euler coarse step (Sec. 3.2)
// on one TX x TY tile of a state, computed in shared memory from a haloed
// region of the input state:
//   S = -(F_{i+1/2} - F_{i-1/2})/dx - (G_{j+1/2} - G_{j-1/2})/dy    slow tendency at q^n,
//        upwind-biased advective fluxes of order 1 or 3, held fixed for the step;
//   n_sound times, tau = Delta t / n_sound, alpha = nu_c dx^2 / tau:
//     u <- u + tau [S_u - c_s (p[i+1]-p[i-1])/(2dx) + alpha1 (div u)_x]
//     w <- w + tau [S_w - c_s (p[j+1]-p[j-1])/(2dy) + alpha2 (div u)_y]
//     p <- p + tau [S_p - c_s ((u[i+1]-u[i-1])/(2dx) + (w[j+1]-w[j-1])/(2dy))]   (new u, w)
// Every substep widens the dependency cone by 2 cells (1 for the velocities,
// 1 for the pressure) and the slow tendency by the flux radius r, so the
// tile loads a halo H = r + 2 n_sound - 1 and shrinks the valid region as
// the substeps proceed; nothing is written to memory between substeps.
//
// scheme = 1 replaces the split step by one non-split RK-3 step of length
// Delta t of the same operators (upwind advection of order 1 or 3, centred
// acoustics, damping with alpha = nu_c dx^2 / Delta t): the coarse
// propagator of the paper's instability demonstrations (Sec. 3.1).  Each
// stage widens the cone by the flux radius r, so the halo is H = 3 r.
#pragma once

#include "common.cuh"

namespace pr {

constexpr int COARSE_MAXH = 12;

template <typename T>
__device__ __forceinline__ T upwind_flux(int order, T U, const T* f, int i, int st) {
    // interface i+1/2 along stride st
    if (order == 1) return U >= T(0) ? U * f[i] : U * f[i + st];
    const T aU = U >= T(0) ? U : -U;
    return U * (T(7) * (f[i + st] + f[i]) - (f[i + 2 * st] + f[i - st])) * (T(1) / T(12)) +
           aU * ((f[i + 2 * st] - f[i - st]) - T(3) * (f[i + st] - f[i])) * (T(1) / T(12));
}

// The same flux from the four values along the stencil line (f_{i-1}, f_i,
// f_{i+1}, f_{i+2}): one expression for both, so both round alike.
template <typename T>
__device__ __forceinline__ T upwind_flux3_pts(T U, T fm1, T f0, T fp1, T fp2) {
    const T aU = U >= T(0) ? U : -U;
    return U * (T(7) * (fp1 + f0) - (fp2 + fm1)) * (T(1) / T(12)) +
           aU * ((fp2 - fm1) - T(3) * (fp1 - f0)) * (T(1) / T(12));
}

// Coefficients of the split coarse step in arithmetic T.
template <typename T>
struct CoarseT {
    T U, V, inv_dx, inv_dy, tau, csx, csy, dxx, dxy1, dyy, dxy2;
    int n_sound, order;
};
template <typename T>
__device__ __forceinline__ CoarseT<T> coarse_t(const CoarseCoef& cd) {
    return {(T)cd.U, (T)cd.V, (T)cd.inv_dx, (T)cd.inv_dy, (T)cd.tau, (T)cd.csx, (T)cd.csy,
            (T)cd.dxx, (T)cd.dxy1, (T)cd.dyy, (T)cd.dxy2, cd.n_sound, cd.order};
}

// Forward-backward acoustic substep of one cell from its neighbourhood (x+-1
// and y+-1 of each field, the corners of the other velocity for the damping
// cross terms; ab names x then y offsets, p = +1, m = -1).  Written once and
// used by the tile kernel and the distributed serial chain alike.
template <typename T>
__device__ __forceinline__ T fb_new_u(const CoarseT<T>& c, T su, T u0, T uxp, T uxm, T pxp, T pxm, T wpp, T wpm,
                                      T wmp, T wmm) {
    const T du = su - c.csx * (pxp - pxm) + c.dxx * (uxp - T(2) * u0 + uxm) + c.dxy1 * ((wpp - wpm) - (wmp - wmm));
    return u0 + c.tau * du;
}
template <typename T>
__device__ __forceinline__ T fb_new_w(const CoarseT<T>& c, T sw, T w0, T wyp, T wym, T pyp, T pym, T upp, T ump,
                                      T upm, T umm) {
    const T dw = sw - c.csy * (pyp - pym) + c.dyy * (wyp - T(2) * w0 + wym) + c.dxy2 * ((upp - ump) - (upm - umm));
    return w0 + c.tau * dw;
}
template <typename T>
__device__ __forceinline__ T fb_new_p(const CoarseT<T>& c, T sp, T p0, T uxp, T uxm, T wyp, T wym) {
    return p0 + c.tau * (sp - (c.csx * (uxp - uxm) + c.csy * (wyp - wym)));
}

// First-order slow tendency of one field from its upwind differences (the
// y-difference skipped when the advection has no y-component anywhere).
template <typename T>
__device__ __forceinline__ T slow_first_order(T ax, T ay, T dxu, T dyu, bool ynone) {
    T v = ax * dxu;
    if (!ynone) v += ay * dyu;
    return v;
}

// Shared memory (elements) of one tile: 6 arrays of (TX + 2H) x (TY + 2H).
template <int TX, int TY>
__host__ __device__ constexpr int coarse_tile_smem_elems(int H) {
    return 6 * (TX + 2 * H) * (TY + 2 * H);
}

// out tile (tx0, ty0) = one coarse step of in, in arithmetic T (double or
// float, loaded from Tin and stored as Tout); NT threads cooperate; sm holds
// coarse_tile_smem_elems<TX,TY>(H) elements of T.  Contains __syncthreads().
// src is read with plain (coherent) loads: the serial chain passes states
// that other CTAs wrote earlier in the same launch.
template <int TX, int TY, int NT, typename T = double, typename Tin = double, typename Tout = double>
__device__ __forceinline__ void coarse_tile(const Tin* src, Tout* __restrict__ dst, int nx, int ny,
                                            const CoarseCoef& cd, int H, int tx0, int ty0, T* __restrict__ sm) {
    const int RX = TX + 2 * H, RY = TY + 2 * H, NR = RX * RY;
    T* u = sm;
    T* w = u + NR;
    T* p = w + NR;
    T* su = p + NR;
    T* sw = su + NR;
    T* sp = sw + NR;
    const long ncell = (long)nx * ny;
    const CoarseT<T> c = coarse_t<T>(cd);
    // advection velocity of the cell at local (lr, lc): constant, or with the
    // solid-body rotation (Eq. adVel) at the cell's periodic position -- the
    // x-velocity is that of the row, the y-velocity that of the column
    auto vel = [&](int lr, int lc, T& Ur, T& Vc) {
        Ur = c.U;
        Vc = c.V;
        if (cd.omega != 0.0) {
            const int gy = pwrap(ty0 - H + lr, ny), gx = pwrap(tx0 - H + lc, nx);
            Ur += (T)(cd.omega * ((gy + 0.5) * cd.dy - cd.hly));
            Vc -= (T)(cd.omega * ((gx + 0.5) * cd.dx - cd.hlx));
        }
    };

    for (int idx = threadIdx.x; idx < NR; idx += NT) {
        int ly = idx / RX, lx = idx - ly * RX;
        long g = (long)pwrap(ty0 - H + ly, ny) * nx + pwrap(tx0 - H + lx, nx);
        u[idx] = (T)src[g];
        w[idx] = (T)src[ncell + g];
        p[idx] = (T)src[2 * ncell + g];
    }
    __syncthreads();

    const int ra = c.order == 1 ? 1 : 2;
    constexpr int MAXC = ((TX + 2 * COARSE_MAXH) * (TY + 2 * COARSE_MAXH) + NT - 1) / NT;
    if (cd.scheme == 1) {
        // L(a) at index i: upwind advection, centred acoustics, grad-div damping
        auto tend = [&](const T* au, const T* aw, const T* ap, int lr, int lc, T& Lu, T& Lw, T& Lp) {
            const int i = lr * RX + lc;
            const T* fs[3] = {au, aw, ap};
            T t[3], Ur, Vc;
            vel(lr, lc, Ur, Vc);
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                const T* a = fs[f];
                const T Fe = upwind_flux<T>(c.order, Ur, a, i, 1), Fw = upwind_flux<T>(c.order, Ur, a, i - 1, 1);
                const T Gn = upwind_flux<T>(c.order, Vc, a, i, RX), Gs = upwind_flux<T>(c.order, Vc, a, i - RX, RX);
                t[f] = -(Fe - Fw) * c.inv_dx - (Gn - Gs) * c.inv_dy;
            }
            Lu = t[0] - c.csx * (ap[i + 1] - ap[i - 1]) + c.dxx * (au[i + 1] - T(2) * au[i] + au[i - 1]) +
                 c.dxy1 * ((aw[i + 1 + RX] - aw[i + 1 - RX]) - (aw[i - 1 + RX] - aw[i - 1 - RX]));
            Lw = t[1] - c.csy * (ap[i + RX] - ap[i - RX]) + c.dyy * (aw[i + RX] - T(2) * aw[i] + aw[i - RX]) +
                 c.dxy2 * ((au[i + 1 + RX] - au[i - 1 + RX]) - (au[i + 1 - RX] - au[i - 1 - RX]));
            Lp = t[2] - (c.csx * (au[i + 1] - au[i - 1]) + c.csy * (aw[i + RX] - aw[i - RX]));
        };
        const T c1 = c.tau / T(3), c2 = c.tau / T(2), c3 = c.tau;
        {   // stage 1: s = q + tau/3 L(q) on the region shrunk by ra
            const int W1 = RX - 2 * ra, H1 = RY - 2 * ra, N1 = W1 * H1;
            for (int t = threadIdx.x; t < N1; t += NT) {
                const int r = t / W1;
                const int i = (r + ra) * RX + (t - r * W1) + ra;
                T Lu, Lw, Lp;
                tend(u, w, p, r + ra, t - r * W1 + ra, Lu, Lw, Lp);
                su[i] = u[i] + c1 * Lu;
                sw[i] = w[i] + c1 * Lw;
                sp[i] = p[i] + c1 * Lp;
            }
        }
        __syncthreads();
        {   // stage 2: s <- q + tau/2 L(s) on the region shrunk by 2 ra (the tile
            // plus ra <= 2 cells around it), staged in registers
            constexpr int MAXR = ((TX + 4) * (TY + 4) + NT - 1) / NT;
            const int sh = 2 * ra, W2 = RX - 2 * sh, H2 = RY - 2 * sh, N2 = W2 * H2;
            T ru[MAXR], rw[MAXR], rp[MAXR];
#pragma unroll
            for (int k = 0; k < MAXR; ++k) {
                const int t = threadIdx.x + k * NT;
                if (t < N2) {
                    const int r = t / W2;
                    const int i = (r + sh) * RX + (t - r * W2) + sh;
                    T Lu, Lw, Lp;
                    tend(su, sw, sp, r + sh, t - r * W2 + sh, Lu, Lw, Lp);
                    ru[k] = u[i] + c2 * Lu;
                    rw[k] = w[i] + c2 * Lw;
                    rp[k] = p[i] + c2 * Lp;
                }
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < MAXR; ++k) {
                const int t = threadIdx.x + k * NT;
                if (t < N2) {
                    const int r = t / W2;
                    const int i = (r + sh) * RX + (t - r * W2) + sh;
                    su[i] = ru[k];
                    sw[i] = rw[k];
                    sp[i] = rp[k];
                }
            }
        }
        __syncthreads();
        // stage 3: q' = q + tau L(s) on the tile, written to memory
        for (int t = threadIdx.x; t < TX * TY; t += NT) {
            const int r = t / TX, cx = t - r * TX;
            const int gx = tx0 + cx, gy = ty0 + r;
            if (gx < nx && gy < ny) {
                const int i = (r + H) * RX + cx + H;
                T Lu, Lw, Lp;
                tend(su, sw, sp, r + H, cx + H, Lu, Lw, Lp);
                const long g = (long)gy * nx + gx;
                dst[g] = (Tout)(u[i] + c3 * Lu);
                dst[ncell + g] = (Tout)(w[i] + c3 * Lw);
                dst[2 * ncell + g] = (Tout)(p[i] + c3 * Lp);
            }
        }
        __syncthreads();   // the shared buffers may be reused right after
        return;
    }
    // slow (advective) tendency on the region shrunk by ra
    {
        const int W1 = RX - 2 * ra, H1 = RY - 2 * ra, N1 = W1 * H1;
        // first order: both x-interfaces of a cell move with the row's velocity
        // and both y-interfaces with the column's, so the flux difference is the
        // velocity times the upwind difference of the field (y skipped when
        // the advection has no y-component anywhere)
        const bool ynone = cd.V == 0.0 && cd.omega == 0.0;
        for (int t = threadIdx.x; t < N1; t += NT) {
            int r = t / W1;
            int i = (r + ra) * RX + (t - r * W1) + ra;
            T* fs[3] = {u, w, p};
            T* ss[3] = {su, sw, sp};
            T Ur, Vc;
            vel(r + ra, t - r * W1 + ra, Ur, Vc);
            if (c.order == 1) {
                const T ax = -Ur * c.inv_dx, ay = -Vc * c.inv_dy;
                const int sx = Ur >= T(0) ? -1 : 1, sy = Vc >= T(0) ? -RX : RX;
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    const T* a = fs[f];
                    const T dx_ = sx < 0 ? a[i] - a[i - 1] : a[i + 1] - a[i];
                    const T dy_ = ynone ? T(0) : (sy < 0 ? a[i] - a[i - RX] : a[i + RX] - a[i]);
                    ss[f][i] = slow_first_order<T>(ax, ay, dx_, dy_, ynone);
                }
            } else {
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    const T* a = fs[f];
                    const T Fe = upwind_flux3_pts<T>(Ur, a[i - 1], a[i], a[i + 1], a[i + 2]);
                    const T Fw = upwind_flux3_pts<T>(Ur, a[i - 2], a[i - 1], a[i], a[i + 1]);
                    const T Gn = upwind_flux3_pts<T>(Vc, a[i - RX], a[i], a[i + RX], a[i + 2 * RX]);
                    const T Gs = upwind_flux3_pts<T>(Vc, a[i - 2 * RX], a[i - RX], a[i], a[i + RX]);
                    ss[f][i] = -(Fe - Fw) * c.inv_dx - (Gn - Gs) * c.inv_dy;
                }
            }
        }
    }
    __syncthreads();

    for (int m = 0; m < c.n_sound; ++m) {
        // forward: velocities on the region shrunk by ra + 2m
        const int sh = ra + 2 * m;
        const int W2 = RX - 2 * sh, H2 = RY - 2 * sh, N2 = W2 * H2;
        T nu[MAXC], nw[MAXC];
#pragma unroll
        for (int k = 0; k < MAXC; ++k) {
            int t = threadIdx.x + k * NT;
            if (t < N2) {
                int r = t / W2;
                int i = (r + sh) * RX + (t - r * W2) + sh;
                nu[k] = fb_new_u<T>(c, su[i], u[i], u[i + 1], u[i - 1], p[i + 1], p[i - 1], w[i + 1 + RX],
                                    w[i + 1 - RX], w[i - 1 + RX], w[i - 1 - RX]);
                nw[k] = fb_new_w<T>(c, sw[i], w[i], w[i + RX], w[i - RX], p[i + RX], p[i - RX], u[i + 1 + RX],
                                    u[i - 1 + RX], u[i + 1 - RX], u[i - 1 - RX]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < MAXC; ++k) {
            int t = threadIdx.x + k * NT;
            if (t < N2) {
                int r = t / W2;
                int i = (r + sh) * RX + (t - r * W2) + sh;
                u[i] = nu[k];
                w[i] = nw[k];
            }
        }
        __syncthreads();
        // backward: pressure with the new velocities on the region shrunk by ra + 2m + 1
        const int sp1 = sh + 1;
        const int W3 = RX - 2 * sp1, H3 = RY - 2 * sp1, N3 = W3 * H3;
        for (int t = threadIdx.x; t < N3; t += NT) {
            int r = t / W3;
            int i = (r + sp1) * RX + (t - r * W3) + sp1;
            p[i] = fb_new_p<T>(c, sp[i], p[i], u[i + 1], u[i - 1], w[i + RX], w[i - RX]);
        }
        __syncthreads();
    }

    for (int t = threadIdx.x; t < TX * TY; t += NT) {
        int r = t / TX, cx = t - r * TX;
        int gx = tx0 + cx, gy = ty0 + r;
        if (gx < nx && gy < ny) {
            int i = (r + H) * RX + cx + H;
            long g = (long)gy * nx + gx;
            dst[g] = (Tout)u[i];
            dst[ncell + g] = (Tout)w[i];
            dst[2 * ncell + g] = (Tout)p[i];
        }
    }
    __syncthreads();   // the shared buffers may be reused right after
}

}  // namespace pr
