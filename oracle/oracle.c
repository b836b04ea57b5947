/*
 * oracle.c -- plain, serial, FP64 CPU oracle for Krylov-subspace-enhanced
 * Parareal (KSE-Parareal) on the linear 2D acoustic-advection system
 * (Ruprecht & Krause, arXiv 1510.02237).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg.  It is deliberately slow and literal: every
 * function follows one passage of the paper, in the paper's order, with no
 * blocking, fusion or reordering.  It shares no code with the CUDA path.
 *
 * Readings of passages the paper leaves open (each also listed in the
 * design notes of the repository):
 *   - flux stencils of order 1..6 are the standard upwind/centred interface
 *     fluxes the paper cites (Wicker & Skamarock 2002) -- Sec. 3, flux form;
 *   - the divergence-damping term alpha*(div u)_x is discretised as the
 *     difference of an interface divergence (compact second difference plus
 *     4-point cross difference) -- Sec. 3.2, Eq. dampingCoeff;
 *   - RK-3 is the Wicker-Skamarock three-stage form (dt/3, dt/2, dt);
 *   - the forward-backward substep updates the velocities first and then
 *     the pressure with the new velocities; the slow (advective) tendency is
 *     evaluated once per coarse step and held fixed -- Sec. 3.2;
 *   - the subspace update is a Householder QR of the columns in insertion
 *     order that drops column j when |R_jj| <= eta * ||a_j|| (the paper uses
 *     pivoted DGEQP3 without stating a rank rule) -- Sec. 2.2, Eq. subspaceUpdate.
 *
 * The parallel predictor can run on several host threads (OpenMP over
 * slices, the paper's own parallel structure, Sec. 2.1); everything else is
 * serial, as in the paper, and the results do not depend on the threads.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ helpers */

static int wrap(int i, int n) {
    while (i < 0) i += n;
    while (i >= n) i -= n;
    return i;
}

#define AT(q, f, j, i) (q)[(long)(f) * ncell + (long)wrap((j), ny) * nx + wrap((i), nx)]

/* Advective interface flux F_{i+1/2} = U * q_{i+1/2} of order 1..6.
 * Arguments are the values at i-2, i-1, i, i+1, i+2, i+3 along the line.
 * Orders 1, 3, 5 are upwind-biased, orders 2, 4, 6 centred. */
static double adv_flux(int order, double U, double qm2, double qm1, double q0,
                       double qp1, double qp2, double qp3) {
    double aU = fabs(U);
    switch (order) {
    case 1:
        return U >= 0.0 ? U * q0 : U * qp1;
    case 2:
        return U * (q0 + qp1) / 2.0;
    case 3:
        return U * (7.0 * (qp1 + q0) - (qp2 + qm1)) / 12.0
             + aU * ((qp2 - qm1) - 3.0 * (qp1 - q0)) / 12.0;
    case 4:
        return U * (7.0 * (qp1 + q0) - (qp2 + qm1)) / 12.0;
    case 5:
        return U * (37.0 * (qp1 + q0) - 8.0 * (qp2 + qm1) + (qp3 + qm2)) / 60.0
             - aU * ((qp3 - qm2) - 5.0 * (qp2 - qm1) + 10.0 * (qp1 - q0)) / 60.0;
    case 6:
    default:
        return U * (37.0 * (qp1 + q0) - 8.0 * (qp2 + qm1) + (qp3 + qm2)) / 60.0;
    }
}

/* Advection velocity (Sec. 3.2, Eq. adVel): the constant (U, V) plus the
 * solid-body rotation omega (y - ly/2, -(x - lx/2)).  Its x-component depends
 * on y only and its y-component on x only, so the velocity at every
 * x-interface of row j is the value at the row's cell centres, and at every
 * y-interface of column i the value at the column's cell centres. */
static double u_row(const orc_problem* pb, int j) {
    const double dy = pb->ly / pb->ny;
    return pb->U + pb->omega * ((j + 0.5) * dy - 0.5 * pb->ly);
}
static double v_col(const orc_problem* pb, int i) {
    const double dx = pb->lx / pb->nx;
    return pb->V - pb->omega * ((i + 0.5) * dx - 0.5 * pb->lx);
}

/* x-interface advective flux of field f at (i+1/2, j) */
static double fx_adv(const orc_problem* pb, const double* q, int order, int f, int j, int i) {
    const int nx = pb->nx, ny = pb->ny;
    const long ncell = (long)nx * ny;
    return adv_flux(order, u_row(pb, j), AT(q, f, j, i - 2), AT(q, f, j, i - 1), AT(q, f, j, i),
                    AT(q, f, j, i + 1), AT(q, f, j, i + 2), AT(q, f, j, i + 3));
}

/* y-interface advective flux of field f at (i, j+1/2) */
static double fy_adv(const orc_problem* pb, const double* q, int order, int f, int j, int i) {
    const int nx = pb->nx, ny = pb->ny;
    const long ncell = (long)nx * ny;
    return adv_flux(order, v_col(pb, i), AT(q, f, j - 2, i), AT(q, f, j - 1, i), AT(q, f, j, i),
                    AT(q, f, j + 1, i), AT(q, f, j + 2, i), AT(q, f, j + 3, i));
}

/* Interface divergence of (u, w) at the x-interface (i+1/2, j): compact
 * du/dx plus the average of the centred dw/dy of cells i and i+1. */
static double div_xface(const orc_problem* pb, const double* q, int j, int i) {
    const int nx = pb->nx, ny = pb->ny;
    const long ncell = (long)nx * ny;
    const double dx = pb->lx / nx, dy = pb->ly / ny;
    double dudx = (AT(q, 0, j, i + 1) - AT(q, 0, j, i)) / dx;
    double dwdy = ((AT(q, 1, j + 1, i) - AT(q, 1, j - 1, i))
                 + (AT(q, 1, j + 1, i + 1) - AT(q, 1, j - 1, i + 1))) / (4.0 * dy);
    return dudx + dwdy;
}

/* Interface divergence of (u, w) at the y-interface (i, j+1/2). */
static double div_yface(const orc_problem* pb, const double* q, int j, int i) {
    const int nx = pb->nx, ny = pb->ny;
    const long ncell = (long)nx * ny;
    const double dx = pb->lx / nx, dy = pb->ly / ny;
    double dwdy = (AT(q, 1, j + 1, i) - AT(q, 1, j, i)) / dy;
    double dudx = ((AT(q, 0, j, i + 1) - AT(q, 0, j, i - 1))
                 + (AT(q, 0, j + 1, i + 1) - AT(q, 0, j + 1, i - 1))) / (4.0 * dx);
    return dwdy + dudx;
}

/* Flux-form tendency of Sec. 3:
 *   d/dt q_ij = -(F_{i+1/2} - F_{i-1/2})/dx - (G_{j+1/2} - G_{j-1/2})/dy
 * with advective fluxes of the given order, 2nd-order centred acoustic
 * fluxes (c_s times the interface average), and divergence damping
 * alpha1 (div u)_x, alpha2 (div u)_y on the momentum equations. */
static void tendency(const orc_problem* pb, const double* q, double* L, int order,
                     int with_adv, int with_fast, double alpha1, double alpha2) {
    const int nx = pb->nx, ny = pb->ny;
    const long ncell = (long)nx * ny;
    const double dx = pb->lx / nx, dy = pb->ly / ny, cs = pb->cs;
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            double t[3] = {0.0, 0.0, 0.0};
            if (with_adv) {
                for (int f = 0; f < 3; ++f) {
                    double Fe = fx_adv(pb, q, order, f, j, i), Fw = fx_adv(pb, q, order, f, j, i - 1);
                    double Gn = fy_adv(pb, q, order, f, j, i), Gs = fy_adv(pb, q, order, f, j - 1, i);
                    t[f] += -(Fe - Fw) / dx - (Gn - Gs) / dy;
                }
            }
            if (with_fast) {
                /* acoustic fluxes: u <- c_s p in x, w <- c_s p in y, p <- c_s u in x and c_s w in y */
                double Pe = cs * (AT(q, 2, j, i) + AT(q, 2, j, i + 1)) / 2.0;
                double Pw = cs * (AT(q, 2, j, i - 1) + AT(q, 2, j, i)) / 2.0;
                double Pn = cs * (AT(q, 2, j, i) + AT(q, 2, j + 1, i)) / 2.0;
                double Ps = cs * (AT(q, 2, j - 1, i) + AT(q, 2, j, i)) / 2.0;
                double Ue = cs * (AT(q, 0, j, i) + AT(q, 0, j, i + 1)) / 2.0;
                double Uw = cs * (AT(q, 0, j, i - 1) + AT(q, 0, j, i)) / 2.0;
                double Wn = cs * (AT(q, 1, j, i) + AT(q, 1, j + 1, i)) / 2.0;
                double Ws = cs * (AT(q, 1, j - 1, i) + AT(q, 1, j, i)) / 2.0;
                t[0] += -(Pe - Pw) / dx;
                t[1] += -(Pn - Ps) / dy;
                t[2] += -(Ue - Uw) / dx - (Wn - Ws) / dy;
                /* divergence damping */
                t[0] += alpha1 * (div_xface(pb, q, j, i) - div_xface(pb, q, j, i - 1)) / dx;
                t[1] += alpha2 * (div_yface(pb, q, j, i) - div_yface(pb, q, j - 1, i)) / dy;
            }
            for (int f = 0; f < 3; ++f) L[(long)f * ncell + (long)j * nx + i] = t[f];
        }
    }
}

/* ------------------------------------------------------------ fine propagator */

/* L_f(q): order adv_order_f advection, acoustics, damping with
 * alpha = nu_f dx^2 / delta t (Eq. dampingCoeff with tau = delta t). */
void orc_fine_rhs(const orc_problem* pb, const double* q, double* L) {
    const double dx = pb->lx / pb->nx, dy = pb->ly / pb->ny;
    double a1 = pb->nu_f * dx * dx / pb->dt_f, a2 = pb->nu_f * dy * dy / pb->dt_f;
    tendency(pb, q, L, pb->adv_order_f, 1, 1, a1, a2);
}

/* Three-stage RK-3: q* = q + dt/3 L(q); q** = q + dt/2 L(q*); q' = q + dt L(q**). */
static void rk3_step(const orc_problem* pb, double* q, double* s, double* L, int order,
                     double dt, double a1, double a2) {
    const long d = 3L * pb->nx * pb->ny;
    const double c[3] = {dt / 3.0, dt / 2.0, dt};
    tendency(pb, q, L, order, 1, 1, a1, a2);
    for (long n = 0; n < d; ++n) s[n] = q[n] + c[0] * L[n];
    tendency(pb, s, L, order, 1, 1, a1, a2);
    for (long n = 0; n < d; ++n) s[n] = q[n] + c[1] * L[n];
    tendency(pb, s, L, order, 1, 1, a1, a2);
    for (long n = 0; n < d; ++n) q[n] = q[n] + c[2] * L[n];
}

void orc_fine_steps(const orc_problem* pb, const double* q_in, double* q_out, int nsteps) {
    const long d = 3L * pb->nx * pb->ny;
    const double dx = pb->lx / pb->nx, dy = pb->ly / pb->ny;
    double a1 = pb->nu_f * dx * dx / pb->dt_f, a2 = pb->nu_f * dy * dy / pb->dt_f;
    double* s = (double*)malloc(sizeof(double) * d);
    double* L = (double*)malloc(sizeof(double) * d);
    double* q = (double*)malloc(sizeof(double) * d);
    memcpy(q, q_in, sizeof(double) * d);
    for (int n = 0; n < nsteps; ++n) rk3_step(pb, q, s, L, pb->adv_order_f, pb->dt_f, a1, a2);
    memcpy(q_out, q, sizeof(double) * d);
    free(q);
    free(L);
    free(s);
}

void orc_fine_prop(const orc_problem* pb, const double* q_in, double* q_out) {
    orc_fine_steps(pb, q_in, q_out, pb->n_f);
}

/* ---------------------------------------------------------- coarse propagator */

/* One partially split forward-Euler step with forward-backward acoustic
 * substeps (Sec. 3.2): slow (advective) tendency S = adv(q^n) once, then
 * n_sound substeps of length tau = Delta t / n_sound:
 *   u <- u + tau [S_u - c_s p_x + alpha1 (div u)_x]
 *   w <- w + tau [S_w - c_s p_y + alpha2 (div u)_y]
 *   p <- p + tau [S_p - c_s (u_x + w_y)]      (new u, w)
 * with alpha = nu_c dx^2 / tau. */
static void split_fe_step(const orc_problem* pb, double* q, double* S, double* T) {
    const int nx = pb->nx, ny = pb->ny;
    const long ncell = (long)nx * ny, d = 3 * ncell;
    const double dx = pb->lx / nx, dy = pb->ly / ny;
    const double tau = pb->dt_g / pb->n_sound;
    const double a1 = pb->nu_c * dx * dx / tau, a2 = pb->nu_c * dy * dy / tau;
    tendency(pb, q, S, pb->adv_order_c, 1, 0, 0.0, 0.0);
    for (int m = 0; m < pb->n_sound; ++m) {
        /* forward: momentum from the old (u, w, p) */
        tendency(pb, q, T, pb->adv_order_c, 0, 1, a1, a2);
        for (long n = 0; n < 2 * ncell; ++n) q[n] = q[n] + tau * (S[n] + T[n]);
        /* backward: pressure from the new (u, w) */
        tendency(pb, q, T, pb->adv_order_c, 0, 1, a1, a2);
        for (long n = 2 * ncell; n < d; ++n) q[n] = q[n] + tau * (S[n] + T[n]);
    }
}

void orc_coarse_steps(const orc_problem* pb, const double* q_in, double* q_out, int nsteps) {
    const long d = 3L * pb->nx * pb->ny;
    const double dx = pb->lx / pb->nx, dy = pb->ly / pb->ny;
    double* q = (double*)malloc(sizeof(double) * d);
    double* s = (double*)malloc(sizeof(double) * d);
    double* L = (double*)malloc(sizeof(double) * d);
    memcpy(q, q_in, sizeof(double) * d);
    for (int n = 0; n < nsteps; ++n) {
        if (pb->coarse_scheme == 1) {
            /* non-split RK-3 with the coarse advective order, tau = Delta t */
            double a1 = pb->nu_c * dx * dx / pb->dt_g, a2 = pb->nu_c * dy * dy / pb->dt_g;
            rk3_step(pb, q, s, L, pb->adv_order_c, pb->dt_g, a1, a2);
        } else {
            split_fe_step(pb, q, s, L);
        }
    }
    memcpy(q_out, q, sizeof(double) * d);
    free(L);
    free(s);
    free(q);
}

void orc_coarse_prop(const orc_problem* pb, const double* q_in, double* q_out) {
    orc_coarse_steps(pb, q_in, q_out, pb->n_g);
}

/* ------------------------------------------------------------ subspace basis */
/* Householder QR of the columns in insertion order (Sec. 2.2).  Column j of
 * the explicit basis is H_1 ... H_j e_j; appending a reflector leaves the
 * earlier columns unchanged, so the basis of a grown column set equals the
 * one a fresh factorisation of all columns would produce, bit for bit.  The
 * fine images of the basis follow by linearity (Eq. Genhance):
 * A_sel = Q R  =>  F(Q) = F(A_sel) R^{-1}. */
struct orc_basis {
    long d;
    int cap, m;
    double* V;    /* reflector vectors, cap x d (full length, zeros above) */
    double* tau;  /* reflector scalars                                      */
    double* R;    /* cap x cap, column-major upper triangular               */
    double* Q;    /* d x cap explicit orthonormal basis                     */
    double* FQ;   /* d x cap fine images of the basis                       */
};

orc_basis* orc_basis_create(long d, int cap) {
    orc_basis* b = (orc_basis*)calloc(1, sizeof(orc_basis));
    b->d = d;
    b->cap = cap;
    b->V = (double*)calloc((size_t)cap * d, sizeof(double));
    b->tau = (double*)calloc((size_t)cap, sizeof(double));
    b->R = (double*)calloc((size_t)cap * cap, sizeof(double));
    b->Q = (double*)calloc((size_t)cap * d, sizeof(double));
    b->FQ = (double*)calloc((size_t)cap * d, sizeof(double));
    return b;
}

void orc_basis_free(orc_basis* b) {
    if (!b) return;
    free(b->V);
    free(b->tau);
    free(b->R);
    free(b->Q);
    free(b->FQ);
    free(b);
}

int orc_basis_rank(const orc_basis* b) { return b->m; }

/* x <- H_l x = x - tau_l v_l (v_l^T x) */
static void apply_reflector(const orc_basis* b, int l, double* x) {
    const long d = b->d;
    const double* v = b->V + (long)l * d;
    double s = 0.0;
    for (long n = l; n < d; ++n) s += v[n] * x[n];
    s *= b->tau[l];
    for (long n = l; n < d; ++n) x[n] -= s * v[n];
}

int orc_basis_add(orc_basis* b, const double* a, const double* fa, double eta, double* ratio) {
    const long d = b->d;
    const int m = b->m;
    double anorm = 0.0;
    for (long n = 0; n < d; ++n) anorm += a[n] * a[n];
    anorm = sqrt(anorm);
    double* x = (double*)malloc(sizeof(double) * d);
    memcpy(x, a, sizeof(double) * d);
    for (int l = 0; l < m; ++l) apply_reflector(b, l, x);
    double tail = 0.0;
    for (long n = m; n < d; ++n) tail += x[n] * x[n];
    tail = sqrt(tail);
    double rat = anorm > 0.0 ? tail / anorm : 0.0;
    if (ratio) *ratio = rat;
    if (m >= b->cap || m >= d || anorm == 0.0 || tail <= eta * anorm) {
        free(x);
        return 0;
    }
    /* reflector that maps x[m:] to alpha e_m, alpha = -sign(x_m) ||x[m:]|| */
    double alpha = x[m] >= 0.0 ? -tail : tail;
    double* v = b->V + (long)m * d;
    memset(v, 0, sizeof(double) * d);
    for (long n = m; n < d; ++n) v[n] = x[n];
    v[m] -= alpha;
    double vv = 0.0;
    for (long n = m; n < d; ++n) vv += v[n] * v[n];
    b->tau[m] = 2.0 / vv;
    /* column m of R: x[0..m-1] above the diagonal, alpha on it */
    double* Rc = b->R + (long)m * b->cap;
    for (int l = 0; l < m; ++l) Rc[l] = x[l];
    Rc[m] = alpha;
    b->m = m + 1;
    /* explicit basis column: Q e_m = H_0 ... H_m e_m */
    double* q = b->Q + (long)m * d;
    memset(q, 0, sizeof(double) * d);
    q[m] = 1.0;
    for (int l = m; l >= 0; --l) apply_reflector(b, l, q);
    /* its fine image by forward substitution: F(a) = sum_{l<=m} F(Q_l) R_lm */
    double* fq = b->FQ + (long)m * d;
    for (long n = 0; n < d; ++n) fq[n] = fa[n];
    for (int l = 0; l < m; ++l) {
        const double* fl = b->FQ + (long)l * d;
        for (long n = 0; n < d; ++n) fq[n] -= Rc[l] * fl[n];
    }
    for (long n = 0; n < d; ++n) fq[n] /= alpha;
    free(x);
    return 1;
}

void orc_basis_get_q(const orc_basis* b, double* Q) {
    memcpy(Q, b->Q, sizeof(double) * (size_t)b->m * b->d);
}

void orc_basis_get_fq(const orc_basis* b, double* FQ) {
    memcpy(FQ, b->FQ, sizeof(double) * (size_t)b->m * b->d);
}

/* c = Q^T q;  Pq = Q c;  F(Pq) = sum_l c_l F(Q_l)   (Eq. Genhance) */
static void basis_coeffs(const orc_basis* b, const double* q, double* c) {
    for (int l = 0; l < b->m; ++l) {
        const double* ql = b->Q + (long)l * b->d;
        double s = 0.0;
        for (long n = 0; n < b->d; ++n) s += ql[n] * q[n];
        c[l] = s;
    }
}

void orc_basis_project(const orc_basis* b, const double* q, double* Pq, double* FPq) {
    const long d = b->d;
    double* c = (double*)malloc(sizeof(double) * (b->m > 0 ? b->m : 1));
    basis_coeffs(b, q, c);
    for (long n = 0; n < d; ++n) {
        Pq[n] = 0.0;
        FPq[n] = 0.0;
    }
    for (int l = 0; l < b->m; ++l) {
        const double* ql = b->Q + (long)l * d;
        const double* fl = b->FQ + (long)l * d;
        for (long n = 0; n < d; ++n) {
            Pq[n] += c[l] * ql[n];
            FPq[n] += c[l] * fl[n];
        }
    }
    free(c);
}

/* Modified coarse propagator (Eq. modifiedCoarse):
 *   K(q) = G((I - P) q) + F(P q),  F(P q) from the stored images. */
static void kse_coarse(const orc_problem* pb, const orc_basis* b, const double* q, double* out,
                       double* Pq, double* FPq, double* r) {
    const long d = 3L * pb->nx * pb->ny;
    orc_basis_project(b, q, Pq, FPq);
    for (long n = 0; n < d; ++n) r[n] = q[n] - Pq[n];
    orc_coarse_prop(pb, r, out);
    for (long n = 0; n < d; ++n) out[n] = out[n] + FPq[n];
}

/* ------------------------------------------------------------------ Parareal */

static int g_threads = 1;

int orc_set_threads(int n) {
    const int old = g_threads;
    g_threads = n > 0 ? n : 1;
    return old;
}

int orc_parareal(const orc_problem* pb, const double* q0, int K, int variant,
                 double eta, int cap, double r_tol, double* q_all, double* r_hist, int* rank_hist,
                 int* kept, double* ratio) {
    const int N = pb->n_slices;
    const long d = 3L * pb->nx * pb->ny;
    double* qt = (double*)malloc(sizeof(double) * (size_t)N * d);        /* fine images q~_{i+1} */
    double* qold = (double*)malloc(sizeof(double) * (size_t)(N + 1) * d); /* q^k                 */
    double* kn = (double*)malloc(sizeof(double) * d);
    double* ko = (double*)malloc(sizeof(double) * d);
    double* w1 = (double*)malloc(sizeof(double) * d);
    double* w2 = (double*)malloc(sizeof(double) * d);
    double* w3 = (double*)malloc(sizeof(double) * d);
    orc_basis* b = orc_basis_create(d, cap > 0 ? cap : 1);
    if (!qt || !qold || !kn || !ko || !w1 || !w2 || !w3 || !b) return -1;

    /* initialisation: q_0^0 = q0, q_{i+1}^0 = G(q_i^0) */
    memcpy(q_all, q0, sizeof(double) * d);
    for (int i = 0; i < N; ++i) orc_coarse_prop(pb, q_all + (long)i * d, q_all + (long)(i + 1) * d);

    for (int k = 0; k < K; ++k) {
        /* parallel predictor: q~_{i+1}^k = F(q_i^k), one slice per iteration of
         * an OpenMP loop as in the paper's implementation when threads > 1 */
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads) if (g_threads > 1)
        for (int i = 0; i < N; ++i) orc_fine_prop(pb, q_all + (long)i * d, qt + (long)i * d);
        /* subspace update S^{k-1} -> S^k with q_i^k and their images */
        if (variant == 0) {
            for (int i = 0; i < N; ++i) {
                double rt = 0.0;
                int kp = orc_basis_add(b, q_all + (long)i * d, qt + (long)i * d, eta, &rt);
                if (kept) kept[k * N + i] = kp;
                if (ratio) ratio[k * N + i] = rt;
            }
        }
        /* sequential correction:
         * q_{i+1}^{k+1} = K(q_i^{k+1}) + q~_{i+1}^k - K(q_i^k)  (Alg. 2), evaluated as
         * q~ + (K_new - K_old); original Parareal uses G in place of K (Alg. 1). */
        memcpy(qold, q_all, sizeof(double) * (size_t)(N + 1) * d);
        for (int i = 0; i < N; ++i) {
            const double* qn = q_all + (long)i * d;
            const double* qo = qold + (long)i * d;
            if (variant == 0) {
                kse_coarse(pb, b, qn, kn, w1, w2, w3);
                kse_coarse(pb, b, qo, ko, w1, w2, w3);
            } else {
                orc_coarse_prop(pb, qn, kn);
                orc_coarse_prop(pb, qo, ko);
            }
            double* out = q_all + (long)(i + 1) * d;
            const double* t = qt + (long)i * d;
            for (long n = 0; n < d; ++n) out[n] = t[n] + (kn[n] - ko[n]);
        }
        /* error estimate r^k = max_i ||q_i^{k+1} - q_i^k||_2, i = 1..N */
        double rmax = 0.0;
        for (int i = 1; i <= N; ++i) {
            double s = 0.0;
            for (long n = 0; n < d; ++n) {
                double e = q_all[(long)i * d + n] - qold[(long)i * d + n];
                s += e * e;
            }
            s = sqrt(s);
            if (s > rmax) rmax = s;
        }
        if (r_hist) r_hist[k] = rmax;
        if (rank_hist) rank_hist[k] = orc_basis_rank(b);
        /* optional stopping rule of Sec. 2.1: stop once r^k <= r_tol */
        if (r_tol > 0.0 && rmax <= r_tol) {
            K = k + 1;
            break;
        }
    }
    orc_basis_free(b);
    free(w3);
    free(w2);
    free(w1);
    free(ko);
    free(kn);
    free(qold);
    free(qt);
    return K;
}

void orc_serial_fine(const orc_problem* pb, const double* q0, double* q_all) {
    const long d = 3L * pb->nx * pb->ny;
    memcpy(q_all, q0, sizeof(double) * d);
    for (int i = 0; i < pb->n_slices; ++i) orc_fine_prop(pb, q_all + (long)i * d, q_all + (long)(i + 1) * d);
}
