/*
 * oracle.h -- plain, serial, FP64 CPU oracle for Krylov-subspace-enhanced
 * Parareal on the linear 2D acoustic-advection system.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header or constant with the CUDA product path.
 *
 * State layout: q[f*ny*nx + j*nx + i], f = 0 (u), 1 (w), 2 (p); i is the
 * x index (contiguous), j the y index.  d = 3*nx*ny.  Periodic in x and y.
 */
#ifndef ORC_ORACLE_H
#define ORC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny;          /* cells in x and y                                  */
    double lx, ly;       /* domain lengths (unit square: 1, 1)                */
    double U, V;         /* constant advection velocity (Eq. acousticAd)      */
    double cs;           /* speed of sound                                    */
    double nu_f, nu_c;   /* divergence-damping factors (Eq. dampingCoeff)     */
    int n_sound;         /* acoustic substeps per coarse step (Sec. 3.2)      */
    double dt_f, dt_g;   /* fine step delta t, coarse step Delta t            */
    int n_f, n_g;        /* fine / coarse steps per time slice                */
    int n_slices;        /* N_c = N_p                                         */
    int adv_order_f;     /* advective flux order of F (1..6)                  */
    int adv_order_c;     /* advective flux order of G (1..6)                  */
    int coarse_scheme;   /* 0: split forward Euler / forward-backward; 1: RK-3 */
    double omega;        /* solid-body rotation rate: the advection velocity is
                            (U + omega (y - ly/2), V - omega (x - lx/2)),
                            Eq. adVel with gamma = omega (0: constant U, V)   */
} orc_problem;

/* ---- spatial operator and propagators ---- */
void orc_fine_rhs(const orc_problem* pb, const double* q, double* L);
void orc_fine_steps(const orc_problem* pb, const double* q_in, double* q_out, int nsteps);
void orc_fine_prop(const orc_problem* pb, const double* q_in, double* q_out);          /* F: n_f steps */
void orc_coarse_steps(const orc_problem* pb, const double* q_in, double* q_out, int nsteps);
void orc_coarse_prop(const orc_problem* pb, const double* q_in, double* q_out);        /* G: n_g steps */

/* ---- subspace S^k with orthonormal basis and fine images ---- */
typedef struct orc_basis orc_basis;
orc_basis* orc_basis_create(long d, int cap);
void   orc_basis_free(orc_basis* b);
int    orc_basis_rank(const orc_basis* b);
/* Append column a (with fine image fa); returns 1 if kept, 0 if dropped.
 * *ratio receives |R_jj| / ||a|| (residual against the kept columns). */
int    orc_basis_add(orc_basis* b, const double* a, const double* fa, double eta, double* ratio);
void   orc_basis_get_q(const orc_basis* b, double* Q);     /* d x rank, column-major */
void   orc_basis_get_fq(const orc_basis* b, double* FQ);   /* d x rank, column-major */
/* Pq = P q, FPq = F(P q) computed by linearity from the stored images (Eq. Genhance). */
void   orc_basis_project(const orc_basis* b, const double* q, double* Pq, double* FPq);

/* ---- Parareal (Alg. 1 / Alg. 2) ---- */
/* variant: 0 = KSE-Parareal (Alg. 2), 1 = original Parareal (Alg. 1).
 * r_tol > 0 stops after the first iteration with r^k <= r_tol (Sec. 2.1).
 * q_all: (N+1)*d output iterates q_n^K.  r_hist[K], rank_hist[K] outputs.
 * kept / ratio: optional (K*N) per processed column (may be NULL).
 * Returns the number of iterations performed, or -1 if allocation failed. */
int orc_parareal(const orc_problem* pb, const double* q0, int K, int variant,
                 double eta, int cap, double r_tol, double* q_all, double* r_hist, int* rank_hist,
                 int* kept, double* ratio);

/* q_all[n] = F^n(q0), n = 0..N (serial fine reference). */
void orc_serial_fine(const orc_problem* pb, const double* q0, double* q_all);

/* Threads for the parallel predictor of Alg. 2 (the loop over slices that
 * the paper runs with OpenMP, Sec. 2.1 and Sec. 3.2): 1 (the default) runs it
 * serially.  Each slice's fine propagation is independent, so the results do
 * not depend on the thread count.  Returns the previous value. */
int orc_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
