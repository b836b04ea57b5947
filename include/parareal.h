/*
 * parareal.h -- C ABI of the GB300 (sm_103a) KSE-Parareal library for the
 * linear 2D acoustic-advection system (Ruprecht & Krause, "Explicit
 * Parallel-in-time Integration of a Linear Acoustic-Advection System",
 * arXiv 1510.02237).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - A state q holds d = 3*nx*ny doubles laid out [field][y][x] with x
 *    contiguous; fields are (u, w, p) = the paper's (u, v, pi) of
 *    Eq. acousticAd.  The domain is periodic, [0,lx) x [0,ly), cells of size
 *    dx = lx/nx, dy = ly/ny (Sec. 3, flux form on equal rectangular cells).
 *  - A batch of n states is n*d contiguous doubles.
 *  - Pointers named *_dev are CUDA device pointers owned by the caller; the
 *    library never frees or retains them beyond the call.  Host pointers are
 *    ordinary (pageable or pinned) host memory, also owned by the caller.
 *  - All device work is enqueued on the handle's stream (pr_options.stream,
 *    a cudaStream_t; NULL means the legacy default stream).  Calls return
 *    after enqueueing unless stated otherwise; results are valid once the
 *    stream has reached that point.
 *  - Every call returns a pr_status; no exception crosses the ABI.  On an
 *    error the handle keeps a message readable with parareal_last_error().
 *    PR_EINVAL leaves the handle unchanged.  After PR_ECUDA the handle's
 *    device state is unspecified and it should be destroyed.
 *  - One handle per host thread; handles are independent.
 */
#ifndef PARAREAL_H
#define PARAREAL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pr_solver pr_solver; /* opaque: owns iterates, fine images, basis Q and D = F(Q) - G(Q) */

typedef enum {
    PR_OK = 0,
    PR_EINVAL = -1,     /* bad argument (sizes, NaN, unsupported option)      */
    PR_ENOMEM = -2,     /* device or host allocation failed                   */
    PR_ECUDA = -3,      /* a CUDA runtime call or kernel launch failed        */
    PR_ETIMEOUT = -4,   /* a bounded device wait gave up                      */
    PR_ESTATE = -5,     /* call not valid in the handle's current state       */
    PR_ECANCELLED = -6  /* request cancelled                                  */
} pr_status;

enum { PR_FP64 = 0, PR_FP32 = 1, PR_FP32X = 2 };   /* arithmetic of the fine sweep:
                                                      FP64; FP32 state and stages;
                                                      FP32 tendencies and stages with
                                                      an FP64 state (q^{n+1} = q^n +
                                                      dt L(q**) formed in FP64)      */
enum { PR_KSE = 0, PR_ORIGINAL = 1 };              /* Alg. 2 / Alg. 1                */
enum { PR_IMAGES_LINEARITY = 0, PR_IMAGES_DIRECT = 1 };  /* how F(Q) is formed          */
enum { PR_PROJ_FP64 = 0, PR_PROJ_SPLIT_BF16 = 1 };  /* arithmetic of the projections
                                                      Q^T V and V - Q C of the
                                                      subspace update: FP64 units,
                                                      or FP64-accurate products on
                                                      the BF16 tensor cores (each
                                                      FP64 column split into 8
                                                      exact 7-bit digit slices)     */
enum { PR_BATCH_STREAMS = 0, PR_BATCH_PERSISTENT = 1 };  /* fine sweeps of a batch graph */
enum { PR_COARSE_SPLIT_FE = 0, PR_COARSE_RK3 = 1 };  /* coarse propagator G: partially
                                                      split forward Euler with
                                                      forward-backward acoustic
                                                      substeps (Sec. 3.2), or
                                                      non-split RK-3 of the same
                                                      operators (Sec. 3.1 demos)  */
#define PR_MAX_ITERS 128

typedef struct {
    int32_t nx, ny;   /* cells in x and y; nx, ny >= 4                          */
    double lx, ly;    /* domain lengths; <= 0 means 1.0                         */
} pr_grid;

typedef struct {
    double T;              /* end time of the single parallel step (default 1.0) */
    double nu_f;           /* fine divergence damping factor, Eq. dampingCoeff (0.005) */
    double nu_c;           /* coarse divergence damping factor (0.1)             */
    int32_t n_sound;       /* acoustic substeps per coarse step, Sec. 3.2 (4)    */
    int32_t adv_order_f;   /* advective flux order of F: 6 (centred)             */
    int32_t adv_order_c;   /* advective flux order of G: 1 (upwind)              */
    double V;              /* y component of the advection velocity (0.0)        */
    int32_t K_max;         /* largest K passed to parareal_solve (default N)     */
    int32_t krylov_cap;    /* max dim of S^k; 0 = sum_{k<K_max} (N - k)          */
    double drop_tol;       /* eta: drop a column whose residual after projection
                              is <= eta * its norm (1e-10)                       */
    int32_t fine_prec;     /* PR_FP64, PR_FP32 or PR_FP32X arithmetic inside F   */
    int32_t variant;       /* PR_KSE (Alg. 2) or PR_ORIGINAL (Alg. 1)            */
    int32_t corr_prec;     /* PR_FP64: serial correction evaluated literally in
                              FP64; PR_FP32: evaluated by linearity as
                              G(delta) + D Q^T delta, delta = q_i^{k+1} - q_i^k,
                              in FP32 (coarse images G(q_i^k) also in FP32),
                              accumulated into q in FP64                          */
    double r_tol;          /* > 0: stop a parallel step once r^k <= r_tol (Sec. 2.1);
                              0: always K_iters iterations                        */
    int32_t n_windows;     /* M_p: [0, T] is solved as n_windows consecutive
                              parallel steps of N_slices slices each (Sec. 2.1),
                              each started from the previous step's q_N (1)      */
    int32_t images;        /* PR_IMAGES_LINEARITY: F(Q) - G(Q) carried through the
                              Gram-Schmidt transform of the iterates' images, as
                              in Eq. Genhance (no extra fine sweeps); its
                              rounding error grows with 1/|R_jj| when iterates
                              are nearly dependent.  PR_IMAGES_DIRECT: F and G
                              applied to each new orthonormal basis vector (one
                              extra fine and coarse propagation per new
                              column), rounding error independent of the
                              conditioning.  corr_prec = PR_FP32 and fine_prec
                              other than PR_FP64 always use PR_IMAGES_DIRECT.    */
    int32_t sm_limit;      /* > 0: the handle's grid-synchronised kernels use at
                              most this many SMs, so solves of several handles on
                              different streams run side by side (0: all SMs)    */
    void* stream;          /* cudaStream_t, or NULL                              */
    int32_t proj_prec;     /* PR_PROJ_FP64 or PR_PROJ_SPLIT_BF16: how the
                              subspace update (Eq. subspaceUpdate) forms Q^T V
                              and V - Q C, and how K(q_i^k) forms Q^T q
                              (Eq. modifiedCoarse).  PR_PROJ_SPLIT_BF16
                              orthogonalises the new columns in blocks of 16
                              with these products on the tensor cores, to FP64
                              accuracy, and with images by linearity also the
                              image update Z - D C (norms, the drop rule, the
                              in-block Gram-Schmidt and the serial chain's
                              products stay FP64); it needs 3*nx*ny to be a
                              multiple of 8 and adds about 32*cap*3*nx*ny bytes
                              of digit slices to the footprint (48*cap*3*nx*ny
                              with images by linearity; default PR_PROJ_FP64) */
    int32_t coarse_scheme; /* PR_COARSE_SPLIT_FE (default): one coarse step is a
                              partially split forward-Euler step with n_sound
                              forward-backward acoustic substeps and damping
                              alpha = nu_c dx^2 / (Delta t / n_sound);
                              PR_COARSE_RK3: one coarse step is a non-split RK-3
                              step of length Delta t of the upwind advection
                              (adv_order_c), centred acoustics and damping with
                              alpha = nu_c dx^2 / Delta t (n_sound unused) -- the
                              coarse propagator of the paper's instability
                              demonstrations (Sec. 3.1, first-order upwind)      */
    double omega;          /* solid-body rotation rate (Eq. adVel, gamma): the
                              advection velocity is (U + omega (y - ly/2),
                              V - omega (x - lx/2)); in flux form every
                              x-interface of a row moves with the row's
                              x-velocity and every y-interface of a column with
                              the column's y-velocity.  0 (default): constant
                              (U, V).  The paper's workload: U = V = 0,
                              omega = pi, c_s = 30                              */
    int32_t batch_fine;    /* in batch graphs (parareal_batch_create):
                              PR_BATCH_STREAMS (default) runs this handle's
                              solve on its own stream; PR_BATCH_PERSISTENT puts
                              its fine sweeps into the batch's persistent
                              launches (used when every handle of the batch asks
                              for it and runs PR_FP32X with V = 0, no rotation,
                              KSE-Parareal in one parallel step)               */
} pr_options;

typedef struct {
    int32_t K;                   /* iterations performed, summed over the parallel
                                    steps; entries below are in that order        */
    int32_t rank[PR_MAX_ITERS];  /* dim S^k after the update of iteration k      */
    double r[PR_MAX_ITERS];      /* r^k = max_i ||q_i^{k+1} - q_i^k||_2 (Sec. 2.1) */
    float ms_total;              /* device time of the whole solve (CUDA events)  */
    int32_t n_windows;           /* parallel steps solved                          */
    int32_t K_window[PR_MAX_ITERS]; /* iterations performed in each parallel step */
    double min_ratio[PR_MAX_ITERS]; /* smallest |R_jj|/||a_j|| among the columns kept
                                    in iteration k: the conditioning of the new
                                    basis directions (rounding in F(Q) formed by
                                    linearity grows like 1/min_ratio); 1 if none */
} pr_report;

/* Phase timing of solves, measured with CUDA events on the handle's stream
 * (no synchronisation while solving).  Phases follow Alg. 2: the serial
 * coarse initialisation, then per iteration the parallel fine predictor, the
 * coarse images G(q_i^k), the subspace update, and the serial correction
 * (K(q_i^{k+1}) - K(q_i^k) through the linearity of K, so K(q_i^k) itself is
 * not formed). */
typedef struct {
    int32_t n_solves;        /* solves accumulated since the last reset           */
    double ms_init;          /* serial coarse initialisation                      */
    double ms_fine;          /* fine predictor F (all RK-3 step launches)         */
    double ms_coarse;        /* coarse images G(q_i^k)                            */
    double ms_krylov;        /* subspace update (sum of the next 3)               */
    double ms_gs_block;      /*   Gram-Schmidt against the existing basis         */
    double ms_gs_intra;      /*   Gram-Schmidt within the new columns, appends    */
    double ms_kold;          /*   direct images F(Q_j) - G(Q_j) of the new columns
                              *   (PR_IMAGES_DIRECT, FP32 fine sweeps); ~0 else   */
    double ms_chain;         /* serial correction                                 */
    double ms_total;         /* sum of the solves' device time                    */
    double fine_cell_steps;  /* cells x RK-3 steps computed by the fine predictor */
    int64_t fine_launches;   /* RK-3 step kernel launches of the fine predictor   */
} pr_timing;

/* Fill *opt with the defaults listed above (the paper's values, Sec. 3.2). */
pr_status parareal_default_options(pr_options* opt);

/* Create a solver for  q_t = f(q)  (Eq. ODE) from the spatial discretisation
 * of Eq. acousticAd with constant advection velocity (U, opt->V) and sound
 * speed c_s.  The interval [0, T] is split into N_slices time slices of
 * length T/N_slices (Sec. 2.1); the fine propagator F uses dt_f (RK-3) and
 * the coarse propagator G uses dt_g (partially split forward Euler with
 * forward-backward acoustic substeps, Sec. 3.2).  T/N_slices must be an
 * integer multiple of dt_f and of dt_g within 1e-9 relative (PR_EINVAL
 * otherwise).  Allocates every device buffer the solve needs; later calls
 * do not allocate.  *out receives the handle (NULL on failure). */
pr_status parareal_create(const pr_grid* g, double U, double c_s, double dt_f, double dt_g,
                          int32_t N_slices, const pr_options* opt, pr_solver** out);

/* Release the handle and its device memory (synchronises its stream). */
pr_status parareal_destroy(pr_solver* h);

/* Message of the last error on h ("" if none).  Valid until the next call on h.
 * h == NULL returns the message of the calling host thread's last failed
 * parareal_create. */
const char* parareal_last_error(const pr_solver* h);

/* Bytes of device memory a handle with these parameters holds. */
size_t parareal_footprint_bytes(const pr_grid* g, int32_t N_slices, const pr_options* opt);

/* KSE-Parareal, Alg. 2 (or Alg. 1 with variant = PR_ORIGINAL):
 * initialise q_{i+1}^0 = G(q_i^0) serially, then K_iters iterations of
 * parallel fine predictor, subspace update (Eq. subspaceUpdate) and serial
 * correction q_{i+1}^{k+1} = q~_{i+1}^k + (K(q_i^{k+1}) - K(q_i^k)) with the
 * modified coarse propagator K of Eq. modifiedCoarse.
 *   u0_dev : device, d doubles, the initial value q_0.
 *   K_iters: 0 <= K_iters <= opt.K_max iterations per parallel step (fewer
 *            when opt.r_tol stops the step early; that check synchronises
 *            the stream once per iteration).
 *   q_out_dev: device, (N+1)*d doubles receiving q_n^K, n = 0..N, of the last
 *            parallel step; may be NULL.
 *   qT_dev : device, d doubles receiving the value at T; may be NULL.
 *   rep    : host; if non-NULL the call synchronises the stream and fills it.
 * The subspace S^K remains in the handle for krylov_project(). */
pr_status parareal_solve(pr_solver* h, const double* u0_dev, int32_t K_iters, double* q_out_dev,
                         double* qT_dev, pr_report* rep);

/* parareal_solve with host buffers: copies u0_host (d doubles) to the device,
 * solves, and copies q_N^K back to qT_host (d doubles).  Synchronous. */
pr_status parareal_solve_host(pr_solver* h, const double* u0_host, int32_t K_iters, double* qT_host,
                              pr_report* rep);

/* Fine propagator F over one slice (N_f = (T/N)/dt_f RK-3 steps, Sec. 3.2)
 * applied independently to n states: q_out[i] = F(q_in[i]), the parallel
 * predictor of Alg. 2.  q_in_dev / q_out_dev: device, n*d doubles each,
 * must not overlap.  1 <= n <= N_slices. */
pr_status parareal_fine_sweep(pr_solver* h, const double* q_in_dev, double* q_out_dev, int32_t n);

/* Serial coarse sweep (initialisation of Alg. 2): q_out[i] = G^{i+1}(q0),
 * i = 0..N-1.  q0_dev: d doubles; q_out_dev: N*d doubles (device). */
pr_status parareal_coarse_sweep(pr_solver* h, const double* q0_dev, double* q_out_dev);

/* Coarse propagator G over one slice applied independently to n states. */
pr_status parareal_coarse_apply(pr_solver* h, const double* q_in_dev, double* q_out_dev, int32_t n);

/* Empty the handle's subspace (S = {}). */
pr_status krylov_reset(pr_solver* h);

/* Subspace update S -> S + span{V_j} (Sec. 2.2, Eq. subspaceUpdate) with the
 * fine images FV_j = F(V_j): the columns are orthogonalised in order against
 * the current basis (block classical Gram-Schmidt, applied twice) and then
 * against each other; column j is dropped when its residual is <= drop_tol
 * times its norm or the basis is full.  The same transformation applied to
 * F(V_j) - G(V_j) keeps D = F(Q) - G(Q) exact by linearity.
 *   V_dev, FV_dev: device, m*d doubles each.  kept_host: optional host array
 *   of m flags (synchronises when non-NULL).  1 <= m <= N_slices. */
pr_status krylov_update(pr_solver* h, const double* V_dev, const double* FV_dev, int32_t m,
                        int32_t* kept_host);

/* Current dim S (synchronises). */
pr_status krylov_rank(pr_solver* h, int32_t* rank);

/* Projection onto the current subspace (Sec. 2.2): Pq = Q Q^T q and, by
 * linearity (Eq. Genhance), FPq = F(P q) = D (Q^T q) + G(P q).  q_dev, Pq_dev,
 * FPq_dev: device, d doubles each; Pq_dev or FPq_dev may be NULL. */
pr_status krylov_project(pr_solver* h, const double* q_dev, double* Pq_dev, double* FPq_dev);

/* Record phase events for up to max_solves subsequent solves (allocates the
 * events; max_solves = 0 disables and frees them).  Resets the accumulators. */
pr_status parareal_timing_enable(pr_solver* h, int32_t max_solves);

/* Synchronise the stream and return the phase times accumulated over the
 * solves recorded since the last reset; reset != 0 starts a new accumulation. */
pr_status parareal_timing_read(pr_solver* h, pr_timing* t, int32_t reset);

/* Measurement utility with no counterpart in the paper: fused multiply-add
 * throughput of the current device in FLOP/s for prec = PR_FP64 or PR_FP32
 * (8 independent FMA chains per thread, 8 CTAs of 256 threads per SM, iters
 * x 32 FMAs per thread), the denominator of the ALU roofline.  Allocates a
 * small device buffer, synchronises the legacy default stream. */
pr_status parareal_alu_probe(int32_t prec, int32_t iters, double* flops_per_s);

/* ---- autotuning of the fine-step launch shape (no counterpart in the
 *      paper: it only chooses how the same arithmetic is laid out on the GPU) */

typedef struct {
    int32_t kernel;           /* 0: nothing to tune (FP64 fine sweep, or V != 0);
                                 1: shared-memory tile kernel (FP32X, or FP32 with
                                    nx not a multiple of 128);
                                 2: row-streamed kernel (FP32, V = 0, nx a
                                    multiple of 128)                              */
    int32_t choice;           /* kernel 1: tile index (TX x TY cells per CTA:
                                 0 = 32x8, 1 = 64x8, 2 = 64x16, 3 = 128x8);
                                 kernel 2: smallest row range per CTA;  -1: none  */
    int32_t cached;           /* 1: taken from the process-wide cache, not timed  */
    int32_t n_candidates;     /* candidates timed (0 when cached)                 */
    int32_t candidates[8];    /* tile indices or rows per CTA, in timing order    */
    float us_per_step[8];     /* device time of one RK-3 step over all N slices   */
} pr_tuning;

/* Time the candidate launch shapes of the handle's FP32 fine step on its own
 * fine-stage buffers (their contents are overwritten; nothing is allocated
 * on the device), keep the fastest for the handle's later sweeps and record
 * it in a process-wide cache keyed by (device, nx, ny, N_slices, fine_prec,
 * V != 0), so handles of the same shape take it without timing.  Every
 * candidate computes the same values cell by cell: results do not depend on
 * the choice, bit for bit.  Synchronises the handle's stream; not for use
 * while the stream is being captured.  out (host, optional) receives the
 * choice and the timings.  PR_ECUDA if a launch failed. */
pr_status parareal_autotune(pr_solver* h, pr_tuning* out);

/* ---- batches of independent solves (no counterpart in the paper: the
 *      instances are independent problems; this only schedules them) ---- */

/* Solve n independent problems side by side: each handle's solve is
 * enqueued on the handle's own stream (handles must have distinct non-NULL
 * streams to overlap; use pr_options.sm_limit so their grid-synchronised
 * kernels fit next to each other), then every stream is synchronised.
 * u0_dev[i], qT_dev[i]: device, d_i doubles; K[i] iterations. */
pr_status parareal_solve_batch(pr_solver* const* hs, int32_t n, const double* const* u0_dev, const int32_t* K,
                               double* const* qT_dev);

typedef struct pr_batch pr_batch;
/* Capture the n solves of parareal_solve_batch (same arguments, which stay
 * bound to the batch: refill u0_dev[i] before each launch) into one CUDA
 * graph that forks from `stream` into the handles' streams and joins back.
 * When every handle has batch_fine = PR_BATCH_PERSISTENT and runs the
 * FP32-tendency fine sweep (PR_FP32X) with V = 0, no rotation, KSE-Parareal
 * and one parallel step, the solves advance in lockstep phase by phase and
 * their fine sweeps (the predictor of every iteration and the fine images of
 * the new basis columns) run as one persistent cooperative launch per phase
 * over all the (state, tile) items of the handles still iterating; the rest
 * of each solve runs on the handle's stream.  Results equal the handles'
 * solo solves bit for bit either way.  Handles must be distinct, with
 * non-NULL streams other than `stream`; handles sharing a stream run one
 * after the other.  Requires r_tol = 0 on every handle.  Allocates the
 * graph, and for persistent fine sweeps one stream, one barrier word and the
 * work tables. */
pr_status parareal_batch_create(pr_solver* const* hs, int32_t n, const double* const* u0_dev, const int32_t* K,
                                double* const* qT_dev, void* stream, pr_batch** out);
/* Enqueue one replay of the batch graph on its stream (asynchronous). */
pr_status parareal_batch_launch(pr_batch* b);
pr_status parareal_batch_destroy(pr_batch* b);

/* Allocation-free fine sweep, for callers that cannot allocate device memory
 * where they need F: code running while a stream is captured into a CUDA
 * graph (cudaMalloc is not permitted there), runtimes that route every
 * device allocation through their own pool, and hosts that may not allocate
 * after start-up.  The paper has no counterpart.  For constant advection
 * velocity (U, V) in PR_FP64 or PR_FP32 it computes what parareal_fine_sweep
 * computes on a handle with the same parameters (n_steps RK-3 steps of the
 * fine tendency on n independent states); it has no rotation (omega) and no
 * PR_FP32X mode.  It needs no handle: every input and output comes from the
 * caller and the RK-3 intermediates live in a file-scope device array of
 * 32 MiB (two 16 MiB halves) that every GPU loading the library holds until
 * the process exits.  It always runs the shared-memory tile kernel, which
 * has no device-side waits, so nothing is left to report after it returns.
 *   g, U, V, c_s, nu_f, dt_f: as for parareal_create (nx, ny >= 4).
 *   n_steps: RK-3 steps (>= 1); fine_prec: PR_FP64 or PR_FP32.
 *   q_in_dev / q_out_dev: device, n*d doubles each, not overlapping.
 *   n: 1..65535 states with n*d*(8 for FP64, 4 for FP32) <= 16 MiB, i.e.
 *      n*d <= 2097152 (FP64) or 4194304 (FP32); larger sizes return
 *      PR_EINVAL and print the limit to stderr.
 *   stream: cudaStream_t or NULL.  Returns after enqueueing.
 * The first call on each device looks up the array's device address (with
 * that device current) and must come before any stream capture; later calls
 * made outside capture look it up again.  Calls share
 * the array: calls whose work overlaps on the GPU race and must be
 * serialised by the caller.  No allocation of any kind is made. */
pr_status parareal_fine_sweep_static(const pr_grid* g, double U, double V, double c_s, double nu_f,
                                     double dt_f, int32_t n_steps, int32_t fine_prec,
                                     const double* q_in_dev, double* q_out_dev, int32_t n, void* stream);

/* FP64-accurate tall-skinny products on the BF16 tensor cores, the same
 * kernels the subspace update uses with PR_PROJ_SPLIT_BF16 (Eq.
 * subspaceUpdate, Eq. modifiedCoarse: the projection coefficients Q^T q and
 * the update q - Q c), exposed for direct use and testing.  All matrices are
 * column-major FP64 device buffers.  Each column of both operands is written
 * as 2^E times 8 digits of 7 bits, the 43 leading digit products are summed
 * exactly in FP32 over chunks of 256 contraction elements and the chunks are
 * combined in FP64: per term the error is at most 2^-55 (max|a| |b_k| +
 * |a_k| max|b|) + 2^-58 max|a| max|b| (a, b the two columns), plus the FP64
 * rounding of the combination.
 *   tn:  C (m x n, ld ldc) = A^T B,  A: k x m (ld lda), B: k x n (ld ldb).
 *   nn:  Y (k x n, ld ldy) <- Y - A B,  A: k x m (ld lda), B: m x n (ld ldb).
 * k must be a multiple of 8 (>= 8), 1 <= m <= 16384, n >= 1.  Not the solve's
 * allocation-free path: each call allocates its digit buffers, enqueues on
 * `stream` (cudaStream_t or NULL), synchronises it and frees them.  Returns
 * PR_EINVAL for bad sizes or NULL pointers, PR_ENOMEM, PR_ECUDA, or
 * PR_ETIMEOUT if a pipeline wait of the kernel gave up. */
pr_status parareal_split_gemm_tn(const double* A, int64_t lda, int32_t m, const double* B, int64_t ldb,
                                 int32_t n, int64_t k, double* C, int64_t ldc, void* stream);
pr_status parareal_split_gemm_nn(const double* A, int64_t lda, int32_t m, const double* B, int64_t ldb,
                                 int32_t n, int64_t k, double* Y, int64_t ldy, void* stream);

/* Self-test of the library's bounded device waits (no counterpart in the
 * paper): launches a cooperative kernel whose grid barrier can never complete
 * (it expects one CTA more than the grid has).  Every wait gives up after its
 * poll limit (well under a few seconds), records the failure and returns, so
 * the call returns PR_ETIMEOUT and the CUDA context stays usable.  *seconds
 * (optional) receives the device time until the waits gave up. */
pr_status parareal_selftest_wait_timeout(void* stream, double* seconds);

/* Process-wide number of CUDA kernels this library has launched. */
uint64_t parareal_kernel_launches(void);

/* Synchronise the handle's stream and report whether the work enqueued on
 * it so far completed cleanly: PR_OK, PR_ETIMEOUT if a bounded device-side
 * wait gave up (a grid barrier, a tensor-core pipeline or row-ring wait;
 * results since then are invalid and the handle should be destroyed), or
 * PR_ECUDA.  For callers of the asynchronous calls (parareal_solve without a
 * report, batches, servers); the paper has no counterpart. */
pr_status parareal_status(pr_solver* h);

#ifdef __cplusplus
}
#endif
#endif /* PARAREAL_H */
