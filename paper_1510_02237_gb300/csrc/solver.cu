// solver.cu -- the solver handle, the KSE-Parareal driver (Alg. 2 / Alg. 1)
// and the extern "C" entry points declared in include/parareal.h.
//
// Device data layout (all FP64 unless noted, column = one state of d values):
//   q    (N+1) x d   iterates q_n^k, updated in place by the serial correction
//   qt   N x d       fine images q~_{i+1}^k = F(q_i^k)   (slot i)
//   gv   N x d       coarse images G(q_i^k)              (slot i)
//   dlt64 d          delta_i = q_i^{k+1} - q_i^k of the serial correction
//   Q, D d x cap     orthonormal basis of S^k and D = F(Q) - G(Q); by linearity
//                    K(q) = G(q - Q Q^T q) + F(Q) Q^T q = G(q) + D (Q^T q), so
//                    K(q_i^{k+1}) - K(q_i^k) = G(delta_i) + D (Q^T delta_i)
//   wv, wz N x d     Gram-Schmidt work columns and their D-images
//   fine/coarse ping-pong buffers (FP64, and FP32 when the fine sweep runs in FP32)
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "parareal.h"
#include "split_gemm.h"

using namespace pr;

static std::atomic<uint64_t> g_launches{0};
extern "C" uint64_t parareal_kernel_launches(void);
void pr::count_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

// Ring of CUDA events recording the phase boundaries of up to max_solves solves:
// [start, init end, then per iteration: fine end, coarse end, krylov end, chain end].
// With the tensor-core projection the in-block Gram-Schmidt of every 16-column
// sub-block is bracketed by a pair of events (sub, per solve and iteration
// up to sub_per_iter pairs) so that it can be told apart from the projections.
struct TimingRing {
    int max_solves = 0, per_solve = 0, n = 0;
    std::vector<cudaEvent_t> ev;
    std::vector<int> K;
    std::vector<long> fine_launches;
    int sub_per_iter = 0;
    std::vector<cudaEvent_t> sub;
    std::vector<int> nsub;   // pairs recorded, per solve and iteration
};

struct pr_solver {
    int nx = 0, ny = 0, N = 0, n_f = 0, n_g = 0, K_max = 0, cap = 0;
    long d = 0;
    double U = 0, V = 0, cs = 0, dt_f = 0, dt_g = 0, lx = 1, ly = 1;
    pr_options opt{};
    cudaStream_t stream = nullptr;
    FineCoef<double> fc64{};
    FineCoef<float> fc32{};
    FineCoefK fck{};
    double* fb2 = nullptr;
    CoarseCoef cc{};
    double *q = nullptr, *qt = nullptr, *gv = nullptr, *dlt64 = nullptr;
    double *Q = nullptr, *D = nullptr, *wv = nullptr, *wz = nullptr;
    double *fb0 = nullptr, *fb1 = nullptr, *cb0 = nullptr, *cb1 = nullptr, *gtmp = nullptr;
    float *f32a = nullptr, *f32b = nullptr;
    double *C = nullptr, *cvec = nullptr, *partial = nullptr;
    double *anorm2 = nullptr, *res2 = nullptr, *rhist = nullptr, *nres2 = nullptr;
    double *gbuf = nullptr, *resp = nullptr, *ratios = nullptr;   // ratios: PR_MAX_ITERS x N
    float *Q32 = nullptr, *D32 = nullptr, *dlt = nullptr, *gbuf32 = nullptr;
    int* r_it = nullptr;
    int *r = nullptr, *r_old = nullptr, *kept = nullptr, *ranks = nullptr, *zero = nullptr, *nk = nullptr;
    double *G = nullptr, *Rinv = nullptr;   // 64 x 64 Gram matrix and R^-1 of the block Cholesky QR
    int* kept_hist = nullptr;                       // PR_MAX_ITERS x N kept flags
    int M_hist[PR_MAX_ITERS] = {};
    GridBar* gbar = nullptr;
    SplitGemm sg;                 // tensor-core projection state (proj_prec = PR_PROJ_SPLIT_BF16)
    bool use_sg = false;
    long partial_elems = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    TimingRing tr;
    long fine_launch_acc = 0;   // fine-predictor kernel launches of the current solve
    FineLaunch fl;              // launch shape of the FP32 fine steps (parareal_autotune)
    std::string err;
};

static thread_local std::string g_create_err;   // per host thread: concurrent creates do not race

static pr_status set_err(pr_solver* h, pr_status st, const std::string& msg) {
    if (h) h->err = msg; else g_create_err = msg;
    return st;
}

#define CKC(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return set_err(h, PR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));        \
    } while (0)

#define CKS(call)                                                                                   \
    do {                                                                                            \
        pr_status s_ = (call);                                                                      \
        if (s_ != PR_OK) return s_;                                                                 \
    } while (0)

// ------------------------------------------------------------------ sizes

static int default_cap(int N, int K_max) {
    long c = 0;
    for (int k = 0; k < K_max; ++k) c += N - k;
    return (int)(c > 0 ? c : 1);
}

// Whether the KSE path forms the basis images by linearity (Eq. Genhance)
// rather than directly: FP64 fine sweep, FP64 correction, not forced direct.
static bool linear_images(const pr_options& o) {
    return o.variant == PR_KSE && o.corr_prec != PR_FP32 && o.images != PR_IMAGES_DIRECT && o.fine_prec == PR_FP64;
}

struct Sizes {
    long d;
    int cap;
    long partial;
    size_t bytes;
};

static Sizes compute_sizes(int nx, int ny, int N, int K_max, const pr_options& o) {
    Sizes s{};
    s.d = 3L * nx * ny;
    int cap = o.krylov_cap > 0 ? o.krylov_cap : default_cap(N, K_max);
    if (cap > s.d) cap = (int)s.d;
    s.cap = cap < 1 ? 1 : cap;
    s.partial = tswork_elems(s.d, s.cap, N);
    const long pg = tswork_elems(s.d, 64, 64);   // Gram matrices of the block Cholesky QR
    if (pg > s.partial) s.partial = pg;
    size_t dd = sizeof(double);
    size_t b = 0;
    b += dd * (size_t)(N + 1) * s.d;           // q
    b += dd * (size_t)N * s.d * 3;             // qt, gv, wv
    b += dd * (size_t)s.d;                     // FP64 delta of the serial correction
    b += dd * (size_t)N * s.d;                 // wz
    b += dd * (size_t)s.cap * s.d * 2;         // Q, D
    b += dd * (size_t)N * s.d * 2;             // coarse ping-pong
    if (o.fine_prec == PR_FP32)
        b += sizeof(float) * (size_t)N * s.d * 2;
    else if (o.fine_prec == PR_FP32X)
        b += dd * (size_t)N * s.d * 2;
    else
        b += dd * (size_t)N * s.d * 3;         // fine stage buffers
    b += dd * (size_t)s.d * 3;                 // gtmp, chain coarse ping-pong
    if (o.corr_prec == PR_FP32)
        b += sizeof(float) * ((size_t)s.cap * s.d * 2 + (size_t)s.d * 3);   // Q32, D32, delta, ping-pong
    b += dd * (size_t)chain_resp_elems(N);
    b += dd * ((size_t)s.cap * N + s.cap);     // C, cvec
    b += dd * 2 * 64 * 64;                     // G, Rinv
    b += dd * (size_t)s.partial;
    b += dd * (size_t)(N + (N + 1) + PR_MAX_ITERS + 1);
    b += sizeof(int) * (size_t)(3 + N + PR_MAX_ITERS);
    if (o.proj_prec == PR_PROJ_SPLIT_BF16) b += sg_bytes(s.d, s.cap, linear_images(o));
    s.bytes = b;
    return s;
}

// ------------------------------------------------------------------ propagators

// F on n states.  With a slice map (first: the first step, rest: later steps)
// only the slices the map admits are propagated (see SliceMap).
static pr_status fine_apply(pr_solver* h, const double* in, double* out, int n, const SliceMap* first = nullptr,
                            const SliceMap* rest = nullptr) {
    const long d = h->d;
    const bool hv = h->V != 0.0 || h->opt.omega != 0.0;
    cudaStream_t s = h->stream;
    const int nf = h->n_f;
    const SliceMap m0 = first ? *first : SliceMap(), m1 = rest ? *rest : SliceMap();
    if (h->opt.fine_prec == PR_FP32X) {
        const double* a = in;
        for (int st = 0; st < nf; ++st) {
            double* b = st == nf - 1 ? out : (st % 2 == 0 ? h->fb0 : h->fb1);
            CKC(launch_fine_step_acc64(a, b, d, n, h->nx, h->ny, hv, h->fc32, s, st == 0 ? m0 : m1, h->fl));
            a = b;
        }
        return PR_OK;
    }
    if (h->opt.fine_prec == PR_FP32) {
        if (nf == 1) {
            CKC((launch_fine_step<float, double, double>(in, d, out, d, n, h->nx, h->ny, hv, h->fc32, s, m0, h->fl)));
            return PR_OK;
        }
        if (h->fl.rows && fine_rows_eligible(h->nx, hv)) {
            // FP32 copies of the input first, so that the first step also runs
            // on the row-streamed kernel (an FP64 input would be converted at
            // every read): one conversion pass, then FP32 -> FP32
            SliceMap mc = m0;
            mc.in_map = false;
            CKC(launch_to_fp32_states(in, d, h->f32b, d, n, d, m0, s));
            CKC((launch_fine_step<float, float, float>(h->f32b, d, h->f32a, d, n, h->nx, h->ny, hv, h->fc32, s, mc,
                                                       h->fl)));
        } else {
            CKC((launch_fine_step<float, double, float>(in, d, h->f32a, d, n, h->nx, h->ny, hv, h->fc32, s, m0,
                                                        h->fl)));
        }
        float* a = h->f32a;
        float* b = h->f32b;
        for (int st = 1; st < nf - 1; ++st) {
            CKC((launch_fine_step<float, float, float>(a, d, b, d, n, h->nx, h->ny, hv, h->fc32, s, m1, h->fl)));
            float* t = a; a = b; b = t;
        }
        CKC((launch_fine_step<float, float, double>(a, d, out, d, n, h->nx, h->ny, hv, h->fc32, s, m1, h->fl)));
        return PR_OK;
    }
    if (h->fb2 && !first) {
        FineSweepArgs a{};
        a.in = in;
        a.out = out;
        a.w1 = h->fb0;
        a.w2 = h->fb1;
        a.w3 = h->fb2;
        a.n = n;
        a.nx = h->nx;
        a.ny = h->ny;
        a.nsteps = nf;
        a.c = h->fck;
        a.gb = h->gbar;
        a.max_sms = h->opt.sm_limit;
        CKC(fine_sweep_coop(a, hv, s));
        return PR_OK;
    }
    if (nf == 1) {
        CKC((launch_fine_step<double, double, double>(in, d, out, d, n, h->nx, h->ny, hv, h->fc64, s, m0)));
        return PR_OK;
    }
    CKC((launch_fine_step<double, double, double>(in, d, h->fb0, d, n, h->nx, h->ny, hv, h->fc64, s, m0)));
    double* a = h->fb0;
    double* b = h->fb1;
    for (int st = 1; st < nf - 1; ++st) {
        CKC((launch_fine_step<double, double, double>(a, d, b, d, n, h->nx, h->ny, hv, h->fc64, s, m1)));
        double* t = a; a = b; b = t;
    }
    CKC((launch_fine_step<double, double, double>(a, d, out, d, n, h->nx, h->ny, hv, h->fc64, s, m1)));
    return PR_OK;
}

static pr_status coarse_apply(pr_solver* h, const double* in, double* out, int n, bool fp32 = false,
                              const SliceMap* first = nullptr, const SliceMap* rest = nullptr) {
    const long d = h->d;
    cudaStream_t s = h->stream;
    const SliceMap m0 = first ? *first : SliceMap(), m1 = rest ? *rest : SliceMap();
    if (h->n_g == 1) {
        CKC(launch_coarse_step(in, out, d, n, h->nx, h->ny, h->cc, s, fp32, m0));
        return PR_OK;
    }
    CKC(launch_coarse_step(in, h->cb0, d, n, h->nx, h->ny, h->cc, s, fp32, m0));
    double* a = h->cb0;
    double* b = h->cb1;
    for (int st = 1; st < h->n_g - 1; ++st) {
        CKC(launch_coarse_step(a, b, d, n, h->nx, h->ny, h->cc, s, fp32, m1));
        double* t = a; a = b; b = t;
    }
    CKC(launch_coarse_step(a, out, d, n, h->nx, h->ny, h->cc, s, fp32, m1));
    return PR_OK;
}

// ------------------------------------------------------------------ subspace update

// One classical Gram-Schmidt pass of the mm columns v (and their D-images z)
// against the basis columns [0, *r_old): C = Q^T v, v <- v - Q C, z <- z - D C,
// on the FP64 units or with the tensor-core projections.
static pr_status block_pass(pr_solver* h, double* v, double* z, int mm) {
    const long d = h->d;
    const int cap = h->cap;
    cudaStream_t s = h->stream;
    TsWork w{h->partial, h->partial_elems};
    if (h->use_sg) {
        CKC(sg_cgs_pass(&h->sg, v, d, mm, h->r_old, s));
        if (z && h->sg.Dr) {
            CKC(sg_update_images(&h->sg, z, d, mm, h->r_old, s));
        } else if (z) {
            CKC(gemm_nn(h->D, d, nullptr, h->r_old, cap, h->sg.C, h->sg.cap_pad, z, d, z, d, mm, d, -1.0, s));
        }
    } else {
        CKC(gemm_tn(h->Q, d, nullptr, h->r_old, cap, v, d, mm, d, h->C, cap, w, s));
        CKC(gemm_nn(h->Q, d, nullptr, h->r_old, cap, h->C, cap, v, d, v, d, mm, d, -1.0, s));
        if (z) CKC(gemm_nn(h->D, d, nullptr, h->r_old, cap, h->C, cap, z, d, z, d, mm, d, -1.0, s));
    }
    return PR_OK;
}

// Append the m columns V (with fine images FV and coarse images GV) to the
// subspace, in order (Eq. subspaceUpdate), by block Gram-Schmidt with
// reorthogonalisation of the orthonormalised block (the BCGS2 of Barlow and
// Smoktunowicz), in blocks of B columns (16 with the tensor-core
// projections, 64 otherwise):
//   1. one projection pass of the block against the basis present at entry;
//   2. classical Gram-Schmidt twice within the block, column by column, with
//      the drop rule on the residual ratio; the kept columns, normalised,
//      are compacted in place;
//   3. a second projection pass of that orthonormal block against the basis;
//   4. Cholesky QR of the block (its Gram matrix is I up to rounding) and
//      the append.
// Step 3 restores orthogonality to the basis that step 2 loses when the
// block's own columns are nearly dependent (in-block ratios of 1e-6 leave
// components of size eps / 1e-6 along the old basis, and they compound from
// block to block); the drop decisions and ratios come from step 2.  The
// D-images Z = FV - GV receive exactly the same transformations, so
// D = F(Q) - G(Q).
template <typename Mark, typename SubMark>
static pr_status krylov_block(pr_solver* h, const double* V, const double* FV, const double* GV, int m, Mark mark,
                              SubMark sub_mark, double* ratio = nullptr) {
    const long d = h->d;
    const int cap = h->cap;
    cudaStream_t s = h->stream;
    TsWork w{h->partial, h->partial_elems};
    const bool images = FV != nullptr;   // carry D = F(Q) - G(Q) along (Eq. Genhance)
    CKC(cudaMemcpyAsync(h->wv, V, sizeof(double) * m * d, cudaMemcpyDeviceToDevice, s));
    if (images) CKC(sub(FV, GV, h->wz, (long)m * d, s));
    CKC(colnorm2(h->wv, d, m, d, h->anorm2, w, s));
    const int B = h->use_sg ? SG_N : 64;
    for (int j0 = 0; j0 < m; j0 += B) {
        const int mm = m - j0 < B ? m - j0 : B;
        double* v = h->wv + (long)j0 * d;
        double* z = images ? h->wz + (long)j0 * d : nullptr;
        CKC(cudaMemcpyAsync(h->r_old, h->r, sizeof(int), cudaMemcpyDeviceToDevice, s));
        CKS(block_pass(h, v, z, mm));
        CKC(sub_mark(0));
        CKC(intra_block(v, z, d, mm, h->anorm2 + j0, h->r_old, h->r, cap, h->opt.drop_tol, h->Q, h->D,
                        h->kept + j0, ratio ? ratio + j0 : nullptr, w, h->gbar, s, h->opt.sm_limit, true));
        CKC(sub_mark(1));
        CKC(sub_int(h->r, h->r_old, h->nk, s));
        CKS(block_pass(h, v, z, mm));
        CKC(cholqr_block(v, z, d, mm, h->nk, h->use_sg ? h->sg.C : h->C, h->use_sg ? h->sg.cap_pad : cap, h->r_old,
                         h->G, h->Rinv, h->Q, h->D, h->r_old, s));
        if (h->use_sg) {
            CKC(sg_append(&h->sg, h->Q, d, h->r_old, h->r, 0, mm, s));
            if (images && h->sg.Dr) CKC(sg_append_images(&h->sg, h->D, d, h->r_old, h->r, 0, mm, s));
        }
    }
    CKC(mark());
    return PR_OK;
}

static cudaError_t no_mark() { return cudaSuccess; }
static cudaError_t no_sub_mark(int) { return cudaSuccess; }

// ------------------------------------------------------------------ the solve

static ChainArgs chain_args(pr_solver* h, int i_begin, int i_end, const double* qt, const double* kold,
                            const int* r_dev, double* res2) {
    ChainArgs a{};
    a.q = h->q;
    a.qt = qt;
    a.kold = kold;
    a.Q = h->Q;
    a.D = h->D;
    a.r_dev = r_dev;
    a.ccap = h->cap;
    a.i_begin = i_begin;
    a.i_end = i_end;
    a.d = h->d;
    a.nx = h->nx;
    a.ny = h->ny;
    a.cc = h->cc;
    a.n_g = h->n_g;
    a.H = coarse_halo(h->cc);
    a.gbuf = h->gbuf;
    a.cvec = h->cvec;
    a.part = h->partial;
    a.resp = h->resp;
    a.res2 = res2;
    a.gb = h->gbar;
    a.max_blocks = h->opt.sm_limit;
    return a;
}

// One solve of Alg. 2 / Alg. 1 (one parallel step), split into the phases
// between which a batch runs the fine sweeps of all its handles in one
// launch: begin (the serial coarse initialisation), then per iteration
// fine (the parallel predictor), update (the subspace update), images_fine
// (the fine images of the new basis columns, where they are formed
// directly), correct (their coarse images, the serial correction, r^k).  The
// solo solve runs the phases in this order on the handle's stream; a batch
// runs exactly the same phases, so its results are the solo results bit for
// bit.
struct SolveRun {
    pr_solver* h;
    int K, rbase, k = 0, iter = 0, evi = 0;
    bool kse, mixed, direct, gacc, d64;
    cudaEvent_t* ev = nullptr;
    SliceMap img_first, img_rest;   // slice maps of the images sweep

    SolveRun(pr_solver* h_, int K_, int rbase_, bool timing) : h(h_), K(K_), rbase(rbase_) {
        kse = h->opt.variant == PR_KSE;
        mixed = h->opt.corr_prec == PR_FP32;
        // FP32 fine images cannot be divided by small residuals: non-FP64 fine sweeps use direct images
        direct = mixed || h->opt.images == PR_IMAGES_DIRECT || h->opt.fine_prec != PR_FP64;
        // The FP64 KSE path with images by linearity needs the coarse images
        // G(q_i^k) of the new columns.  G(q_i^0) = q_{i+1}^0 bit for bit; later
        // the delta-form correction adds G(delta_i) to them (linearity of G), so
        // no coarse sweep over the columns is needed.
        gacc = kse && !mixed && !direct;
        d64 = kse && !mixed;
        img_first.beg = img_rest.beg = h->r_it;
        img_first.end = img_rest.end = h->r;
        img_first.in_map = true;
        if (timing && h->tr.n < h->tr.max_solves) {
            ev = h->tr.ev.data() + (size_t)h->tr.n * h->tr.per_solve;
            h->tr.K[h->tr.n] = K;
            h->tr.fine_launches[h->tr.n] = 0;
            h->tr.n += 1;
        }
    }
    cudaError_t mark() { return ev ? cudaEventRecord(ev[evi++], h->stream) : cudaSuccess; }
    cudaError_t sub_mark(int) {
        if (!ev) return cudaSuccess;
        const size_t base = ((size_t)(h->tr.n - 1) * h->K_max + iter) * (size_t)h->tr.sub_per_iter;
        int& ns = h->tr.nsub[(size_t)(h->tr.n - 1) * h->K_max + iter];
        if (ns >= 2 * h->tr.sub_per_iter) return cudaSuccess;
        return cudaEventRecord(h->tr.sub[2 * base + ns++], h->stream);
    }
    int M() const { return h->N - k; }       // active slices of iteration k (slices i < k are converged)
    double* qa() const { return h->q + (long)k * h->d; }
    double* qta() const { return h->qt + (long)k * h->d; }
    bool has_images_fine() const { return kse && direct; }

    pr_status begin() {
        const long d = h->d;
        const int N = h->N;
        cudaStream_t s = h->stream;
        CKC(mark());
        // initialisation: q_{i+1}^0 = G(q_i^0), serially (q[0] already holds u0)
        CKC(chain_coop(chain_args(h, 0, N, nullptr, nullptr, nullptr, nullptr), s));
        CKC(fill_int(h->r, 0, 1, s));
        if (gacc) CKC(cudaMemcpyAsync(h->gv, h->q + d, sizeof(double) * (size_t)N * d, cudaMemcpyDeviceToDevice, s));
        CKC(mark());
        if (ev)
            for (int j = 0; j < h->K_max; ++j) h->tr.nsub[(size_t)(h->tr.n - 1) * h->K_max + j] = 0;
        return PR_OK;
    }
    // parallel predictor: q~_{i+1}^k = F(q_i^k).  Slices i < k satisfy
    // q_i^{k} = q_i^{k-1} bit for bit (the correction of a converged slice is
    // K(q) - K(q) = 0), so their fine images, their columns (already in S)
    // and their corrections are skipped.
    pr_status fine() {
        iter = k;
        const uint64_t l0 = parareal_kernel_launches();
        CKS(fine_apply(h, qa(), qta(), M()));
        if (ev) h->tr.fine_launches[h->tr.n - 1] += (long)(parareal_kernel_launches() - l0);
        return PR_OK;
    }
    pr_status update() {
        const long d = h->d;
        const int N = h->N;
        cudaStream_t s = h->stream;
        // coarse images G(q_i^k): K_old of the FP64 original Parareal (the
        // KSE images by linearity have them from the correction, above)
        if (!kse && !mixed) CKS(coarse_apply(h, qa(), h->gv + (long)k * d, M()));
        CKC(mark());
        if (kse) {
            CKC(cudaMemcpyAsync(h->r_it, h->r, sizeof(int), cudaMemcpyDeviceToDevice, s));
            auto mk = [&]() { return mark(); };
            auto smk = [&](int i) { return sub_mark(i); };
            CKS(krylov_block(h, qa(), direct ? nullptr : qta(), h->gv + (long)k * d, M(), mk, smk,
                             h->ratios + (long)(rbase + k) * N));
            CKC(cudaMemcpyAsync(h->kept_hist + (long)(rbase + k) * N, h->kept, sizeof(int) * M(),
                                cudaMemcpyDeviceToDevice, s));
            h->M_hist[rbase + k] = M();
            CKC(mark());
        } else {
            CKC(mark());
            CKC(mark());
        }
        return PR_OK;
    }
    // Images of the columns appended since *r_it computed directly as
    // D_j = F(Q_j) - G(Q_j) (the quantity Eq. Genhance forms by linearity,
    // here without dividing rounding errors by small residuals |R_jj|):
    // images_fine forms F(Q_j) (at most M columns, the exact count known only
    // on the device), correct forms G(Q_j) and D.  Mixed precision uses the
    // FP32 propagators and refreshes the FP32 copies of Q and D used by the
    // serial correction.
    pr_status images_fine() { return fine_apply(h, h->Q, h->wv, M(), &img_first, &img_rest); }
    pr_status correct(int* K_done) {
        const long d = h->d;
        const int N = h->N;
        const int a = k;
        cudaStream_t s = h->stream;
        TsWork w{h->partial, h->partial_elems};
        if (kse) {
            if (direct) {
                // D_j = F(Q_j) - G(Q_j) for the new columns
                CKS(coarse_apply(h, h->Q, h->wz, M(), mixed, &img_first, &img_rest));
                CKC(sub_mapped(h->wv, h->wz, h->D, d, M(), h->r_it, h->r, s));
                if (mixed) CKC(to_fp32_cols(h->Q, h->D, h->Q32, h->D32, d, h->r_it, h->r, M(), s));
            }
            CKC(cudaMemcpyAsync(h->ranks + rbase + k, h->r, sizeof(int), cudaMemcpyDeviceToDevice, s));
        }
        CKC(mark());
        // serial correction
        CKC(cudaMemsetAsync(h->res2, 0, sizeof(double) * (N + 1), s));
        // q_{i+1}^{k+1} = q~_{i+1}^k + K(q_i^{k+1}) - K(q_i^k) (Alg. 2; K = G
        // for Alg. 1) evaluated through the linearity of K as
        // q~ + G(delta) + D Q^T delta, delta = q_i^{k+1} - q_i^k: in FP32 with
        // FP32 copies of Q and D in mixed precision, in FP64 for the KSE
        // correction otherwise; the FP64 original Parareal subtracts
        // K_old = G(q_i^k) literally
        CKC(copy_resid(h->qt + (long)a * d, h->q + (long)(a + 1) * d, d, h->res2 + a + 1, w, s,
                       mixed ? h->dlt : nullptr, d64 ? h->dlt64 : nullptr));
        ChainArgs ca = chain_args(h, a + 1, N, h->qt, kse || mixed ? nullptr : h->gv, kse ? h->r : nullptr,
                                  h->res2);
        if (mixed) {
            ca.dlt = h->dlt;
            ca.Q32 = h->Q32;
            ca.D32 = h->D32;
            ca.gbuf32 = h->gbuf32;
        } else if (d64) {
            ca.dlt64 = h->dlt64;
            if (gacc) ca.gacc = h->gv;
        }
        CKC(chain_coop(ca, s));
        CKC(max_sqrt(h->res2 + 1, N, h->rhist + rbase + k, s));
        CKC(mark());
        *K_done = k + 1;
        ++k;
        return PR_OK;
    }
};

static pr_status solve_impl(pr_solver* h, int K, int rbase, int* K_done) {
    SolveRun run(h, K, rbase, true);
    CKS(run.begin());
    while (run.k < K) {
        CKS(run.fine());
        CKC(run.mark());
        CKS(run.update());
        if (run.has_images_fine()) CKS(run.images_fine());
        const int k = run.k;
        CKS(run.correct(K_done));
        if (h->opt.r_tol > 0) {
            // stopping rule of Sec. 2.1 (one synchronisation per iteration)
            double r = 0.0;
            CKC(cudaMemcpyAsync(&r, h->rhist + rbase + k, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            CKC(cudaStreamSynchronize(h->stream));
            if (r <= h->opt.r_tol) break;
        }
    }
    return PR_OK;
}

static void timing_free(pr_solver* h) {
    for (cudaEvent_t e : h->tr.ev) cudaEventDestroy(e);
    for (cudaEvent_t e : h->tr.sub) cudaEventDestroy(e);
    h->tr = TimingRing();
}

// After a synchronisation: PR_ETIMEOUT if a bounded device wait gave up.
static pr_status check_device_waits(pr_solver* h) {
    int err = 0;
    CKC(cudaMemcpy(&err, &h->gbar->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err == 2) return set_err(h, PR_ECUDA, "the serial chain read a basis rank above the cap; results invalid");
    if (err) return set_err(h, PR_ETIMEOUT, "a grid barrier wait gave up; results of this handle are invalid");
    if (h->opt.fine_prec != PR_FP64 && fine_rows_wait_error(false) > 0)
        return set_err(h, PR_ETIMEOUT, "a fine-sweep row-load wait gave up; FP32 fine sweeps since then are invalid");
    if (h->use_sg) {
        CKC(cudaMemcpy(&err, h->sg.err, sizeof(int), cudaMemcpyDeviceToHost));
        if (err) return set_err(h, PR_ETIMEOUT, "a tensor-core pipeline wait gave up; results of this handle are invalid");
    }
    return PR_OK;
}

// All parallel steps (Sec. 2.1): window w starts from q_N of window w-1.
// q[0] holds u0 on entry.  Iteration records are kept in order, up to
// PR_MAX_ITERS of them.
static pr_status solve_windows(pr_solver* h, int K, std::vector<int>& Kw) {
    const long d = h->d;
    int rbase = 0;
    Kw.clear();
    for (int w = 0; w < h->opt.n_windows; ++w) {
        if (w > 0)
            CKC(cudaMemcpyAsync(h->q, h->q + (long)h->N * d, sizeof(double) * d, cudaMemcpyDeviceToDevice, h->stream));
        const int Kc = rbase + K <= PR_MAX_ITERS ? K : (PR_MAX_ITERS - rbase > 0 ? PR_MAX_ITERS - rbase : 0);
        int done = 0;
        CKS(solve_impl(h, K, Kc < K ? PR_MAX_ITERS - K : rbase, &done));
        Kw.push_back(done);
        rbase += Kc < K ? 0 : done;
    }
    return PR_OK;
}

static pr_status fill_report(pr_solver* h, const std::vector<int>& Kw, pr_report* rep) {
    CKC(cudaStreamSynchronize(h->stream));
    CKS(check_device_waits(h));
    std::memset(rep, 0, sizeof(*rep));
    int K = 0;
    for (int x : Kw) K += x;
    if (K > PR_MAX_ITERS) K = PR_MAX_ITERS;
    rep->K = K;
    rep->n_windows = (int)Kw.size();
    for (size_t w = 0; w < Kw.size() && w < PR_MAX_ITERS; ++w) rep->K_window[w] = Kw[w];
    for (int k = 0; k < PR_MAX_ITERS; ++k) rep->min_ratio[k] = 1.0;
    if (K > 0) {
        CKC(cudaMemcpy(rep->r, h->rhist, sizeof(double) * K, cudaMemcpyDeviceToHost));
        if (h->opt.variant == PR_KSE) {
            CKC(cudaMemcpy(rep->rank, h->ranks, sizeof(int) * K, cudaMemcpyDeviceToHost));
            std::vector<double> rat((size_t)K * h->N);
            std::vector<int> kp((size_t)K * h->N);
            CKC(cudaMemcpy(rat.data(), h->ratios, sizeof(double) * rat.size(), cudaMemcpyDeviceToHost));
            CKC(cudaMemcpy(kp.data(), h->kept_hist, sizeof(int) * kp.size(), cudaMemcpyDeviceToHost));
            for (int k = 0; k < K; ++k)
                for (int j = 0; j < h->M_hist[k]; ++j)
                    if (kp[(size_t)k * h->N + j] && rat[(size_t)k * h->N + j] < rep->min_ratio[k])
                        rep->min_ratio[k] = rat[(size_t)k * h->N + j];
        }
    }
    float ms = 0.f;
    CKC(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    rep->ms_total = ms;
    return PR_OK;
}

// ------------------------------------------------------------------ C ABI

static bool is_fin(double x) { return std::isfinite(x); }

template <typename T>
static FineCoef<T> make_fine_coef(double U, double V, double cs, double dx, double dy, double nu, double dt,
                                  double omega, double lx, double ly) {
    const double a1 = nu * dx * dx / dt, a2 = nu * dy * dy / dt;
    FineCoef<T> c;
    c.omx = (T)(omega / (60.0 * dx));
    c.omy = (T)(omega / (60.0 * dy));
    c.dx = (T)dx;
    c.dy = (T)dy;
    c.hlx = (T)(0.5 * lx);
    c.hly = (T)(0.5 * ly);
    c.ax6 = (T)(U / (60.0 * dx));
    c.ay6 = (T)(V / (60.0 * dy));
    c.csx = (T)(cs / (2.0 * dx));
    c.csy = (T)(cs / (2.0 * dy));
    c.dxx = (T)(a1 / (dx * dx));
    c.dxy1 = (T)(a1 / (4.0 * dx * dy));
    c.dyy = (T)(a2 / (dy * dy));
    c.dxy2 = (T)(a2 / (4.0 * dx * dy));
    c.c1 = (T)(dt / 3.0);
    c.c2 = (T)(dt / 2.0);
    c.c3 = (T)dt;
    return c;
}

extern "C" {

pr_status parareal_default_options(pr_options* o) {
    if (!o) return PR_EINVAL;
    std::memset(o, 0, sizeof(*o));
    o->T = 1.0;
    o->nu_f = 0.005;
    o->nu_c = 0.1;
    o->n_sound = 4;
    o->adv_order_f = 6;
    o->adv_order_c = 1;
    o->V = 0.0;
    o->K_max = 0;
    o->krylov_cap = 0;
    o->drop_tol = 1e-10;
    o->fine_prec = PR_FP64;
    o->variant = PR_KSE;
    o->corr_prec = PR_FP64;
    o->r_tol = 0.0;
    o->n_windows = 1;
    o->images = PR_IMAGES_LINEARITY;
    o->sm_limit = 0;
    o->stream = nullptr;
    o->coarse_scheme = PR_COARSE_SPLIT_FE;
    o->batch_fine = PR_BATCH_STREAMS;
    return PR_OK;
}

static pr_status validate(const pr_grid* g, double U, double c_s, double dt_f, double dt_g, int N,
                          const pr_options& o, int* n_f, int* n_g) {
    pr_solver* h = nullptr;
    if (!g) return set_err(h, PR_EINVAL, "grid is NULL");
    if (g->nx < 4 || g->ny < 4) return set_err(h, PR_EINVAL, "nx and ny must be >= 4");
    if ((long)g->nx * g->ny > (1L << 28)) return set_err(h, PR_EINVAL, "grid too large");
    if (N < 1 || N > 4096) return set_err(h, PR_EINVAL, "N_slices must be in [1, 4096]");
    if (!is_fin(U) || !is_fin(c_s) || !is_fin(o.V) || c_s < 0) return set_err(h, PR_EINVAL, "U, V, c_s must be finite, c_s >= 0");
    if (!(dt_f > 0) || !(dt_g > 0) || !is_fin(dt_f) || !is_fin(dt_g)) return set_err(h, PR_EINVAL, "dt_f, dt_g must be > 0");
    if (!(o.T > 0) || !is_fin(o.T)) return set_err(h, PR_EINVAL, "T must be > 0");
    if (!is_fin(o.nu_f) || !is_fin(o.nu_c) || o.nu_f < 0 || o.nu_c < 0) return set_err(h, PR_EINVAL, "nu_f, nu_c must be >= 0");
    if (o.adv_order_f != 6) return set_err(h, PR_EINVAL, "adv_order_f must be 6");
    if (o.adv_order_c != 1 && o.adv_order_c != 3) return set_err(h, PR_EINVAL, "adv_order_c must be 1 or 3");
    if (o.n_sound < 1) return set_err(h, PR_EINVAL, "n_sound must be >= 1");
    if (!is_fin(o.omega)) return set_err(h, PR_EINVAL, "omega must be finite");
    if (o.coarse_scheme != PR_COARSE_SPLIT_FE && o.coarse_scheme != PR_COARSE_RK3)
        return set_err(h, PR_EINVAL, "coarse_scheme must be PR_COARSE_SPLIT_FE or PR_COARSE_RK3");
    if (o.coarse_scheme == PR_COARSE_SPLIT_FE && (o.adv_order_c == 1 ? 1 : 2) + 2 * o.n_sound - 1 > 12)
        return set_err(h, PR_EINVAL, "n_sound too large for the fused coarse step (halo > 12)");
    if (o.fine_prec != PR_FP64 && o.fine_prec != PR_FP32 && o.fine_prec != PR_FP32X)
        return set_err(h, PR_EINVAL, "fine_prec must be PR_FP64, PR_FP32 or PR_FP32X");
    if (o.variant != PR_KSE && o.variant != PR_ORIGINAL) return set_err(h, PR_EINVAL, "variant must be PR_KSE or PR_ORIGINAL");
    if (o.corr_prec != PR_FP64 && o.corr_prec != PR_FP32) return set_err(h, PR_EINVAL, "corr_prec must be PR_FP64 or PR_FP32");
    if (!(o.r_tol >= 0) || !is_fin(o.r_tol)) return set_err(h, PR_EINVAL, "r_tol must be >= 0");
    if (o.n_windows < 1 || o.n_windows > 1000000) return set_err(h, PR_EINVAL, "n_windows must be >= 1");
    if (o.images != PR_IMAGES_LINEARITY && o.images != PR_IMAGES_DIRECT) return set_err(h, PR_EINVAL, "images must be PR_IMAGES_LINEARITY or PR_IMAGES_DIRECT");
    if (o.sm_limit < 0) return set_err(h, PR_EINVAL, "sm_limit must be >= 0");
    if (o.proj_prec != PR_PROJ_FP64 && o.proj_prec != PR_PROJ_SPLIT_BF16)
        return set_err(h, PR_EINVAL, "proj_prec must be PR_PROJ_FP64 or PR_PROJ_SPLIT_BF16");
    if (o.proj_prec == PR_PROJ_SPLIT_BF16 && (3L * g->nx * g->ny) % 8 != 0)
        return set_err(h, PR_EINVAL, "PR_PROJ_SPLIT_BF16 needs 3*nx*ny to be a multiple of 8");
    if (!(o.drop_tol >= 0) || !is_fin(o.drop_tol)) return set_err(h, PR_EINVAL, "drop_tol must be >= 0");
    if (o.K_max < 0 || o.K_max > PR_MAX_ITERS || o.K_max > N) return set_err(h, PR_EINVAL, "K_max must be in [0, min(N, 128)]");
    if (o.krylov_cap < 0 || o.krylov_cap > 1600) return set_err(h, PR_EINVAL, "krylov_cap must be in [0, 1600]");
    const double DT = o.T / ((double)N * o.n_windows);
    double nf = DT / dt_f, ng = DT / dt_g;
    long inf = std::lround(nf), ing = std::lround(ng);
    if (inf < 1 || std::fabs(inf * dt_f - DT) > 1e-9 * DT) return set_err(h, PR_EINVAL, "T/(N n_windows) is not an integer multiple of dt_f");
    if (ing < 1 || std::fabs(ing * dt_g - DT) > 1e-9 * DT) return set_err(h, PR_EINVAL, "T/(N n_windows) is not an integer multiple of dt_g");
    if (inf > 100000 || ing > 100000) return set_err(h, PR_EINVAL, "too many steps per slice");
    *n_f = (int)inf;
    *n_g = (int)ing;
    return PR_OK;
}

size_t parareal_footprint_bytes(const pr_grid* g, int32_t N_slices, const pr_options* opt) {
    pr_options o;
    if (opt) o = *opt; else parareal_default_options(&o);
    if (!g || g->nx < 1 || g->ny < 1 || N_slices < 1) return 0;
    int K_max = o.K_max > 0 ? o.K_max : N_slices;
    return compute_sizes(g->nx, g->ny, N_slices, K_max, o).bytes;
}

pr_status parareal_create(const pr_grid* g, double U, double c_s, double dt_f, double dt_g, int32_t N_slices,
                          const pr_options* opt, pr_solver** out) {
    if (!out) return set_err(nullptr, PR_EINVAL, "out is NULL");
    *out = nullptr;
    pr_options o;
    if (opt) o = *opt; else parareal_default_options(&o);
    int n_f = 0, n_g = 0;
    CKS(validate(g, U, c_s, dt_f, dt_g, N_slices, o, &n_f, &n_g));
    pr_solver* h = new (std::nothrow) pr_solver();
    if (!h) return set_err(nullptr, PR_ENOMEM, "host allocation failed");
    h->nx = g->nx;
    h->ny = g->ny;
    h->lx = g->lx > 0 ? g->lx : 1.0;
    h->ly = g->ly > 0 ? g->ly : 1.0;
    h->N = N_slices;
    h->n_f = n_f;
    h->n_g = n_g;
    h->K_max = o.K_max > 0 ? o.K_max : N_slices;
    h->U = U;
    h->V = o.V;
    h->cs = c_s;
    h->dt_f = dt_f;
    h->dt_g = dt_g;
    h->opt = o;
    h->stream = (cudaStream_t)o.stream;
    Sizes sz = compute_sizes(h->nx, h->ny, h->N, h->K_max, o);
    h->d = sz.d;
    h->cap = sz.cap;
    h->partial_elems = sz.partial;
    const double dx = h->lx / h->nx, dy = h->ly / h->ny;
    h->fc64 = make_fine_coef<double>(U, o.V, c_s, dx, dy, o.nu_f, dt_f, o.omega, h->lx, h->ly);
    h->fc32 = make_fine_coef<float>(U, o.V, c_s, dx, dy, o.nu_f, dt_f, o.omega, h->lx, h->ly);
    h->fck = make_fine_coef_k(U, o.V, c_s, dx, dy, o.nu_f, dt_f, o.omega, h->lx, h->ly);
    const double tau = o.coarse_scheme == PR_COARSE_RK3 ? dt_g : dt_g / o.n_sound;
    const double a1 = o.nu_c * dx * dx / tau, a2 = o.nu_c * dy * dy / tau;
    h->cc.U = U;
    h->cc.V = o.V;
    h->cc.inv_dx = 1.0 / dx;
    h->cc.inv_dy = 1.0 / dy;
    h->cc.tau = tau;
    h->cc.csx = c_s / (2.0 * dx);
    h->cc.csy = c_s / (2.0 * dy);
    h->cc.dxx = a1 / (dx * dx);
    h->cc.dxy1 = a1 / (4.0 * dx * dy);
    h->cc.dyy = a2 / (dy * dy);
    h->cc.dxy2 = a2 / (4.0 * dx * dy);
    h->cc.n_sound = o.n_sound;
    h->cc.order = o.adv_order_c;
    h->cc.scheme = o.coarse_scheme == PR_COARSE_RK3 ? 1 : 0;
    h->cc.omega = o.omega;
    h->cc.dx = dx;
    h->cc.dy = dy;
    h->cc.hlx = 0.5 * h->lx;
    h->cc.hly = 0.5 * h->ly;

    const long d = h->d;
    const int N = h->N;
    auto dalloc = [&](double** p, size_t n) { return cudaMalloc((void**)p, sizeof(double) * (n ? n : 1)); };
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    chk(dalloc(&h->q, (size_t)(N + 1) * d));
    chk(dalloc(&h->qt, (size_t)N * d));
    chk(dalloc(&h->gv, (size_t)N * d));
    chk(dalloc(&h->dlt64, (size_t)d));
    chk(dalloc(&h->wv, (size_t)N * d));
    chk(dalloc(&h->wz, (size_t)N * d));
    chk(dalloc(&h->Q, (size_t)h->cap * d));
    chk(dalloc(&h->D, (size_t)h->cap * d));
    chk(dalloc(&h->cb0, (size_t)N * d));
    chk(dalloc(&h->cb1, (size_t)N * d));
    if (o.fine_prec == PR_FP32) {
        chk(cudaMalloc((void**)&h->f32a, sizeof(float) * (size_t)N * d));
        chk(cudaMalloc((void**)&h->f32b, sizeof(float) * (size_t)N * d));
    } else if (o.fine_prec == PR_FP32X) {
        chk(dalloc(&h->fb0, (size_t)N * d));
        chk(dalloc(&h->fb1, (size_t)N * d));
    } else {
        chk(dalloc(&h->fb0, (size_t)N * d));
        chk(dalloc(&h->fb1, (size_t)N * d));
        chk(dalloc(&h->fb2, (size_t)N * d));
    }
    chk(dalloc(&h->gtmp, (size_t)d));
    chk(dalloc(&h->gbuf, (size_t)2 * d));
    chk(dalloc(&h->ratios, (size_t)PR_MAX_ITERS * N));
    chk(dalloc(&h->resp, (size_t)chain_resp_elems(N)));
    chk(dalloc(&h->C, (size_t)h->cap * N));
    chk(dalloc(&h->cvec, (size_t)h->cap));
    chk(dalloc(&h->partial, (size_t)h->partial_elems));
    chk(dalloc(&h->anorm2, (size_t)N));
    chk(dalloc(&h->res2, (size_t)N + 1));
    chk(dalloc(&h->rhist, (size_t)PR_MAX_ITERS));
    chk(dalloc(&h->nres2, 1));
    chk(cudaMalloc((void**)&h->r, sizeof(int) * 8));
    chk(dalloc(&h->G, 64 * 64));
    chk(dalloc(&h->Rinv, 64 * 64));
    if (o.corr_prec == PR_FP32) {
        chk(cudaMalloc((void**)&h->Q32, sizeof(float) * (size_t)h->cap * d));
        chk(cudaMalloc((void**)&h->D32, sizeof(float) * (size_t)h->cap * d));
        chk(cudaMalloc((void**)&h->dlt, sizeof(float) * (size_t)d));
        chk(cudaMalloc((void**)&h->gbuf32, sizeof(float) * (size_t)2 * d));
    }
    chk(cudaMalloc((void**)&h->kept, sizeof(int) * N));
    chk(cudaMalloc((void**)&h->ranks, sizeof(int) * PR_MAX_ITERS));
    chk(cudaMalloc((void**)&h->kept_hist, sizeof(int) * PR_MAX_ITERS * N));
    chk(cudaMalloc((void**)&h->gbar, sizeof(GridBar)));
    if (e == cudaSuccess) {
        h->r_old = h->r + 1;
        h->zero = h->r + 2;
        h->r_it = h->r + 3;
        h->nk = h->r + 4;
        chk(cudaMemset(h->r, 0, sizeof(int) * 8));
        chk(cudaMemset(h->ranks, 0, sizeof(int) * PR_MAX_ITERS));
        chk(cudaMemset(h->gbar, 0, sizeof(GridBar)));
        chk(cudaMemset(h->rhist, 0, sizeof(double) * PR_MAX_ITERS));
        chk(cudaEventCreate(&h->ev0));
        chk(cudaEventCreate(&h->ev1));
    }
    if (e == cudaSuccess && o.proj_prec == PR_PROJ_SPLIT_BF16) {
        chk(sg_init(&h->sg, d, h->cap, linear_images(o)));
        h->use_sg = e == cudaSuccess;
    }
    if (e != cudaSuccess) {
        std::string msg = std::string("device allocation failed: ") + cudaGetErrorString(e);
        cudaGetLastError();
        parareal_destroy(h);
        return set_err(nullptr, e == cudaErrorMemoryAllocation ? PR_ENOMEM : PR_ECUDA, msg);
    }
    *out = h;
    return PR_OK;
}

pr_status parareal_destroy(pr_solver* h) {
    if (!h) return PR_EINVAL;
    if (h->stream || h->q) cudaStreamSynchronize(h->stream);
    double* ds[] = {h->q, h->qt, h->gv, h->dlt64, h->Q, h->D, h->wv, h->wz, h->fb0, h->fb1, h->fb2, h->cb0, h->cb1,
                    h->gtmp, h->C, h->cvec, h->partial, h->anorm2, h->res2, h->rhist, h->nres2,
                    h->gbuf, h->resp, h->ratios, h->G, h->Rinv};
    for (double* p : ds) if (p) cudaFree(p);
    float* fs[] = {h->Q32, h->D32, h->dlt, h->gbuf32};
    for (float* p : fs) if (p) cudaFree(p);
    if (h->f32a) cudaFree(h->f32a);
    if (h->f32b) cudaFree(h->f32b);
    if (h->r) cudaFree(h->r);
    if (h->kept) cudaFree(h->kept);
    if (h->ranks) cudaFree(h->ranks);
    if (h->kept_hist) cudaFree(h->kept_hist);
    if (h->gbar) cudaFree(h->gbar);
    if (h->use_sg) sg_free(&h->sg);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    timing_free(h);
    delete h;
    return PR_OK;
}

const char* parareal_last_error(const pr_solver* h) { return h ? h->err.c_str() : g_create_err.c_str(); }

pr_status parareal_solve(pr_solver* h, const double* u0_dev, int32_t K, double* q_out_dev, double* qT_dev,
                         pr_report* rep) {
    if (!h) return PR_EINVAL;
    if (!u0_dev) return set_err(h, PR_EINVAL, "u0 is NULL");
    if (K < 0 || K > h->K_max) return set_err(h, PR_EINVAL, "K_iters out of [0, K_max]");
    const long d = h->d;
    CKC(cudaEventRecord(h->ev0, h->stream));
    CKC(cudaMemcpyAsync(h->q, u0_dev, sizeof(double) * d, cudaMemcpyDeviceToDevice, h->stream));
    std::vector<int> Kw;
    CKS(solve_windows(h, K, Kw));
    CKC(cudaEventRecord(h->ev1, h->stream));
    if (q_out_dev)
        CKC(cudaMemcpyAsync(q_out_dev, h->q, sizeof(double) * (h->N + 1) * d, cudaMemcpyDeviceToDevice, h->stream));
    if (qT_dev)
        CKC(cudaMemcpyAsync(qT_dev, h->q + (long)h->N * d, sizeof(double) * d, cudaMemcpyDeviceToDevice, h->stream));
    if (rep) CKS(fill_report(h, Kw, rep));
    return PR_OK;
}

pr_status parareal_solve_host(pr_solver* h, const double* u0_host, int32_t K, double* qT_host, pr_report* rep) {
    if (!h) return PR_EINVAL;
    if (!u0_host || !qT_host) return set_err(h, PR_EINVAL, "host buffers must be non-NULL");
    if (K < 0 || K > h->K_max) return set_err(h, PR_EINVAL, "K_iters out of [0, K_max]");
    const long d = h->d;
    CKC(cudaEventRecord(h->ev0, h->stream));
    CKC(cudaMemcpyAsync(h->q, u0_host, sizeof(double) * d, cudaMemcpyHostToDevice, h->stream));
    std::vector<int> Kw;
    CKS(solve_windows(h, K, Kw));
    CKC(cudaMemcpyAsync(qT_host, h->q + (long)h->N * d, sizeof(double) * d, cudaMemcpyDeviceToHost, h->stream));
    CKC(cudaEventRecord(h->ev1, h->stream));
    CKC(cudaStreamSynchronize(h->stream));
    CKS(check_device_waits(h));
    if (rep) CKS(fill_report(h, Kw, rep));
    return PR_OK;
}

pr_status parareal_fine_sweep(pr_solver* h, const double* q_in_dev, double* q_out_dev, int32_t n) {
    if (!h) return PR_EINVAL;
    if (!q_in_dev || !q_out_dev) return set_err(h, PR_EINVAL, "NULL buffer");
    if (n < 1 || n > h->N) return set_err(h, PR_EINVAL, "n must be in [1, N_slices]");
    return fine_apply(h, q_in_dev, q_out_dev, n);
}

pr_status parareal_coarse_apply(pr_solver* h, const double* q_in_dev, double* q_out_dev, int32_t n) {
    if (!h) return PR_EINVAL;
    if (!q_in_dev || !q_out_dev) return set_err(h, PR_EINVAL, "NULL buffer");
    if (n < 1 || n > h->N) return set_err(h, PR_EINVAL, "n must be in [1, N_slices]");
    return coarse_apply(h, q_in_dev, q_out_dev, n);
}

pr_status parareal_coarse_sweep(pr_solver* h, const double* q0_dev, double* q_out_dev) {
    if (!h) return PR_EINVAL;
    if (!q0_dev || !q_out_dev) return set_err(h, PR_EINVAL, "NULL buffer");
    const long d = h->d;
    CKS(coarse_apply(h, q0_dev, q_out_dev, 1));
    for (int i = 1; i < h->N; ++i)
        CKS(coarse_apply(h, q_out_dev + (long)(i - 1) * d, q_out_dev + (long)i * d, 1));
    return PR_OK;
}

pr_status krylov_reset(pr_solver* h) {
    if (!h) return PR_EINVAL;
    CKC(fill_int(h->r, 0, 1, h->stream));
    return PR_OK;
}

pr_status krylov_update(pr_solver* h, const double* V_dev, const double* FV_dev, int32_t m, int32_t* kept_host) {
    if (!h) return PR_EINVAL;
    if (!V_dev || !FV_dev) return set_err(h, PR_EINVAL, "NULL buffer");
    if (m < 1 || m > h->N) return set_err(h, PR_EINVAL, "m must be in [1, N_slices]");
    CKS(coarse_apply(h, V_dev, h->gv, m));
    CKS(krylov_block(h, V_dev, FV_dev, h->gv, m, no_mark, no_sub_mark));
    if (kept_host) {
        CKC(cudaMemcpyAsync(kept_host, h->kept, sizeof(int) * m, cudaMemcpyDeviceToHost, h->stream));
        CKC(cudaStreamSynchronize(h->stream));
        CKS(check_device_waits(h));
    }
    return PR_OK;
}

pr_status krylov_rank(pr_solver* h, int32_t* rank) {
    if (!h || !rank) return PR_EINVAL;
    CKC(cudaMemcpyAsync(rank, h->r, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CKC(cudaStreamSynchronize(h->stream));
    return PR_OK;
}

pr_status krylov_project(pr_solver* h, const double* q_dev, double* Pq_dev, double* FPq_dev) {
    if (!h) return PR_EINVAL;
    if (!q_dev) return set_err(h, PR_EINVAL, "q is NULL");
    const long d = h->d;
    cudaStream_t s = h->stream;
    TsWork w{h->partial, h->partial_elems};
    double* pq = Pq_dev ? Pq_dev : h->wv;
    CKC(gemm_tn(h->Q, d, nullptr, h->r, h->cap, q_dev, d, 1, d, h->cvec, h->cap, w, s));
    CKC(gemm_nn(h->Q, d, nullptr, h->r, h->cap, h->cvec, h->cap, nullptr, d, pq, d, 1, d, 1.0, s));
    if (FPq_dev) {
        CKS(coarse_apply(h, pq, h->gtmp, 1));
        CKC(gemm_nn(h->D, d, nullptr, h->r, h->cap, h->cvec, h->cap, h->gtmp, d, FPq_dev, d, 1, d, 1.0, s));
    }
    return PR_OK;
}

pr_status parareal_timing_enable(pr_solver* h, int32_t max_solves) {
    if (!h) return PR_EINVAL;
    if (max_solves < 0 || max_solves > 100000) return set_err(h, PR_EINVAL, "max_solves out of range");
    CKC(cudaStreamSynchronize(h->stream));
    timing_free(h);
    if (max_solves == 0) return PR_OK;
    h->tr.max_solves = max_solves;
    h->tr.per_solve = 2 + 6 * h->K_max;
    h->tr.ev.assign((size_t)max_solves * h->tr.per_solve, nullptr);
    h->tr.K.assign((size_t)max_solves, 0);
    h->tr.fine_launches.assign((size_t)max_solves, 0);
    h->tr.sub_per_iter = (h->N + (h->use_sg ? SG_N : 64) - 1) / (h->use_sg ? SG_N : 64);
    h->tr.sub.assign((size_t)max_solves * h->K_max * 2 * h->tr.sub_per_iter, nullptr);
    h->tr.nsub.assign((size_t)max_solves * h->K_max, 0);
    for (auto& e : h->tr.sub) {
        cudaError_t x = cudaEventCreate(&e);
        if (x != cudaSuccess) {
            timing_free(h);
            return set_err(h, PR_ECUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(x));
        }
    }
    for (auto& e : h->tr.ev) {
        cudaError_t x = cudaEventCreate(&e);
        if (x != cudaSuccess) {
            timing_free(h);
            return set_err(h, PR_ECUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(x));
        }
    }
    return PR_OK;
}

pr_status parareal_timing_read(pr_solver* h, pr_timing* t, int32_t reset) {
    if (!h || !t) return PR_EINVAL;
    CKC(cudaStreamSynchronize(h->stream));
    CKS(check_device_waits(h));
    std::memset(t, 0, sizeof(*t));
    const long ncell = (long)h->nx * h->ny;
    for (int sidx = 0; sidx < h->tr.n; ++sidx) {
        cudaEvent_t* ev = h->tr.ev.data() + (size_t)sidx * h->tr.per_solve;
        const int K = h->tr.K[sidx];
        float ms = 0.f;
        CKC(cudaEventElapsedTime(&ms, ev[0], ev[1]));
        t->ms_init += ms;
        t->ms_total += ms;
        for (int k = 0; k < K; ++k) {
            double* acc[6] = {&t->ms_fine, &t->ms_coarse, &t->ms_gs_block, &t->ms_gs_intra, &t->ms_kold, &t->ms_chain};
            for (int ph = 0; ph < 6; ++ph) {
                CKC(cudaEventElapsedTime(&ms, ev[1 + 6 * k + ph], ev[2 + 6 * k + ph]));
                *acc[ph] += ms;
                if (ph >= 2 && ph <= 4) t->ms_krylov += ms;
                t->ms_total += ms;
            }
            if (h->tr.sub_per_iter > 0) {
                // in-block Gram-Schmidt segments inside the projection phase
                const size_t it = (size_t)sidx * h->K_max + k;
                const int ns = h->tr.nsub[it];
                cudaEvent_t* se = h->tr.sub.data() + 2 * it * h->tr.sub_per_iter;
                for (int p = 0; p + 1 < ns; p += 2) {
                    CKC(cudaEventElapsedTime(&ms, se[p], se[p + 1]));
                    t->ms_gs_block -= ms;
                    t->ms_gs_intra += ms;
                }
            }
            t->fine_cell_steps += (double)(h->N - k) * h->n_f * ncell;
        }
        t->fine_launches += h->tr.fine_launches[sidx];
        t->n_solves += 1;
    }
    if (reset) h->tr.n = 0;
    return PR_OK;
}

uint64_t parareal_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

pr_status parareal_status(pr_solver* h) {
    if (!h) return PR_EINVAL;
    CKC(cudaStreamSynchronize(h->stream));
    return check_device_waits(h);
}

// ------------------------------------------------------------------ autotuning

}  // extern "C"

namespace {
// Process-wide cache of tuned launch shapes: (device, nx, ny, N, fine_prec,
// V != 0) -> (kernel kind, choice).
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int>, std::pair<int, int>> g_tune;
}  // namespace

extern "C" {

pr_status parareal_autotune(pr_solver* h, pr_tuning* out) {
    if (!h) return PR_EINVAL;
    pr_tuning t;
    std::memset(&t, 0, sizeof(t));
    t.choice = -1;
    const bool hv = h->V != 0.0 || h->opt.omega != 0.0;
    const int prec = h->opt.fine_prec;
    int kind = 0;
    if (prec == PR_FP32X)
        kind = hv ? 0 : 1;
    else if (prec == PR_FP32)
        kind = fine_rows_eligible(h->nx, hv) ? 2 : (hv ? 0 : 1);
    t.kernel = kind;
    if (kind == 0) {
        if (out) *out = t;
        return PR_OK;
    }
    int dev = 0;
    CKC(cudaGetDevice(&dev));
    const auto key = std::make_tuple(dev, h->nx, h->ny, h->N, prec, (int)hv);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end() && it->second.first == kind) {
            if (kind == 1) h->fl.tile = it->second.second; else h->fl.min_rows = it->second.second;
            t.choice = it->second.second;
            t.cached = 1;
            if (out) *out = t;
            return PR_OK;
        }
    }
    const int nc = kind == 1 ? kFineTiles : 4;
    const int rows_cand[4] = {8, 16, 32, 64};
    const long d = h->d;
    const size_t elems = (size_t)h->N * d;
    cudaStream_t s = h->stream;
    if (prec == PR_FP32X)
        CKC(cudaMemsetAsync(h->fb0, 0, sizeof(double) * elems, s));
    else
        CKC(cudaMemsetAsync(h->f32a, 0, sizeof(float) * elems, s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CKC(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return set_err(h, PR_ECUDA, "cudaEventCreate failed");
    }
    const int reps = 20;
    float best = 0.f;
    int bi = 0;
    cudaError_t err = cudaSuccess;
    for (int c = 0; c < nc && err == cudaSuccess; ++c) {
        FineLaunch fl = h->fl;
        if (kind == 1) fl.tile = c; else fl.min_rows = rows_cand[c];
        t.candidates[c] = kind == 1 ? c : rows_cand[c];
        for (int r = 0; r <= reps && err == cudaSuccess; ++r) {
            if (r == 1) err = cudaEventRecord(e0, s);
            if (err != cudaSuccess) break;
            if (prec == PR_FP32X)
                err = launch_fine_step_acc64(h->fb0, h->fb1, d, h->N, h->nx, h->ny, hv, h->fc32, s, SliceMap(), fl);
            else
                err = launch_fine_step<float, float, float>(h->f32a, d, h->f32b, d, h->N, h->nx, h->ny, hv, h->fc32,
                                                            s, SliceMap(), fl);
        }
        if (err == cudaSuccess) err = cudaEventRecord(e1, s);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        t.us_per_step[c] = 1e3f * ms / reps;
        if (c == 0 || t.us_per_step[c] < best) {
            best = t.us_per_step[c];
            bi = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return set_err(h, PR_ECUDA, std::string("autotune: ") + cudaGetErrorString(err));
    CKS(check_device_waits(h));
    t.n_candidates = nc;
    t.choice = t.candidates[bi];
    if (kind == 1) h->fl.tile = t.choice; else h->fl.min_rows = t.choice;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = std::make_pair(kind, t.choice);
    }
    if (out) *out = t;
    return PR_OK;
}

// ------------------------------------------------------------------ batches

pr_status parareal_solve_batch(pr_solver* const* hs, int32_t n, const double* const* u0_dev, const int32_t* K,
                               double* const* qT_dev) {
    if (!hs || !u0_dev || !K || !qT_dev || n < 1) return PR_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!hs[i] || !u0_dev[i] || !qT_dev[i] || K[i] < 0 || K[i] > hs[i]->K_max) return PR_EINVAL;
    for (int i = 0; i < n; ++i) CKS(parareal_solve(hs[i], u0_dev[i], K[i], nullptr, qT_dev[i], nullptr));
    for (int i = 0; i < n; ++i) {
        pr_solver* h = hs[i];
        CKC(cudaStreamSynchronize(h->stream));
        CKS(check_device_waits(h));
    }
    return PR_OK;
}

}  // extern "C"

struct pr_batch {
    std::vector<pr_solver*> hs;
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> ev;   // fork + one join per handle (+ one for the batched launches)
    bool lockstep = false;         // fine sweeps batched per group of handles of one shape
    struct Group {
        std::vector<int> idx;              // handles of the group
        cudaStream_t stream = nullptr;     // the group's batched fine launches
        GridBar* gb = nullptr;
        cudaEvent_t ev = nullptr;
        int sm_limit = 0;                  // SMs of its batched launches (0: all)
        std::vector<long> first, count, total;   // per batched launch: its items and work indices
        std::vector<int> maxnf;
    };
    std::vector<Group> groups;
    FineBatchItem* items = nullptr;   // device: the work tables of all batched launches
};

static void batch_free(pr_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto& g : b->groups) {
        if (g.gb) cudaFree(g.gb);
        if (g.ev) cudaEventDestroy(g.ev);
        if (g.stream) cudaStreamDestroy(g.stream);
    }
    if (b->items) cudaFree(b->items);
    for (cudaEvent_t e : b->ev)
        if (e) cudaEventDestroy(e);
    delete b;
}

// A batch whose handles all ask for persistent fine sweeps and run the
// FP32-tendency fine sweep (PR_FP32X) of constant velocity with V = 0 and
// KSE-Parareal in one parallel step runs its fine sweeps batched: the solves
// advance in lockstep phase by phase (see SolveRun); at each fine phase (the
// predictor of iteration k, the fine images of the new basis columns) the
// sweeps of every handle still iterating run as one persistent cooperative
// launch over all their (state, tile) items, forked from and joined back
// into the handles' streams.
static bool batch_lockstep_ok(pr_solver* const* hs, int n) {
    for (int i = 0; i < n; ++i) {
        const pr_solver* h = hs[i];
        if (h->opt.batch_fine != PR_BATCH_PERSISTENT || h->opt.fine_prec != PR_FP32X || h->V != 0.0 || h->opt.omega != 0.0 || h->opt.variant != PR_KSE ||
            h->opt.n_windows != 1)
            return false;
    }
    return true;
}

static FineBatchItem batch_item(pr_solver* h, const double* in, double* out, int n, const SliceMap* first,
                                const SliceMap* rest) {
    FineBatchItem it{};
    it.in = in;
    it.out = out;
    it.w0 = h->fb0;
    it.w1 = h->fb1;
    if (first) it.first = *first;
    if (rest) it.rest = *rest;
    it.c = h->fc32;
    it.d = h->d;
    it.nx = h->nx;
    it.ny = h->ny;
    it.n = n;
    it.nf = h->n_f;
    fine_batch_tiles(h->nx, h->ny, &it.tiles_x, &it.tiles);
    return it;
}

// Groups, their streams and barriers, and the work tables (per group and
// iteration k: the predictor q_i^k -> q~_{i+1}^k over N - k states and the
// fine images Q[:, *r_it ..] -> wv of at most N - k columns, one item per
// handle of the group still iterating), built and uploaded before capture.
static cudaError_t batch_setup(pr_batch* b, const int32_t* K) {
    const int n = (int)b->hs.size();
    // one group over all handles (grouping by problem shape, each group with
    // its own persistent launches side by side, measured slower: 64 uneven
    // instances took 1.60 s against 1.17 s in one group)
    b->groups.emplace_back();
    for (int i = 0; i < n; ++i) b->groups.back().idx.push_back(i);
    std::vector<FineBatchItem> tab;
    for (auto& g : b->groups) {
        cudaError_t e = cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc((void**)&g.gb, sizeof(GridBar));
        if (e == cudaSuccess) e = cudaMemset(g.gb, 0, sizeof(GridBar));
        if (e != cudaSuccess) return e;
        int Kmax = 0;
        for (int i : g.idx) Kmax = K[i] > Kmax ? K[i] : Kmax;
        for (int k = 0; k < Kmax; ++k) {
            for (int images = 0; images < 2; ++images) {
                g.first.push_back((long)tab.size());
                long tile0 = 0;
                int mnf = 0;
                for (int i : g.idx) {
                    if (k >= K[i]) continue;
                    pr_solver* h = b->hs[i];
                    const int M = h->N - k;
                    FineBatchItem it;
                    if (images) {
                        SliceMap first, rest;
                        first.beg = rest.beg = h->r_it;
                        first.end = rest.end = h->r;
                        first.in_map = true;
                        it = batch_item(h, h->Q, h->wv, M, &first, &rest);
                    } else {
                        it = batch_item(h, h->q + (long)k * h->d, h->qt + (long)k * h->d, M, nullptr, nullptr);
                    }
                    it.tile0 = tile0;
                    tile0 += (long)it.n * it.tiles;
                    mnf = it.nf > mnf ? it.nf : mnf;
                    tab.push_back(it);
                }
                g.count.push_back((long)tab.size() - g.first.back());
                g.total.push_back(tile0);
                g.maxnf.push_back(mnf);
            }
        }
    }
    cudaError_t e = cudaMalloc((void**)&b->items, sizeof(FineBatchItem) * (tab.empty() ? 1 : tab.size()));
    if (e == cudaSuccess && !tab.empty())
        e = cudaMemcpy(b->items, tab.data(), sizeof(FineBatchItem) * tab.size(), cudaMemcpyHostToDevice);
    return e;
}

// Capture body of a lockstep batch (the caller has begun capture on b->stream
// and recorded b->ev[0] there).
static pr_status batch_capture_lockstep(pr_batch* b, const double* const* u0_dev, const int32_t* K,
                                        double* const* qT_dev) {
    pr_solver* h = b->hs[0];   // errors are reported on the first handle
    for (auto& g : b->groups) {
        int Kmax = 0;
        for (int i : g.idx) Kmax = K[i] > Kmax ? K[i] : Kmax;
        CKC(cudaStreamWaitEvent(g.stream, b->ev[0], 0));
        std::vector<SolveRun> runs;
        runs.reserve(g.idx.size());
        for (int i : g.idx) {
            pr_solver* hi = b->hs[i];
            CKC(cudaStreamWaitEvent(hi->stream, b->ev[0], 0));
            CKC(cudaEventRecord(hi->ev0, hi->stream));
            CKC(cudaMemcpyAsync(hi->q, u0_dev[i], sizeof(double) * hi->d, cudaMemcpyDeviceToDevice, hi->stream));
            runs.emplace_back(hi, K[i], 0, false);
            CKS(runs.back().begin());
        }
        // a batched fine phase: join the handles still iterating, one launch, fork
        auto batched = [&](int k, int li) -> pr_status {
            for (int i : g.idx) {
                if (k >= K[i]) continue;
                CKC(cudaEventRecord(b->ev[i + 1], b->hs[i]->stream));
                CKC(cudaStreamWaitEvent(g.stream, b->ev[i + 1], 0));
            }
            CKC(fine_batch_coop(b->items + g.first[li], (int)g.count[li], g.total[li], g.maxnf[li], g.gb,
                                g.stream, g.sm_limit));
            CKC(cudaEventRecord(g.ev, g.stream));
            for (int i : g.idx)
                if (k < K[i]) CKC(cudaStreamWaitEvent(b->hs[i]->stream, g.ev, 0));
            return PR_OK;
        };
        for (int k = 0; k < Kmax; ++k) {
            CKS(batched(k, 2 * k));
            for (size_t j = 0; j < g.idx.size(); ++j) {
                if (k >= K[g.idx[j]]) continue;
                CKC(runs[j].mark());
                CKS(runs[j].update());
            }
            CKS(batched(k, 2 * k + 1));
            int done = 0;
            for (size_t j = 0; j < g.idx.size(); ++j)
                if (k < K[g.idx[j]]) CKS(runs[j].correct(&done));
        }
        for (int i : g.idx) {
            pr_solver* hi = b->hs[i];
            CKC(cudaEventRecord(hi->ev1, hi->stream));
            CKC(cudaMemcpyAsync(qT_dev[i], hi->q + (long)hi->N * hi->d, sizeof(double) * hi->d,
                                cudaMemcpyDeviceToDevice, hi->stream));
            CKC(cudaEventRecord(b->ev[i + 1], hi->stream));
            CKC(cudaStreamWaitEvent(b->stream, b->ev[i + 1], 0));
        }
        CKC(cudaEventRecord(g.ev, g.stream));
        CKC(cudaStreamWaitEvent(b->stream, g.ev, 0));
    }
    return PR_OK;
}

extern "C" {

pr_status parareal_batch_create(pr_solver* const* hs, int32_t n, const double* const* u0_dev, const int32_t* K,
                                double* const* qT_dev, void* stream, pr_batch** out) {
    pr_solver* h = nullptr;
    if (!out) return set_err(h, PR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!hs || !u0_dev || !K || !qT_dev || n < 1) return set_err(h, PR_EINVAL, "NULL or empty batch");
    for (int i = 0; i < n; ++i) {
        if (!hs[i] || !u0_dev[i] || !qT_dev[i] || K[i] < 0 || K[i] > hs[i]->K_max)
            return set_err(h, PR_EINVAL, "invalid batch entry");
        if (hs[i]->opt.r_tol > 0) return set_err(h, PR_EINVAL, "batch graphs need r_tol = 0");
        if (!hs[i]->stream || hs[i]->stream == (cudaStream_t)stream)
            return set_err(h, PR_EINVAL, "every handle needs a non-NULL stream other than the batch stream");
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return set_err(h, PR_EINVAL, "handles must be distinct");
    }
    pr_batch* b = new (std::nothrow) pr_batch();
    if (!b) return set_err(h, PR_ENOMEM, "host allocation failed");
    b->hs.assign(hs, hs + n);
    b->stream = (cudaStream_t)stream;
    b->lockstep = batch_lockstep_ok(hs, n);
    b->ev.assign((size_t)n + 1, nullptr);
    cudaError_t e = cudaSuccess;
    for (auto& x : b->ev)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
    if (e == cudaSuccess && b->lockstep) e = batch_setup(b, K);
    if (e != cudaSuccess) {
        batch_free(b);
        return set_err(h, PR_ECUDA, std::string("batch set-up: ") + cudaGetErrorString(e));
    }
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev[0], b->stream);
    pr_status st = PR_OK;
    if (b->lockstep && e == cudaSuccess) {
        st = batch_capture_lockstep(b, u0_dev, K, qT_dev);
    } else {
        for (int i = 0; i < n && e == cudaSuccess && st == PR_OK; ++i) {
            e = cudaStreamWaitEvent(hs[i]->stream, b->ev[0], 0);
            if (e != cudaSuccess) break;
            st = parareal_solve(hs[i], u0_dev[i], K[i], nullptr, qT_dev[i], nullptr);
            if (st != PR_OK) break;
            e = cudaEventRecord(b->ev[i + 1], hs[i]->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev[i + 1], 0);
        }
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e == cudaSuccess) e = e2;
    b->graph = g;
    if (st != PR_OK || e != cudaSuccess) {
        std::string msg = st != PR_OK ? std::string("capture of a solve failed: ") + parareal_last_error(hs[0])
                                      : std::string("stream capture: ") + cudaGetErrorString(e);
        cudaGetLastError();
        batch_free(b);
        return set_err(h, st != PR_OK ? st : PR_ECUDA, msg);
    }
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
        batch_free(b);
        return set_err(h, PR_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    *out = b;
    return PR_OK;
}

pr_status parareal_batch_launch(pr_batch* b) {
    pr_solver* h = nullptr;
    if (!b) return PR_EINVAL;
    cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) return set_err(h, PR_ECUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
    return PR_OK;
}

pr_status parareal_batch_destroy(pr_batch* b) {
    if (!b) return PR_EINVAL;
    cudaStreamSynchronize(b->stream);
    batch_free(b);
    return PR_OK;
}

}  // extern "C"
