// common.cuh -- internal definitions shared by the CUDA translation units of
// the KSE-Parareal library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

namespace pr {

// Kernels whose dynamic shared memory depends on the problem set the
// process-wide per-kernel limit to the launch's own size right before the
// launch.  Both happen under this lock, so a concurrent host thread (one
// handle per thread) cannot lower the limit between another thread's set and
// its launch.
inline std::mutex& smem_launch_lock() {
    static std::mutex m;
    return m;
}
inline cudaError_t set_dynamic_smem(const void* fn, size_t bytes) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Count n kernel launches (process-wide, reported by parareal_kernel_launches).
void count_launches(int n);

// Per-device memo of a pair of small non-negative launch parameters (a, b),
// one atomic 64-bit word per device so that concurrent host threads (one
// handle per thread) read either nothing or a consistent pair.
struct DevMemo {
    std::atomic<unsigned long long> w[64];
    bool get(int dev, int* a, int* b) const {
        if (dev < 0 || dev >= 64) return false;
        const unsigned long long x = w[dev].load(std::memory_order_acquire);
        if (!(x >> 63)) return false;
        *a = (int)((x >> 32) & 0x7fffffffu);
        *b = (int)(x & 0xffffffffu);
        return true;
    }
    void put(int dev, int a, int b) {
        if (dev < 0 || dev >= 64 || a < 0 || b < 0) return;
        w[dev].store((1ull << 63) | ((unsigned long long)(unsigned)a << 32) | (unsigned)b,
                     std::memory_order_release);
    }
};

// Periodic index for offsets that may exceed one period (tiny grids).
__host__ __device__ __forceinline__ int pwrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// Coefficients of the fine tendency L_f (Sec. 3 flux form, 6th-order
// centred advection, 2nd-order centred acoustics, compact grad-div damping).
template <typename T>
struct FineCoef {
    T ax6;    // U / (60 dx): multiplies the 6-point x advective difference
    T ay6;    // V / (60 dy)
    T csx;    // c_s / (2 dx)
    T csy;    // c_s / (2 dy)
    T dxx;    // alpha1 / dx^2
    T dxy1;   // alpha1 / (4 dx dy)
    T dyy;    // alpha2 / dy^2
    T dxy2;   // alpha2 / (4 dx dy)
    T c1, c2, c3;   // RK-3 stage lengths dt/3, dt/2, dt
    // Solid-body rotation (Eq. adVel): the velocity is (U + omega (y - ly/2),
    // V - omega (x - lx/2)), so row j advects with ax6 + omx yc(j) and column
    // i with ay6 - omy xc(i), yc(j) = (j + 1/2) dy - ly/2, xc(i) likewise.
    T omx = T(0);   // omega / (60 dx)
    T omy = T(0);   // omega / (60 dy)
    T dx = T(0), dy = T(0), hlx = T(0), hly = T(0);   // cell sizes, lx/2, ly/2
};
// Cell-centre coordinates relative to the domain centre (periodic index).
template <typename T>
__host__ __device__ __forceinline__ T xcen(const FineCoef<T>& c, int i) { return (T(i) + T(0.5)) * c.dx - c.hlx; }
template <typename T>
__host__ __device__ __forceinline__ T ycen(const FineCoef<T>& c, int j) { return (T(j) + T(0.5)) * c.dy - c.hly; }

// Coefficients of one partially split coarse step (Sec. 3.2).
struct CoarseCoef {
    double U, V;        // advection velocity (upwind direction from the sign)
    double inv_dx, inv_dy;
    double tau;         // acoustic substep Delta t / n_sound
    double csx, csy;    // c_s / (2 dx), c_s / (2 dy)
    double dxx, dxy1;   // alpha1 / dx^2, alpha1 / (4 dx dy); alpha = nu_c dx^2 / tau
    double dyy, dxy2;   // alpha2 / dy^2, alpha2 / (4 dx dy)
    int n_sound;
    int order;          // 1 or 3 (upwind-biased advective flux)
    double omega = 0.0;                 // rotation: U + omega yc(j), V - omega xc(i)
    double dx = 0, dy = 0, hlx = 0, hly = 0;   // cell sizes, lx/2, ly/2
    int scheme = 0;     // 0: partially split forward Euler; 1: non-split RK-3 with
                        //    tau = Delta t and alpha = nu_c dx^2 / Delta t
};

// ------------------------------------------------------------ launchers
// Each returns a cudaError_t from the launch.

// Optional device-side slice mapping of a batched launch: slices z >= *end -
// *beg are skipped; with in_map (out_map) the input (output) slice is
// *beg + z instead of z.  Lets a launch act on a column range the host does
// not know (e.g. the columns the last subspace update kept).
struct SliceMap {
    const int* beg = nullptr;
    const int* end = nullptr;
    bool in_map = false, out_map = false;
};

// Launch shape of the FP32 fine step, chosen by the autotuner
// (parareal_autotune) or left at the built-in heuristic.
//   tile:     shared-memory tile kernel (V = 0): -1 heuristic, else an index
//             into fine_tile_shapes (TX x TY cells per CTA);
//   min_rows: row-streamed kernel: smallest row range per CTA (the grid is
//             min(resident CTAs, n*ny / min_rows)).
struct FineLaunch {
    int tile = -1;
    int min_rows = 16;
    bool rows = true;   // false: never the row-streamed kernel (it has bounded waits)
};
constexpr int kFineTiles = 4;
extern const int fine_tile_shapes[kFineTiles][2];

// One RK-3 step on n states.  in/out element types select FP64 or FP32
// arithmetic (T) with conversion at the boundary.  instride/outstride are
// element strides between consecutive states.
template <typename T, typename Tin, typename Tout>
cudaError_t launch_fine_step(const Tin* in, long instride, Tout* out, long outstride, int n, int nx,
                             int ny, bool has_v, const FineCoef<T>& c, cudaStream_t s,
                             const SliceMap& sm = SliceMap(), const FineLaunch& fl = FineLaunch());

// One RK-3 step in FP32 arithmetic streamed row by row (fine_rows.cu), for
// FP32 input, V = 0 and nx a multiple of 128 up to 1024 with 16-byte aligned
// states.  Returns false (nothing launched) outside that case; otherwise
// *err holds the launch status.
template <typename Tin, typename Tout>
bool launch_fine_rows(const Tin* in, long instride, Tout* out, long outstride, int n, int nx, int ny, bool has_v,
                      const FineCoef<float>& c, cudaStream_t s, const SliceMap& map, cudaError_t* err,
                      int min_rows = 16);

// Process-wide flag of the row-streamed kernel (synchronising read): 1 once a
// wait for one of its TMA row loads gave up (results since then invalid),
// -1 if it could not be read; reset clears it.
int fine_rows_wait_error(bool reset);

// One RK-3 step with FP32 tendencies and stages on an FP64 state: the last
// stage forms q^{n+1} = q^n + dt L(q**) in FP64 (fine_prec = PR_FP32X).
cudaError_t launch_fine_step_acc64(const double* in, double* out, long stride, int n, int nx, int ny, bool has_v,
                                  const FineCoef<float>& c, cudaStream_t s, const SliceMap& sm = SliceMap(),
                                  const FineLaunch& fl = FineLaunch());
// true when an FP32-input step of this shape runs on the row-streamed kernel
bool fine_rows_eligible(int nx, bool has_v);
// FP32 copies of n FP64 states (slice z of the output from slice z, or with
// map.in_map slice *map.beg + z, of the input; slices z >= *end - *beg of a
// map are skipped).
cudaError_t launch_to_fp32_states(const double* in, long instride, float* out, long outstride, int n, long d,
                                  const SliceMap& map, cudaStream_t s);

// One coarse step (slow tendency + n_sound forward-backward substeps) on n
// states, FP64 arithmetic or FP32 arithmetic (fp32) on FP64 data.
cudaError_t launch_coarse_step(const double* in, double* out, long stride, int n, int nx, int ny,
                               const CoarseCoef& c, cudaStream_t s, bool fp32 = false,
                               const SliceMap& sm = SliceMap());
int coarse_halo(const CoarseCoef& c);

// -------- tall-skinny FP64 linear algebra over d-long columns (column-major)
// Column ranges are read from device memory ([*c0_dev, *c1_dev), c0_dev may be
// NULL for 0) so a whole solve can be enqueued without host synchronisation;
// ccap is the host-side upper bound used to size grids.
struct TsWork {
    double* partial;   // scratch for per-chunk partial sums
    long elems;        // its capacity in doubles (>= tswork_elems(...))
};
long tswork_elems(long nrows, int ccap, int mmax);

// C[c, j] = sum_rows A[row, c0 + c] * X[row, j]   (C column-major with leading dim ldc)
cudaError_t gemm_tn(const double* A, long lda, const int* c0_dev, const int* c1_dev, int ccap,
                    const double* X, long ldx, int m, long nrows, double* C, int ldc, const TsWork& w,
                    cudaStream_t s);
// Y[:, j] = B[:, j] + sgn * sum_c A[:, c0 + c] C[c, j]   (B may alias Y; B == NULL means 0)
cudaError_t gemm_nn(const double* A, long lda, const int* c0_dev, const int* c1_dev, int ccap,
                    const double* C, int ldc, const double* B, long ldb, double* Y, long ldy, int m,
                    long nrows, double sgn, cudaStream_t s);
// out[j] = sum_rows X[row, j]^2
cudaError_t colnorm2(const double* X, long ldx, int m, long nrows, double* out, const TsWork& w,
                     cudaStream_t s);
// dst <- src with *res2 = ||src - dst_old||^2 (and delta = src - dst_old in FP32,
// delta64 the same in FP64, where non-NULL)
cudaError_t copy_resid(const double* src, double* dst, long n, double* res2, const TsWork& w, cudaStream_t s,
                       float* delta = nullptr, double* delta64 = nullptr);
// FP32 copies of basis columns [*c0_dev, *c1_dev) of Q and D (at most maxcols columns)
cudaError_t to_fp32_cols(const double* Q, const double* D, float* Q32, float* D32, long d, const int* c0_dev,
                         const int* c1_dev, int maxcols, cudaStream_t s);
// *out = max_i sqrt(res2[i])
cudaError_t max_sqrt(const double* res2, int n, double* out, cudaStream_t s);
cudaError_t sub(const double* a, const double* b, double* out, long n, cudaStream_t s);
// out[(*beg + j) d + i] = a[j d + i] - b[j d + i] for slices j < *end - *beg (at most maxn)
cudaError_t sub_mapped(const double* a, const double* b, double* out, long d, int maxn, const int* beg,
                       const int* end, cudaStream_t s);
cudaError_t fill_int(int* p, int v, int n, cudaStream_t s);

// Grid-barrier state of a cooperative launch (zeroed before each launch).
struct GridBar {
    unsigned count;   // monotonic arrival counter of grid_barrier (zeroed before each launch)
    int err;   // set to 1 when a barrier wait gave up
    unsigned gcount[3];   // monotonic counters of grid_barrier_group (zeroed before a launch using them)
};
// In-order Gram-Schmidt (twice) within a block of m <= 64 columns that are
// already orthogonal to the basis columns [0, *r_old_dev), the drop rule
// against the original column norms a2[j] and the append, in one cooperative
// launch.  gb->err != 0 afterwards (sticky) means a barrier wait gave up and
// the result is invalid.
// ratio[j] (optional) receives ||residual_j|| / ||a_j||.
// max_blocks > 0 caps the cooperative grid (one CTA per SM).
// compact: the kept columns (normalised) are written in order to the first
// slots of wv (and wz) instead of Q[:, *r_dev] (and D); *r_dev still counts them.
cudaError_t intra_block(double* wv, double* wz, long d, int m, const double* a2, const int* r_old_dev,
                        int* r_dev, int cap, double eta, double* Q, double* D, int* kept, double* ratio,
                        const TsWork& w, GridBar* gb, cudaStream_t s, int max_blocks = 0, bool compact = false);
// Re-orthonormalisation of n = *nk_dev <= m <= 64 nearly orthonormal columns
// W = Q1 - Q C2 (ld d; Q1 orthonormal, C2 = Q^T Q1 with *r2_dev rows, ld ldc2)
// by Cholesky QR: G = W^T W = I - C2^T C2 = R^T R (G, Rinv: 64 x 64 scratch),
// the result W R^-1 written to Q[:, *off_dev + j] (and Z R^-1 to D when
// Z != NULL).
cudaError_t cholqr_block(double* W, double* Z, long d, int m, const int* nk_dev, const double* C2, int ldc2,
                         const int* r2_dev, double* G, double* Rinv, double* Q, double* D, const int* off_dev,
                         cudaStream_t s);
cudaError_t sub_int(const int* a, const int* b, int* out, cudaStream_t s);


// Serial correction of Alg. 2 over slices [i_begin, i_end) in one cooperative
// launch (chain.cu):  q_{i+1} = qt_i + ((G(q_i) + D Q^T q_i) - kold_i).
// qt, kold may be NULL (zero) and r_dev NULL (no basis): with all three NULL
// it is the serial coarse sweep q_{i+1} = G(q_i).
struct ChainArgs {
    double* q;            // (N+1) x d iterates; q_i read, q_{i+1} written
    const double* qt;     // slot i: fine image q~_{i+1}, or NULL
    const double* kold;   // slot i: K(q_i^k), or NULL
    const double* Q;      // basis, d x cap
    const double* D;      // F(Q) - G(Q), d x cap
    const int* r_dev;     // number of basis columns, or NULL for none
    int ccap;             // basis capacity (partial-sum stride)
    int i_begin, i_end;
    long d;
    int nx, ny;
    CoarseCoef cc;
    int n_g, H;
    double* gbuf;         // 2 x d coarse ping-pong
    double* cvec;         // >= ccap coefficients
    double* part;         // >= 1024 x ccap partial sums
    double* resp;         // >= chain_resp_elems(N) residual partials
    double* res2;         // res2[i+1] = ||q_{i+1} change||^2, or NULL
    GridBar* gb;
    // FP32 delta form (dlt != NULL): q_{i+1} = qt_i + (G(delta_i) + D32 Q32^T delta_i)
    float* dlt;           // d values: delta_i on entry to slice i, delta_{i+1} after it
    const float* Q32;     // FP32 copies of Q and D
    const float* D32;
    float* gbuf32;        // 2 x d FP32 coarse ping-pong
    // FP64 delta form (dlt64 != NULL): the same with Q, D, gbuf and delta in FP64
    double* dlt64;
    // with the FP64 delta form, optional: slot i holds G(q_i^k) on entry and
    // receives G(q_i^{k+1}) = G(q_i^k) + G(delta_i) (linearity of G)
    double* gacc;
    int max_blocks;       // > 0: cap on the cooperative grid (one CTA per SM)
};
cudaError_t chain_coop(const ChainArgs& a, cudaStream_t s);
long chain_resp_elems(int n_slices);


// FP64 fine sweep in one cooperative launch (fine_coop.cu).  Coefficients
// already multiplied by the stage length c_k (k = 0, 1, 2: dt/3, dt/2, dt)
// and signed as they enter q^n + c_k L.
// One handle's fine sweep inside a batched launch (FP32 tendencies on FP64
// states, V = 0, no rotation): n states from in to out in nf RK-3 steps
// through the ping-pong buffers w0, w1 (step t writes out when t = nf - 1,
// else w0 for even t and w1 for odd t), with the slice maps of its first and
// of its later steps; d = 3 nx ny; its tiles are the work indices
// [tile0, tile0 + n * tiles).
struct FineBatchItem {
    const double* in;
    double* out;
    double *w0, *w1;
    SliceMap first, rest;
    FineCoef<float> c;
    long d;
    int nx, ny, n, nf;
    int tiles_x, tiles;
    long tile0;
};
// Output tiles per state of the batched sweep's tile shape.
void fine_batch_tiles(int nx, int ny, int* tiles_x, int* tiles);
// All nf steps of all items in one cooperative launch with a bounded grid
// barrier between steps (items sorted by tile0; total = sum of n * tiles),
// on max_sms SMs (0: all), so that several batched launches can run side by
// side.
cudaError_t fine_batch_coop(const FineBatchItem* items_dev, int nitems, long total, int max_nf, GridBar* gb,
                            cudaStream_t s, int max_sms);

struct FineCoefK {
    double adx[3], ady[3], csx[3], csy[3], dxx[3], dxy1[3], dyy[3], dxy2[3];
    // products of the above used by the V = 0 marching kernel, formed on the
    // host so the kernel reads them as constant operands: u's x-terms on raw
    // neighbours (45 A + Cx, Cx - 45 A, -9 A, 9 A, -A, -2 Cx), 45 A, -9 A, -2 Cy
    double up1[3], um1[3], up2[3], um2[3], um3[3], u00[3], a45[3], am9[3], cy2[3];
    // rotation (Eq. adVel): row j advects with adx + aomx yc(j), column i with
    // ady + aomy xc(i); yc, xc cell-centre coordinates about the domain centre
    double aomx[3], aomy[3];
    double dx, dy, hlx, hly;
};
FineCoefK make_fine_coef_k(double U, double V, double cs, double dx, double dy, double nu, double dt,
                           double omega = 0.0, double lx = 1.0, double ly = 1.0);
struct FineSweepArgs {
    const double* in;    // n x d, not modified
    double* out;         // n x d
    double *w1, *w2, *w3;  // n x d work buffers each (distinct from in and out)
    int n, nx, ny, nsteps;
    FineCoefK c;
    GridBar* gb;
    int max_sms;           // > 0: cap on the SMs used (CTAs = SMs x CTAs per SM)
};
cudaError_t fine_sweep_coop(const FineSweepArgs& a, bool has_v, cudaStream_t s);

}  // namespace pr
