// krylov.cu -- FP64 tall-skinny linear algebra of the subspace update and
// the modified coarse propagator (Sec. 2.2: Eq. subspaceUpdate,
// Eq. modifiedCoarse, Eq. Genhance) and the serial Parareal correction
// (Alg. 2).
//
// All matrices are column-major with d-long columns (one state per column).
// Reductions over the d rows are split into fixed row chunks; every chunk
// writes a partial result and a second kernel sums the chunks in a fixed
// order, so results are bitwise reproducible run to run and independent of
// what else runs on the GPU (no atomics in any reduction).
#include "common.cuh"
#include "grid_barrier.cuh"

namespace pr {
namespace {

constexpr int TN_CB = 32;     // columns of A per CTA (gemm_tn)
constexpr int TN_JB = 16;     // columns of X per CTA (gemm_tn)
constexpr int TN_KT = 32;     // rows per shared-memory tile
constexpr int GV_CB = 64;     // columns of A per CTA (gemv_tn)
constexpr int NN_JB = 16;     // output columns per thread (gemm_nn)

// Columns [c0, c1) read from device memory, clamped to [0, ccap] (the
// buffers and shared-memory tiles hold ccap columns).
__device__ __forceinline__ int cols_avail(const int* c0_dev, const int* c1_dev, int ccap) {
    int c0 = c0_dev ? *c0_dev : 0;
    const int n = *c1_dev - c0;
    return n < 0 ? 0 : (n > ccap ? ccap : n);
}

// partial[chunk][c * m + j] = sum over the chunk's rows of A[row, c0 + c] * X[row, j]
__global__ void __launch_bounds__(256) k_gemm_tn_partial(const double* __restrict__ A, long lda,
                                                         const int* c0_dev, const int* c1_dev,
                                                         const double* __restrict__ X, long ldx,
                                                         int m, long nrows, int rpc, int ccap,
                                                         double* __restrict__ partial) {
    __shared__ double As[TN_KT][TN_CB + 1];
    __shared__ double Xs[TN_KT][TN_JB + 1];
    const int ncols = cols_avail(c0_dev, c1_dev, ccap);
    const int c0 = c0_dev ? *c0_dev : 0;
    const int cb = blockIdx.y * TN_CB, jb = blockIdx.z * TN_JB;
    if (cb >= ncols) return;
    const long r0 = (long)blockIdx.x * rpc;
    const long r1 = min(nrows, r0 + rpc);
    const int tx = threadIdx.x & 31;      // column of A within the block
    const int ty = threadIdx.x >> 5;      // 8 groups of output columns j
    double acc[TN_JB / 8] = {0.0, 0.0};
    for (long rt = r0; rt < r1; rt += TN_KT) {
        // load A tile: rows rt..rt+31, columns cb..cb+31 (coalesced along rows)
        for (int e = threadIdx.x; e < TN_KT * TN_CB; e += 256) {
            int cc = e / TN_KT, rr = e - cc * TN_KT;
            long row = rt + rr;
            int col = cb + cc;
            As[rr][cc] = (row < r1 && col < ncols) ? A[row + (long)(c0 + col) * lda] : 0.0;
        }
        for (int e = threadIdx.x; e < TN_KT * TN_JB; e += 256) {
            int jj = e / TN_KT, rr = e - jj * TN_KT;
            long row = rt + rr;
            int j = jb + jj;
            Xs[rr][jj] = (row < r1 && j < m) ? X[row + (long)j * ldx] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int rr = 0; rr < TN_KT; ++rr) {
            double a = As[rr][tx];
#pragma unroll
            for (int k = 0; k < TN_JB / 8; ++k) acc[k] += a * Xs[rr][ty + 8 * k];
        }
        __syncthreads();
    }
    double* P = partial + (long)blockIdx.x * ccap * m;
    const int col = cb + tx;
    if (col < ncols) {
#pragma unroll
        for (int k = 0; k < TN_JB / 8; ++k) {
            int j = jb + ty + 8 * k;
            if (j < m) P[(long)col * m + j] = acc[k];
        }
    }
}

// m == 1: warp per column, lanes over rows (coalesced), x chunk in shared memory
__global__ void __launch_bounds__(256) k_gemv_tn_partial(const double* __restrict__ A, long lda,
                                                         const int* c0_dev, const int* c1_dev,
                                                         const double* __restrict__ x, long nrows,
                                                         int rpc, int ccap, double* __restrict__ partial) {
    extern __shared__ double xs[];
    const int ncols = cols_avail(c0_dev, c1_dev, ccap);
    const int c0 = c0_dev ? *c0_dev : 0;
    const int cb = blockIdx.y * GV_CB;
    if (cb >= ncols) return;
    const long r0 = (long)blockIdx.x * rpc;
    const int nr = (int)min((long)rpc, nrows - r0);
    for (int e = threadIdx.x; e < nr; e += 256) xs[e] = x[r0 + e];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int cend = min(ncols, cb + GV_CB);
    double* P = partial + (long)blockIdx.x * ccap;
    for (int col = cb + wid; col < cend; col += 8) {
        const double* a = A + r0 + (long)(c0 + col) * lda;
        double s = 0.0;
        for (int e = lane; e < nr; e += 32) s += a[e] * xs[e];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) P[col] = s;
    }
}

// out[idx] = sum_chunk partial[chunk][idx], idx < n_dev_cols * m (fixed chunk order)
__global__ void k_reduce_chunks(const double* __restrict__ partial, int nchunk, long pstride,
                                const int* c0_dev, const int* c1_dev, int m, double* __restrict__ out,
                                int ldo, int ccap) {
    const int ncols = c1_dev ? cols_avail(c0_dev, c1_dev, ccap) : 1;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ncols * m) return;
    double s = 0.0;
    for (int k = 0; k < nchunk; ++k) s += partial[(long)k * pstride + idx];
    const int c = idx / m, j = idx - c * m;
    out[c + (long)j * ldo] = s;
}

// Y[:, j] = B[:, j] + sgn * sum_{c < ncols} A[:, c0 + c] C[c, j]
__global__ void __launch_bounds__(256) k_gemm_nn(const double* __restrict__ A, long lda,
                                                 const int* c0_dev, const int* c1_dev,
                                                 const double* __restrict__ C, int ldc,
                                                 const double* B, long ldb, double* Y, long ldy,
                                                 int m, long nrows, double sgn, int ccap) {
    extern __shared__ double Cs[];   // ccap x NN_JB
    const int ncols = cols_avail(c0_dev, c1_dev, ccap);
    const int c0 = c0_dev ? *c0_dev : 0;
    const int jb = blockIdx.y * NN_JB;
    const int nj = min(NN_JB, m - jb);
    for (int e = threadIdx.x; e < ncols * NN_JB; e += 256) {
        int c = e / NN_JB, jj = e - c * NN_JB;
        Cs[e] = (jj < nj) ? sgn * C[c + (long)(jb + jj) * ldc] : 0.0;
    }
    __syncthreads();
    const long row = (long)blockIdx.x * 256 + threadIdx.x;
    if (row >= nrows) return;
    double acc[NN_JB];
#pragma unroll
    for (int k = 0; k < NN_JB; ++k) acc[k] = 0.0;
    for (int c = 0; c < ncols; ++c) {
        double a = A[row + (long)(c0 + c) * lda];
#pragma unroll
        for (int k = 0; k < NN_JB; ++k) acc[k] += a * Cs[c * NN_JB + k];
    }
#pragma unroll
    for (int k = 0; k < NN_JB; ++k)
        if (k < nj) Y[row + (long)(jb + k) * ldy] = (B ? B[row + (long)(jb + k) * ldb] : 0.0) + acc[k];
}

// block-level fixed-order sum of 256 values
__device__ __forceinline__ double block_sum256(double v, double* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        for (int k = 0; k < 8; ++k) s += red[k];
    }
    return s;   // valid in thread 0
}

// partial[chunk * m + j] = sum over the chunk's rows of X[row, j]^2  (grid.y = j)
__global__ void __launch_bounds__(256) k_colnorm2_partial(const double* __restrict__ X, long ldx, int m,
                                                          long nrows, int rpc, double* __restrict__ partial) {
    __shared__ double red[8];
    const int j = blockIdx.y;
    const long r0 = (long)blockIdx.x * rpc;
    const long r1 = min(nrows, r0 + rpc);
    double s = 0.0;
    for (long r = r0 + threadIdx.x; r < r1; r += 256) {
        double v = X[r + (long)j * ldx];
        s += v * v;
    }
    s = block_sum256(s, red);
    if (threadIdx.x == 0) partial[(long)blockIdx.x * m + j] = s;
}

__global__ void k_copy_resid(const double* __restrict__ src, double* __restrict__ dst, long n,
                             double* __restrict__ partial, float* __restrict__ delta, double* __restrict__ delta64) {
    __shared__ double red[8];
    const long row = (long)blockIdx.x * 256 + threadIdx.x;
    double s = 0.0;
    if (row < n) {
        double y = src[row];
        double e = y - dst[row];
        s = e * e;
        dst[row] = y;
        if (delta) delta[row] = (float)e;
        if (delta64) delta64[row] = e;
    }
    s = block_sum256(s, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_sum_partials(const double* __restrict__ partial, int n, double* out) {
    __shared__ double red[8];
    double s = 0.0;
    // fixed assignment of partials to threads and fixed combination order
    for (int k = threadIdx.x; k < n; k += 256) s += partial[k];
    s = block_sum256(s, red);
    if (threadIdx.x == 0) *out = s;
}

__global__ void k_max_sqrt(const double* res2, int n, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < n; ++i) m = fmax(m, sqrt(res2[i]));
        *out = m;
    }
}

__global__ void k_sub(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ o, long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        o[i] = a[i] - b[i];
}

__global__ void k_to_fp32_cols(const double* __restrict__ Q, const double* __restrict__ D, float* __restrict__ Q32,
                               float* __restrict__ D32, long d, const int* c0_dev, const int* c1_dev) {
    const int col = (c0_dev ? *c0_dev : 0) + blockIdx.y;
    if (col >= *c1_dev) return;
    for (long row = (long)blockIdx.x * blockDim.x + threadIdx.x; row < d; row += (long)gridDim.x * blockDim.x) {
        Q32[row + (long)col * d] = (float)Q[row + (long)col * d];
        D32[row + (long)col * d] = (float)D[row + (long)col * d];
    }
}

__global__ void k_sub_mapped(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out,
                             long d, const int* beg, const int* end) {
    const int j = blockIdx.y;
    const int b0 = *beg;
    if (j >= *end - b0) return;
    double* o = out + (long)(b0 + j) * d;
    const double* x = a + (long)j * d;
    const double* y = b + (long)j * d;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (long)gridDim.x * blockDim.x)
        o[i] = x[i] - y[i];
}

__global__ void k_fill_int(int* p, int v, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}


// In-order classical Gram-Schmidt (twice) of each of m columns against the
// columns kept earlier in this block, the drop rule and the append, all in
// one cooperative launch.  Every CTA owns a fixed range of rows; dot products
// are summed per CTA in a fixed order and published; after a barrier every
// CTA sums the CTA partials in the same order, so all CTAs hold identical
// coefficients and take identical decisions.  Partial buffers alternate
// between two halves, so one barrier per reduction suffices.
constexpr int IB_NT = 512;
__global__ void __launch_bounds__(IB_NT) k_intra_block(double* wv, double* wz, long d, int m,
                                                      const double* __restrict__ a2, const int* r_old_dev,
                                                      int* r_dev, int cap, double eta, double* Qb, double* Db,
                                                      int* kept, double* ratio, double* __restrict__ part,
                                                      int pstride, GridBar* gb, bool compact) {
    __shared__ double cs[64];
    __shared__ double sred[IB_NT / 32][17];
    __shared__ double s_res2;   // pstride >= 64: slot 63 carries ||v||^2 partials (nn <= 63)
    const unsigned nb = gridDim.x;
    const int b = blockIdx.x;
    const long rpb = (d + nb - 1) / nb;
    const long r0 = min(d, (long)b * rpb), r1 = min(d, r0 + rpb);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = IB_NT / 32;
    const int c0 = *r_old_dev;
    int rl = *r_dev;
    // Kept columns go to Q[:, rl] (and D) or, compacted, to slot rl - c0 of
    // the work block itself (Qb = wv, Db = wz): in both cases column c of the
    // block's kept set is at Q[(c0 + c) d] below.
    double* Q = compact ? Qb - (long)c0 * d : Qb;
    double* D = (compact && Db) ? Db - (long)c0 * d : Db;
    int buf = 0;
    double* P0 = part;
    double* P1 = part + (long)nb * pstride;
    for (int j = 0; j < m; ++j) {
        double* v = wv + (long)j * d;
        double* z = wz ? wz + (long)j * d : nullptr;   // no D bookkeeping when wz is NULL
        const int nn = rl - c0;   // columns kept so far in this block
        // Two passes of classical Gram-Schmidt against those columns.  The
        // second pass also reduces ||v||^2: with c2 = Q^T v and Q^T Q = I the
        // residual is ||v - Q c2||^2 = ||v||^2 - ||c2||^2, where ||c2|| is
        // already at rounding level after the first pass (no cancellation).
        // Without earlier columns only ||v||^2 is reduced.
        const int npass = nn > 0 ? 2 : 1;
        double res2 = 0.0;
        for (int pass = 0; pass < npass; ++pass) {
            double* P = buf ? P1 : P0;
            const bool last = pass == npass - 1;
            // This CTA's partial dot products with the nn kept columns (and
            // ||v||^2 in the last pass).  Up to 16 columns: every thread walks
            // its rows once, reading v once and the columns together (many
            // loads in flight), then the CTA sums the thread values in a
            // fixed order.  More columns: one warp per column.
            if (nn > 16) {
                for (int l = wid; l < nn; l += nw) {
                    const double s = warp_dot(Q + (long)(c0 + l) * d, v, r0, r1);
                    if (lane == 0) P[(long)b * pstride + l] = s;
                }
                if (last) {
                    double s = 0.0;
                    for (long row = r0 + threadIdx.x; row < r1; row += IB_NT) s += v[row] * v[row];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                    if (lane == 0) sred[wid][16] = s;
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        double t = 0.0;
                        for (int q = 0; q < nw; ++q) t += sred[q][16];
                        P[(long)b * pstride + 63] = t;
                    }
                }
            } else
            for (int l0 = 0; l0 < nn || (last && l0 == 0); l0 += 16) {
                const int lc = min(16, nn - l0);
                const bool norm = last && l0 == 0;
                double acc[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) acc[k] = 0.0;
                double nv = 0.0;
                for (long row = r0 + threadIdx.x; row < r1; row += IB_NT) {
                    const double x = v[row];
                    if (norm) nv += x * x;
                    const double* q = Q + (long)(c0 + l0) * d + row;
                    // groups of 4 columns behind uniform branches: at most 3
                    // predicated-off products per row instead of 16 - lc
#pragma unroll
                    for (int g = 0; g < 16; g += 4) {
                        if (g < lc) {
#pragma unroll
                            for (int k = g; k < g + 4; ++k)
                                if (k < lc) acc[k] += q[(long)k * d] * x;
                        }
                    }
                }
                // warp sums of the 16 accumulators (recursive halving); lane L
                // ends with the sum for column kof(L), in a fixed order
                {
                    const int kof = warp_sum16(acc);
                    if ((lane & 1) == 0 && kof < lc) sred[wid][kof] = acc[0];
                }
                if (norm) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) nv += __shfl_xor_sync(0xffffffffu, nv, o);
                    if (lane == 0) sred[wid][16] = nv;
                }
                __syncthreads();
                if ((int)threadIdx.x < lc) {
                    double t = 0.0;
                    for (int w = 0; w < nw; ++w) t += sred[w][threadIdx.x];
                    P[(long)b * pstride + l0 + threadIdx.x] = t;
                }
                if (norm && threadIdx.x == 32) {
                    double t = 0.0;
                    for (int w = 0; w < nw; ++w) t += sred[w][16];
                    P[(long)b * pstride + 63] = t;
                }
                __syncthreads();
            }
            if (!grid_barrier(gb, nb)) return;
            {
                // every CTA sums all CTAs' partials of the nn coefficients (and
                // of ||v||^2 in the last pass) with the loads in flight together:
                // 16 threads per value, each summing every 16th CTA's partial in
                // order, then a fixed butterfly over the 16 lanes
                const int nval = nn + (last ? 1 : 0);
                for (int v0 = 0; v0 < nval; v0 += IB_NT / 16) {
                    const int vi = v0 + (int)(threadIdx.x >> 4), sub = threadIdx.x & 15;
                    double s = 0.0;
                    if (vi < nval) {
                        const double* pp = P + (vi < nn ? vi : 63);
#pragma unroll 8
                        for (unsigned k = sub; k < nb; k += 16) s += __ldcg(pp + (long)k * pstride);
                    }
#pragma unroll
                    for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                    if (sub == 0 && vi < nval) {
                        if (vi < nn) cs[vi] = s;
                        else s_res2 = s;
                    }
                }
            }
            buf ^= 1;
            __syncthreads();
            if (last) {
                double c2 = 0.0;
                for (int l = 0; l < nn; ++l) c2 += cs[l] * cs[l];
                res2 = fmax(s_res2 - c2, 0.0);
            }
            for (long row = r0 + threadIdx.x; row < r1 && nn > 0; row += IB_NT) {
                double av = 0.0, az = 0.0;
                if (z) {
#pragma unroll 4
                    for (int l = 0; l < nn; ++l) {
                        av += Q[row + (long)(c0 + l) * d] * cs[l];
                        az += D[row + (long)(c0 + l) * d] * cs[l];
                    }
                    z[row] -= az;
                } else {
#pragma unroll 4
                    for (int l = 0; l < nn; ++l) av += Q[row + (long)(c0 + l) * d] * cs[l];
                }
                v[row] -= av;
            }
            __syncthreads();   // the next dot products read these rows with another thread mapping
        }
        const double res = sqrt(res2), an = sqrt(a2[j]);
        const bool keep = (res > eta * an) && (an > 0.0) && (rl < cap);
        if (keep) {
            const double inv = 1.0 / res;
            for (long row = r0 + threadIdx.x; row < r1; row += IB_NT) {
                Q[row + (long)rl * d] = v[row] * inv;
                if (z) D[row + (long)rl * d] = z[row] * inv;
            }
            ++rl;
        }
        __syncthreads();       // the appended column is read by the next column's dot products
        if (b == 0 && threadIdx.x == 0) {
            kept[j] = keep ? 1 : 0;
            if (ratio) ratio[j] = an > 0.0 ? res / an : 0.0;
        }
    }
    if (b == 0 && threadIdx.x == 0) *r_dev = rl;
}

}  // namespace

// *out = *a - *b
__global__ void k_sub_int(const int* a, const int* b, int* out) { *out = *a - *b; }

// Cholesky factor of the Gram matrix G = W^T W of n = *n_dev <= 64 nearly
// orthonormal columns, G = R^T R with R upper triangular, and R^{-1}
// (upper, ld 64, zero below the diagonal, columns >= n zero), in one CTA.  A non-positive pivot
// (impossible for nearly orthonormal W) yields NaN, so that it cannot pass
// silently.
__global__ void k_cholqr(const double* __restrict__ G, int ldg, const int* n_dev, double* __restrict__ Rinv) {
    __shared__ double R[64][65];
    const int n = min(*n_dev, 64);
    for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) {
        const int i = idx % 64, j = idx / 64;
        R[i][j] = (i <= j && j < n) ? G[i + (long)j * ldg] : 0.0;
        Rinv[i + 64L * j] = 0.0;
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            double t = R[k][k];
            for (int p = 0; p < k; ++p) t -= R[p][k] * R[p][k];
            R[k][k] = t > 0.0 ? sqrt(t) : __longlong_as_double(0x7FF8000000000000ll);
        }
        __syncthreads();
        for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) {
            double t = R[k][j];
            for (int p = 0; p < k; ++p) t -= R[p][k] * R[p][j];
            R[k][j] = t / R[k][k];
        }
        __syncthreads();
    }
    // R X = I by back substitution, one column of X = R^-1 per thread
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double* x = Rinv + 64L * j;
        for (int i = j; i >= 0; --i) {
            double t = i == j ? 1.0 : 0.0;
            for (int p = i + 1; p <= j; ++p) t -= R[i][p] * x[p];
            x[i] = t / R[i][i];
        }
    }
}

// Gram matrix of the reprojected block W = Q1 - Q C (Q1: in-block
// orthonormal columns, Q: the orthonormal basis, C = Q^T Q1 with *r_dev rows):
// W^T W = Q1^T Q1 - C^T C = I - C^T C up to rounding, because Q1^T Q1 = I and
// Q^T Q = I to working accuracy.  G[i + 64 j] for i, j < *n_dev, one CTA per
// column j, entries summed over the rows of C in a fixed order.
__global__ void k_gram_c(const double* __restrict__ C, int ldc, const int* r_dev, const int* n_dev, double* G) {
    __shared__ double part[4][64];
    const int j = blockIdx.x;
    const int n = min(*n_dev, 64), r = *r_dev;
    const int i = threadIdx.x & 63, grp = threadIdx.x >> 6;   // 4 groups of 64 threads
    double s = 0.0;
    if (j < n && i < n)
        for (int l = grp; l < r; l += 4) s += C[l + (long)i * ldc] * C[l + (long)j * ldc];
    part[grp][i] = s;
    __syncthreads();
    if (grp == 0 && j < n && i < n)
        G[i + 64L * j] = (i == j ? 1.0 : 0.0) - ((part[0][i] + part[1][i]) + (part[2][i] + part[3][i]));
}

// out[:, *off_dev + j] = sum_{i <= j} W[:, i] Rinv[i, j] for j < *n_dev
// (Rinv upper, ld 64): one row per thread, 16 output columns at a time.
__global__ void k_apply_upper(const double* __restrict__ W, long d, const double* __restrict__ Rinv,
                              const int* n_dev, double* out, const int* off_dev) {
    __shared__ double Rs[64 * 64];
    const int n = min(*n_dev, 64);
    for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) Rs[idx] = Rinv[idx];
    __syncthreads();
    double* o = out + (long)(*off_dev) * d;
    for (long row = (long)blockIdx.x * blockDim.x + threadIdx.x; row < d; row += (long)gridDim.x * blockDim.x) {
        for (int j0 = 0; j0 < n; j0 += 16) {
            double acc[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) acc[k] = 0.0;
            const int iend = min(n, j0 + 16);
            for (int i = 0; i < iend; ++i) {
                const double w = W[row + (long)i * d];
#pragma unroll
                for (int k = 0; k < 16; ++k) acc[k] += w * Rs[i + 64 * (j0 + k)];
            }
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if (j0 + k < n) o[row + (long)(j0 + k) * d] = acc[k];
        }
    }
}

constexpr int TN_RPC = 512;   // rows per chunk, gemm_tn
constexpr int GV_RPC = 1024;  // rows per chunk, gemv_tn
constexpr int NRM_RPC = 4096; // rows per chunk, column norms

static inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

long tswork_elems(long nrows, int ccap, int mmax) {
    long a = (long)cdiv(nrows, TN_RPC) * ccap * (mmax > 1 ? mmax : 1);
    long b = (long)cdiv(nrows, GV_RPC) * ccap;
    long c = (long)cdiv(nrows, NRM_RPC) * (mmax > 1 ? mmax : 1);
    long d = (long)cdiv(nrows, 256);
    d = d > 2L * 512 * 64 ? d : 2L * 512 * 64;   // intra-block partials: 2 halves x CTAs x 64
    long m = a > b ? a : b;
    m = m > c ? m : c;
    return m > d ? m : d;
}

cudaError_t gemm_tn(const double* A, long lda, const int* c0_dev, const int* c1_dev, int ccap,
                    const double* X, long ldx, int m, long nrows, double* C, int ldc, const TsWork& w,
                    cudaStream_t s) {
    if (m <= 0 || ccap <= 0) return cudaSuccess;
    if (m == 1) {
        const int nchunk = cdiv(nrows, GV_RPC);
        if ((long)nchunk * ccap > w.elems) return cudaErrorInvalidValue;
        dim3 grid(nchunk, cdiv(ccap, GV_CB));
        k_gemv_tn_partial<<<grid, 256, GV_RPC * sizeof(double), s>>>(A, lda, c0_dev, c1_dev, X, nrows,
                                                                    GV_RPC, ccap, w.partial);
        count_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_reduce_chunks<<<cdiv(ccap, 256), 256, 0, s>>>(w.partial, nchunk, ccap, c0_dev, c1_dev, 1, C, ldc, ccap);
        count_launches(1);
        return cudaGetLastError();
    }
    const int nchunk = cdiv(nrows, TN_RPC);
    if ((long)nchunk * ccap * m > w.elems) return cudaErrorInvalidValue;
    dim3 grid(nchunk, cdiv(ccap, TN_CB), cdiv(m, TN_JB));
    k_gemm_tn_partial<<<grid, 256, 0, s>>>(A, lda, c0_dev, c1_dev, X, ldx, m, nrows, TN_RPC, ccap, w.partial);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_chunks<<<cdiv((long)ccap * m, 256), 256, 0, s>>>(w.partial, nchunk, (long)ccap * m, c0_dev,
                                                            c1_dev, m, C, ldc, ccap);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t gemm_nn(const double* A, long lda, const int* c0_dev, const int* c1_dev, int ccap,
                    const double* C, int ldc, const double* B, long ldb, double* Y, long ldy, int m,
                    long nrows, double sgn, cudaStream_t s) {
    if (m <= 0 || ccap <= 0) return cudaSuccess;
    const size_t smem = sizeof(double) * (size_t)ccap * NN_JB;
    std::lock_guard<std::mutex> lk(smem_launch_lock());
    cudaError_t e = set_dynamic_smem((const void*)k_gemm_nn, smem);
    if (e != cudaSuccess) return e;
    dim3 grid(cdiv(nrows, 256), cdiv(m, NN_JB));
    k_gemm_nn<<<grid, 256, smem, s>>>(A, lda, c0_dev, c1_dev, C, ldc, B, ldb, Y, ldy, m, nrows, sgn, ccap);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t colnorm2(const double* X, long ldx, int m, long nrows, double* out, const TsWork& w,
                     cudaStream_t s) {
    const int nchunk = cdiv(nrows, NRM_RPC);
    if ((long)nchunk * m > w.elems) return cudaErrorInvalidValue;
    k_colnorm2_partial<<<dim3(nchunk, m), 256, 0, s>>>(X, ldx, m, nrows, NRM_RPC, w.partial);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_chunks<<<cdiv(m, 256), 256, 0, s>>>(w.partial, nchunk, m, nullptr, nullptr, m, out, 1, 1);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t copy_resid(const double* src, double* dst, long n, double* res2, const TsWork& w, cudaStream_t s,
                       float* delta, double* delta64) {
    const int nb = cdiv(n, 256);
    if (nb > w.elems) return cudaErrorInvalidValue;
    k_copy_resid<<<nb, 256, 0, s>>>(src, dst, n, w.partial, delta, delta64);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sum_partials<<<1, 256, 0, s>>>(w.partial, nb, res2);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t max_sqrt(const double* res2, int n, double* out, cudaStream_t s) {
    k_max_sqrt<<<1, 32, 0, s>>>(res2, n, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t sub(const double* a, const double* b, double* out, long n, cudaStream_t s) {
    int nb = cdiv(n, 256);
    if (nb > 4096) nb = 4096;
    k_sub<<<nb, 256, 0, s>>>(a, b, out, n);
    count_launches(1);
    return cudaGetLastError();
}

int intra_block_grid() {
    static DevMemo memo;   // [device] -> (SMs, CTAs per SM)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    int sms = 0, per = 0;
    if (!memo.get(dev, &sms, &per)) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_intra_block, IB_NT, 0);
        memo.put(dev, sms, per);
    }
    return sms * (per < 1 ? 0 : 1);
}

cudaError_t intra_block(double* wv, double* wz, long d, int m, const double* a2, const int* r_old_dev,
                        int* r_dev, int cap, double eta, double* Q, double* D, int* kept, double* ratio,
                        const TsWork& w, GridBar* gb, cudaStream_t s, int max_blocks, bool compact) {
    if (compact) {
        Q = wv;
        D = wz;
    }
    if (m < 1 || m > 64) return cudaErrorInvalidValue;
    int nb = intra_block_grid();
    if (max_blocks > 0 && nb > max_blocks) nb = max_blocks;
    if (nb < 1) return cudaErrorInvalidConfiguration;
    int pstride = 64;
    if ((long)2 * nb * pstride > w.elems) return cudaErrorInvalidValue;
    // arrival counter to zero; the sticky error word is kept
    cudaError_t e = cudaMemsetAsync(&gb->count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    double* part = w.partial;
    void* args[] = {&wv, &wz, &d, &m, (void*)&a2, (void*)&r_old_dev, &r_dev, &cap, &eta, &Q, &D, &kept, &ratio,
                    &part, &pstride, &gb, &compact};
    e = cudaLaunchCooperativeKernel((const void*)k_intra_block, dim3(nb), dim3(IB_NT), args, 0, s);
    count_launches(1);
    return e;
}

cudaError_t to_fp32_cols(const double* Q, const double* D, float* Q32, float* D32, long d, const int* c0_dev,
                         const int* c1_dev, int maxcols, cudaStream_t s) {
    if (maxcols < 1) return cudaSuccess;
    int nb = cdiv(d, 256);
    if (nb > 256) nb = 256;
    k_to_fp32_cols<<<dim3(nb, maxcols), 256, 0, s>>>(Q, D, Q32, D32, d, c0_dev, c1_dev);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t sub_mapped(const double* a, const double* b, double* out, long d, int maxn, const int* beg,
                       const int* end, cudaStream_t s) {
    if (maxn < 1) return cudaSuccess;
    int nb = cdiv(d, 256);
    if (nb > 256) nb = 256;
    k_sub_mapped<<<dim3(nb, maxn), 256, 0, s>>>(a, b, out, d, beg, end);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t cholqr_block(double* W, double* Z, long d, int m, const int* nk_dev, const double* C2, int ldc2,
                         const int* r2_dev, double* G, double* Rinv, double* Q, double* D, const int* off_dev,
                         cudaStream_t s) {
    if (m < 1 || m > 64) return cudaErrorInvalidValue;
    // G = W^T W = I - C2^T C2 over the kept columns, R^-1 of its Cholesky
    // factor, then Q[:, off + j] = (W R^-1)_j and D likewise
    k_gram_c<<<m, 256, 0, s>>>(C2, ldc2, r2_dev, nk_dev, G);
    k_cholqr<<<1, 64, 0, s>>>(G, 64, nk_dev, Rinv);
    count_launches(1);
    int nb = cdiv(d, 256);
    if (nb > 4 * 152) nb = 4 * 152;
    k_apply_upper<<<nb, 256, 0, s>>>(W, d, Rinv, nk_dev, Q, off_dev);
    count_launches(2);
    if (Z) {
        k_apply_upper<<<nb, 256, 0, s>>>(Z, d, Rinv, nk_dev, D, off_dev);
        count_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t sub_int(const int* a, const int* b, int* out, cudaStream_t s) {
    k_sub_int<<<1, 1, 0, s>>>(a, b, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t fill_int(int* p, int v, int n, cudaStream_t s) {
    k_fill_int<<<cdiv(n, 256), 256, 0, s>>>(p, v, n);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pr
