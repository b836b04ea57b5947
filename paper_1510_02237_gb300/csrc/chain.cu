// chain.cu -- the serial correction of Alg. 2 for a run of consecutive
// slices in one cooperative launch:
//
//   for i = i_begin .. i_end-1:
//     c         = Q^T x_i                                 (Eq. modifiedCoarse, P x = Q c)
//     K(x_i)    = G(x_i) + D c,   D = F(Q) - G(Q)          (Eq. Genhance by linearity)
//     q_{i+1}   = q~_{i+1} + K(x_i) [- K_old_i]            (Alg. 2)
//     res2[i+1] = ||q_{i+1}^{new} - q_{i+1}^{old}||^2       (for r^k, Sec. 2.1)
//
// KSE correction: x_i = delta_i = q_i^{k+1} - q_i^k (K is linear, so
// K(q_i^{k+1}) - K(q_i^k) = K(delta_i)), and the update produces delta_{i+1}.
// Literal form (x_i = q_i): with no basis, no fine images and no K_old it is
// the serial coarse sweep q_{i+1} = G(q_i) of the initialisation; with
// K_old = G(q_i^k) and no basis it is the correction of the original
// Parareal (Alg. 1).
//
// k_chain (below) serves every form; the FP64 delta form with the split
// coarse step runs in k_chain_split (further below).  In k_chain every CTA
// owns a fixed range of rows for the dot products and the update and a set
// of 16 x 16 tiles for the coarse steps.  Per slice: phase A
// computes the CTA's partial dot products and the first coarse step; after a
// barrier the coefficients are reduced (each CTA sums a share of them over
// all CTA partials in a fixed order) while the second coarse step runs;
// after a barrier every CTA updates its rows; a last barrier publishes
// q_{i+1} before the next slice's coarse step reads its halos.  All waits are
// bounded (grid_barrier).
#include <type_traits>

#include "coarse_tile.cuh"
#include "grid_barrier.cuh"

namespace pr {
namespace {

constexpr int CH_NT = 512, CH_TX = 16, CH_TY = 16;

// FP32 dot product of a and x over rows [r0, r1) by one warp, accumulated in
// FP32 in a fixed order (deterministic).  With vec (both columns 16-byte
// aligned at r0, r0 a multiple of 4) four float4 loads per operand are in
// flight per lane.
__device__ __forceinline__ float warp_dot_f32(const float* __restrict__ a, const float* x, long r0,
                                              long r1, bool vec) {
    const int lane = threadIdx.x & 31;
    float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
    long tail = r0;
    if (vec) {
        const float4* a4 = reinterpret_cast<const float4*>(a + r0);
        const float4* x4 = reinterpret_cast<const float4*>(x + r0);
        const long n4 = (r1 - r0) >> 2;
        long i = lane;
        for (; i + 96 < n4; i += 128) {
            const float4 p0 = __ldg(a4 + i), p1 = __ldg(a4 + i + 32), p2 = __ldg(a4 + i + 64), p3 = __ldg(a4 + i + 96);
            const float4 y0 = x4[i], y1 = x4[i + 32], y2 = x4[i + 64], y3 = x4[i + 96];
            t0 += p0.x * y0.x + p0.y * y0.y + p0.z * y0.z + p0.w * y0.w;
            t1 += p1.x * y1.x + p1.y * y1.y + p1.z * y1.z + p1.w * y1.w;
            t2 += p2.x * y2.x + p2.y * y2.y + p2.z * y2.z + p2.w * y2.w;
            t3 += p3.x * y3.x + p3.y * y3.y + p3.z * y3.z + p3.w * y3.w;
        }
        for (; i < n4; i += 32) {
            const float4 p0 = __ldg(a4 + i), y0 = x4[i];
            t0 += p0.x * y0.x + p0.y * y0.y + p0.z * y0.z + p0.w * y0.w;
        }
        tail = r0 + 4 * n4;
    }
    for (long row = tail + lane; row < r1; row += 32) t0 += a[row] * x[row];
    float t = (t0 + t1) + (t2 + t3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

// DELTA = false: the literal correction in FP64 (T = double),
//   q_{i+1} = q~_{i+1} + ((G(q_i) + D Q^T q_i) - K_old_i)
// (K_old = G(q_i^k) for the original Parareal, or no basis and no K_old: the
// serial coarse sweep).
// DELTA = true: the KSE correction through the linearity of K,
//   q_{i+1} = q~_{i+1} + (G(delta_i) + D Q^T delta_i),  delta_i = q_i^{k+1} - q_i^k,
// in T = float (FP32 copies of Q and D) or T = double; delta_{i+1} is
// produced by the update itself.  Its rounding scales with ||delta||, not
// ||q||, a converged slice (delta = 0) gets exactly no correction, and the
// sum into q stays FP64.
template <bool DELTA, typename T>
__global__ void __launch_bounds__(CH_NT) k_chain(ChainArgs A) {
    static_assert(DELTA || std::is_same<T, double>::value, "the literal form is FP64");
    constexpr bool F32 = std::is_same<T, float>::value;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    __shared__ double red[CH_NT / 32];
    const unsigned nb = gridDim.x;
    const int b = blockIdx.x;
    const long d = A.d;
    const long rpb = ((d + nb - 1) / nb + 31) / 32 * 32;   // rows per CTA, a multiple of 32
    const long r0 = min(d, (long)b * rpb), r1 = min(d, r0 + rpb);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = CH_NT / 32;
    int ncols = A.r_dev ? *A.r_dev : 0;
    if (ncols < 0 || ncols > A.ccap) {   // cannot happen: the rank never exceeds the cap
        if (threadIdx.x == 0) atomicExch(&A.gb->err, 2);
        return;
    }
    const int ntx = (A.nx + CH_TX - 1) / CH_TX, nty = (A.ny + CH_TY - 1) / CH_TY, ntiles = ntx * nty;
    const int cpb = (ncols + (int)nb - 1) / (int)nb;
    const T* Qm = F32 ? reinterpret_cast<const T*>(A.Q32) : reinterpret_cast<const T*>(A.Q);
    const T* Dm = F32 ? reinterpret_cast<const T*>(A.D32) : reinterpret_cast<const T*>(A.D);
    T* gbuf = F32 ? reinterpret_cast<T*>(A.gbuf32) : reinterpret_cast<T*>(A.gbuf);
    T* dlt = F32 ? reinterpret_cast<T*>(A.dlt) : reinterpret_cast<T*>(A.dlt64);

    for (int i = A.i_begin; i < A.i_end; ++i) {
        const double* qi = A.q + (long)i * d;
        double* qn = A.q + (long)(i + 1) * d;
        const T* x = DELTA ? dlt : reinterpret_cast<const T*>(qi);
        // phase A: this CTA's partial dot products c_l = sum_rows Q[row, l] x[row]
        for (int l = wid; l < ncols; l += nw) {
            double s;
            if (F32) {
                s = (double)warp_dot_f32(reinterpret_cast<const float*>(Qm) + (long)l * d,
                                         reinterpret_cast<const float*>(x), r0, r1, (d & 3) == 0);
            } else {
                s = warp_dot(reinterpret_cast<const double*>(Qm) + (long)l * d, reinterpret_cast<const double*>(x),
                             r0, r1);
            }
            if (lane == 0) A.part[(long)b * A.ccap + l] = s;
        }
        // coarse steps G(x), one barrier after each
        const T* gin = x;
        for (int st = 0; st < A.n_g; ++st) {
            T* gout = gbuf + (long)(st & 1) * d;
            for (int t = b; t < ntiles; t += nb) {
                const int ty = t / ntx, tx = t - ty * ntx;
                coarse_tile<CH_TX, CH_TY, CH_NT, T, T, T>(gin, gout, A.nx, A.ny, A.cc, A.H, tx * CH_TX,
                                                          ty * CH_TY, sm);
            }
            if (!grid_barrier(A.gb, nb)) return;
            if (st == 0 && ncols > 0) {
                // this CTA's share of the coefficients, summed over all CTAs in order
                const int l1 = min(ncols, (b + 1) * cpb);
                for (int l = b * cpb + wid; l < l1; l += nw) {
                    const double s = warp_sum_strided(A.part + l, nb, A.ccap);
                    if (lane == 0) A.cvec[l] = s;
                }
                if (A.n_g == 1 && !grid_barrier(A.gb, nb)) return;
            }
            gin = gout;
        }
        // update of this CTA's rows
        T* cs = sm;
        for (int l = threadIdx.x; l < ncols; l += CH_NT) cs[l] = (T)__ldcg(A.cvec + l);
        __syncthreads();
        const double* qt = A.qt ? A.qt + (long)i * d : nullptr;
        const double* ko = A.kold ? A.kold + (long)i * d : nullptr;
        double* ga = (DELTA && !F32 && A.gacc) ? A.gacc + (long)i * d : nullptr;
        double s = 0.0;
        if (F32 && (d & 3) == 0) {
            // four consecutive rows per thread: 16-byte loads of D32, eight
            // basis columns in flight
            const float* gq = reinterpret_cast<const float*>(gin);
            for (long row = r0 + 4 * threadIdx.x; row < r1; row += 4 * CH_NT) {
                float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                const float4* Dr = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(Dm) + row);
                const long st = d >> 2;
#pragma unroll 8
                for (int l = 0; l < ncols; ++l) {
                    const float4 dv = __ldg(Dr + (long)l * st);
                    const float cl = (float)cs[l];
                    acc.x += dv.x * cl;
                    acc.y += dv.y * cl;
                    acc.z += dv.z * cl;
                    acc.w += dv.w * cl;
                }
                const float av[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const long rw = row + u;
                    const double y = qt[rw] + (double)(gq[rw] + av[u]);
                    const double e = y - qn[rw];
                    s += e * e;
                    qn[rw] = y;
                    dlt[rw] = (T)e;
                }
            }
        } else
        for (long row = r0 + threadIdx.x; row < r1; row += CH_NT) {
            T acc = T(0);
            const T* Dr = Dm + row;
#pragma unroll 8
            for (int l = 0; l < ncols; ++l) acc += __ldg(Dr + (long)l * d) * cs[l];
            double y;
            if (DELTA) {
                y = qt[row] + (double)(gin[row] + acc);
            } else {
                const double knew = (double)gin[row] + (double)acc;
                y = (qt ? qt[row] : 0.0) + (knew - (ko ? ko[row] : 0.0));
            }
            const double e = y - qn[row];
            s += e * e;
            qn[row] = y;
            if (DELTA) dlt[row] = (T)e;
            if (ga) ga[row] += (double)gin[row];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[wid] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < nw; ++k) t += red[k];
            A.resp[(long)i * nb + b] = t;
        }
        if (!grid_barrier(A.gb, nb)) return;
    }
    if (A.res2 && b == 0) {
        for (int i = A.i_begin + wid; i < A.i_end; i += nw) {
            const double t = warp_sum_strided(A.resp + (long)i * nb, nb, 1);
            if (lane == 0) A.res2[i + 1] = t;
        }
    }
}

// ------------------------------------------------------------ split groups
// The FP64 KSE correction (delta form) with the partially split coarse step,
// with the coarse steps and the products in two thread groups of every CTA
// that run side by side.  CTA b owns one tile of the grid (16 columns by th
// rows, th chosen so that the tiles fit on the CTAs; CTAs past the last tile
// own none) and the rows of its cells in all three fields:
//   coarse group (warps 0..3): the n_g coarse steps of delta_i on the tile,
//     one phase per acoustic substep: the state on the tile and a 2-cell ring
//     (3 for third-order fluxes) is loaded into shared memory, the forward
//     half (velocities) is computed on the tile and a 1-cell ring, the
//     backward half (pressure) on the tile, the tile is written out, and the
//     group's grid barrier separates the phases; the slow tendencies of the
//     tile and ring stay in shared memory through a step; two states
//     alternate in memory;
//   product group (warps 4..15): the partial dot products Q^T delta_i over a
//     fixed row range, the group's grid barrier, the CTA's share of the
//     coefficient sums, the group's grid barrier, and D c on the tile's rows.
// The groups join (CTA barrier), every thread updates the tile's rows, and a
// full grid barrier ends the slice.  Each cell's arithmetic is the tile
// kernel's (the shared fb_new_* helpers; a ring cell's forward values are
// those its owner computes), and each dot product, coefficient sum and D c
// row is summed in the tile kernel's order, so the iterates are the same bit
// for bit; only the order of the residual partial sums differs.  The literal
// form without a basis (the coarse initialisation, the original Parareal, the
// coarse sweep) has no products: there all 16 warps form the coarse group.
constexpr int CS_NT = 512, CS_NW = CS_NT / 32, CS_CW = 4;   // threads, warps, coarse warps
constexpr int CS_TW = 16;   // tile width

// Tiling of an nx x ny grid on nb CTAs: tiles of tw0 x th0 (the last column
// and row of tiles may be narrower), tw0 = 16, 32, 64 or 128 columns (nx if
// narrower), whichever gives the smallest loaded region (tile + ring) with at
// most nb tiles; ntx = 0 when no width fits.
struct SplitTiles {
    int tw0, th0, ntx, nty, LR;
};
__host__ __device__ inline SplitTiles split_tiles(int nx, int ny, int nb, int order) {
    SplitTiles best{};
    best.LR = order == 3 ? 3 : 2;
    long best_area = -1;
    for (int w = CS_TW; w <= 8 * CS_TW; w *= 2) {
        SplitTiles t{};
        t.LR = best.LR;
        t.tw0 = nx < w ? nx : w;
        t.ntx = (nx + t.tw0 - 1) / t.tw0;
        const int ntymax = t.ntx <= nb ? nb / t.ntx : 0;
        if (ntymax < 1) continue;
        t.th0 = (ny + ntymax - 1) / ntymax;
        t.nty = (ny + t.th0 - 1) / t.th0;
        const long area = (long)(t.tw0 + 2 * t.LR) * (t.th0 + 2 * t.LR);
        if (best_area < 0 || area < best_area) {
            best = t;
            best_area = area;
        }
        if (nx <= w) break;
    }
    return best;
}
// shared-memory doubles: the loaded state (3 fields, tile + ring LR), the slow
// tendencies and the forward velocities (tile + ring 1), D c of the tile's
// rows, the coefficients
__host__ __device__ inline long split_smem_doubles(const SplitTiles& t, int ccap) {
    const long rw = t.tw0 + 2 * t.LR, rh = t.th0 + 2 * t.LR, hw = t.tw0 + 2, hh = t.th0 + 2;
    return 3 * rw * rh + 5 * hw * hh + 3L * t.tw0 * t.th0 + (ccap > 0 ? ccap : 1);
}

__device__ __forceinline__ double ldg2(const double* p) { return __ldcg(p); }   // written by other CTAs

// warp_dot with x read from L2 (x's rows were written by other CTAs)
__device__ __forceinline__ double warp_dot_x_l2(const double* a, const double* x, long r0, long r1) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    long row = r0 + lane;
    for (; row + 96 < r1; row += 128) {
        const double a0 = a[row], a1 = a[row + 32], a2 = a[row + 64], a3 = a[row + 96];
        const double b0 = __ldcg(x + row), b1 = __ldcg(x + row + 32), b2 = __ldcg(x + row + 64),
                     b3 = __ldcg(x + row + 96);
        s += a0 * b0;
        s += a1 * b1;
        s += a2 * b2;
        s += a3 * b3;
    }
    for (; row < r1; row += 32) s += a[row] * __ldcg(x + row);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// CW: warps of the coarse group; CW = CS_NW (no product group) for the literal
// form without a basis, where D c = 0.
template <bool DELTA, int CW>
__global__ void __launch_bounds__(CS_NT, 1) k_chain_split(ChainArgs A) {
    constexpr int CT = 32 * CW, PT = CS_NT - CT, PW = PT / 32 > 0 ? PT / 32 : 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[CS_NT / 32];
    __shared__ int s_okc, s_okp, s_okf, s_fail;
    const unsigned nb = gridDim.x;
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const long d = A.d, ncell = d / 3;
    const int nx = A.nx, ny = A.ny;
    const SplitTiles T = split_tiles(nx, ny, (int)nb, A.cc.order);
    int tx0 = 0, ty0 = 0, tw = 0, th = 0;
    if (b < T.ntx * T.nty) {
        const int ty = b / T.ntx, tx = b - ty * T.ntx;
        tx0 = tx * T.tw0;
        ty0 = ty * T.th0;
        tw = min(T.tw0, nx - tx0);
        th = min(T.th0, ny - ty0);
    }
    const int ncl = tw * th, nclx = T.tw0 * T.th0;
    const int LR = T.LR, RW = tw + 2 * LR, RH = th + 2 * LR, HW = tw + 2, HH = th + 2;
    const int RSZ = (T.tw0 + 2 * LR) * (T.th0 + 2 * LR), HSZ = (T.tw0 + 2) * (T.th0 + 2);
    double* st = reinterpret_cast<double*>(smraw);   // [3][RSZ] state on the tile + ring LR
    double* S = st + 3 * RSZ;                        // [3][HSZ] slow tendencies, tile + ring 1
    double* fu = S + 3 * HSZ;                        // [HSZ] forward u, tile + ring 1
    double* fw = fu + HSZ;                           // [HSZ] forward w
    double* dc = fw + HSZ;                           // [3][nclx] D c on the tile's rows
    double* cs = dc + 3 * nclx;                      // [ccap] coefficients
    const int ncols = A.r_dev ? *A.r_dev : 0;
    if (ncols < 0 || ncols > A.ccap) {   // cannot happen: the rank never exceeds the cap
        if (tid == 0) atomicExch(&A.gb->err, 2);
        return;
    }
    if (tid == 0) s_fail = 0;
    __syncthreads();
    // rows of the dot products: the tile kernel's contiguous ranges
    const long rpb = ((d + nb - 1) / nb + 31) / 32 * 32;
    const long r0 = min(d, (long)b * rpb), r1 = min(d, r0 + rpb);
    const CoarseT<double> cc = coarse_t<double>(A.cc);
    const bool ynone = A.cc.V == 0.0 && A.cc.omega == 0.0;
    double* bufA = A.gbuf;
    double* bufB = A.gbuf + d;
    // global row of local cell k of the tile, field f
    auto tile_row = [&](int f, int k) {
        const int ly = k / tw, lx = k - ly * tw;
        return (long)f * ncell + (long)(ty0 + ly) * nx + tx0 + lx;
    };

    // the buffer holding G(delta_i) after the coarse group: every step starts
    // in the buffer other than its input and alternates with each substep
    const double* R = nullptr;   // the input is neither work state
    for (int st_ = 0; st_ < A.n_g; ++st_) {
        const double* n0 = (R == bufA) ? bufB : bufA;
        R = (cc.n_sound & 1) ? n0 : ((n0 == bufA) ? bufB : bufA);
    }

    for (int i = A.i_begin; i < A.i_end; ++i) {
        // the state K acts on: delta_i, or q_i itself (literal form)
        const double* xin = DELTA ? A.dlt64 : A.q + (long)i * d;
        if (wid < CW) {
            // ---------------------------------------------------- coarse group
            const int ct = tid;
            const double* X = xin;
            bool ok = true;
            for (int gs = 0; gs < A.n_g && ok; ++gs) {
                const double* cur = X;
                double* nxt = (X == bufA) ? bufB : bufA;
                for (int m = 0; m < cc.n_sound && ok; ++m) {
                    // the state on the tile and its ring (periodic); four cells
                    // per thread at a time, their loads in flight together
                    for (int e0 = ct; e0 < RW * RH; e0 += 4 * CT) {
                        double vu[4], vw[4], vp[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int e = e0 + q * CT;
                            if (e < RW * RH) {
                                const int ly = e / RW, lx = e - ly * RW;
                                const long g = (long)pwrap(ty0 - LR + ly, ny) * nx + pwrap(tx0 - LR + lx, nx);
                                vu[q] = ldg2(cur + g);
                                vw[q] = ldg2(cur + ncell + g);
                                vp[q] = ldg2(cur + 2 * ncell + g);
                            }
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int e = e0 + q * CT;
                            if (e < RW * RH) {
                                st[e] = vu[q];
                                st[RSZ + e] = vw[q];
                                st[2 * RSZ + e] = vp[q];
                            }
                        }
                    }
                    named_barrier(1, CT);
                    if (m == 0) {
                        // slow tendencies of the step's input (cur == X) on the tile + ring 1
                        for (int e = ct; e < HW * HH; e += CT) {
                            const int hy = e / HW, hx = e - hy * HW;
                            const int si = (hy + LR - 1) * RW + hx + LR - 1;
                            double Ur = cc.U, Vc = cc.V;
                            if (A.cc.omega != 0.0) {
                                const int gy = pwrap(ty0 - 1 + hy, ny), gx = pwrap(tx0 - 1 + hx, nx);
                                Ur += (double)(A.cc.omega * ((gy + 0.5) * A.cc.dy - A.cc.hly));
                                Vc -= (double)(A.cc.omega * ((gx + 0.5) * A.cc.dx - A.cc.hlx));
                            }
#pragma unroll
                            for (int f = 0; f < 3; ++f) {
                                const double* a = st + f * RSZ;
                                double v;
                                if (cc.order == 1) {
                                    const double ax = -Ur * cc.inv_dx, ay = -Vc * cc.inv_dy;
                                    const double dx_ = Ur >= 0.0 ? a[si] - a[si - 1] : a[si + 1] - a[si];
                                    const double dy_ = ynone ? 0.0 : (Vc >= 0.0 ? a[si] - a[si - RW] : a[si + RW] - a[si]);
                                    v = slow_first_order<double>(ax, ay, dx_, dy_, ynone);
                                } else {
                                    const double Fe = upwind_flux3_pts<double>(Ur, a[si - 1], a[si], a[si + 1], a[si + 2]);
                                    const double Fw = upwind_flux3_pts<double>(Ur, a[si - 2], a[si - 1], a[si], a[si + 1]);
                                    const double Gn = upwind_flux3_pts<double>(Vc, a[si - RW], a[si], a[si + RW],
                                                                               a[si + 2 * RW]);
                                    const double Gs = upwind_flux3_pts<double>(Vc, a[si - 2 * RW], a[si - RW], a[si],
                                                                               a[si + RW]);
                                    v = -(Fe - Fw) * cc.inv_dx - (Gn - Gs) * cc.inv_dy;
                                }
                                S[f * HSZ + e] = v;
                            }
                        }
                        named_barrier(1, CT);
                    }
                    // forward: velocities on the tile + ring 1
                    {
                        const double* u = st;
                        const double* w = st + RSZ;
                        const double* p = st + 2 * RSZ;
                        for (int e = ct; e < HW * HH; e += CT) {
                            const int hy = e / HW, hx = e - hy * HW;
                            const int si = (hy + LR - 1) * RW + hx + LR - 1;
                            fu[e] = fb_new_u<double>(cc, S[e], u[si], u[si + 1], u[si - 1], p[si + 1], p[si - 1],
                                                     w[si + 1 + RW], w[si + 1 - RW], w[si - 1 + RW], w[si - 1 - RW]);
                            fw[e] = fb_new_w<double>(cc, S[HSZ + e], w[si], w[si + RW], w[si - RW], p[si + RW],
                                                     p[si - RW], u[si + 1 + RW], u[si - 1 + RW], u[si + 1 - RW],
                                                     u[si - 1 - RW]);
                        }
                    }
                    named_barrier(1, CT);
                    // backward: pressure on the tile; the tile's new state is written out
                    for (int k = ct; k < ncl; k += CT) {
                        const int ly = k / tw, lx = k - ly * tw;
                        const int e = (ly + 1) * HW + lx + 1, si = (ly + LR) * RW + lx + LR;
                        const double pn = fb_new_p<double>(cc, S[2 * HSZ + e], st[2 * RSZ + si], fu[e + 1], fu[e - 1],
                                                           fw[e + HW], fw[e - HW]);
                        const long g = (long)(ty0 + ly) * nx + tx0 + lx;
                        nxt[g] = fu[e];
                        nxt[ncell + g] = fw[e];
                        nxt[2 * ncell + g] = pn;
                    }
                    const bool last = gs == A.n_g - 1 && m == cc.n_sound - 1;
                    if (!last && !grid_barrier_group(A.gb, 0, nb, 1, CT, ct == 0, &s_okc)) {
                        ok = false;
                        break;
                    }
                    cur = nxt;
                    nxt = (nxt == bufA) ? bufB : bufA;
                }
                X = cur;
            }
            if (!ok) s_fail = 1;
        } else if constexpr (PT > 0) {
            // ---------------------------------------------------- product group
            const int pt = tid - CT, pw = pt >> 5;
            const double* x = xin;
            bool ok = true;
            for (int l = pw; l < ncols; l += PW) {
                const double s = warp_dot_x_l2(A.Q + (long)l * d, x, r0, r1);
                if (lane == 0) A.part[(long)b * A.ccap + l] = s;
            }
            ok = grid_barrier_group(A.gb, 1, nb, 2, PT, pt == 0, &s_okp);
            if (ok && ncols > 0) {
                const int cpb = (ncols + (int)nb - 1) / (int)nb;
                const int l1 = min(ncols, (b + 1) * cpb);
                for (int l = b * cpb + pw; l < l1; l += PW) {
                    const double s = warp_sum_strided(A.part + l, nb, A.ccap);
                    if (lane == 0) A.cvec[l] = s;
                }
            }
            if (ok) ok = grid_barrier_group(A.gb, 1, nb, 2, PT, pt == 0, &s_okp);
            if (ok) {
                for (int l = pt; l < ncols; l += PT) cs[l] = __ldcg(A.cvec + l);
                named_barrier(2, PT);
                for (int k = pt; k < 3 * ncl; k += PT) {
                    const int f = k / ncl, kk = k - f * ncl;
                    const double* Dr = A.D + tile_row(f, kk);
                    double acc = 0.0;
#pragma unroll 8
                    for (int l = 0; l < ncols; ++l) acc += __ldg(Dr + (long)l * d) * cs[l];
                    dc[f * nclx + kk] = acc;
                }
            }
            if (!ok) s_fail = 1;
        }
        __syncthreads();   // join: G(delta_i) and D c of the tile's rows are complete
        if (s_fail) return;
        const double* qt = A.qt ? A.qt + (long)i * d : nullptr;
        const double* ko = A.kold ? A.kold + (long)i * d : nullptr;
        double* qn = A.q + (long)(i + 1) * d;
        double* dl = A.dlt64;
        double* ga = (DELTA && A.gacc) ? A.gacc + (long)i * d : nullptr;
        double s = 0.0;
        for (int k = tid; k < 3 * ncl; k += CS_NT) {
            const int f = k / ncl, kk = k - f * ncl;
            const long row = tile_row(f, kk);
            const double gin = R[row];
            const double dcv = PT > 0 ? dc[f * nclx + kk] : 0.0;   // (no product group: no basis)
            double y;
            if (DELTA) {
                y = qt[row] + (gin + dcv);
            } else {
                const double knew = gin + dcv;
                y = (qt ? qt[row] : 0.0) + (knew - (ko ? ko[row] : 0.0));
            }
            const double e = y - qn[row];
            s += e * e;
            qn[row] = y;
            if (DELTA) dl[row] = e;
            if (ga) ga[row] += gin;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[wid] = s;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int k = 0; k < CS_NT / 32; ++k) t += red[k];
            A.resp[(long)i * nb + b] = t;
        }
        if (!grid_barrier_group(A.gb, 2, nb, 0, CS_NT, tid == 0, &s_okf)) return;
    }
    if (A.res2 && b == 0) {
        for (int i = A.i_begin + wid; i < A.i_end; i += CS_NT / 32) {
            const double t = warp_sum_strided(A.resp + (long)i * nb, nb, 1);
            if (lane == 0) A.res2[i + 1] = t;
        }
    }
}

size_t chain_smem_bytes(int H, int ccap, bool f32) {
    const size_t el = f32 ? sizeof(float) : sizeof(double);
    size_t a = el * coarse_tile_smem_elems<CH_TX, CH_TY>(H);
    size_t c = el * (size_t)(ccap > 0 ? ccap : 1);
    return a > c ? a : c;
}

}  // namespace

template <bool DELTA, typename T>
int chain_grid(int H, int ccap) {
    static DevMemo memo;   // [device] -> (shared-memory bytes, blocks)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    const int key = (int)chain_smem_bytes(H, ccap, std::is_same<T, float>::value);
    int k0 = -1, blocks = 0;
    if (memo.get(dev, &k0, &blocks) && k0 == key) return blocks;
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    {
        std::lock_guard<std::mutex> lk(smem_launch_lock());
        if (set_dynamic_smem((const void*)k_chain<DELTA, T>, key) != cudaSuccess) return 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_chain<DELTA, T>, CH_NT, key);
    }
    blocks = per >= 1 ? sms : 0;
    memo.put(dev, key, blocks);
    return blocks;
}

long chain_resp_elems(int n_slices) { return (long)(n_slices + 1) * 1024; }

namespace {

size_t split_smem_bytes(int nx, int ny, int nb, int order, int ccap) {
    const SplitTiles t = split_tiles(nx, ny, nb, order);
    if (t.ntx * t.nty < 1 || t.ntx * t.nty > nb) return 0;
    return sizeof(double) * (size_t)split_smem_doubles(t, ccap);
}

// CTAs of the split-group chain (one per SM), or 0 when it does not fit
template <bool DELTA, int CW>
int split_grid(size_t smem) {
    static DevMemo memo;   // [device] -> (shared-memory bytes, blocks)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    int k0 = -1, blocks = 0;
    if (memo.get(dev, &k0, &blocks) && k0 == (int)smem) return blocks;
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    {
        std::lock_guard<std::mutex> lk(smem_launch_lock());
        if (set_dynamic_smem((const void*)k_chain_split<DELTA, CW>, smem) != cudaSuccess) return 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_chain_split<DELTA, CW>, CS_NT, smem);
    }
    blocks = per >= 1 ? sms : 0;
    memo.put(dev, (int)smem, blocks);
    return blocks;
}

}  // namespace

cudaError_t chain_coop(const ChainArgs& a, cudaStream_t s) {
    if (a.i_end <= a.i_begin) return cudaSuccess;
    if (a.dlt && a.dlt64) return cudaErrorInvalidValue;
    const bool split_delta = a.dlt64 && a.qt, split_literal = !a.dlt && !a.dlt64;
    if ((split_delta || split_literal) && a.cc.scheme == 0 && a.cc.n_sound >= 1 && a.n_g >= 1) {
        // FP64 with the split coarse step: coarse steps and products side by
        // side in two thread groups (one CTA per SM)
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorInvalidDevice;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int nb = a.max_blocks > 0 && a.max_blocks < sms ? a.max_blocks : sms;
        const size_t smem = nb >= 1 ? split_smem_bytes(a.nx, a.ny, nb, a.cc.order, a.ccap) : 0;
        // the literal form without a basis (the coarse initialisation, the
        // original Parareal, the coarse sweep): all warps in the coarse group
        const bool coarse_only = split_literal && !a.r_dev;
        const void* fn = split_delta  ? (const void*)k_chain_split<true, CS_CW>
                         : coarse_only ? (const void*)k_chain_split<false, CS_NW>
                                       : (const void*)k_chain_split<false, CS_CW>;
        const int fit = split_delta  ? split_grid<true, CS_CW>(smem)
                        : coarse_only ? split_grid<false, CS_NW>(smem)
                                      : split_grid<false, CS_CW>(smem);
        if (smem > 0 && smem <= 200 * 1024 && fit >= nb) {
            cudaError_t e = cudaMemsetAsync(&a.gb->count, 0, sizeof(unsigned), s);
            if (e == cudaSuccess) e = cudaMemsetAsync(a.gb->gcount, 0, sizeof(a.gb->gcount), s);
            if (e != cudaSuccess) return e;
            ChainArgs arg = a;
            void* args[] = {&arg};
            std::lock_guard<std::mutex> lk(smem_launch_lock());
            e = set_dynamic_smem(fn, smem);
            if (e != cudaSuccess) return e;
            e = cudaLaunchCooperativeKernel(fn, dim3(nb), dim3(CS_NT), args, smem, s);
            count_launches(1);
            return e;
        }
    }
    const bool f32 = a.dlt != nullptr, d64 = a.dlt64 != nullptr;
    int nb = f32 ? chain_grid<true, float>(a.H, a.ccap)
                 : (d64 ? chain_grid<true, double>(a.H, a.ccap) : chain_grid<false, double>(a.H, a.ccap));
    if (a.max_blocks > 0 && nb > a.max_blocks) nb = a.max_blocks;
    if (nb < 1 || nb > 1024) return cudaErrorInvalidConfiguration;
    const size_t smem = chain_smem_bytes(a.H, a.ccap, f32);
    const void* fn = f32 ? (const void*)k_chain<true, float>
                         : (d64 ? (const void*)k_chain<true, double> : (const void*)k_chain<false, double>);
    cudaError_t e = cudaMemsetAsync(&a.gb->count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    ChainArgs arg = a;
    void* args[] = {&arg};
    std::lock_guard<std::mutex> lk(smem_launch_lock());
    e = set_dynamic_smem(fn, smem);
    if (e != cudaSuccess) return e;
    e = cudaLaunchCooperativeKernel(fn, dim3(nb), dim3(CH_NT), args, smem, s);
    count_launches(1);
    return e;
}

}  // namespace pr
