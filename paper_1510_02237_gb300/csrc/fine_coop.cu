// fine_coop.cu -- FP64 fine propagator F as one cooperative launch: all
// three RK-3 stages of all N_f steps for n states, a grid barrier between
// stages, no halo recomputation (the FP64 pipe, not memory, bounds FP64
// stencil work on GB300, so the stages are not fused).
//
// Per stage k (stage lengths c_k = dt/3, dt/2, dt) and cell:
//   out = q^n + c_k L(in),   L = the flux-form tendency of Sec. 3 with the
//   6th-order centred advection difference, 2nd-order centred acoustics and
//   the compact grad-div damping (Sec. 3.2, Eq. dampingCoeff).
// c_k is folded into every coefficient, so each term costs one FMA.
//
// GB300 issues FP64 arithmetic at 1/64 of the FP32 rate (one warp
// instruction per ~64 cycles per SM sub-partition), while shuffles, loads and
// integer work issue at full rate: the FP64 instruction count per cell is the
// cost, everything else is nearly free.  Constant velocity with V = 0 (the
// benchmark problems) runs k_fine_march: every warp walks down a contiguous
// range of rows of 32-column segments (lane = column), x-neighbours come by
// shuffles from the lane values and a 6-cell halo held by lanes 0..5, and
// the x-differences of u and w are computed once per row and reused by the
// rows above and below (the cross terms of the damping are differences of
// them), 33 FP64 instructions per cell and stage.  Rows are split evenly over
// all warps of the grid, so every SM sub-partition gets the same work.
// V != 0 and the rotation run k_fine_coop<true> on 32-cell work items.
#include "grid_barrier.cuh"

namespace pr {
namespace {

constexpr int FC_NT = 512;

__device__ __forceinline__ int wrapp(int i, int n) { return i >= n ? i - n : i; }   // needs n >= 4
__device__ __forceinline__ int wrapm(int i, int n) { return i < 0 ? i + n : i; }

template <bool HV>
// in and qn are written by other CTAs earlier in the same launch (ordered by
// the grid barriers), so they are read through the coherent path, not the
// read-only one: no __restrict__ on them.
__device__ __forceinline__ void stage_seg(const double* in, const double* qn,
                                          double* __restrict__ out, long base, int y, int xs, int nx, int ny,
                                          long ncell, const FineCoefK& c, int k) {
    const int lane = threadIdx.x & 31;
    const double* u = in + base;
    const double* w = u + ncell;
    const double* p = w + ncell;
    const long R0 = (long)y * nx, Rm = (long)wrapm(y - 1, ny) * nx, Rp = (long)wrapp(y + 1, ny) * nx;
    long Rm2 = 0, Rm3 = 0, Rp2 = 0, Rp3 = 0;
    if (HV) {
        Rm2 = (long)wrapm(y - 2, ny) * nx;
        Rm3 = (long)wrapm(y - 3, ny) * nx;
        Rp2 = (long)wrapp(y + 2, ny) * nx;
        Rp3 = (long)wrapp(y + 3, ny) * nx;
    }
    // advection coefficients of this row (x) and, below, of each column (y):
    // constant, or varying with the solid-body rotation (Eq. adVel), which
    // the host runs as HV (a rotation has both components)
    const double A = HV ? c.adx[k] + c.aomx[k] * ((y + 0.5) * c.dy - c.hly) : c.adx[k];
    const double Bx = c.csx[k], By = c.csy[k];
    const double Cx = c.dxx[k], Ex = c.dxy1[k], Cy = c.dyy[k], Ey = c.dxy2[k];
    const double* qu = qn + base;
    const double* qw = qu + ncell;
    const double* qp = qw + ncell;
    double* ou = out + base;
    double* ow = ou + ncell;
    double* op = ow + ncell;
    {
        const int x = xs + lane;
        if (x >= nx) return;
        const double Ay = HV ? c.ady[k] + c.aomy[k] * ((x + 0.5) * c.dx - c.hlx) : 0.0;
        const int xm1 = wrapm(x - 1, nx), xm2 = wrapm(x - 2, nx), xm3 = wrapm(x - 3, nx);
        const int xp1 = wrapp(x + 1, nx), xp2 = wrapp(x + 2, nx), xp3 = wrapp(x + 3, nx);
        // x-advection differences (6th-order centred flux difference)
        const double du6 = (u[R0 + xp3] - u[R0 + xm3]) - 9.0 * (u[R0 + xp2] - u[R0 + xm2]) + 45.0 * (u[R0 + xp1] - u[R0 + xm1]);
        const double dw6 = (w[R0 + xp3] - w[R0 + xm3]) - 9.0 * (w[R0 + xp2] - w[R0 + xm2]) + 45.0 * (w[R0 + xp1] - w[R0 + xm1]);
        const double dp6 = (p[R0 + xp3] - p[R0 + xm3]) - 9.0 * (p[R0 + xp2] - p[R0 + xm2]) + 45.0 * (p[R0 + xp1] - p[R0 + xm1]);
        const double dux = u[R0 + xp1] - u[R0 + xm1];
        const double dwy = w[Rp + x] - w[Rm + x];
        const double dpx = p[R0 + xp1] - p[R0 + xm1];
        const double dpy = p[Rp + x] - p[Rm + x];
        const double lapu = (u[R0 + xp1] + u[R0 + xm1]) - 2.0 * u[R0 + x];
        const double lapw = (w[Rp + x] + w[Rm + x]) - 2.0 * w[R0 + x];
        const double crw = (w[Rp + xp1] - w[Rm + xp1]) - (w[Rp + xm1] - w[Rm + xm1]);
        const double cru = (u[Rp + xp1] - u[Rp + xm1]) - (u[Rm + xp1] - u[Rm + xm1]);
        double nu = qu[R0 + x] + A * du6;
        double nw = qw[R0 + x] + A * dw6;
        double np = qp[R0 + x] + A * dp6;
        if (HV) {
            nu += Ay * ((u[Rp3 + x] - u[Rm3 + x]) - 9.0 * (u[Rp2 + x] - u[Rm2 + x]) + 45.0 * (u[Rp + x] - u[Rm + x]));
            nw += Ay * ((w[Rp3 + x] - w[Rm3 + x]) - 9.0 * (w[Rp2 + x] - w[Rm2 + x]) + 45.0 * dwy);
            np += Ay * ((p[Rp3 + x] - p[Rm3 + x]) - 9.0 * (p[Rp2 + x] - p[Rm2 + x]) + 45.0 * dpy);
        }
        nu += Bx * dpx;
        nu += Cx * lapu;
        nu += Ex * crw;
        nw += By * dpy;
        nw += Cy * lapw;
        nw += Ey * cru;
        np += Bx * dux;
        np += By * dwy;
        ou[R0 + x] = nu;
        ow[R0 + x] = nw;
        op[R0 + x] = np;
    }
}

template <bool HV>
__global__ void __launch_bounds__(FC_NT) k_fine_coop(FineSweepArgs a) {
    const unsigned nb = gridDim.x;
    const long ncell = (long)a.nx * a.ny;
    const long d = 3 * ncell;
    const int nseg = (a.nx + 31) >> 5;                 // 32-cell segments per grid row
    const int nitems = a.n * a.ny * nseg;
    // each CTA takes a contiguous range of work items (consecutive segments
    // and rows of a slice), so the y-neighbour rows a warp reads were mostly
    // brought into L1 by the CTA's other warps; its warps share the range
    // round-robin
    const int it0 = (int)((long)nitems * blockIdx.x / nb), it1 = (int)((long)nitems * (blockIdx.x + 1) / nb);
    const int wq = threadIdx.x >> 5, nwq = FC_NT >> 5;
    const double* cur = a.in;
    for (int t = 0; t < a.nsteps; ++t) {
        double* s1 = (cur == a.w1) ? a.w2 : a.w1;
        double* s2 = a.w3;
        double* dst = (t == a.nsteps - 1) ? a.out : s1;
        const double* srcs[3] = {cur, s1, s2};
        double* dsts[3] = {s1, s2, dst};
        for (int k = 0; k < 3; ++k) {
            for (int it = it0 + wq; it < it1; it += nwq) {
                const int rr = it / nseg, sg = it - rr * nseg;
                const int sl = rr / a.ny, y = rr - sl * a.ny;
                stage_seg<HV>(srcs[k], cur, dsts[k], (long)sl * d, y, sg * 32, a.nx, a.ny, ncell, a.c, k);
            }
            if (t == a.nsteps - 1 && k == 2) break;   // kernel end publishes the result
            if (!grid_barrier(a.gb, nb)) return;
        }
        cur = dst;
    }
}

// ------------------------------------------------------------ V = 0 marching

constexpr int FM_NT = 256;   // 8 warps per CTA, one CTA per SM

// a - b as one FMA by a 1.0 held in a register: exactly the rounded
// difference.  DADD and DFMA take the same FP64 pipe slot; in this kernel the
// FMA form measured 4 % faster, but only with the 1.0 in a register -- as a
// constant-bank operand of the FMAs (a literal or a kernel parameter) it was
// 5 % slower than that.  The 1.0 is therefore read from device memory, which
// the compiler cannot fold.
__device__ double g_march_one = 1.0;
__device__ __forceinline__ double dsub(double a, double b, double one) { return fma(a, one, -b); }

// Stage k on the rows [g0, g1) of the batch's row segments (index
// ((slice * nseg) + segment) * ny + y): out = qn + c_k L(in).  A warp marches
// down its rows with 32 columns per row (one per lane): each row's own values
// are loaded one row ahead of their use, its x-neighbours (periodic offsets
// -3..3 precomputed per lane) are loaded where they are used, from lines the
// row's own loads brought into L1, and the x-differences of a row are reused
// by the rows above and below it.  in, qn and out are written by other CTAs
// earlier in the same launch (ordered by the grid barriers), so they are read
// through the coherent path: no __restrict__, no __ldg.
__device__ __forceinline__ void stage_march(const double* in, const double* qn, double* out, long d, int nx, int ny,
                                            int nseg, long g0, long g1, const FineCoefK& c, int k) {
    const int lane = threadIdx.x & 31;
    const long ncell = (long)nx * ny;
    // k is a compile-time constant after unrolling: the coefficients are
    // constant operands of the FMAs, not registers
    const double A = c.adx[k], Bx = c.csx[k], By = c.csy[k], Ex = c.dxy1[k], Cy = c.dyy[k], Ey = c.dxy2[k];
    // u's x-terms on raw neighbours: A (6-point difference) + Cx (u[x+1] - 2u + u[x-1])
    const double up1 = c.up1[k], um1 = c.um1[k], up2 = c.up2[k], um2 = c.um2[k], um3 = c.um3[k], u00 = c.u00[k];
    const double A45 = c.a45[k], Am9 = c.am9[k], Cy2 = c.cy2[k];
    const double one = g_march_one;
    for (long g = g0; g < g1;) {
        const long col = g / ny;
        const int y0 = (int)(g - col * ny);
        const int y1 = (int)min((long)ny, (long)y0 + (g1 - g));
        g += y1 - y0;
        const int z = (int)(col / nseg), sg = (int)(col - (long)z * nseg);
        const int x0 = 32 * sg, nv = min(32, nx - x0);
        const int xo = x0 + (lane < nv ? lane : 0);   // lanes past a ragged edge compute, never store
        const int xm1 = pwrap(xo - 1, nx), xp1 = pwrap(xo + 1, nx), xm2 = pwrap(xo - 2, nx);
        const int xp2 = pwrap(xo + 2, nx), xm3 = pwrap(xo - 3, nx), xp3 = pwrap(xo + 3, nx);
        const double* src = in + (long)z * d;
        const double* qz = qn + (long)z * d;
        double* dz = out + (long)z * d;
        // the row above the range (only its x-differences and w, p are used)
        const double* rm = src + (long)pwrap(y0 - 1, ny) * nx;
        double d1u_m = dsub(rm[xp1], rm[xm1], one);
        double d1w_m = dsub(rm[ncell + xp1], rm[ncell + xm1], one);
        double w_m = rm[ncell + xo], p_m = rm[2 * ncell + xo];
        // the centre row and the row below: own values in registers
        const double* rc = src + (long)y0 * nx;
        double d1u_c = dsub(rc[xp1], rc[xm1], one);
        double d1w_c = dsub(rc[ncell + xp1], rc[ncell + xm1], one);
        double cu = rc[xo], cw = rc[ncell + xo], cp = rc[2 * ncell + xo];
        const double* rb = src + (long)(y0 + 1 < ny ? y0 + 1 : y0 + 1 - ny) * nx;
        double bu = rb[xo], bw = rb[ncell + xo], bp = rb[2 * ncell + xo];
        long rcx = (long)y0 * nx + xo;
        double qu = qz[rcx], qw = qz[ncell + rcx], qp = qz[2 * ncell + rcx];
        for (int y = y0; y < y1; ++y) {
            const double* rn = src + (long)pwrap(y + 2, ny) * nx;
            const double nu_ = rn[xo], nw_ = rn[ncell + xo], np_ = rn[2 * ncell + xo];
            const long rnx = (long)(y + 1 < ny ? y + 1 : y + 1 - ny) * nx + xo;
            const double qu_n = qz[rnx], qw_n = qz[ncell + rnx], qp_n = qz[2 * ncell + rnx];
            const double d1u_n = dsub(rb[xp1], rb[xm1], one);
            const double d1w_n = dsub(rb[ncell + xp1], rb[ncell + xm1], one);
            const double u1 = rc[xp1], um1v = rc[xm1], u2 = rc[xp2], um2v = rc[xm2], u3 = rc[xp3], um3v = rc[xm3];
            const double* rcw = rc + ncell;
            const double* rcp = rc + 2 * ncell;
            const double d1p = dsub(rcp[xp1], rcp[xm1], one);
            const double d2p = dsub(rcp[xp2], rcp[xm2], one);
            const double d3p = dsub(rcp[xp3], rcp[xm3], one);
            const double d2w = dsub(rcw[xp2], rcw[xm2], one);
            const double d3w = dsub(rcw[xp3], rcw[xm3], one);
            const double dwy = dsub(bw, w_m, one), dpy = dsub(bp, p_m, one);
            const double crw = dsub(d1w_n, d1w_m, one), cru = dsub(d1u_n, d1u_m, one);
            double nu = fma(up1, u1, qu);
            nu = fma(um1, um1v, nu);
            nu = fma(up2, u2, nu);
            nu = fma(um2, um2v, nu);
            nu = fma(A, u3, nu);
            nu = fma(um3, um3v, nu);
            nu = fma(u00, cu, nu);
            nu = fma(Bx, d1p, nu);
            nu = fma(Ex, crw, nu);
            double nw = fma(A45, d1w_c, qw);
            nw = fma(Am9, d2w, nw);
            nw = fma(A, d3w, nw);
            nw = fma(By, dpy, nw);
            nw = fma(Cy, bw, nw);
            nw = fma(Cy, w_m, nw);
            nw = fma(Cy2, cw, nw);
            nw = fma(Ey, cru, nw);
            double np = fma(A45, d1p, qp);
            np = fma(Am9, d2p, np);
            np = fma(A, d3p, np);
            np = fma(Bx, d1u_c, np);
            np = fma(By, dwy, np);
            if (lane < nv) {
                dz[rcx] = nu;
                dz[ncell + rcx] = nw;
                dz[2 * ncell + rcx] = np;
            }
            w_m = cw;
            p_m = cp;
            d1u_m = d1u_c;
            d1w_m = d1w_c;
            rc = rb;
            cu = bu;
            cw = bw;
            cp = bp;
            rb = rn;
            bu = nu_;
            bw = nw_;
            bp = np_;
            d1u_c = d1u_n;
            d1w_c = d1w_n;
            rcx = rnx;
            qu = qu_n;
            qw = qw_n;
            qp = qp_n;
        }
    }
}

// One CTA per SM, stated as the minimum-blocks bound: the compiler then uses
// up to 140 registers and keeps more loads in flight (without the bound it
// chose 104 and the sweep was 5 % slower)
__global__ void __launch_bounds__(FM_NT, 1) k_fine_march(FineSweepArgs a) {
    const unsigned nb = gridDim.x;
    const long d = 3L * a.nx * a.ny;
    const int nseg = (a.nx + 31) >> 5;
    const long rows = (long)a.n * nseg * a.ny;
    const long W = (long)gridDim.x * (FM_NT / 32);
    const long gw = (long)blockIdx.x * (FM_NT / 32) + (threadIdx.x >> 5);
    const long g0 = rows * gw / W, g1 = rows * (gw + 1) / W;
    const double* cur = a.in;
    for (int t = 0; t < a.nsteps; ++t) {
        double* s1 = (cur == a.w1) ? a.w2 : a.w1;
        double* s2 = a.w3;
        double* dst = (t == a.nsteps - 1) ? a.out : s1;
        const double* srcs[3] = {cur, s1, s2};
        double* dsts[3] = {s1, s2, dst};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            stage_march(srcs[k], cur, dsts[k], d, a.nx, a.ny, nseg, g0, g1, a.c, k);
            if (t == a.nsteps - 1 && k == 2) break;   // kernel end publishes the result
            if (!grid_barrier(a.gb, nb)) return;
        }
        cur = dst;
    }
}

int march_blocks(int max_sms) {
    static DevMemo memo;   // [device] -> (SMs, CTAs per SM)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    int nsm = 0, per = 0;
    if (!memo.get(dev, &nsm, &per)) {
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fine_march, FM_NT, 0);
        memo.put(dev, nsm, per);
    }
    if (per < 1) return -1;
    return max_sms > 0 && max_sms < nsm ? max_sms : nsm;   // one CTA per SM
}

template <bool HV>
int coop_blocks(int max_sms) {
    static DevMemo memo;   // [device] -> (SMs, CTAs per SM)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    int nsm = 0, per = 0;
    if (!memo.get(dev, &nsm, &per)) {
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fine_coop<HV>, FC_NT, 0);
        memo.put(dev, nsm, per);
    }
    if (per < 1) return -1;
    const int sms = max_sms > 0 && max_sms < nsm ? max_sms : nsm;
    return sms * per;
}

}  // namespace

FineCoefK make_fine_coef_k(double U, double V, double cs, double dx, double dy, double nu, double dt, double omega,
                           double lx, double ly) {
    const double a1 = nu * dx * dx / dt, a2 = nu * dy * dy / dt;
    const double ck[3] = {dt / 3.0, dt / 2.0, dt};
    FineCoefK c;
    c.dx = dx;
    c.dy = dy;
    c.hlx = 0.5 * lx;
    c.hly = 0.5 * ly;
    for (int k = 0; k < 3; ++k) {
        c.adx[k] = -ck[k] * (U / (60.0 * dx));
        c.ady[k] = -ck[k] * (V / (60.0 * dy));
        c.aomx[k] = -ck[k] * (omega / (60.0 * dx));
        c.aomy[k] = ck[k] * (omega / (60.0 * dy));
        c.csx[k] = -ck[k] * (cs / (2.0 * dx));
        c.csy[k] = -ck[k] * (cs / (2.0 * dy));
        c.dxx[k] = ck[k] * (a1 / (dx * dx));
        c.dxy1[k] = ck[k] * (a1 / (4.0 * dx * dy));
        c.dyy[k] = ck[k] * (a2 / (dy * dy));
        c.dxy2[k] = ck[k] * (a2 / (4.0 * dx * dy));
        const double A = c.adx[k], Cx = c.dxx[k];
        c.up1[k] = 45.0 * A + Cx;
        c.um1[k] = Cx - 45.0 * A;
        c.up2[k] = -9.0 * A;
        c.um2[k] = 9.0 * A;
        c.um3[k] = -A;
        c.u00[k] = -2.0 * Cx;
        c.a45[k] = 45.0 * A;
        c.am9[k] = -9.0 * A;
        c.cy2[k] = -2.0 * c.dyy[k];
    }
    return c;
}

cudaError_t fine_sweep_coop(const FineSweepArgs& a, bool has_v, cudaStream_t s) {
    const int nb = has_v ? coop_blocks<true>(a.max_sms) : march_blocks(a.max_sms);
    if (nb < 1) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaMemsetAsync(&a.gb->count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    FineSweepArgs arg = a;
    void* args[] = {&arg};
    const void* fn = has_v ? (const void*)k_fine_coop<true> : (const void*)k_fine_march;
    e = cudaLaunchCooperativeKernel(fn, dim3(nb), dim3(has_v ? FC_NT : FM_NT), args, 0, s);
    count_launches(1);
    return e;
}

}  // namespace pr
