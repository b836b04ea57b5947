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
// Work items are 32-cell segments of grid rows, one per warp (lanes along x,
// coalesced); each CTA owns a contiguous range of them.
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
    }
    return c;
}

cudaError_t fine_sweep_coop(const FineSweepArgs& a, bool has_v, cudaStream_t s) {
    const int nb = has_v ? coop_blocks<true>(a.max_sms) : coop_blocks<false>(a.max_sms);
    if (nb < 1) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaMemsetAsync(&a.gb->count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    FineSweepArgs arg = a;
    void* args[] = {&arg};
    const void* fn = has_v ? (const void*)k_fine_coop<true> : (const void*)k_fine_coop<false>;
    e = cudaLaunchCooperativeKernel(fn, dim3(nb), dim3(FC_NT), args, 0, s);
    count_launches(1);
    return e;
}

}  // namespace pr
