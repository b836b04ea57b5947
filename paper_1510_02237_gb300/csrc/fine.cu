// fine.cu -- fine propagator F: one RK-3 step of the flux-form
// acoustic-advection tendency (Sec. 3; fine scheme of Sec. 3.2) per launch,
// with the three stages fused in shared memory.
//
// Tendency per cell (x contiguous, periodic):
//   adv   = -U/(60 dx) [(f[i+3]-f[i-3]) - 9(f[i+2]-f[i-2]) + 45(f[i+1]-f[i-1])]  (+ same in y with V)
//           i.e. the difference of 6th-order centred interface fluxes;
//   u_t  += -c_s (p[i+1]-p[i-1])/(2dx) + alpha1 [ (u[i+1]-2u+u[i-1])/dx^2
//           + ((w[i+1,j+1]-w[i+1,j-1]) - (w[i-1,j+1]-w[i-1,j-1]))/(4 dx dy) ]
//   w_t  += -c_s (p[j+1]-p[j-1])/(2dy) + alpha2 [ (w[j+1]-2w+w[j-1])/dy^2 + (same cross term of u) ]
//   p_t  += -c_s [ (u[i+1]-u[i-1])/(2dx) + (w[j+1]-w[j-1])/(2dy) ]
// with alpha = nu_f dx^2 / delta t (Eq. dampingCoeff).
// RK-3: q* = q + dt/3 L(q), q** = q + dt/2 L(q*), q' = q + dt L(q**).
//
// Each CTA owns a TX x TY output tile of one state and loads a halo of
// 3 cells per stage in x (9 in total) and RYH per stage in y (RYH = 1 when
// V = 0, else 3).  Stage 1 is computed on the tile shrunk by one stage
// radius, stage 2 by two, stage 3 on the tile itself, so each step reads the
// state from memory once and writes it once.
#include <type_traits>

#include "common.cuh"
#include "grid_barrier.cuh"

namespace pr {
namespace {

// Advective coefficients (U / 60 dx, V / 60 dy) of the cell at local row lr,
// column lc of a tile whose local origin is global (gy0, gx0): constant, or
// varying with the solid-body rotation at the cell's periodic position.
template <typename T>
__device__ __forceinline__ void adv_coef(const FineCoef<T>& c, int gy0, int gx0, int lr, int lc, int nx, int ny,
                                         T& ax, T& ay) {
    ax = c.ax6;
    ay = c.ay6;
    if (c.omx != T(0)) {
        ax += c.omx * ycen(c, pwrap(gy0 + lr, ny));
        ay -= c.omy * xcen(c, pwrap(gx0 + lc, nx));
    }
}

template <typename T, int RYH>
__device__ __forceinline__ void fine_tend(const T* __restrict__ u, const T* __restrict__ w,
                                          const T* __restrict__ p, int i, int RX,
                                          const FineCoef<T>& c, T ax, T ay, T& Lu, T& Lw, T& Lp) {
    const int S1 = RX;
    T du = (u[i + 3] - u[i - 3]) - T(9) * (u[i + 2] - u[i - 2]) + T(45) * (u[i + 1] - u[i - 1]);
    T dw = (w[i + 3] - w[i - 3]) - T(9) * (w[i + 2] - w[i - 2]) + T(45) * (w[i + 1] - w[i - 1]);
    T dp = (p[i + 3] - p[i - 3]) - T(9) * (p[i + 2] - p[i - 2]) + T(45) * (p[i + 1] - p[i - 1]);
    Lu = -ax * du;
    Lw = -ax * dw;
    Lp = -ax * dp;
    if (RYH == 3) {
        const int S2 = 2 * RX, S3 = 3 * RX;
        T eu = (u[i + S3] - u[i - S3]) - T(9) * (u[i + S2] - u[i - S2]) + T(45) * (u[i + S1] - u[i - S1]);
        T ew = (w[i + S3] - w[i - S3]) - T(9) * (w[i + S2] - w[i - S2]) + T(45) * (w[i + S1] - w[i - S1]);
        T ep = (p[i + S3] - p[i - S3]) - T(9) * (p[i + S2] - p[i - S2]) + T(45) * (p[i + S1] - p[i - S1]);
        Lu -= ay * eu;
        Lw -= ay * ew;
        Lp -= ay * ep;
    }
    Lu -= c.csx * (p[i + 1] - p[i - 1]);
    Lw -= c.csy * (p[i + S1] - p[i - S1]);
    Lp -= c.csx * (u[i + 1] - u[i - 1]) + c.csy * (w[i + S1] - w[i - S1]);
    Lu += c.dxx * (u[i + 1] - T(2) * u[i] + u[i - 1]) +
          c.dxy1 * ((w[i + 1 + S1] - w[i + 1 - S1]) - (w[i - 1 + S1] - w[i - 1 - S1]));
    Lw += c.dyy * (w[i + S1] - T(2) * w[i] + w[i - S1]) +
          c.dxy2 * ((u[i + 1 + S1] - u[i - 1 + S1]) - (u[i + 1 - S1] - u[i - 1 - S1]));
}

// One RK-3 step of the TX x TY output tile at (tx0, ty0) of one state:
// src -> dst (both already offset to the state), in arithmetic T, with the
// three stages in shared memory (smem_raw: 6 (TX + 18) (TY + 6 RYH) values of
// T).  ACC64: the state is FP64 in memory and the last stage adds dt L(q**)
// to the FP64 q^n (the tendencies and the intermediate stages stay in T).
// src is read with plain loads (the batched sweep passes states that other
// CTAs wrote earlier in the same launch).  Contains __syncthreads().
template <typename T, typename Tin, typename Tout, int RYH, int TX, int TY, int NT, bool ACC64>
__device__ __forceinline__ void fine_tile(const Tin* src, Tout* __restrict__ dst, int nx, int ny,
                                          const FineCoef<T>& c, int tx0, int ty0, unsigned char* smem_raw) {
    constexpr int HX = 9, HY = 3 * RYH;
    constexpr int RX = TX + 2 * HX, RY = TY + 2 * HY, NR = RX * RY;
    T* q = reinterpret_cast<T*>(smem_raw);
    T* s = q + 3 * NR;
    const long ncell = (long)nx * ny;

    // load the haloed region (periodic wrap)
    for (int idx = threadIdx.x; idx < NR; idx += NT) {
        int ly = idx / RX, lx = idx - ly * RX;
        long g = (long)pwrap(ty0 - HY + ly, ny) * nx + pwrap(tx0 - HX + lx, nx);
        q[idx] = (T)src[g];
        q[NR + idx] = (T)src[ncell + g];
        q[2 * NR + idx] = (T)src[2 * ncell + g];
    }
    __syncthreads();

    // stage 1: s = q + dt/3 L(q) on the region shrunk by (3, RYH)
    {
        constexpr int W1 = RX - 6, H1 = RY - 2 * RYH, N1 = W1 * H1;
        for (int t = threadIdx.x; t < N1; t += NT) {
            int r = t / W1;
            int i = (r + RYH) * RX + (t - r * W1) + 3;
            T Lu, Lw, Lp, ax, ay;
            adv_coef(c, ty0 - HY, tx0 - HX, r + RYH, t - r * W1 + 3, nx, ny, ax, ay);
            fine_tend<T, RYH>(q, q + NR, q + 2 * NR, i, RX, c, ax, ay, Lu, Lw, Lp);
            s[i] = q[i] + c.c1 * Lu;
            s[NR + i] = q[NR + i] + c.c1 * Lw;
            s[2 * NR + i] = q[2 * NR + i] + c.c1 * Lp;
        }
    }
    __syncthreads();

    // stage 2: s <- q + dt/2 L(s) on the region shrunk by (6, 2 RYH); staged in registers
    {
        constexpr int W2 = RX - 12, H2 = RY - 4 * RYH, N2 = W2 * H2, NPT = (N2 + NT - 1) / NT;
        T ru[NPT], rw[NPT], rp[NPT];
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            int t = threadIdx.x + k * NT;
            if (t < N2) {
                int r = t / W2;
                int i = (r + 2 * RYH) * RX + (t - r * W2) + 6;
                T Lu, Lw, Lp, ax, ay;
                adv_coef(c, ty0 - HY, tx0 - HX, r + 2 * RYH, t - r * W2 + 6, nx, ny, ax, ay);
                fine_tend<T, RYH>(s, s + NR, s + 2 * NR, i, RX, c, ax, ay, Lu, Lw, Lp);
                ru[k] = q[i] + c.c2 * Lu;
                rw[k] = q[NR + i] + c.c2 * Lw;
                rp[k] = q[2 * NR + i] + c.c2 * Lp;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            int t = threadIdx.x + k * NT;
            if (t < N2) {
                int r = t / W2;
                int i = (r + 2 * RYH) * RX + (t - r * W2) + 6;
                s[i] = ru[k];
                s[NR + i] = rw[k];
                s[2 * NR + i] = rp[k];
            }
        }
    }
    __syncthreads();

    // stage 3: q' = q + dt L(s) on the tile, written to global memory
    for (int t = threadIdx.x; t < TX * TY; t += NT) {
        int r = t / TX, cx = t - r * TX;
        int gx = tx0 + cx, gy = ty0 + r;
        if (gx < nx && gy < ny) {
            int i = (r + HY) * RX + cx + HX;
            T Lu, Lw, Lp, ax, ay;
            adv_coef(c, ty0 - HY, tx0 - HX, r + HY, cx + HX, nx, ny, ax, ay);
            fine_tend<T, RYH>(s, s + NR, s + 2 * NR, i, RX, c, ax, ay, Lu, Lw, Lp);
            long g = (long)gy * nx + gx;
            if (ACC64) {
                const double c3 = (double)c.c3;
                dst[g] = (Tout)((double)src[g] + c3 * (double)Lu);
                dst[ncell + g] = (Tout)((double)src[ncell + g] + c3 * (double)Lw);
                dst[2 * ncell + g] = (Tout)((double)src[2 * ncell + g] + c3 * (double)Lp);
            } else {
                dst[g] = (Tout)(q[i] + c.c3 * Lu);
                dst[ncell + g] = (Tout)(q[NR + i] + c.c3 * Lw);
                dst[2 * ncell + g] = (Tout)(q[2 * NR + i] + c.c3 * Lp);
            }
        }
    }
    __syncthreads();   // the shared buffers may be reused right after
}

template <typename T, typename Tin, typename Tout, int RYH, int TX, int TY, int NT, bool ACC64 = false>
__global__ void __launch_bounds__(NT) k_fine_step(const Tin* __restrict__ in, long instride,
                                                   Tout* __restrict__ out, long outstride, int nx,
                                                   int ny, FineCoef<T> c, SliceMap map) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    long zi = blockIdx.z, zo = blockIdx.z;
    if (map.end) {
        const int b0 = *map.beg;
        if ((int)blockIdx.z >= *map.end - b0) return;
        if (map.in_map) zi += b0;
        if (map.out_map) zo += b0;
    }
    fine_tile<T, Tin, Tout, RYH, TX, TY, NT, ACC64>(in + zi * instride, out + zo * outstride, nx, ny, c,
                                                    blockIdx.x * TX, blockIdx.y * TY, smem_raw);
}

template <typename T, typename Tin, typename Tout, int RYH, int TX, int TY, int NT, bool ACC64 = false>
cudaError_t launch_tile(const Tin* in, long instride, Tout* out, long outstride, int n, int nx, int ny,
                        const FineCoef<T>& c, cudaStream_t s, const SliceMap& map) {
    constexpr int RX = TX + 18, RY = TY + 6 * RYH;
    constexpr size_t smem = sizeof(T) * 6 * RX * RY;
    auto kern = k_fine_step<T, Tin, Tout, RYH, TX, TY, NT, ACC64>;
    std::lock_guard<std::mutex> lk(smem_launch_lock());
    cudaError_t e = set_dynamic_smem((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((nx + TX - 1) / TX, (ny + TY - 1) / TY, n);
    kern<<<grid, NT, smem, s>>>(in, instride, out, outstride, nx, ny, c, map);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T, typename Tin, typename Tout, bool ACC64>
cudaError_t launch_tiles(const Tin* in, long instride, Tout* out, long outstride, int n, int nx, int ny, bool has_v,
                         const FineCoef<T>& c, cudaStream_t s, const SliceMap& map, const FineLaunch& fl) {
    const bool big = nx >= 64 && ny >= 16;
    if (has_v) {
        if (big)
            return launch_tile<T, Tin, Tout, 3, 64, 16, 256, ACC64>(in, instride, out, outstride, n, nx, ny, c, s, map);
        return launch_tile<T, Tin, Tout, 3, 32, 8, 256, ACC64>(in, instride, out, outstride, n, nx, ny, c, s, map);
    }
    if constexpr (std::is_same<T, float>::value) {
        const int t = (fl.tile < 0 || fl.tile >= kFineTiles) ? (big ? 2 : 0) : fl.tile;
        switch (t) {
            case 0: return launch_tile<T, Tin, Tout, 1, 32, 8, 256, ACC64>(in, instride, out, outstride, n, nx, ny, c, s, map);
            case 1: return launch_tile<T, Tin, Tout, 1, 64, 8, 256, ACC64>(in, instride, out, outstride, n, nx, ny, c, s, map);
            case 3: return launch_tile<T, Tin, Tout, 1, 128, 8, 256, ACC64>(in, instride, out, outstride, n, nx, ny, c, s, map);
            default: return launch_tile<T, Tin, Tout, 1, 64, 16, 256, ACC64>(in, instride, out, outstride, n, nx, ny, c, s, map);
        }
    } else {   // FP64 tile steps (slice-mapped sweeps) keep the fixed shapes
        if (big) return launch_tile<T, Tin, Tout, 1, 64, 16, 256, ACC64>(in, instride, out, outstride, n, nx, ny, c, s, map);
        return launch_tile<T, Tin, Tout, 1, 32, 8, 256, ACC64>(in, instride, out, outstride, n, nx, ny, c, s, map);
    }
}

// ------------------------------------------------------------ batched sweep

constexpr int FB_TX = 32, FB_TY = 8, FB_NT = 256;
constexpr size_t FB_SMEM = sizeof(float) * 6 * (FB_TX + 18) * (FB_TY + 6);

// The fine sweeps of many handles (uneven grids, slice counts and step
// counts) in one cooperative launch: per step t, every CTA takes work
// indices (item, state, tile) in a grid-stride loop, items whose nf <= t
// are done; a bounded grid barrier separates the steps.  Each tile runs the
// same per-cell arithmetic as the per-handle tile kernel (fine_tile), so the
// results are those of the handles' own sweeps bit for bit.
__global__ void __launch_bounds__(FB_NT) k_fine_batch(const FineBatchItem* __restrict__ items, int nitems,
                                                      long total, int max_nf, GridBar* gb) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const unsigned nb = gridDim.x;
    for (int t = 0; t < max_nf; ++t) {
        for (long w = blockIdx.x; w < total; w += nb) {
            int lo = 0, hi = nitems - 1;   // last item with tile0 <= w
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (items[mid].tile0 <= w) lo = mid; else hi = mid - 1;
            }
            const FineBatchItem& it = items[lo];
            if (t >= it.nf) continue;
            const long lw = w - it.tile0;
            const int z = (int)(lw / it.tiles), tt = (int)(lw - (long)z * it.tiles);
            const int ty = tt / it.tiles_x, tx = tt - ty * it.tiles_x;
            const SliceMap& map = t == 0 ? it.first : it.rest;
            long zi = z, zo = z;
            if (map.end) {
                const int b0 = *map.beg;
                if (z >= *map.end - b0) continue;
                if (map.in_map) zi += b0;
                if (map.out_map) zo += b0;
            }
            const double* a = t == 0 ? it.in : ((t - 1) % 2 == 0 ? it.w0 : it.w1);
            double* b = t == it.nf - 1 ? it.out : (t % 2 == 0 ? it.w0 : it.w1);
            fine_tile<float, double, double, 1, FB_TX, FB_TY, FB_NT, true>(a + zi * it.d, b + zo * it.d, it.nx, it.ny,
                                                                          it.c, tx * FB_TX, ty * FB_TY, smem_raw);
        }
        if (t + 1 < max_nf && !grid_barrier(gb, nb)) return;
    }
}

}  // namespace

// Candidate tile shapes of the autotuner (V = 0): TX x TY output cells per
// CTA of 256 threads.
const int fine_tile_shapes[kFineTiles][2] = {{32, 8}, {64, 8}, {64, 16}, {128, 8}};

template <typename T, typename Tin, typename Tout>
cudaError_t launch_fine_step(const Tin* in, long instride, Tout* out, long outstride, int n, int nx,
                             int ny, bool has_v, const FineCoef<T>& c, cudaStream_t s, const SliceMap& map,
                             const FineLaunch& fl) {
    if constexpr (std::is_same<T, float>::value) {
        cudaError_t e = cudaSuccess;
        if (fl.rows &&
            launch_fine_rows<Tin, Tout>(in, instride, out, outstride, n, nx, ny, has_v, c, s, map, &e, fl.min_rows))
            return e;
    }
    return launch_tiles<T, Tin, Tout, false>(in, instride, out, outstride, n, nx, ny, has_v, c, s, map, fl);
}

namespace {
__global__ void k_to_fp32_states(const double* __restrict__ in, long instride, float* __restrict__ out,
                                 long outstride, int n, long d, SliceMap map) {
    long zb = 0;
    int nact = n;
    if (map.end) {
        nact = min(n, *map.end - *map.beg);
        if (map.in_map) zb = *map.beg;
    }
    const long tot = (long)nact * d;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long)gridDim.x * blockDim.x) {
        const long z = i / d, k = i - z * d;
        out[z * outstride + k] = (float)in[(zb + z) * instride + k];
    }
}
}  // namespace

cudaError_t launch_to_fp32_states(const double* in, long instride, float* out, long outstride, int n, long d,
                                  const SliceMap& map, cudaStream_t s) {
    if (n < 1 || d < 1) return cudaSuccess;
    long blocks = ((long)n * d + 255) / 256;
    if (blocks > 152L * 16) blocks = 152L * 16;
    k_to_fp32_states<<<(unsigned)blocks, 256, 0, s>>>(in, instride, out, outstride, n, d, map);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fine_step_acc64(const double* in, double* out, long stride, int n, int nx, int ny, bool has_v,
                                  const FineCoef<float>& c, cudaStream_t s, const SliceMap& map,
                                  const FineLaunch& fl) {
    return launch_tiles<float, double, double, true>(in, stride, out, stride, n, nx, ny, has_v, c, s, map, fl);
}

template cudaError_t launch_fine_step<double, double, double>(const double*, long, double*, long, int,
                                                              int, int, bool, const FineCoef<double>&,
                                                              cudaStream_t, const SliceMap&, const FineLaunch&);
template cudaError_t launch_fine_step<float, double, float>(const double*, long, float*, long, int, int,
                                                            int, bool, const FineCoef<float>&,
                                                            cudaStream_t, const SliceMap&, const FineLaunch&);
template cudaError_t launch_fine_step<float, float, float>(const float*, long, float*, long, int, int,
                                                           int, bool, const FineCoef<float>&,
                                                           cudaStream_t, const SliceMap&, const FineLaunch&);
template cudaError_t launch_fine_step<float, float, double>(const float*, long, double*, long, int, int,
                                                            int, bool, const FineCoef<float>&,
                                                            cudaStream_t, const SliceMap&, const FineLaunch&);
template cudaError_t launch_fine_step<float, double, double>(const double*, long, double*, long, int,
                                                             int, int, bool, const FineCoef<float>&,
                                                             cudaStream_t, const SliceMap&, const FineLaunch&);

void fine_batch_tiles(int nx, int ny, int* tiles_x, int* tiles) {
    *tiles_x = (nx + FB_TX - 1) / FB_TX;
    *tiles = *tiles_x * ((ny + FB_TY - 1) / FB_TY);
}

cudaError_t fine_batch_coop(const FineBatchItem* items_dev, int nitems, long total, int max_nf, GridBar* gb,
                            cudaStream_t s, int max_sms) {
    if (nitems < 1 || total < 1 || max_nf < 1) return cudaSuccess;
    static DevMemo memo;   // [device] -> (SMs, CTAs per SM)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int sms = 0, per = 0;
    if (!memo.get(dev, &sms, &per)) {
        std::lock_guard<std::mutex> lk(smem_launch_lock());
        e = set_dynamic_smem((const void*)k_fine_batch, FB_SMEM);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fine_batch, FB_NT, FB_SMEM);
        if (e != cudaSuccess) return e;
        memo.put(dev, sms, per);
    }
    if (per < 1) return cudaErrorInvalidConfiguration;
    if (max_sms > 0 && max_sms < sms) sms = max_sms;
    long nb = (long)sms * per;
    if (nb > total) nb = total;
    e = cudaMemsetAsync(&gb->count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&items_dev, &nitems, &total, &max_nf, &gb};
    std::lock_guard<std::mutex> lk(smem_launch_lock());
    e = set_dynamic_smem((const void*)k_fine_batch, FB_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaLaunchCooperativeKernel((const void*)k_fine_batch, dim3((unsigned)nb), dim3(FB_NT), args, FB_SMEM, s);
    count_launches(1);
    return e;
}

}  // namespace pr
