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
// Every CTA owns a fixed range of rows for the dot products and the update
// and a set of 16 x 16 tiles for the coarse steps.  Per slice: phase A
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

cudaError_t chain_coop(const ChainArgs& a, cudaStream_t s) {
    if (a.i_end <= a.i_begin) return cudaSuccess;
    if (a.dlt && a.dlt64) return cudaErrorInvalidValue;
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
