// split_gemm.cu -- FP64-accurate tall-skinny products C = Q^T V and
// V <- V - Q C on the BF16 tensor cores (tcgen05, TMEM accumulators, TMA
// operand tiles), for the Gram-Schmidt passes of the subspace update
// (Eq. subspaceUpdate) and the projection c = Q^T q of Eq. modifiedCoarse.
// The digit representation and the exactness argument are in split_gemm.h.
//
// One kernel, k_split_mma, serves both products.  A CTA owns a tile of 128
// rows of the long operand (basis columns for Q^T V, state rows for V - Q C)
// against all SG_N = 16 columns of the narrow operand, over a range of the
// contraction.  Warp 0 streams the 8 digit slices of both operands through a
// 3-stage TMA pipeline (operand tiles stored pre-swizzled; one 4-D tensor
// load per operand and stage brings all 8 slices -- with one 2-D load per
// slice and tile piece the issue of up to 32 loads per stage, not the
// memory, set the pace), warp 1 issues 8
// MMAs per 16 contraction elements -- one per digit slice of the long operand
// against the stacked slices of the narrow one, 43 digit products in all --
// into 9 FP32 accumulators (double-buffered across 256-element chunks), and warps
// 4-7 drain each chunk from TMEM and combine it in FP64.  Every wait is
// bounded; on expiry the sticky error word is set and the CTA winds down.
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cudaTypedefs.h>

#include "common.cuh"
#include "split_gemm.h"
#include "tc.cuh"

namespace pr {
namespace {

constexpr int SG_NST = 3;                          // pipeline stages
constexpr int SG_NG = SG_S + 1;                    // accumulator groups: s + t = 2 .. S + 2
constexpr int SG_A_TILE = SG_BM * SG_KC * 2;       // bytes per slice tile of the long operand
constexpr int SG_B_TILE = SG_N * SG_KC * 2;        // bytes per slice tile of the narrow operand
// a stage: S tiles of the long operand, S tiles of the narrow operand and one
// tile of zeros after them (written once), so that the narrow operand's
// slices t = 0..S read as one operand of (S + 1) * SG_N rows
constexpr int SG_STAGE = SG_S * SG_A_TILE + (SG_S + 1) * SG_B_TILE;
constexpr int SG_SPC = SG_L / SG_KC;               // stages per exact chunk
constexpr int SG_TMEM_COLS = 512;                  // two accumulator sets (2 x 9 x 16 columns)
constexpr int SG_DSMEM = SG_NST * SG_STAGE + 1024; // + alignment slack for the 64-byte swizzle
// MMA s (the long operand's digit slice s) multiplies the narrow operand's
// slices t = 0 .. S - s stacked along N, so its output columns are the
// accumulator groups g = s + t = s .. S: one MMA per slice instead of one per
// digit pair.  Slice 0 also takes the zero tile (t = S) so that its first MMA
// of a chunk initialises all S + 1 groups.
__host__ __device__ constexpr uint32_t sg_idesc(int s) {
    return tc::idesc_bf16_f32(SG_BM, (s == 0 ? SG_S + 1 : SG_S + 1 - s) * SG_N);
}
constexpr int SG_THREADS = 256;

struct SgArgs {
    int mode;               // 0: partial sums of Q^T V;  1: V <- V - Q C
    const int* rows_dev;    // mode 0: valid rows (basis columns r)
    int rows_host;          // bound on the rows of the long operand (mode 0: cap, mode 1: d)
    const int* k_dev;       // mode 1: contraction length (basis columns); NULL: k_host
    long k_host;            // mode 0: contraction length (d)
    double* ws;             // mode 0: partial sums [split][SG_N][rows_pad]
    int rows_pad;
    double* v;              // mode 1: columns updated in place
    long ldv;
    const int* vexp;        // mode 1: exponents of the narrow operand's columns
    int ncols;              // mode 1: columns to update
    int* err;
};

constexpr int SG_EXP_NAN = 0x7FFF;   // column exponent of a column holding a NaN or an infinity

// Work decomposition of Q^T V for r valid basis columns on `grid` CTAs:
// `tiles` row tiles times `nsplit` contraction ranges of kps elements (a
// multiple of SG_KC), every range non-empty.  Computed on the device from
// the device-side r by the product and by its reduction alike.
__device__ __forceinline__ void tn_layout(int r, long d, int grid, int* tiles, int* nsplit, long* kps) {
    const int t = max(1, (r + SG_BM - 1) / SG_BM);
    const int ns = max(1, grid / t);
    long k = (d + ns - 1) / ns;
    k = (k + SG_KC - 1) / SG_KC * SG_KC;
    *kps = k;
    *nsplit = (int)((d + k - 1) / k);
    *tiles = t;
}

__device__ __forceinline__ void sg_fail(int* err, volatile int* abort_flag) {
    atomicExch(err, 1);
    *abort_flag = 1;
}

// Persistent: CTA b handles work items b, b + gridDim.x, ...  (mode 0: one
// (row tile, contraction range) pair per CTA; mode 1: row tiles of V).  The
// pipeline counters run on across items, so loads of the next item overlap
// the epilogue of the current one.
__global__ void __launch_bounds__(SG_THREADS, 1)
    k_split_mma(const __grid_constant__ CUtensorMap mapA2, const __grid_constant__ CUtensorMap mapA4,
                const __grid_constant__ CUtensorMap mapA6, const __grid_constant__ CUtensorMap mapA8,
                const __grid_constant__ CUtensorMap mapA10, const __grid_constant__ CUtensorMap mapA12,
                const __grid_constant__ CUtensorMap mapA14, const __grid_constant__ CUtensorMap mapA16,
                const __grid_constant__ CUtensorMap mapB, const SgArgs a) {
    extern __shared__ unsigned char sg_raw[];
    __shared__ __align__(8) uint64_t bars[2 * SG_NST + 5];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;
    __shared__ double s_scale[SG_N];   // mode 1: 2^{G_n - 14}

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int n_items, tiles = 1, nsplit = 1, rows;
    long kps = 0, klen = 0;
    if (a.mode == 0) {
        rows = min(*a.rows_dev, a.rows_host);
        if (rows <= 0) return;
        tn_layout(rows, a.k_host, (int)gridDim.x, &tiles, &nsplit, &kps);
        n_items = tiles * nsplit;
    } else {
        klen = a.k_dev ? (long)*a.k_dev : a.k_host;
        if (klen <= 0) return;
        rows = a.rows_host;
        n_items = (rows + SG_BM - 1) / SG_BM;
    }
    if ((int)blockIdx.x >= n_items) return;
    auto item = [&](int i, int& row0, long& kb, long& ke, int& split) {
        if (a.mode == 0) {
            split = i / tiles;
            row0 = (i - split * tiles) * SG_BM;
            kb = (long)split * kps;
            ke = min(a.k_host, kb + kps);
        } else {
            split = 0;
            row0 = i * SG_BM;
            kb = 0;
            ke = klen;
        }
    };

    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(sg_raw) + 1023) &
                                                           ~static_cast<uintptr_t>(1023));
    const uint32_t sbase = tc::smem_u32(base);
    const uint32_t bar0 = tc::smem_u32(bars);
    auto full = [&](int st) { return bar0 + 8u * st; };
    auto empty = [&](int st) { return bar0 + 8u * (SG_NST + st); };
    auto tfull = [&](int b) { return bar0 + 8u * (2 * SG_NST + b); };
    auto tempty = [&](int b) { return bar0 + 8u * (2 * SG_NST + 2 + b); };
    const uint32_t done = bar0 + 8u * (2 * SG_NST + 4);

    if (threadIdx.x == 0) {
        for (int i = 0; i < SG_NST; ++i) {
            tc::mbar_init(full(i), 1);
            tc::mbar_init(empty(i), 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(tfull(b), 1);
            tc::mbar_init(tempty(b), 128);
        }
        tc::mbar_init(done, 1);
        tc::fence_barrier_init();
        s_abort = 0;
    }
    // the zero tile of every stage (never overwritten by the loads)
    for (int st = 0; st < SG_NST; ++st) {
        uint4* z = reinterpret_cast<uint4*>(base + st * SG_STAGE + SG_S * SG_A_TILE + SG_S * SG_B_TILE);
        for (int i = threadIdx.x; i < SG_B_TILE / 16; i += SG_THREADS) z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor cores
    if (threadIdx.x < SG_N)
        s_scale[threadIdx.x] = (a.mode == 1 && a.vexp) ? ldexp(1.0, a.vexp[threadIdx.x] - 14) : 0.0;
    if (warp == 2) {
        tc::tmem_alloc(tc::smem_u32(&tmem_slot), SG_TMEM_COLS);
        tc::tmem_relinquish();
    }
    if (warp == 0 && lane == 0) {
        tc::tma_prefetch_map(&mapA16);
        tc::tma_prefetch_map(&mapB);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    volatile int* abort_flag = &s_abort;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------------------------------------------- TMA producer
            int issued[SG_NST] = {0, 0, 0};
            int it = 0;
            bool ok = true;
            for (int i = blockIdx.x; i < n_items && ok; i += gridDim.x) {
                int row0, split;
                long kb, ke;
                item(i, row0, kb, ke, split);
                const int ns = (int)((ke - kb + SG_KC - 1) / SG_KC);
                // row groups of 8 to load: the tile's valid rows, rounded up to 16
                const int ng = ((min(SG_BM, rows - row0) + 15) / 16) * 2;
                const uint32_t bytes = (uint32_t)SG_S * (uint32_t)(ng * 512 + SG_B_TILE);
                for (int j = 0; j < ns; ++j, ++it) {
                    const int st = it % SG_NST;
                    const uint32_t ph = (uint32_t)(it / SG_NST) & 1u;
                    if (*abort_flag || !tc::mbar_wait(empty(st), ph ^ 1u)) {
                        sg_fail(a.err, abort_flag);
                        ok = false;
                        break;
                    }
                    tc::mbar_expect_tx(full(st), bytes);
                    const int kblk = (int)(kb / SG_KC + j);
                    const uint32_t sa = sbase + st * SG_STAGE;
                    const uint32_t sb = sa + SG_S * SG_A_TILE;
                    // all 8 digit slices of the long operand's ng row groups
                    // (slice s at s * ng units) and of the narrow operand's 2
                    const CUtensorMap* mA = ng == 16 ? &mapA16 : ng == 14 ? &mapA14 : ng == 12 ? &mapA12
                                          : ng == 10 ? &mapA10 : ng == 8 ? &mapA8 : ng == 6 ? &mapA6
                                          : ng == 4 ? &mapA4 : &mapA2;
                    tc::tma_load_4d(sa, mA, 0, row0 / 8, kblk, 0, full(st));
                    tc::tma_load_4d(sb, &mapB, 0, 0, kblk, 0, full(st));
                    issued[st] += 1;
                }
            }
            // every load issued has landed before the CTA may exit
            for (int st = 0; st < SG_NST; ++st)
                if (issued[st] > 0 && !tc::mbar_wait(full(st), (uint32_t)(issued[st] - 1) & 1u))
                    sg_fail(a.err, abort_flag);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------------------------------------------- MMA issuer
            int it = 0, cg = 0;
            bool ok = true;
            for (int i = blockIdx.x; i < n_items && ok; i += gridDim.x) {
                int row0, split;
                long kb, ke;
                item(i, row0, kb, ke, split);
                const int ns = (int)((ke - kb + SG_KC - 1) / SG_KC);
                const int nch = (ns + SG_SPC - 1) / SG_SPC;
                // slice s of the long operand's tile starts s * ng units into the stage
                const uint32_t sl_bytes = (uint32_t)(((min(SG_BM, rows - row0) + 15) / 16) * 2) * 512u;
                for (int c = 0; c < nch && ok; ++c, ++cg) {
                    const int buf = cg & 1;
                    const uint32_t use = (uint32_t)(cg >> 1);
                    if (*abort_flag || !tc::mbar_wait(tempty(buf), (use & 1u) ^ 1u)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t dbase = tmem + (uint32_t)(buf * SG_NG * SG_N);
                    uint32_t init = 0;
                    const int j_end = min(ns, (c + 1) * SG_SPC);
                    for (int j = c * SG_SPC; j < j_end; ++j, ++it) {
                        const int st = it % SG_NST;
                        const uint32_t ph = (uint32_t)(it / SG_NST) & 1u;
                        if (*abort_flag || !tc::mbar_wait(full(st), ph)) {
                            ok = false;
                            break;
                        }
                        tc::fence_after_sync();
                        const uint32_t sa = sbase + st * SG_STAGE;
                        const uint32_t sb = sa + SG_S * SG_A_TILE;
#pragma unroll
                        for (int kk = 0; kk < SG_KC / 16; ++kk) {
                            const uint64_t bd = tc::desc_kmajor_sw64(sb + kk * 32);
#pragma unroll
                            for (int s = 0; s < SG_S; ++s) {
                                const uint64_t ad = tc::desc_kmajor_sw64(sa + s * sl_bytes + kk * 32);
                                // slice 0 (groups 0..S) overwrites at the chunk's first step; the
                                // others then accumulate into groups s..S
                                tc::mma_bf16(dbase + (uint32_t)(s * SG_N), ad, bd, sg_idesc(s), init | (s > 0));
                            }
                            init = 1u;
                        }
                        tc::mma_commit(empty(st));
                    }
                    if (!ok) break;
                    tc::mma_commit(tfull(buf));
                }
            }
            if (!ok) sg_fail(a.err, abort_flag);
            // all MMAs complete before the accumulators are released
            tc::mma_commit(done);
            if (!tc::mbar_wait(done, 0)) sg_fail(a.err, abort_flag);
        }
    } else if (warp >= 4) {
        // -------------------------------------------------------- epilogue
        // Each chunk's group sums are exact integers below 2^23: they are
        // converted to integers and accumulated exactly in two 64-bit words,
        // hi = sum_{g<=3} a_g 2^{7(3-g)} and lo = sum_{g>=4} a_g 2^{7(8-g)},
        // so the value sum_g a_g 2^{-7g} = 2^-21 hi + 2^-56 lo is rounded to
        // FP64 once per output, at the end of the item.
        const int q = warp & 3;
        const uint32_t lane_addr = static_cast<uint32_t>(q * 32) << 16;
        int cg = 0;
        bool ok = true;
        for (int i = blockIdx.x; i < n_items && ok; i += gridDim.x) {
            int row0, split;
            long kb, ke;
            item(i, row0, kb, ke, split);
            const int ns = (int)((ke - kb + SG_KC - 1) / SG_KC);
            const int nch = (ns + SG_SPC - 1) / SG_SPC;
            long long hi[SG_N], lo[SG_N];
            uint32_t nanmask = 0;
#pragma unroll
            for (int n = 0; n < SG_N; ++n) hi[n] = lo[n] = 0;
            // mode 1: the row's values of v, loaded together before the wait
            // (one memory round trip instead of one per column)
            const int vrow = row0 + q * 32 + lane;
            double vold[SG_N];
#pragma unroll
            for (int n = 0; n < SG_N; ++n)
                vold[n] = (a.mode == 1 && vrow < rows && n < a.ncols) ? a.v[vrow + (long)n * a.ldv] : 0.0;
            for (int c = 0; c < nch; ++c, ++cg) {
                const int buf = cg & 1;
                const uint32_t use = (uint32_t)(cg >> 1);
                const bool w = !*abort_flag && tc::mbar_wait(tfull(buf), use & 1u);
                if (!__all_sync(0xffffffffu, w)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
#pragma unroll
                for (int g = 0; g < SG_NG; ++g) {
                    float v[16];
                    tc::tmem_ld16(tmem + lane_addr + (uint32_t)(buf * SG_NG * SG_N + g * SG_N), v);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int n = 0; n < SG_N; ++n) {
                        if (v[n] != v[n]) nanmask |= 1u << n;
                        const long long x = (long long)__float2int_rn(v[n]);
                        if (g <= 3)
                            hi[n] += x * (1ll << (7 * (3 - g)));
                        else
                            lo[n] += x * (1ll << (7 * (8 - g)));
                    }
                }
                tc::fence_before_sync();
                tc::mbar_arrive(tempty(buf));
            }
            if (!ok) break;
            // (double)hi is exact (|hi| < 2^50 for up to 64 chunks); lo may
            // round, below 2^-53 of its own size; the power-of-two scalings
            // are exact, and the combination rounds once.
            const int row = row0 + q * 32 + lane;
            if (a.mode == 0) {
                if (row < rows) {
#pragma unroll
                    for (int n = 0; n < SG_N; ++n) {
                        const double t = (nanmask >> n) & 1u ? __longlong_as_double(0x7FF8000000000000ll)
                                                               : fma((double)hi[n], 0x1p-21, (double)lo[n] * 0x1p-56);
                        a.ws[((long)split * SG_N + n) * a.rows_pad + row] = t;
                    }
                }
            } else if (row < rows) {
#pragma unroll
                for (int n = 0; n < SG_N; ++n) {
                    if (n < a.ncols) {
                        const double t = (nanmask >> n) & 1u ? __longlong_as_double(0x7FF8000000000000ll)
                                                               : fma((double)hi[n], 0x1p-21, (double)lo[n] * 0x1p-56);
                        a.v[row + (long)n * a.ldv] = fma(-t, s_scale[n], vold[n]);
                    }
                }
            }
        }
        if (!ok && lane == 0) sg_fail(a.err, abort_flag);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 2) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, SG_TMEM_COLS);
    }
}

// ------------------------------------------------------------ digit kernels

// |x| as an ordered integer key (bit pattern without the sign).
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7FFFFFFFFFFFFFFFull;
}

// Column exponent E from the largest |x| key: max |x| < 2^{E-1}; 0 for a
// zero column, SG_EXP_NAN if the column holds a NaN or an infinity.
__device__ __forceinline__ int exponent_of_max(unsigned long long mb) {
    if (mb == 0) return 0;
    if ((mb >> 52) == 0x7FF) return SG_EXP_NAN;
    int e = 0;
    frexp(__longlong_as_double(static_cast<long long>(mb)), &e);   // max < 2^e
    return e + 1;
}

// The 8 digits of x in the column scale 2^E, computed exactly in integer
// arithmetic: T = round(x 2^{56-E}) (|T| <= 2^55), then balanced base-128
// digits from the least significant one, d = ((T + 64) mod 128) - 64 in
// [-64, 63], T <- (T - d) / 128; the leading digit is what remains, in
// [-64, 64].  x = 2^E sum_s d_s 2^{-7s} up to 2^{E-57}.
__device__ __forceinline__ void digits8(double x, int E, __nv_bfloat16 (&dg)[SG_S]) {
    if (E == SG_EXP_NAN) {
#pragma unroll
        for (int s = 0; s < SG_S; ++s) dg[s] = __ushort_as_bfloat16((unsigned short)0x7FC0);
        return;
    }
    const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
    const int ex = (int)((bits >> 52) & 0x7FF);
    unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
    if (ex != 0) m |= 1ull << 52;
    const int sh = (ex != 0 ? ex : 1) - 1075 + 56 - E;   // x = m 2^{ex - 1075}
    long long T;
    if (sh >= 0)
        T = static_cast<long long>(m << sh);              // sh <= 2 for |x| < 2^{E-1}
    else if (sh > -63)
        T = static_cast<long long>((m + (1ull << (-sh - 1))) >> (-sh));
    else
        T = 0;
    if (bits >> 63) T = -T;
#pragma unroll
    for (int s = SG_S - 1; s > 0; --s) {
        const long long d = ((T + 64) & 127) - 64;
        dg[s] = __float2bfloat16_rn((float)d);
        T = (T - d) >> 7;
    }
    dg[0] = __float2bfloat16_rn((float)T);
}

// Element offset of (row r8 in [0, 8), contraction index k in [0, 32)) inside
// a 512-byte operand unit: 64-byte rows, 16-byte chunks XOR-swizzled with
// bits 1-2 of the row (the 64-byte swizzle the tensor cores' descriptors name).
__device__ __forceinline__ int unit_elem(int r8, int k) {
    return r8 * 32 + ((((k >> 3) ^ (r8 >> 1)) & 3) << 3) + (k & 7);
}

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long m, unsigned long long* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
    }
    if (lane == 0) red[wid] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t = red[k] > t ? red[k] : t;
        red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// keys[c] = max over a share of the rows of the |x| key of column
// c = c0 + blockIdx.y (c < *c1_dev when given); keys zeroed beforehand.
// Many CTAs per column, so the column maxima stream at full bandwidth.
__global__ void k_col_max(const double* __restrict__ X, long ldx, long nrows, const int* c0_dev, const int* c1_dev,
                          int c0_host, unsigned long long* keys) {
    __shared__ unsigned long long red[33];
    const int c = (c0_dev ? *c0_dev : c0_host) + (int)blockIdx.y;
    if (c1_dev && c >= *c1_dev) return;
    const double* x = X + (long)c * ldx;
    unsigned long long m = 0;
    for (long row = (long)blockIdx.x * blockDim.x + threadIdx.x; row < nrows; row += (long)gridDim.x * blockDim.x) {
        const unsigned long long b = abs_bits(x[row]);
        m = b > m ? b : m;
    }
    m = block_max_u64(m, red);
    if (threadIdx.x == 0 && m > 0) atomicMax(keys + c, m);
}

// Digits of basis columns [c0, c1) (at most SG_N) of Q into both operand
// layouts: Xc (rows = basis columns, contraction = state rows) and Xr (rows =
// state rows, contraction = basis columns); exps[c] from the column maxima
// keys.  A CTA takes 128 state rows: one row per thread forms the digits and
// stores Xc (consecutive threads on consecutive elements of a 64-byte row);
// the digits are staged in shared memory and the Xr stores are issued with
// consecutive threads on consecutive basis columns of a state row.
constexpr int DB_ROWS = 128;
__global__ void __launch_bounds__(DB_ROWS) k_digits_basis(const double* __restrict__ Q, long ldq, long d,
                                                          const int* c0_dev, const int* c1_dev, int c0_host,
                                                          int maxcols, const unsigned long long* __restrict__ keys,
                                                          int* exps, __nv_bfloat16* Xc, __nv_bfloat16* Xr, long nkb,
                                                          int ngl, int nlb, long ngd) {
    __shared__ __nv_bfloat16 tile[SG_S][DB_ROWS][SG_N];
    __shared__ int se[SG_N];
    const int c0 = c0_dev ? *c0_dev : c0_host;
    const int c1 = c1_dev ? min(*c1_dev, c0 + maxcols) : c0 + maxcols;
    const int nc = min(c1 - c0, SG_N);
    if (nc <= 0) return;
    if (threadIdx.x < nc) {
        se[threadIdx.x] = exponent_of_max(keys[c0 + threadIdx.x]);
        if (blockIdx.x == 0) exps[c0 + threadIdx.x] = se[threadIdx.x];
    }
    __syncthreads();
    for (long r0 = (long)blockIdx.x * DB_ROWS; r0 < d; r0 += (long)gridDim.x * DB_ROWS) {
        const long row = r0 + threadIdx.x;
        if (row < d) {
            const long kb = row >> 5;
            const int k = (int)(row & 31);
            for (int j = 0; j < nc; ++j) {
                const int cc = c0 + j;
                __nv_bfloat16 dg[SG_S];
                digits8(Q[row + (long)cc * ldq], se[j], dg);
                const long uc = kb * ngl + (cc >> 3);
                const int ec = unit_elem(cc & 7, k);
#pragma unroll
                for (int s = 0; s < SG_S; ++s) {
                    if (Xc) Xc[((long)s * nkb * ngl + uc) * 256 + ec] = dg[s];
                    tile[s][threadIdx.x][j] = dg[s];
                }
            }
        }
        __syncthreads();
        for (int s = 0; s < SG_S; ++s) {
            for (int idx = threadIdx.x; idx < DB_ROWS * SG_N; idx += DB_ROWS) {
                const int rl = idx / SG_N, j = idx % SG_N;
                const long rw = r0 + rl;
                if (j < nc && rw < d) {
                    const int cc = c0 + j;
                    const long ur = (long)(cc >> 5) * ngd + (rw >> 3);
                    Xr[((long)s * nlb * ngd + ur) * 256 + unit_elem((int)(rw & 7), cc & 31)] = tile[s][rl][j];
                }
            }
        }
        __syncthreads();
    }
}

// Digits of the block V (m columns, ld ldv) into the Vs operand layout
// (SG_N rows = the columns, contraction = state rows); columns j in
// [m, SG_N) are zero.
__global__ void k_digits_block(const double* __restrict__ V, long ldv, long d, int m,
                               const unsigned long long* __restrict__ keys, int* exps, __nv_bfloat16* Vs,
                               long nkb) {
    __shared__ int se[SG_N];
    if (threadIdx.x < SG_N) {
        se[threadIdx.x] = threadIdx.x < m ? exponent_of_max(keys[threadIdx.x]) : 0;
        if (blockIdx.x == 0) exps[threadIdx.x] = se[threadIdx.x];
    }
    __syncthreads();
    for (long row = (long)blockIdx.x * blockDim.x + threadIdx.x; row < d; row += (long)gridDim.x * blockDim.x) {
        for (int j = 0; j < SG_N; ++j) {
            __nv_bfloat16 dg[SG_S];
            if (j < m) {
                digits8(V[row + (long)j * ldv], se[j], dg);
            } else {
#pragma unroll
                for (int s = 0; s < SG_S; ++s) dg[s] = __float2bfloat16_rn(0.f);
            }
            const long u = (row >> 5) * 2 + (j >> 3);
            const int e = unit_elem(j & 7, (int)(row & 31));
#pragma unroll
            for (int s = 0; s < SG_S; ++s) Vs[((long)s * nkb * 2 + u) * 256 + e] = dg[s];
        }
    }
}

// Column j = blockIdx.x of the coefficient block: either C[l, j] =
// 2^{E_l + F_j - 14} sum_splits ws (stored to C; the splits of the product
// launched on tn_grid CTAs, summed in a fixed order), or C given (Cin).  Then
// the folded column C'[l] = 2^{E_l} C[l, j] (l < r; zero up to kpad), its
// exponent G_j and its digits in the Cs operand layout (SG_N rows, contraction
// = basis columns; kpad a multiple of 32).  Columns j >= m are zero.
constexpr int FIN_T = 1024;   // threads of k_finish: 4 groups of 256 rows
__global__ void __launch_bounds__(FIN_T) k_finish(const double* __restrict__ ws, int rows_pad, int tn_grid, long d,
                                                  const int* r_dev, const int* __restrict__ Eq,
                                                  const int* __restrict__ Fv, int m, double* C, int ldc,
                                                  const double* __restrict__ Cin, int ldcin, __nv_bfloat16* Cs,
                                                  int kpad, int* Gc) {
    extern __shared__ double cp[];   // kpad values
    __shared__ double part[4][256];
    __shared__ unsigned long long red[33];
    const int j = blockIdx.x;
    const int r = min(*r_dev, kpad);
    int tiles = 1, nsplit = 1;
    long kps = 0;
    if (ws && r > 0) tn_layout(r, d, tn_grid, &tiles, &nsplit, &kps);
    const int grp = threadIdx.x >> 8, li = threadIdx.x & 255;
    unsigned long long mb = 0;
    for (int l0 = 0; l0 < kpad; l0 += 256) {
        const int l = l0 + li;
        const bool live = j < m && l < r;
        if (ws) {
            // group grp sums the splits k = grp, grp + 4, ... in order
            double s = 0.0;
            if (live) {
                const double* p = ws + (long)j * rows_pad + l;
                const long st = (long)SG_N * rows_pad;
                for (int k = grp; k < nsplit; k += 4) s += p[k * st];
            }
            part[grp][li] = s;
        }
        __syncthreads();
        if (grp == 0 && l < kpad) {
            double v = 0.0;
            if (live) {
                double cc;
                if (ws) {
                    cc = ldexp((part[0][li] + part[1][li]) + (part[2][li] + part[3][li]), Eq[l] + Fv[j] - 14);
                    C[l + (long)j * ldc] = cc;
                } else {
                    cc = Cin[l + (long)j * ldcin];
                }
                v = ldexp(cc, Eq[l]);
            }
            cp[l] = v;
            const unsigned long long b = abs_bits(v);
            mb = b > mb ? b : mb;
        }
        __syncthreads();
    }
    mb = block_max_u64(mb, red);
    const int G = exponent_of_max(mb);
    for (int l = threadIdx.x; l < kpad; l += blockDim.x) {
        __nv_bfloat16 dg[SG_S];
        digits8(cp[l], G, dg);
        const long u = (long)(l >> 5) * 2 + (j >> 3);
        const int e = unit_elem(j & 7, l & 31);
#pragma unroll
        for (int s = 0; s < SG_S; ++s) Cs[((long)s * (kpad >> 5) * 2 + u) * 256 + e] = dg[s];
    }
    if (threadIdx.x == 0) Gc[j] = G;
}

// ------------------------------------------------------------ host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// BF16 2-D map over `units` operand units of 512 bytes (256 elements each,
// stored already in the tensor cores' swizzled layout, so no TMA swizzle), box
// of `box_units` consecutive units, zero fill beyond the end.
// A digit-slice operand of units of 512 bytes ordered [slice][contraction
// block][row group] as a 4-D tensor (256 elements, row groups, blocks,
// slices); a box covers box_units row groups of one block in all 8 slices.
// Row groups past the end read as zeros.
bool make_map(CUtensorMap* m, const void* base, uint64_t groups, uint64_t blocks, uint32_t box_units) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[4] = {256, groups, blocks, (cuuint64_t)SG_S};
    cuuint64_t strides[3] = {512, 512 * groups, 512 * groups * blocks};
    cuuint32_t box[4] = {256, box_units, 1, (cuuint32_t)SG_S};
    cuuint32_t es[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

cudaError_t launch_mma(const CUtensorMap* A, const CUtensorMap& B2, const SgArgs& a, dim3 grid, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(smem_launch_lock());
    const cudaError_t attr = set_dynamic_smem((const void*)k_split_mma, SG_DSMEM);
    if (attr != cudaSuccess) return attr;
    k_split_mma<<<grid, SG_THREADS, SG_DSMEM, s>>>(A[0], A[1], A[2], A[3], A[4], A[5], A[6], A[7], B2, a);
    count_launches(1);
    return cudaGetLastError();
}

inline long cdivl(long a, long b) { return (a + b - 1) / b; }

}  // namespace

size_t sg_bytes(long d, int cap, bool images) {
    const long cap_pad = cdivl(cap, SG_KC) * SG_KC;
    const long grid = 1024;   // bound on the SM count
    size_t b = 0;
    const long dp = cdivl(d, SG_KC) * SG_KC;
    b += 2 * (size_t)SG_S * cap_pad * dp * 2;        // Xc, Xr
    b += (size_t)SG_S * SG_N * dp * 2;               // Vs
    b += (size_t)SG_S * SG_N * cap_pad * 2;          // Cs
    b += sizeof(int) * ((size_t)cap_pad + 2 * SG_N + 1) + sizeof(unsigned long long) * ((size_t)cap_pad + SG_N);
    b += sizeof(double) * ((size_t)grid * cap_pad * SG_N + (size_t)SG_N * cap_pad);
    if (images) {
        b += (size_t)SG_S * cap_pad * dp * 2;        // Dr
        b += (size_t)SG_S * SG_N * cap_pad * 2;      // CsD
        b += sizeof(int) * ((size_t)cap_pad + SG_N) + sizeof(unsigned long long) * (size_t)cap_pad;
    }
    return b;
}

cudaError_t sg_init(SplitGemm* g, long d, int cap, bool images) {
    *g = SplitGemm();
    if (d < 1 || d % 8 != 0 || cap < 1 || cap > 16384) return cudaErrorInvalidValue;
    g->d = d;
    g->cap = cap;
    g->cap_pad = (int)(cdivl(cap, SG_KC) * SG_KC);
    g->grid = sm_count();
    if (g->grid > 1024) g->grid = 1024;
    const long cp = g->cap_pad;
    g->nkb = cdivl(d, SG_KC);
    g->nlb = (int)(cp / SG_KC);
    g->ngl = (int)(cp / 8);
    g->ngd = d / 8;
    const size_t uXc = (size_t)SG_S * g->nkb * g->ngl, uXr = (size_t)SG_S * g->nlb * g->ngd;
    const size_t uVs = (size_t)SG_S * g->nkb * 2, uCs = (size_t)SG_S * g->nlb * 2;
    cudaError_t e;
#define SG_ALLOC(ptr, bytes)                                        \
    if ((e = cudaMalloc((void**)&(ptr), (bytes))) != cudaSuccess) { \
        sg_free(g);                                                 \
        return e;                                                   \
    }                                                               \
    if ((e = cudaMemset((ptr), 0, (bytes))) != cudaSuccess) {       \
        sg_free(g);                                                 \
        return e;                                                   \
    }
    SG_ALLOC(g->Xc, uXc * 512);
    SG_ALLOC(g->Xr, uXr * 512);
    SG_ALLOC(g->Vs, uVs * 512);
    SG_ALLOC(g->Cs, uCs * 512);
    SG_ALLOC(g->Eq, sizeof(int) * cp);
    SG_ALLOC(g->Kq, sizeof(unsigned long long) * cp);
    SG_ALLOC(g->Kv, sizeof(unsigned long long) * SG_N);
    SG_ALLOC(g->Fv, sizeof(int) * SG_N);
    SG_ALLOC(g->Gc, sizeof(int) * SG_N);
    SG_ALLOC(g->err, sizeof(int));
    SG_ALLOC(g->ws, sizeof(double) * (size_t)g->grid * cp * SG_N);
    SG_ALLOC(g->C, sizeof(double) * (size_t)SG_N * cp);
    if (images) {
        SG_ALLOC(g->Dr, uXr * 512);
        SG_ALLOC(g->CsD, uCs * 512);
        SG_ALLOC(g->Ed, sizeof(int) * cp);
        SG_ALLOC(g->GcD, sizeof(int) * SG_N);
        SG_ALLOC(g->Kd, sizeof(unsigned long long) * cp);
    }
#undef SG_ALLOC
    const cudaError_t attr = set_dynamic_smem((const void*)k_finish, 16384 * sizeof(double));
    if (attr != cudaSuccess) {
        sg_free(g);
        return attr;
    }
    bool ok = make_map(&g->mapVs, g->Vs, 2, (uint64_t)g->nkb, 2) && make_map(&g->mapCs, g->Cs, 2, (uint64_t)g->nlb, 2);
    for (int i = 0; i < 8; ++i) {
        const uint32_t box = 2u * (uint32_t)(i + 1);
        ok = ok && make_map(&g->mapXc[i], g->Xc, (uint64_t)g->ngl, (uint64_t)g->nkb, box);
        ok = ok && make_map(&g->mapXr[i], g->Xr, (uint64_t)g->ngd, (uint64_t)g->nlb, box);
        if (images) ok = ok && make_map(&g->mapDr[i], g->Dr, (uint64_t)g->ngd, (uint64_t)g->nlb, box);
    }
    if (images) ok = ok && make_map(&g->mapCsD, g->CsD, 2, (uint64_t)g->nlb, 2);
    if (!ok) {
        sg_free(g);
        return cudaErrorNotSupported;
    }
    return cudaSuccess;
}

void sg_free(SplitGemm* g) {
    cudaFree(g->Xc);
    cudaFree(g->Xr);
    cudaFree(g->Vs);
    cudaFree(g->Cs);
    cudaFree(g->Eq);
    cudaFree(g->Kq);
    cudaFree(g->Kv);
    cudaFree(g->Fv);
    cudaFree(g->Gc);
    cudaFree(g->err);
    cudaFree(g->ws);
    cudaFree(g->C);
    cudaFree(g->Dr);
    cudaFree(g->CsD);
    cudaFree(g->Ed);
    cudaFree(g->GcD);
    cudaFree(g->Kd);
    *g = SplitGemm();
}

static int colmax_blocks(long d) {
    long nb = (d + 256 * 16 - 1) / (256 * 16);
    return (int)(nb < 1 ? 1 : nb > 128 ? 128 : nb);
}

// Column maxima, exponents and digits of columns of X into the Xr layout
// (xr) and, when xc is given, the Xc layout.
static cudaError_t append_digits(SplitGemm* g, const double* X, long ldx, const int* c0_dev, const int* c1_dev,
                                 int c0_host, int maxcols, unsigned long long* keys, int* exps, __nv_bfloat16* xc,
                                 __nv_bfloat16* xr, cudaStream_t s) {
    for (int j0 = 0; j0 < maxcols; j0 += SG_N) {
        // columns [c0 + j0, c0 + j0 + SG_N) of the (device-side) range
        const int nc = maxcols - j0 < SG_N ? maxcols - j0 : SG_N;
        cudaError_t e = cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * g->cap_pad, s);
        if (e != cudaSuccess) return e;
        if (c0_dev) {
            if (j0 > 0) return cudaErrorInvalidValue;   // device ranges: at most SG_N columns per call
            k_col_max<<<dim3(colmax_blocks(g->d), nc), 256, 0, s>>>(X, ldx, g->d, c0_dev, c1_dev, 0, keys);
        } else {
            k_col_max<<<dim3(colmax_blocks(g->d), nc), 256, 0, s>>>(X, ldx, g->d, nullptr, nullptr, c0_host + j0,
                                                                   keys);
        }
        long nb = cdivl(g->d, DB_ROWS);
        if (nb > 8 * 152) nb = 8 * 152;
        k_digits_basis<<<(int)nb, DB_ROWS, 0, s>>>(X, ldx, g->d, c0_dev, c1_dev, c0_host + j0, nc, keys, exps, xc, xr,
                                               g->nkb, g->ngl, g->nlb, g->ngd);
        count_launches(2);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t sg_append(SplitGemm* g, const double* Q, long ldq, const int* c0_dev, const int* c1_dev, int c0_host,
                      int maxcols, cudaStream_t s) {
    return append_digits(g, Q, ldq, c0_dev, c1_dev, c0_host, maxcols, g->Kq, g->Eq, g->Xc, g->Xr, s);
}

cudaError_t sg_append_images(SplitGemm* g, const double* D, long ldd, const int* c0_dev, const int* c1_dev,
                             int c0_host, int maxcols, cudaStream_t s) {
    if (!g->Dr) return cudaErrorInvalidValue;
    return append_digits(g, D, ldd, c0_dev, c1_dev, c0_host, maxcols, g->Kd, g->Ed, nullptr, g->Dr, s);
}

cudaError_t sg_project(SplitGemm* g, const double* v, long ldv, int m, const int* r_dev, cudaStream_t s) {
    if (m < 1 || m > SG_N) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(g->Kv, 0, sizeof(unsigned long long) * SG_N, s);
    if (e != cudaSuccess) return e;
    k_col_max<<<dim3(colmax_blocks(g->d), m), 256, 0, s>>>(v, ldv, g->d, nullptr, nullptr, 0, g->Kv);
    long nb = cdivl(g->d, 256);
    if (nb > 4 * 152) nb = 4 * 152;
    k_digits_block<<<(int)nb, 256, 0, s>>>(v, ldv, g->d, m, g->Kv, g->Fv, g->Vs, g->nkb);
    count_launches(2);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    SgArgs a{};
    a.mode = 0;
    a.rows_dev = r_dev;
    a.rows_host = g->cap;
    a.k_host = g->d;
    a.ws = g->ws;
    a.rows_pad = g->cap_pad;
    a.err = g->err;
    e = launch_mma(g->mapXc, g->mapVs, a, dim3((unsigned)g->grid), s);
    if (e != cudaSuccess) return e;
    k_finish<<<SG_N, FIN_T, sizeof(double) * g->cap_pad, s>>>(g->ws, g->cap_pad, g->grid, g->d, r_dev, g->Eq, g->Fv, m,
                                                            g->C, g->cap_pad, nullptr, 0, g->Cs, g->cap_pad, g->Gc);
    count_launches(1);
    return cudaGetLastError();
}

// v <- v - X C on the tensor cores: X's digits (maps mapA, Xr layout) against
// the folded coefficient digits (map mapB) with their column exponents gc.
static cudaError_t sg_apply(SplitGemm* g, double* v, long ldv, int m, const int* r_dev, const CUtensorMap* mapA,
                            const CUtensorMap& mapB, int* gc, cudaStream_t s) {
    SgArgs a{};
    a.mode = 1;
    a.rows_host = (int)g->d;
    a.k_dev = r_dev;
    a.k_host = g->cap;
    a.v = v;
    a.ldv = ldv;
    a.vexp = gc;
    a.ncols = m;
    a.err = g->err;
    long tiles = cdivl(g->d, SG_BM);
    return launch_mma(mapA, mapB, a, dim3((unsigned)(tiles < g->grid ? tiles : g->grid)), s);
}
static cudaError_t sg_apply_update(SplitGemm* g, double* v, long ldv, int m, const int* r_dev, cudaStream_t s) {
    return sg_apply(g, v, ldv, m, r_dev, g->mapXr, g->mapCs, g->Gc, s);
}

cudaError_t sg_cgs_pass(SplitGemm* g, double* v, long ldv, int m, const int* r_dev, cudaStream_t s) {
    cudaError_t e = sg_project(g, v, ldv, m, r_dev, s);
    if (e != cudaSuccess) return e;
    return sg_apply_update(g, v, ldv, m, r_dev, s);
}

cudaError_t sg_update_images(SplitGemm* g, double* z, long ldz, int m, const int* r_dev, cudaStream_t s) {
    if (m < 1 || m > SG_N || !g->Dr) return cudaErrorInvalidValue;
    // the coefficients of the last projection, folded with D's exponents
    k_finish<<<SG_N, FIN_T, sizeof(double) * g->cap_pad, s>>>(nullptr, 0, 0, g->d, r_dev, g->Ed, nullptr, m, nullptr,
                                                            0, g->C, g->cap_pad, g->CsD, g->cap_pad, g->GcD);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return sg_apply(g, z, ldz, m, r_dev, g->mapDr, g->mapCsD, g->GcD, s);
}
cudaError_t sg_update(SplitGemm* g, double* v, long ldv, int m, const double* C, int ldc, const int* r_dev,
                      cudaStream_t s) {
    if (m < 1 || m > SG_N) return cudaErrorInvalidValue;
    k_finish<<<SG_N, FIN_T, sizeof(double) * g->cap_pad, s>>>(nullptr, 0, 0, g->d, r_dev, g->Eq, nullptr, m, nullptr, 0,
                                                            C, ldc, g->Cs, g->cap_pad, g->Gc);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return sg_apply_update(g, v, ldv, m, r_dev, s);
}

}  // namespace pr

// ------------------------------------------------------------ standalone entry points

#include "parareal.h"

namespace {

struct TmpSplit {
    pr::SplitGemm g;
    int* r_dev = nullptr;
    bool ok = false;
    ~TmpSplit() {
        if (ok) pr::sg_free(&g);
        cudaFree(r_dev);
    }
};

pr_status split_common(TmpSplit& t, const double* A, int64_t lda, int32_t m, int64_t k, cudaStream_t s) {
    cudaError_t e = pr::sg_init(&t.g, (long)k, m);
    if (e == cudaErrorMemoryAllocation) return PR_ENOMEM;
    if (e != cudaSuccess) return PR_ECUDA;
    t.ok = true;
    if (cudaMalloc((void**)&t.r_dev, sizeof(int)) != cudaSuccess) return PR_ENOMEM;
    if (cudaMemcpy(t.r_dev, &m, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return PR_ECUDA;
    if (pr::sg_append(&t.g, A, (long)lda, nullptr, nullptr, 0, m, s) != cudaSuccess) return PR_ECUDA;
    return PR_OK;
}

pr_status split_finish(TmpSplit& t, cudaStream_t s) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return PR_ECUDA;
    int err = 0;
    if (cudaMemcpy(&err, t.g.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return PR_ECUDA;
    return err ? PR_ETIMEOUT : PR_OK;
}

bool split_args_ok(const double* A, int64_t lda, int32_t m, const double* B, int64_t ldb, int32_t n, int64_t k,
                   const double* Y, int64_t ldy, int64_t ldb_min, int64_t ldy_min) {
    if (!A || !B || !Y) return false;
    if (k < 8 || k % 8 != 0 || k > (int64_t)1 << 30 || m < 1 || m > 16384 || n < 1) return false;
    return lda >= k && ldb >= ldb_min && ldy >= ldy_min;
}

}  // namespace

extern "C" pr_status parareal_split_gemm_tn(const double* A, int64_t lda, int32_t m, const double* B, int64_t ldb,
                                            int32_t n, int64_t k, double* C, int64_t ldc, void* stream) {
    if (!split_args_ok(A, lda, m, B, ldb, n, k, C, ldc, k, m)) {
        std::fprintf(stderr, "parareal_split_gemm_tn: invalid sizes, leading dimensions or NULL pointer\n");
        return PR_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    TmpSplit t;
    pr_status st = split_common(t, A, lda, m, k, s);
    if (st != PR_OK) return st;
    for (int j0 = 0; j0 < n; j0 += pr::SG_N) {
        const int mm = n - j0 < pr::SG_N ? n - j0 : pr::SG_N;
        if (pr::sg_project(&t.g, B + (long)j0 * ldb, (long)ldb, mm, t.r_dev, s) != cudaSuccess) return PR_ECUDA;
        if (cudaMemcpy2DAsync(C + (long)j0 * ldc, sizeof(double) * ldc, t.g.C, sizeof(double) * t.g.cap_pad,
                              sizeof(double) * m, mm, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return PR_ECUDA;
    }
    return split_finish(t, s);
}

extern "C" pr_status parareal_split_gemm_nn(const double* A, int64_t lda, int32_t m, const double* B, int64_t ldb,
                                            int32_t n, int64_t k, double* Y, int64_t ldy, void* stream) {
    if (!split_args_ok(A, lda, m, B, ldb, n, k, Y, ldy, m, k)) {
        std::fprintf(stderr, "parareal_split_gemm_nn: invalid sizes, leading dimensions or NULL pointer\n");
        return PR_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    TmpSplit t;
    pr_status st = split_common(t, A, lda, m, k, s);
    if (st != PR_OK) return st;
    for (int j0 = 0; j0 < n; j0 += pr::SG_N) {
        const int mm = n - j0 < pr::SG_N ? n - j0 : pr::SG_N;
        if (pr::sg_update(&t.g, Y + (long)j0 * ldy, (long)ldy, mm, B + (long)j0 * ldb, (int)ldb, t.r_dev, s) !=
            cudaSuccess)
            return PR_ECUDA;
    }
    return split_finish(t, s);
}
