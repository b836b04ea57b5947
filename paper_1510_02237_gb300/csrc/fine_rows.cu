// fine_rows.cu -- fine propagator F in FP32 arithmetic: one RK-3 step of the
// flux-form tendency (Sec. 3: 6th-order centred advection, 2nd-order centred
// acoustics, compact grad-div damping with alpha = nu_f dx^2 / dt, Eq.
// dampingCoeff) for V = 0, streamed row by row.
//
// A CTA of nx/4 threads covers one full grid row: lane l of warp w owns the
// 4 consecutive cells x0 = 4 (32 w + l) .. x0 + 3.  The x-neighbours of a
// cell are in the same lane or the next lanes and come in by warp shuffles;
// the row is periodic, so with one warp per row the shuffle wraps exactly,
// and with several warps the edge lanes take the neighbouring warps' cells
// from shared memory.  With V = 0 one stage has a y-radius of 1, so each CTA
// marches down a range of rows with the three stages skewed by one row:
//
//   iteration j:  s1 = q^n + dt/3 L(q^n) at row j+2;  s2 = q^n + dt/2 L(s1)
//                 at row j+1;  q^{n+1} = q^n + dt L(s2) at row j,
//
// holding the last three rows of s1 and s2 in registers.  The rows of q^n
// arrive by TMA bulk copies (cp.async.bulk, one per field and row) in a ring
// of R rows in shared memory, R - 4 rows ahead of their first use, each slot
// completed on its own mbarrier.  Every state value is read from memory once
// and written once (plus 6 halo rows per row range); stage values never go
// through shared memory.  The grid is persistent: the n*ny rows of the batch
// are split into equal contiguous ranges, one per CTA (a range may continue
// into the next state), and a CTA's ranges form one stream of ring rows.
#include "common.cuh"
#include "tc.cuh"

namespace pr {

// Set (sticky) when a wait for a ring row gave up: results are then invalid.
__device__ int g_rows_wait_err = 0;

namespace {

template <typename T>
__host__ __device__ constexpr int ring_rows() { return 8; }

// Per-stage coefficients, already multiplied by the stage length c_k
// (dt/3, dt/2, dt) and signed as they enter q^n + c_k L.
struct RowCoef {
    float A[3];    // -c_k U/(60 dx): 6-point advective difference
    float Bx[3];   // -c_k c_s/(2 dx)
    float By[3];   // -c_k c_s/(2 dy)
    float Cx[3];   // c_k alpha1/dx^2
    float Ex[3];   // c_k alpha1/(4 dx dy)
    float Cy[3];   // c_k alpha2/dy^2
    float Ey[3];   // c_k alpha2/(4 dx dy)
};

struct Row {
    float4 u, w, p;
    __device__ __forceinline__ float4 f(int i) const { return i == 0 ? u : (i == 1 ? w : p); }
};

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 lds4(const double* p) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    return make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
}
__device__ __forceinline__ void store4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ void store4(double* p, float4 v) {
    double2* q = reinterpret_cast<double2*>(p);
    q[0] = make_double2(v.x, v.y);
    q[1] = make_double2(v.z, v.w);
}

// A row of q^n in the shared-memory ring: fields at p + f nx.  xl / xr: the
// aligned 4-cell chunks just left of the warp's first cell and just right of
// its last cell (periodic).
template <typename T>
struct RingRow {
    const T* p;
    int nx, x0, xl, xr;
    __device__ __forceinline__ float4 own(int f) const { return lds4(p + f * nx + x0); }
    __device__ __forceinline__ float4 left(int f) const { return lds4(p + f * nx + xl); }
    __device__ __forceinline__ float4 right(int f) const { return lds4(p + f * nx + xr); }
};

// Edge chunks of the stage rows held in registers, exchanged between the
// warps of a row: [stage s1/s2][slot][warp][0: lane 0's cells, 1: lane 31's][field].
template <int NW>
struct Edges {
    float4 e[2][4][NW][2][3];
};

// A stage row in registers; left/right read the neighbouring warps' chunks.
struct RegRow {
    const Row& r;
    const float4* L;   // [field] last chunk of the warp to the left
    const float4* R;   // [field] first chunk of the warp to the right
    __device__ __forceinline__ float4 own(int f) const { return r.f(f); }
    __device__ __forceinline__ float4 left(int f) const { return L[f]; }
    __device__ __forceinline__ float4 right(int f) const { return R[f]; }
};

template <int NW>
__device__ __forceinline__ RegRow reg_row(const Row& r, const Edges<NW>& E, int st, int slot, int warp) {
    return RegRow{r, E.e[st][slot][(warp + NW - 1) % NW][1], E.e[st][slot][(warp + 1) % NW][0]};
}

template <int NW>
__device__ __forceinline__ void publish(Edges<NW>& E, int st, int slot, const Row& r, int warp, int lane) {
    if (NW == 1) return;
    if (lane == 0 || lane == 31) {
        float4* e = E.e[st][slot][warp][lane == 0 ? 0 : 1];
        e[0] = r.u;
        e[1] = r.w;
        e[2] = r.p;
    }
}

// Window of one field on the centre row: cells x0-3 .. x0+6 (index i+3 is cell x0+i).
template <int NW, typename Src>
__device__ __forceinline__ void window3(float (&c)[10], const Src& s, int f, int lane) {
    const unsigned all = 0xffffffffu;
    const int lm = (lane + 31) & 31, lp = (lane + 1) & 31;
    const float4 v = s.own(f);
    c[3] = v.x;
    c[4] = v.y;
    c[5] = v.z;
    c[6] = v.w;
    c[0] = __shfl_sync(all, v.y, lm);
    c[1] = __shfl_sync(all, v.z, lm);
    c[2] = __shfl_sync(all, v.w, lm);
    c[7] = __shfl_sync(all, v.x, lp);
    c[8] = __shfl_sync(all, v.y, lp);
    c[9] = __shfl_sync(all, v.z, lp);
    if (NW > 1) {   // warp-uniform (broadcast) reads, selected on the edge lanes
        const float4 l = s.left(f), r = s.right(f);
        const bool l0 = lane == 0, l31 = lane == 31;
        c[0] = l0 ? l.y : c[0];
        c[1] = l0 ? l.z : c[1];
        c[2] = l0 ? l.w : c[2];
        c[7] = l31 ? r.x : c[7];
        c[8] = l31 ? r.y : c[8];
        c[9] = l31 ? r.z : c[9];
    }
}

// Window of one field on a neighbouring row: cells x0-1 .. x0+4 (index i+1 is cell x0+i).
template <int NW, typename Src>
__device__ __forceinline__ void window1(float (&c)[6], const Src& s, int f, int lane) {
    const unsigned all = 0xffffffffu;
    const float4 v = s.own(f);
    c[1] = v.x;
    c[2] = v.y;
    c[3] = v.z;
    c[4] = v.w;
    c[0] = __shfl_sync(all, v.w, (lane + 31) & 31);
    c[5] = __shfl_sync(all, v.x, (lane + 1) & 31);
    if (NW > 1) {
        const float l = s.left(f).w, r = s.right(f).x;
        c[0] = lane == 0 ? l : c[0];
        c[5] = lane == 31 ? r : c[5];
    }
}

// Packed FP32 pair arithmetic (sm_100 family `.f32x2`): two lanes of work per
// instruction.  Pairs of consecutive cells whose values sit in one aligned
// register pair (the own cells 0-1 and 2-3, two shuffled neighbours) cost
// nothing to form; the others are formed by scalar operations.
__device__ __forceinline__ unsigned long long pk(float2 v) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
    return r;
}
__device__ __forceinline__ float2 upk(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {   // a * b + c
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)), "l"(pk(c)));
    return upk(d);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 sp(float a) { return make_float2(a, a); }

// qn + c_k L(X) at the 4 own cells of the centre row, from the rows S (y-1),
// C (y), N (y+1) of the stage input X, as two pairs of cells (0,1), (2,3).
// The terms are accumulated field by field so that only one window is live
// at a time.  Centre windows c[i+3] = cell x0+i (i = -3..6); neighbour-row
// windows a[i+1], b[i+1] = cell x0+i (i = -1..4).
template <int NW, typename SS, typename SC, typename SN>
__device__ __forceinline__ Row stage_row(const SS& S, const SC& C, const SN& N, const Row& qn, const RowCoef& k,
                                         int kk, int lane) {
    const float2 A = sp(k.A[kk]), Bx = sp(k.Bx[kk]), By = sp(k.By[kk]), Cx = sp(k.Cx[kk]), Ex = sp(k.Ex[kk]),
                 Cy = sp(k.Cy[kk]), Ey = sp(k.Ey[kk]), M9 = sp(-9.f), P45 = sp(45.f), M2 = sp(-2.f),
                 M2Cy = sp(-2.f * k.Cy[kk]);
    float2 ru[2] = {f2(qn.u.x, qn.u.y), f2(qn.u.z, qn.u.w)};
    float2 rw[2] = {f2(qn.w.x, qn.w.y), f2(qn.w.z, qn.w.w)};
    float2 rp[2] = {f2(qn.p.x, qn.p.y), f2(qn.p.z, qn.p.w)};
    // 6th-order advective difference of cells (2h, 2h+1) and their centred
    // difference d1 = c[i+1] - c[i-1]
    auto adv = [&](const float (&c)[10], int h, float2& d1) {
        const int m = 2 * h + 3;
        d1 = f2(c[m + 1] - c[m - 1], c[m + 2] - c[m]);
        const float2 d3 = f2(c[m + 3] - c[m - 3], c[m + 4] - c[m - 2]);
        const float2 d2 = sub2(f2(c[m + 2], c[m + 3]), f2(c[m - 2], c[m - 1]));
        return fma2(P45, d1, fma2(M9, d2, d3));
    };
    {   // p on the centre row: advection of p, x-acoustics of u
        float c[10];
        window3<NW>(c, C, 2, lane);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float2 d1;
            const float2 a6 = adv(c, h, d1);
            rp[h] = fma2(A, a6, rp[h]);
            ru[h] = fma2(Bx, d1, ru[h]);
        }
    }
    {   // u on the centre row: advection, x-damping of u, x-acoustics of p
        float c[10];
        window3<NW>(c, C, 0, lane);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int m = 2 * h + 3;
            float2 d1;
            const float2 a6 = adv(c, h, d1);
            ru[h] = fma2(A, a6, ru[h]);
            const float2 lap = fma2(M2, f2(c[m], c[m + 1]), f2(c[m + 1] + c[m - 1], c[m + 2] + c[m]));
            ru[h] = fma2(Cx, lap, ru[h]);
            rp[h] = fma2(Bx, d1, rp[h]);
        }
    }
    {   // w on the centre row: advection, centre of the y-damping of w
        float c[10];
        window3<NW>(c, C, 1, lane);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int m = 2 * h + 3;
            float2 d1;
            const float2 a6 = adv(c, h, d1);
            rw[h] = fma2(A, a6, rw[h]);
            rw[h] = fma2(M2Cy, f2(c[m], c[m + 1]), rw[h]);
        }
    }
    {   // w on the neighbouring rows: cross damping of u, y-damping of w, y-acoustics of p
        float a[6], b[6];
        window1<NW>(a, S, 1, lane);
        window1<NW>(b, N, 1, lane);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int m = 2 * h + 1;   // index of cell 2h
            const float2 hb = f2(b[m + 1] - b[m - 1], b[m + 2] - b[m]);
            const float2 ha = f2(a[m + 1] - a[m - 1], a[m + 2] - a[m]);
            ru[h] = fma2(Ex, sub2(hb, ha), ru[h]);
            const float2 bc = f2(b[m], b[m + 1]), ac = f2(a[m], a[m + 1]);
            rw[h] = fma2(Cy, add2(bc, ac), rw[h]);
            rp[h] = fma2(By, sub2(bc, ac), rp[h]);
        }
    }
    {   // u on the neighbouring rows: cross damping of w
        float a[6], b[6];
        window1<NW>(a, S, 0, lane);
        window1<NW>(b, N, 0, lane);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int m = 2 * h + 1;
            const float2 hb = f2(b[m + 1] - b[m - 1], b[m + 2] - b[m]);
            const float2 ha = f2(a[m + 1] - a[m - 1], a[m + 2] - a[m]);
            rw[h] = fma2(Ey, sub2(hb, ha), rw[h]);
        }
    }
    {   // p on the neighbouring rows: y-acoustics of w
        const float4 sa = S.own(2), sb = N.own(2);
        rw[0] = fma2(By, sub2(f2(sb.x, sb.y), f2(sa.x, sa.y)), rw[0]);
        rw[1] = fma2(By, sub2(f2(sb.z, sb.w), f2(sa.z, sa.w)), rw[1]);
    }
    return Row{make_float4(ru[0].x, ru[0].y, ru[1].x, ru[1].y), make_float4(rw[0].x, rw[0].y, rw[1].x, rw[1].y),
               make_float4(rp[0].x, rp[0].y, rp[1].x, rp[1].y)};
}

template <int NW>
__device__ __forceinline__ void cta_sync() {
    if (NW > 1)
        __syncthreads();
    else
        __syncwarp();
}

// Row range [r, r + L) of the batch's rows (row index = state * ny + y) that
// stays within one state.
struct Seg {
    long z;
    int ya, L;
};
__device__ __forceinline__ Seg segment(long r, long r1, int ny) {
    Seg s;
    s.z = r / ny;
    s.ya = (int)(r - s.z * ny);
    s.L = (int)min((long)(ny - s.ya), r1 - r);
    return s;
}
__device__ __forceinline__ int wrap_row(int y, int ny) {
    y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
    return (y < 0 || y >= ny) ? pwrap(y, ny) : y;   // tiny grids: offsets beyond one period
}

template <int NW, typename Tin, typename Tout>
__global__ void __launch_bounds__(32 * NW, (NW >= 8 ? 1 : 12 / NW))
    k_fine_rows(const Tin* __restrict__ in, long instride, Tout* __restrict__ out, long outstride, int n, int nx,
                int ny, RowCoef k, SliceMap map) {
    constexpr int R = ring_rows<Tin>();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Tin* ring = reinterpret_cast<Tin*>(smem_raw);                       // R x 3 x nx
    const uint32_t bar0 = tc::smem_u32(smem_raw + (size_t)R * 3 * nx * sizeof(Tin));
    __shared__ Edges<NW> E;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x0 = 4 * threadIdx.x;
    const int xl = (128 * warp + nx - 4) % nx, xr = (128 * warp + 128) % nx;
    const long ncell = (long)nx * ny;
    const uint32_t row_bytes = (uint32_t)(nx * sizeof(Tin));
    int nact = n;
    long beg = 0;
    if (map.end) {
        const int b0 = *map.beg;
        nact = min(n, *map.end - b0);
        beg = b0;
    }
    if (nact <= 0) return;
    const long rows = (long)nact * ny;
    const long G = gridDim.x;
    const long r0 = rows * blockIdx.x / G, r1 = rows * (blockIdx.x + 1) / G;
    if (r0 >= r1) return;
    int T_total = 0;   // ring rows of all ranges: L + 6 each
    for (long r = r0; r < r1;) {
        const Seg s = segment(r, r1, ny);
        T_total += s.L + 6;
        r += s.L;
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < R; ++i) tc::mbar_init(bar0 + 8 * i, 1);
        tc::fence_barrier_init();
    }
    __syncthreads();

    // producer (thread 0 issues; the cursor is kept by every thread alike)
    int pt = 0, p_base = 0;
    long p_r = r0;
    Seg ps = segment(r0, r1, ny);
    auto produce = [&](int limit) {
        if (limit > T_total - 1) limit = T_total - 1;
        for (; pt <= limit; ++pt) {
            if (pt >= p_base + ps.L + 6) {
                p_base += ps.L + 6;
                p_r += ps.L;
                ps = segment(p_r, r1, ny);
            }
            if (threadIdx.x == 0) {
                const int y = wrap_row(ps.ya - 3 + (pt - p_base), ny);
                const int slot = pt & (R - 1);
                const uint32_t bar = bar0 + 8 * slot;
                const Tin* src = in + (map.in_map ? ps.z + beg : ps.z) * instride + (long)y * nx;
                Tin* dst = ring + (size_t)slot * 3 * nx;
                tc::mbar_expect_tx(bar, 3 * row_bytes);
#pragma unroll
                for (int f = 0; f < 3; ++f) tc::bulk_load(tc::smem_u32(dst + f * nx), src + f * ncell, row_bytes, bar);
            }
        }
    };
    auto wait_row = [&](int t) {   // ring row of stream index t has landed
        if (!tc::mbar_wait(bar0 + 8 * (t & (R - 1)), (uint32_t)((t / R) & 1)) && lane == 0)
            atomicExch(&g_rows_wait_err, 1);
    };
    auto qrow = [&](int t) { return RingRow<Tin>{ring + (size_t)(t & (R - 1)) * 3 * nx, nx, x0, xl, xr}; };
    produce(R - 1);

    int base = 0;   // stream index of the current range's row -3
    for (long r = r0; r < r1;) {
        const Seg s = segment(r, r1, ny);
        if (r > r0) {    // every warp is done with the previous range: its ring rows are free
            cta_sync<NW>();
            produce(base + R - 1);
        }
        r += s.L;
        Tout* dst = out + (map.out_map ? s.z + beg : s.z) * outstride + x0;
        Row A1{}, B1{}, C1{}, A2{}, B2{}, C2{};
        // s1 row j+2 from q^n rows j+1, j+2, j+3
        auto s1_step = [&](int j) {
            wait_row(base + j + 6);
            const RingRow<Tin> q2 = qrow(base + j + 5);
            const Row qn2{q2.own(0), q2.own(1), q2.own(2)};
            C1 = stage_row<NW>(qrow(base + j + 4), q2, qrow(base + j + 6), qn2, k, 0, lane);
            publish<NW>(E, 0, (j + 6) & 3, C1, warp, lane);
        };
        // s2 row j+1 from s1 rows j, j+1, j+2
        auto s2_step = [&](int j) {
            const RingRow<Tin> q1 = qrow(base + j + 4);
            const Row qn1{q1.own(0), q1.own(1), q1.own(2)};
            C2 = stage_row<NW>(reg_row<NW>(A1, E, 0, (j + 4) & 3, warp), reg_row<NW>(B1, E, 0, (j + 5) & 3, warp),
                               reg_row<NW>(C1, E, 0, (j + 6) & 3, warp), qn1, k, 1, lane);
            publish<NW>(E, 1, (j + 5) & 3, C2, warp, lane);
        };
        // q^{n+1} row j from s2 rows j-1, j, j+1
        auto out_step = [&](int j) {
            const RingRow<Tin> q0 = qrow(base + j + 3);
            const long ro = (long)(s.ya + j) * nx;
            const RegRow a = reg_row<NW>(A2, E, 1, (j + 3) & 3, warp), b = reg_row<NW>(B2, E, 1, (j + 4) & 3, warp),
                         c = reg_row<NW>(C2, E, 1, (j + 5) & 3, warp);
            const Row qn0{q0.own(0), q0.own(1), q0.own(2)};
            const Row o = stage_row<NW>(a, b, c, qn0, k, 2, lane);
            store4(dst + ro, o.u);
            store4(dst + ncell + ro, o.w);
            store4(dst + 2 * ncell + ro, o.p);
        };
        wait_row(base);
        wait_row(base + 1);
        // iterations -4..-1 fill the pipeline (s1 rows -2..1, s2 rows -1..0)
        for (int j = -4; j < 0; ++j) {
            s1_step(j);
            cta_sync<NW>();
            produce(base + R - 1);
            if (j >= -2) s2_step(j);
            cta_sync<NW>();
            A1 = B1;
            B1 = C1;
            A2 = B2;
            B2 = C2;
        }
#pragma unroll 1
        for (int j = 0; j < s.L; ++j) {
            s1_step(j);
            cta_sync<NW>();
            // every warp is done with iteration j-1: ring rows before row j are free
            produce(base + j + 3 + R - 1);
            s2_step(j);
            cta_sync<NW>();
            out_step(j);
            A1 = B1;
            B1 = C1;
            A2 = B2;
            B2 = C2;
        }
        base += s.L + 6;
    }
}

template <int NW, typename Tin, typename Tout>
cudaError_t launch_nw(const Tin* in, long instride, Tout* out, long outstride, int n, int nx, int ny,
                      const RowCoef& k, cudaStream_t s, const SliceMap& map, int min_rows) {
    static DevMemo memo;   // [device] -> (SMs, CTAs per SM)
    constexpr int R = ring_rows<Tin>();
    const size_t smem = (size_t)R * 3 * nx * sizeof(Tin) + 8 * R;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    auto kern = k_fine_rows<NW, Tin, Tout>;
    std::lock_guard<std::mutex> lk(smem_launch_lock());
    e = set_dynamic_smem((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    int sms = 0, per = 0;
    if (!memo.get(dev, &sms, &per)) {
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 32 * NW, smem);
        if (e != cudaSuccess) return e;
        memo.put(dev, sms, per);
    }
    if (per < 1) return cudaErrorInvalidConfiguration;
    // at least min_rows rows per CTA (default 16) keep the 6 halo rows of a range cheap
    if (min_rows < 1) min_rows = 1;
    const long rows = (long)n * ny;
    long G = (rows + min_rows - 1) / min_rows;
    if (G > (long)sms * per) G = (long)sms * per;
    if (G < 1) G = 1;
    kern<<<(unsigned)G, 32 * NW, smem, s>>>(in, instride, out, outstride, n, nx, ny, k, map);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

int fine_rows_wait_error(bool reset) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_rows_wait_err, sizeof(int)) != cudaSuccess) return -1;
    if (reset && v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_rows_wait_err, &z, sizeof(int));
    }
    return v;
}

bool fine_rows_eligible(int nx, bool has_v) {
    const int nw = nx / 128;
    return !has_v && nx % 128 == 0 && (nw == 1 || nw == 2 || nw == 4 || nw == 8);
}

template <typename Tin, typename Tout>
bool launch_fine_rows(const Tin* in, long instride, Tout* out, long outstride, int n, int nx, int ny, bool has_v,
                      const FineCoef<float>& c, cudaStream_t s, const SliceMap& map, cudaError_t* err,
                      int min_rows) {
    if constexpr (sizeof(Tin) != sizeof(float)) {
        // FP64 input: the per-read conversions to FP32 would run at the FP64
        // rate, so the shared-memory tile kernel (one conversion per cell) serves it
        return false;
    } else {
    const int nw = nx / 128;
    if (!fine_rows_eligible(nx, has_v) || ny < 1 || n < 1) return false;
    if (((uintptr_t)in | (uintptr_t)out) % 16 != 0 || instride % 4 != 0 || outstride % 4 != 0) return false;
    RowCoef k;
    const double ck[3] = {(double)c.c1, (double)c.c2, (double)c.c3};
    for (int i = 0; i < 3; ++i) {
        k.A[i] = (float)(-ck[i] * (double)c.ax6);
        k.Bx[i] = (float)(-ck[i] * (double)c.csx);
        k.By[i] = (float)(-ck[i] * (double)c.csy);
        k.Cx[i] = (float)(ck[i] * (double)c.dxx);
        k.Ex[i] = (float)(ck[i] * (double)c.dxy1);
        k.Cy[i] = (float)(ck[i] * (double)c.dyy);
        k.Ey[i] = (float)(ck[i] * (double)c.dxy2);
    }
    switch (nw) {
        case 1: *err = launch_nw<1, Tin, Tout>(in, instride, out, outstride, n, nx, ny, k, s, map, min_rows); break;
        case 2: *err = launch_nw<2, Tin, Tout>(in, instride, out, outstride, n, nx, ny, k, s, map, min_rows); break;
        case 4: *err = launch_nw<4, Tin, Tout>(in, instride, out, outstride, n, nx, ny, k, s, map, min_rows); break;
        default: *err = launch_nw<8, Tin, Tout>(in, instride, out, outstride, n, nx, ny, k, s, map, min_rows); break;
    }
    return true;
    }
}

template bool launch_fine_rows<double, double>(const double*, long, double*, long, int, int, int, bool, const FineCoef<float>&,
                                        cudaStream_t, const SliceMap&, cudaError_t*, int);
template bool launch_fine_rows<double, float>(const double*, long, float*, long, int, int, int, bool, const FineCoef<float>&,
                                        cudaStream_t, const SliceMap&, cudaError_t*, int);
template bool launch_fine_rows<float, float>(const float*, long, float*, long, int, int, int, bool, const FineCoef<float>&,
                                        cudaStream_t, const SliceMap&, cudaError_t*, int);
template bool launch_fine_rows<float, double>(const float*, long, double*, long, int, int, int, bool, const FineCoef<float>&,
                                        cudaStream_t, const SliceMap&, cudaError_t*, int);

}  // namespace pr
