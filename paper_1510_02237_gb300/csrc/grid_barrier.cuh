// grid_barrier.cuh -- bounded barrier over all CTAs of a cooperative launch.
#pragma once

#include "common.cuh"

namespace pr {

// Poll ctr with acquire loads until it reaches target (counters only grow
// within a launch).  Gives up -- sets *err to 1 and returns 0 -- after one
// second by the global timer (or 2^26 polls), and returns 0 at once when
// another wait has set the error word.
__device__ __forceinline__ int poll_until(unsigned* ctr, unsigned target, volatile int* verr, int* err) {
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (unsigned long long it = 1;; ++it) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if ((int)(v - target) >= 0) return 1;
        if ((it & 255) == 0) {
            if (*verr != 0) return 0;
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t - t0 > 1000000000ull || it > (1ull << 26)) {
                atomicExch(err, 1);
                return 0;
            }
        }
    }
}

// Barrier over all CTAs of a cooperative launch, on the monotonic counter
// gb->count (zeroed before every launch that uses it): thread 0 of each CTA
// adds one with release semantics and polls with acquire loads until the
// counter reaches the next multiple of nblocks.  The spin is bounded
// (poll_until): after a second it sets the error word and returns false, so
// a fault elsewhere can never hang the GPU; a set error word makes every
// later barrier return false at once.
__device__ __forceinline__ bool grid_barrier(GridBar* gb, unsigned nblocks) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int* verr = &gb->err;
        int ok = 0;
        if (*verr == 0) {
            unsigned old;
            asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(&gb->count) : "memory");
            const unsigned target = (old / nblocks + 1) * nblocks;
            ok = poll_until(&gb->count, target, verr, &gb->err);
        }
        s_ok = ok && *verr == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

// A barrier over one group of nthr threads (a multiple of 32, calling it
// together) in every CTA, on the monotonic counter gb->gcount[slot] (zero at
// launch): the group meets at named barrier bar_id (0 with all threads of
// the CTA), its first thread (leader) adds one with release semantics and
// polls with acquire loads until the counter reaches the next multiple of
// nblocks, the group meets again.  Two groups of a CTA can synchronise with
// their peers independently.  Bounded like grid_barrier, on the same error
// word; s_ok is a shared-memory word of the group.
__device__ __forceinline__ void named_barrier(int bar_id, int nthr) {
    asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(nthr) : "memory");
}
__device__ __forceinline__ bool grid_barrier_group(GridBar* gb, int slot, unsigned nblocks, int bar_id, int nthr,
                                                   bool leader, volatile int* s_ok) {
    named_barrier(bar_id, nthr);
    if (leader) {
        volatile int* verr = &gb->err;
        unsigned* ctr = &gb->gcount[slot];
        int ok = 0;
        if (*verr == 0) {
            unsigned old;
            asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(ctr) : "memory");
            const unsigned target = (old / nblocks + 1) * nblocks;
            ok = poll_until(ctr, target, verr, &gb->err);
        }
        *s_ok = ok && *verr == 0;
    }
    named_barrier(bar_id, nthr);
    return *s_ok != 0;
}

// Sum of the nb values base[k * stride], k = 0..nb-1, by one warp: lane j adds
// k = j, j+32, ... in order, then a fixed xor-shuffle tree combines the lanes.
// Deterministic, the same in every CTA; the loads are independent, so they
// are in flight together.  Reads bypass L1 (written by other CTAs).
__device__ __forceinline__ double warp_sum_strided(const double* base, unsigned nb, long stride) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (unsigned k = lane; k < nb; k += 32) s += __ldcg(base + (long)k * stride);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Warp sums of 16 per-lane values by recursive halving: at each step a lane
// keeps half of its values and adds its partner's copy of them (16 shuffles
// instead of 80).  Returns kof; afterwards acc[0] of every even lane holds the
// warp sum of value kof, summed in a fixed order.
__device__ __forceinline__ int warp_sum16(double (&acc)[16]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int h = 8, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const double send = up ? acc[i] : acc[i + h];
            const double keep = up ? acc[i + h] : acc[i];
            acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
    return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

// Dot product of a and b over rows [r0, r1) by one warp: lane j takes rows
// r0 + j + 32 t in order, four rows per iteration with their loads issued
// together, then a fixed xor-shuffle tree.  Deterministic.
__device__ __forceinline__ double warp_dot(const double* a, const double* b, long r0,
                                           long r1) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    long row = r0 + lane;
    for (; row + 96 < r1; row += 128) {
        const double a0 = a[row], a1 = a[row + 32], a2 = a[row + 64], a3 = a[row + 96];
        const double b0 = b[row], b1 = b[row + 32], b2 = b[row + 64], b3 = b[row + 96];
        s += a0 * b0;
        s += a1 * b1;
        s += a2 * b2;
        s += a3 * b3;
    }
    for (; row < r1; row += 32) s += a[row] * b[row];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

}  // namespace pr
