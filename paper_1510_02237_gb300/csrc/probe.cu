// probe.cu -- FMA throughput probe used as the ALU roofline denominator.
// Every thread runs 8 independent fused multiply-add chains; the grid fills
// every SM several times over.  Not part of the method.
#include "common.cuh"
#include "parareal.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T* out, int iters, T b, T c) {
    T a0 = (T)threadIdx.x * (T)1e-3, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
    T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            a0 = a0 * b + c; a1 = a1 * b + c; a2 = a2 * b + c; a3 = a3 * b + c;
            a4 = a4 * b + c; a5 = a5 * b + c; a6 = a6 * b + c; a7 = a7 * b + c;
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

template <typename T>
pr_status run_probe(int iters, double* flops_per_s) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PR_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PR_ECUDA;
    const int blocks = sms * 8, threads = 256;
    T* out = nullptr;
    if (cudaMalloc((void**)&out, sizeof(T) * blocks * threads) != cudaSuccess) return PR_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    pr_status st = PR_OK;
    float ms = 0.f;
    for (int rep = 0; rep < 2 && st == PR_OK; ++rep) {   // first run warms up
        cudaEventRecord(e0, 0);
        k_fma_probe<T><<<blocks, threads, 0, 0>>>(out, iters, (T)0.999999, (T)1e-7);
        pr::count_launches(1);
        cudaEventRecord(e1, 0);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) st = PR_ECUDA;
        cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (st == PR_OK) *flops_per_s = 2.0 * 8 * 4 * (double)iters * blocks * threads / (ms * 1e-3);
    return st;
}

}  // namespace

extern "C" pr_status parareal_alu_probe(int32_t prec, int32_t iters, double* flops_per_s) {
    if (!flops_per_s || iters < 1 || (prec != PR_FP64 && prec != PR_FP32)) return PR_EINVAL;
    return prec == PR_FP64 ? run_probe<double>(iters, flops_per_s) : run_probe<float>(iters, flops_per_s);
}

// ---------------------------------------------------------------- bounded-wait self-test
#include "grid_barrier.cuh"

namespace {

// Every CTA waits at a grid barrier that expects one CTA more than the grid
// has: the barrier can never complete, so each wait must give up after its
// poll limit, set the error word and return.
__global__ void k_wait_selftest(pr::GridBar* gb, unsigned expected) {
    pr::grid_barrier(gb, expected);
}

}  // namespace

extern "C" pr_status parareal_selftest_wait_timeout(void* stream, double* seconds) {
    pr::GridBar* gb = nullptr;
    if (cudaMalloc((void**)&gb, sizeof(pr::GridBar)) != cudaSuccess) return PR_ENOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    pr_status st = PR_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    if (cudaMemsetAsync(gb, 0, sizeof(pr::GridBar), s) != cudaSuccess) st = PR_ECUDA;
    if (st == PR_OK) {
        unsigned blocks = 2, expected = 3;
        void* args[] = {&gb, &expected};
        cudaEventRecord(e0, s);
        if (cudaLaunchCooperativeKernel((const void*)k_wait_selftest, dim3(blocks), dim3(32), args, 0, s) != cudaSuccess)
            st = PR_ECUDA;
        pr::count_launches(1);
        cudaEventRecord(e1, s);
    }
    int err = 0;
    if (st == PR_OK && cudaStreamSynchronize(s) != cudaSuccess) st = PR_ECUDA;
    if (st == PR_OK && cudaMemcpy(&err, &gb->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) st = PR_ECUDA;
    float ms = 0.f;
    if (st == PR_OK) cudaEventElapsedTime(&ms, e0, e1);
    if (seconds) *seconds = ms * 1e-3;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(gb);
    if (st != PR_OK) return st;
    return err ? PR_ETIMEOUT : PR_OK;
}
