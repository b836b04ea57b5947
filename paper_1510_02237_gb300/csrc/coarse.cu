// coarse.cu -- coarse propagator G over a batch of states: one launch per
// partially split forward-Euler coarse step (Sec. 3.2); the step itself is
// coarse_tile() (coarse_tile.cuh), one 32 x 16 tile per CTA.
#include "coarse_tile.cuh"

namespace pr {
namespace {

constexpr int CTX = 32, CTY = 16, CNT = 256;

__global__ void __launch_bounds__(CNT) k_coarse_step(const double* __restrict__ in, double* __restrict__ out,
                                                     long stride, int nx, int ny, CoarseCoef c, int H) {
    extern __shared__ __align__(16) double sm[];
    coarse_tile<CTX, CTY, CNT>(in + (long)blockIdx.z * stride, out + (long)blockIdx.z * stride, nx, ny, c, H,
                               blockIdx.x * CTX, blockIdx.y * CTY, sm);
}

}  // namespace

int coarse_halo(const CoarseCoef& c) { return (c.order == 1 ? 1 : 2) + 2 * c.n_sound - 1; }

cudaError_t launch_coarse_step(const double* in, double* out, long stride, int n, int nx, int ny,
                               const CoarseCoef& c, cudaStream_t s) {
    const int H = coarse_halo(c);
    if (H > COARSE_MAXH) return cudaErrorInvalidValue;
    const size_t smem = sizeof(double) * coarse_tile_smem_doubles<CTX, CTY>(H);
    cudaError_t e = cudaFuncSetAttribute(k_coarse_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((nx + CTX - 1) / CTX, (ny + CTY - 1) / CTY, n);
    k_coarse_step<<<grid, CNT, smem, s>>>(in, out, stride, nx, ny, c, H);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pr
