// coarse.cu -- coarse propagator G over a batch of states: one launch per
// partially split forward-Euler coarse step (Sec. 3.2); the step itself is
// coarse_tile() (coarse_tile.cuh), one 32 x 16 tile per CTA, in FP64 or (for
// the mixed-precision solve) FP32 arithmetic with FP64 input and output.
#include "coarse_tile.cuh"

namespace pr {
namespace {

constexpr int CTX = 32, CTY = 16, CNT = 256;

template <typename T>
__global__ void __launch_bounds__(CNT) k_coarse_step(const double* __restrict__ in, double* __restrict__ out,
                                                     long stride, int nx, int ny, CoarseCoef c, int H, SliceMap map) {
    extern __shared__ __align__(16) unsigned char smc[];
    long zi = blockIdx.z, zo = blockIdx.z;
    if (map.end) {
        const int b0 = *map.beg;
        if ((int)blockIdx.z >= *map.end - b0) return;
        if (map.in_map) zi += b0;
        if (map.out_map) zo += b0;
    }
    coarse_tile<CTX, CTY, CNT, T>(in + zi * stride, out + zo * stride, nx, ny, c, H, blockIdx.x * CTX,
                                  blockIdx.y * CTY, reinterpret_cast<T*>(smc));
}

}  // namespace

int coarse_halo(const CoarseCoef& c) {
    const int r = c.order == 1 ? 1 : 2;
    return c.scheme == 1 ? 3 * r : r + 2 * c.n_sound - 1;
}

cudaError_t launch_coarse_step(const double* in, double* out, long stride, int n, int nx, int ny,
                               const CoarseCoef& c, cudaStream_t s, bool fp32, const SliceMap& map) {
    const int H = coarse_halo(c);
    if (H > COARSE_MAXH) return cudaErrorInvalidValue;
    dim3 grid((nx + CTX - 1) / CTX, (ny + CTY - 1) / CTY, n);
    const size_t elems = coarse_tile_smem_elems<CTX, CTY>(H);
    if (fp32) {
        const size_t smem = sizeof(float) * elems;
        cudaError_t e = cudaFuncSetAttribute(k_coarse_step<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_coarse_step<float><<<grid, CNT, smem, s>>>(in, out, stride, nx, ny, c, H, map);
    } else {
        const size_t smem = sizeof(double) * elems;
        cudaError_t e = cudaFuncSetAttribute(k_coarse_step<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_coarse_step<double><<<grid, CNT, smem, s>>>(in, out, stride, nx, ny, c, H, map);
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pr
