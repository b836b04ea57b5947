// coarse.cu -- coarse propagator G over a batch of states: one launch per
// partially split forward-Euler coarse step (Sec. 3.2); the step itself is
// coarse_tile() (coarse_tile.cuh), one tile per CTA, in FP64 or (for the
// mixed-precision solve) FP32 arithmetic with FP64 input and output.
//
// The fused substeps recompute a halo of H cells around each tile, which
// costs 2.0x the tile's own work at 32 x 16 and 1.45x at 64 x 32.  Batches
// with enough 64 x 32 tiles to give every SM two take the large tile (one
// 512-thread CTA per SM in FP64: 11 % faster at 256 x 128 x 32, 21 % at
// 512 x 256 x 64); smaller batches keep 32 x 16 tiles, whose shorter
// per-tile latency matters more there.
#include "coarse_tile.cuh"

namespace pr {
namespace {

template <int TX, int TY, int NT, typename T>
__global__ void __launch_bounds__(NT) k_coarse_step(const double* __restrict__ in, double* __restrict__ out,
                                                    long stride, int nx, int ny, CoarseCoef c, int H, SliceMap map) {
    extern __shared__ __align__(16) unsigned char smc[];
    long zi = blockIdx.z, zo = blockIdx.z;
    if (map.end) {
        const int b0 = *map.beg;
        if ((int)blockIdx.z >= *map.end - b0) return;
        if (map.in_map) zi += b0;
        if (map.out_map) zo += b0;
    }
    coarse_tile<TX, TY, NT, T>(in + zi * stride, out + zo * stride, nx, ny, c, H, blockIdx.x * TX,
                               blockIdx.y * TY, reinterpret_cast<T*>(smc));
}

template <int TX, int TY, int NT, typename T>
cudaError_t launch_shape(const double* in, double* out, long stride, int n, int nx, int ny, const CoarseCoef& c,
                         int H, cudaStream_t s, const SliceMap& map) {
    const dim3 grid((nx + TX - 1) / TX, (ny + TY - 1) / TY, n);
    const size_t smem = sizeof(T) * coarse_tile_smem_elems<TX, TY>(H);
    std::lock_guard<std::mutex> lk(smem_launch_lock());
    cudaError_t e = set_dynamic_smem((const void*)k_coarse_step<TX, TY, NT, T>, smem);
    if (e != cudaSuccess) return e;
    k_coarse_step<TX, TY, NT, T><<<grid, NT, smem, s>>>(in, out, stride, nx, ny, c, H, map);
    count_launches(1);
    return cudaGetLastError();
}

// SMs and opt-in shared memory per block of the current device
bool device_limits(int* sms, int* smem_optin) {
    static DevMemo memo;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    if (memo.get(dev, sms, smem_optin)) return true;
    if (cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return false;
    memo.put(dev, *sms, *smem_optin);
    return true;
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
    int sms = 0, smem_optin = 0;
    if (!device_limits(&sms, &smem_optin)) return cudaErrorInvalidDevice;
    const long big_tiles = (long)((nx + 63) / 64) * ((ny + 31) / 32) * n;
    const size_t big_smem = (fp32 ? sizeof(float) : sizeof(double)) * coarse_tile_smem_elems<64, 32>(H);
    const bool big = big_tiles >= 2L * sms && big_smem <= (size_t)smem_optin;
    if (fp32)
        return big ? launch_shape<64, 32, 512, float>(in, out, stride, n, nx, ny, c, H, s, map)
                   : launch_shape<32, 16, 256, float>(in, out, stride, n, nx, ny, c, H, s, map);
    return big ? launch_shape<64, 32, 512, double>(in, out, stride, n, nx, ny, c, H, s, map)
               : launch_shape<32, 16, 256, double>(in, out, stride, n, nx, ny, c, H, s, map);
}

}  // namespace pr
