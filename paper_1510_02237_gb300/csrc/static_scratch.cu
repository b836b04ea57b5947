// static_scratch.cu -- allocation-free fine sweep.
//
// Some callers cannot allocate device memory at the point where they need F:
// code running while a CUDA stream is being captured into a graph (where
// cudaMalloc is not allowed), runtimes that own all device memory through
// their own pool and forbid other allocations, and embedded or real-time
// hosts that may not allocate after start-up.  parareal_fine_sweep_static()
// serves them: it takes every input and output from the caller and keeps the
// ping-pong intermediates of the RK-3 steps in one file-scope device array,
// g_fine_scratch, instead of a handle's buffers.
//
// The array is 32 MiB, split into two halves of 16 MiB; every GPU on which
// the library's device code is loaded holds it until the process exits.
// Host code cannot use the array's name as a device address, so the first
// call on each device (with that device current) looks the address up with
// cudaGetSymbolAddress and caches it; make that first call before any stream
// capture begins.  Later calls outside capture look it up again (cheap).
// The sweep runs the shared-memory tile kernel, which has no device-side
// waits, so a call has no deferred error to report.  All calls share the
// array: calls whose work overlaps on the GPU (other streams, other host
// threads) race on it and must be serialised by the caller.  Nothing in it needs to start at zero --
// every step overwrites the whole part of the half it uses before reading it.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "common.cuh"
#include "parareal.h"

using namespace pr;

namespace {

constexpr size_t kHalfBytes = 16u << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_fine_scratch[2 * kHalfBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_fine_scratch on the current device.  Set up on the
// first call on each device; looked up again on every call made outside
// stream capture (cheap), so a module reloaded after cudaDeviceReset is
// followed; during capture the cached address is used.
pr_status scratch_for_current_device(cudaStream_t s, void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PR_ECUDA;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return PR_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev] || cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_fine_scratch);
        if (e != cudaSuccess || !p) {
            std::fprintf(stderr, "parareal_fine_sweep_static: cudaGetSymbolAddress failed: %s\n",
                         cudaGetErrorString(e));
            return PR_ECUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return PR_OK;
}

template <typename T>
FineCoef<T> coef(double U, double V, double cs, double dx, double dy, double nu, double dt) {
    const double a1 = nu * dx * dx / dt, a2 = nu * dy * dy / dt;
    FineCoef<T> c;
    c.ax6 = (T)(U / (60.0 * dx));
    c.ay6 = (T)(V / (60.0 * dy));
    c.csx = (T)(cs / (2.0 * dx));
    c.csy = (T)(cs / (2.0 * dy));
    c.dxx = (T)(a1 / (dx * dx));
    c.dxy1 = (T)(a1 / (4.0 * dx * dy));
    c.dyy = (T)(a2 / (dy * dy));
    c.dxy2 = (T)(a2 / (4.0 * dx * dy));
    c.c1 = (T)(dt / 3.0);
    c.c2 = (T)(dt / 2.0);
    c.c3 = (T)dt;
    return c;
}

pr_status reject(const char* msg) {
    std::fprintf(stderr, "parareal_fine_sweep_static: %s\n", msg);
    return PR_EINVAL;
}

template <typename T>
pr_status sweep(const double* in, double* out, int n, int nx, int ny, int nsteps, bool hv, const FineCoef<T>& c,
                unsigned char* scratch, cudaStream_t s) {
    const long d = 3L * nx * ny;
    // shared-memory tile kernel only: the row-streamed FP32 kernel's bounded
    // waits report through a process-wide word that this call cannot return
    FineLaunch fl;
    fl.rows = false;
    const SliceMap all;
    if (nsteps == 1)
        return launch_fine_step<T, double, double>(in, d, out, d, n, nx, ny, hv, c, s, all, fl) == cudaSuccess
                   ? PR_OK
                   : PR_ECUDA;
    T* a = reinterpret_cast<T*>(scratch);
    T* b = reinterpret_cast<T*>(scratch + kHalfBytes);
    if (launch_fine_step<T, double, T>(in, d, a, d, n, nx, ny, hv, c, s, all, fl) != cudaSuccess) return PR_ECUDA;
    for (int st = 1; st < nsteps - 1; ++st) {
        if (launch_fine_step<T, T, T>(a, d, b, d, n, nx, ny, hv, c, s, all, fl) != cudaSuccess) return PR_ECUDA;
        T* t = a;
        a = b;
        b = t;
    }
    return launch_fine_step<T, T, double>(a, d, out, d, n, nx, ny, hv, c, s, all, fl) == cudaSuccess ? PR_OK
                                                                                         : PR_ECUDA;
}

}  // namespace

extern "C" pr_status parareal_fine_sweep_static(const pr_grid* g, double U, double V, double c_s, double nu_f,
                                                double dt_f, int32_t n_steps, int32_t fine_prec,
                                                const double* q_in_dev, double* q_out_dev, int32_t n,
                                                void* stream) {
    if (!g || !q_in_dev || !q_out_dev) return reject("NULL argument");
    if (g->nx < 4 || g->ny < 4) return reject("nx and ny must be >= 4");
    if (n < 1 || n > 65535) return reject("n must be in [1, 65535]");
    if (n_steps < 1) return reject("n_steps must be >= 1");
    if (fine_prec != PR_FP64 && fine_prec != PR_FP32) return reject("fine_prec must be PR_FP64 or PR_FP32");
    if (!std::isfinite(U) || !std::isfinite(V) || !std::isfinite(c_s) || !std::isfinite(nu_f) || nu_f < 0 ||
        !(dt_f > 0) || !std::isfinite(dt_f))
        return reject("U, V, c_s, nu_f must be finite (nu_f >= 0) and dt_f > 0");
    const long d = 3L * g->nx * g->ny;
    const size_t elem = fine_prec == PR_FP64 ? sizeof(double) : sizeof(float);
    if ((double)n * (double)d * (double)elem > (double)kHalfBytes)
        return reject("n * 3 * nx * ny intermediate values exceed the 16 MiB static scratch half "
                      "(2097152 doubles or 4194304 floats)");
    cudaStream_t s = (cudaStream_t)stream;
    void* scratch = nullptr;
    pr_status st = scratch_for_current_device(s, &scratch);
    if (st != PR_OK) return st;
    const double lx = g->lx > 0 ? g->lx : 1.0, ly = g->ly > 0 ? g->ly : 1.0;
    const double dx = lx / g->nx, dy = ly / g->ny;
    const bool hv = V != 0.0;
    unsigned char* sc = static_cast<unsigned char*>(scratch);
    if (fine_prec == PR_FP64)
        return sweep<double>(q_in_dev, q_out_dev, n, g->nx, g->ny, n_steps, hv,
                             coef<double>(U, V, c_s, dx, dy, nu_f, dt_f), sc, s);
    return sweep<float>(q_in_dev, q_out_dev, n, g->nx, g->ny, n_steps, hv,
                        coef<float>(U, V, c_s, dx, dy, nu_f, dt_f), sc, s);
}
