// Relative Poisson residual ||f - A_h u|| / ||f|| computed without any device
// allocation: its scratch (per-plane partial sums) lives in a file-scope
// device array that every GPU loading this library holds until the process
// exits.  Meant for callers that must not call cudaMalloc: code whose device
// memory is owned entirely by another allocator (a framework's caching pool
// or a fixed memory budget), and code on a latency-critical path where an
// allocation's implicit device synchronisation or possible failure under
// memory pressure is not acceptable.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "jacobi_internal.h"

namespace jac {
namespace {

constexpr int kMaxPlanes = JACOBI_NOALLOC_MAX_NZ;
constexpr int kThreads = 256;

// [0, kMaxPlanes): sum of r^2 of plane z; [kMaxPlanes, 2 kMaxPlanes): sum of
// f^2 of plane z; [2 kMaxPlanes], [2 kMaxPlanes + 1]: the two totals.
// Every element a call reads was written earlier in the same call, so
// nothing needs clearing between calls.
__device__ __align__(256) double g_noalloc_scratch[2 * kMaxPlanes + 2];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double sh[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) t = __dadd_rn(t, sh[w]);
    return t;
}

// Block z sums r^2 and f^2 over interior plane z+1 (fixed order).
__global__ void __launch_bounds__(kThreads) plane_sums_kernel(const double *u, const double *f, int nx, int ny,
                                                              double inv_h2, double *scratch)
{
    const long long NXP = nx + 2, plane = NXP * (ny + 2);
    const int z = blockIdx.x + 1;
    double rr = 0.0, ff = 0.0;
    for (int c = threadIdx.x; c < nx * ny; c += kThreads) {
        const long long i = z * plane + (long long)(c / nx + 1) * NXP + (c % nx + 1);
        double s = __dadd_rn(u[i - 1], u[i + 1]);
        s = __dadd_rn(s, u[i - NXP]);
        s = __dadd_rn(s, u[i + NXP]);
        s = __dadd_rn(s, u[i - plane]);
        s = __dadd_rn(s, u[i + plane]);
        const double au = __dmul_rn(__dsub_rn(__dmul_rn(6.0, u[i]), s), inv_h2);
        const double r = __dsub_rn(f[i], au);
        rr = __fma_rn(r, r, rr);
        ff = __fma_rn(f[i], f[i], ff);
    }
    const double tr = block_sum(rr);
    __syncthreads();
    const double tf = block_sum(ff);
    if (threadIdx.x == 0) {
        scratch[blockIdx.x] = tr;
        scratch[kMaxPlanes + blockIdx.x] = tf;
    }
}

__global__ void totals_kernel(int nz, double *scratch)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double r = 0.0, f = 0.0;
        for (int z = 0; z < nz; ++z) {
            r = __dadd_rn(r, scratch[z]);
            f = __dadd_rn(f, scratch[kMaxPlanes + z]);
        }
        scratch[2 * kMaxPlanes] = r;
        scratch[2 * kMaxPlanes + 1] = f;
    }
}

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
int scratch_address(double **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return JACOBI_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return JACOBI_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_ptr[dev]) {
        double *p = nullptr;
        if (cudaGetSymbolAddress((void **)&p, g_noalloc_scratch) != cudaSuccess) return JACOBI_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return JACOBI_OK;
}

}  // namespace
}  // namespace jac

extern "C" int jacobi_poisson_residual_noalloc(const void *u, const void *f, int nx, int ny, int nz, double hgrid,
                                               jacobi_stream_t stream, double *rel)
{
    if (!u || !f || !rel || !(hgrid > 0.0) || nx < 1 || ny < 1 || nz < 1) return JACOBI_ERR_ARG;
    if (nz > jac::kMaxPlanes || (long long)nx * ny > 2147483647ll) return JACOBI_ERR_ARG;
    double *scratch = nullptr;
    int st = jac::scratch_address(&scratch);
    if (st != JACOBI_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const double h2 = hgrid * hgrid;
    jac::plane_sums_kernel<<<nz, jac::kThreads, 0, s>>>(static_cast<const double *>(u),
                                                         static_cast<const double *>(f), nx, ny, 1.0 / h2, scratch);
    jac::totals_kernel<<<1, 32, 0, s>>>(nz, scratch);
    double tot[2] = {0.0, 0.0};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tot, scratch + 2 * jac::kMaxPlanes, sizeof(tot), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return JACOBI_ERR_CUDA;
    *rel = (tot[1] > 0.0) ? std::sqrt(tot[0]) / std::sqrt(tot[1]) : 0.0;
    return JACOBI_OK;
}
