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

// Device address of the scratch array in the current device's context.  It is
// looked up on every call (no allocation, a table lookup in the runtime):
// an address kept from an earlier call would go stale if the context were
// reset and the module loaded again.
int scratch_address(double **out)
{
    double *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return JACOBI_ERR_CUDA;
    *out = p;
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
    const double *pu = static_cast<const double *>(u), *pf = static_cast<const double *>(f);
    const double inv_h2 = 1.0 / h2;
    // Launched through cudaLaunchKernelEx so that each launch's own status is
    // checked (cudaGetLastError could report an unrelated earlier error).
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nz);
    cfg.blockDim = dim3(jac::kThreads);
    cfg.stream = s;
    cudaError_t e = cudaLaunchKernelEx(&cfg, jac::plane_sums_kernel, pu, pf, nx, ny, inv_h2, scratch);
    if (e == cudaSuccess) {
        cfg.gridDim = dim3(1);
        cfg.blockDim = dim3(32);
        e = cudaLaunchKernelEx(&cfg, jac::totals_kernel, nz, scratch);
    }
    double tot[2] = {0.0, 0.0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tot, scratch + 2 * jac::kMaxPlanes, sizeof(tot), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return JACOBI_ERR_CUDA;
    *rel = (tot[1] > 0.0) ? std::sqrt(tot[0]) / std::sqrt(tot[1]) : 0.0;
    return JACOBI_OK;
}
