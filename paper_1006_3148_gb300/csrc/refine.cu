// Poisson problem -Lap_h u = f (7-point Laplacian, Dirichlet halo) on top of
// the Jacobi sweeps:
//   jacobi_poisson_residual  r = f - A_h u and ||r||/||f|| in FP64
//   jacobi_poisson_jacobi    plain FP64 Jacobi with source term h^2 f
//   jacobi_refine            mixed-precision iterative refinement: FP64
//                            residual and update, FP32 inner Jacobi sweeps on
//                            the correction
// The inner sweeps (and the plain FP64 Jacobi) are single-pass sweep
// kernels with the source term, replayed from a CUDA graph of K sweeps: a
// small grid stays in L2 and each sweep costs one kernel, with no host
// launch per sweep.
// Sums of squares are reduced in a fixed order (per-thread grid-stride
// order, then a fixed tree per block, then the block partials in index
// order), so results do not depend on timing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "checked.cuh"
#include "jacobi_internal.h"

namespace jac {
namespace {

constexpr int kRedBlocks = 304;  // fixed reduction layout (2 x 152 SMs)
constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double sh[kRedThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kRedThreads / 32; ++w) t = __dadd_rn(t, sh[w]);
    return t;
}

// Interior cell c (0 <= c < nx*ny*nz, x fastest) -> array index.
__device__ __forceinline__ long long cell_index(long long c, int nx, int ny)
{
    const long long x = c % nx, y = (c / nx) % ny, z = c / ((long long)nx * ny);
    return ((z + 1) * (ny + 2) + (y + 1)) * (long long)(nx + 2) + (x + 1);
}

// partials[b] = sum of f^2 over the cells of block b.
__global__ void __launch_bounds__(kRedThreads) sumsq_kernel(const double *f, int nx, int ny, int nz,
                                                            double *partials, int *status, long long shrink)
{
    const long long n = (long long)nx * ny * nz;
    const long long S = checked_grid_elems(nx, ny, nz, shrink);
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)kRedThreads + threadIdx.x; c < n; c += (long long)kRedBlocks * kRedThreads) {
        const long long i = cell_index(c, nx, ny);
        const double v = in_bounds(i, 1, S, status) ? f[i] : 0.0;
        acc = __fma_rn(v, v, acc);
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// r = f - A_h u (A_h u = (6u - neighbour sum, order of Eq. 1) / h^2, the
// division replaced by the product with 1/h^2); optionally writes the
// source term of the correction, g = RN_f32(h^2 r); partial sums of r^2.
__global__ void __launch_bounds__(kRedThreads) residual_kernel(const double *u, const double *f, float *g, int nx,
                                                               int ny, int nz, double h2, double inv_h2,
                                                               double *partials, int *status, long long shrink)
{
    const long long n = (long long)nx * ny * nz;
    const long long NXP = nx + 2, plane = NXP * (ny + 2);
    const long long S = checked_grid_elems(nx, ny, nz, shrink);
    auto U = [&](long long i) { return in_bounds(i, 1, S, status) ? u[i] : 0.0; };
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)kRedThreads + threadIdx.x; c < n; c += (long long)kRedBlocks * kRedThreads) {
        const long long i = cell_index(c, nx, ny);
        double s = __dadd_rn(U(i - 1), U(i + 1));
        s = __dadd_rn(s, U(i - NXP));
        s = __dadd_rn(s, U(i + NXP));
        s = __dadd_rn(s, U(i - plane));
        s = __dadd_rn(s, U(i + plane));
        const double au = __dmul_rn(__dsub_rn(__dmul_rn(6.0, U(i)), s), inv_h2);
        const double r = __dsub_rn(in_bounds(i, 1, S, status) ? f[i] : 0.0, au);
        if (g && in_bounds(i, 1, S, status)) g[i] = __double2float_rn(__dmul_rn(h2, r));
        acc = __fma_rn(r, r, acc);
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void reduce_partials_kernel(const double *partials, int n, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < n; ++b) t = __dadd_rn(t, partials[b]);
        *out = t;
    }
}

// u += (double) e on the interior.
__global__ void update_kernel(double *u, const float *e, int nx, int ny, int nz, int *status, long long shrink)
{
    const long long n = (long long)nx * ny * nz;
    const long long S = checked_grid_elems(nx, ny, nz, shrink);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const long long i = cell_index(c, nx, ny);
        if (in_bounds(i, 1, S, status)) u[i] = __dadd_rn(u[i], (double)e[i]);
    }
}

// g = h^2 f (FP64) on the interior.
__global__ void scale_kernel(const double *f, double *g, double h2, int nx, int ny, int nz, int *status,
                             long long shrink)
{
    const long long n = (long long)nx * ny * nz;
    const long long S = checked_grid_elems(nx, ny, nz, shrink);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const long long i = cell_index(c, nx, ny);
        if (in_bounds(i, 1, S, status)) g[i] = __dmul_rn(h2, f[i]);
    }
}

size_t cells(const jacobi_plan_s *h) { return (size_t)(h->nx + 2) * (h->ny + 2) * (size_t)(h->nz + 2); }

int ensure_common(jacobi_plan_s *h)
{
    if (!h->partials && cudaMalloc(&h->partials, sizeof(double) * (kRedBlocks + 1)) != cudaSuccess)
        return JACOBI_ERR_ALLOC;
    if (!h->h_sum && cudaMallocHost(&h->h_sum, sizeof(double)) != cudaSuccess) return JACOBI_ERR_ALLOC;
    return JACOBI_OK;
}

// Launch shape of the single-pass sweep kernel for this grid: two x cells
// per thread for FP32 grids of even nx (the FP64 form gains nothing on an
// FP64-pipe-bound sweep), 32 x 8 threads, and the most planes per thread
// (8, 4, 2, 1) that still leaves about two waves of 2048 threads per SM.
PlainArgs inner_args(const jacobi_plan_s *h, int dtype, const void *rhs, bool *x2)
{
    PlainArgs a;
    a.nx = h->nx;
    a.ny = h->ny;
    a.nz = h->nz;
    a.rhs = rhs;
    a.tx = 32;
    a.ty = 8;
    a.status = h->d_status;
    a.shrink = h->check_shrink;
    *x2 = (dtype == JACOBI_F32 && h->nx % 2 == 0);
    const long long row = *x2 ? 32ll * (((h->nx + 2) / 2 + 31) / 32) : 32ll * ((h->nx + 31) / 32);
    const long long want = 2ll * std::max(h->sms, 1) * 2048;
    a.kz = 1;
    for (int kz : {8, 4, 2}) {
        if (row * h->ny * ((h->nz + kz - 1) / kz) >= want) {
            a.kz = kz;
            break;
        }
    }
    return a;
}

cudaError_t sweep_once(const jacobi_plan_s *h, int dtype, PlainArgs a, bool x2, const void *src, void *dst,
                       cudaStream_t s)
{
    a.src = src;
    a.dst = dst;
    return x2 ? plain_x2_launch(dtype, a, s) : plain_launch(dtype, a, s);
}

// A graph of K sweeps A -> B -> A ... with source term G, cached on the
// handle by (dtype, K, A, B, G).  K is even, so the graph leaves its result
// in A and can be replayed.
int ensure_inner(jacobi_plan_s *h, int dtype, int K, void *A, void *B, const void *G)
{
    if (h->inner_exec && h->inner_dtype == dtype && h->inner_K == K && h->inner_A == A && h->inner_B == B &&
        h->inner_G == G)
        return JACOBI_OK;
    if (h->inner_exec) cudaGraphExecDestroy(h->inner_exec);
    h->inner_exec = nullptr;
    bool x2 = false;
    const PlainArgs a = inner_args(h, dtype, G, &x2);
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return JACOBI_ERR_CUDA;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int t = 0; t < K; ++t) {
            const cudaError_t le = sweep_once(h, dtype, a, x2, (t % 2 == 0) ? A : B, (t % 2 == 0) ? B : A, cs);
            if (le != cudaSuccess && e == cudaSuccess) e = le;
        }
        const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = ce;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->inner_exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        h->inner_exec = nullptr;
        return JACOBI_ERR_CUDA;
    }
    h->inner_dtype = dtype;
    h->inner_K = K;
    h->inner_A = A;
    h->inner_B = B;
    h->inner_G = G;
    return JACOBI_OK;
}

// T sweeps A -> B -> ... with source term G on stream s (halos of A and B
// already equal): ceil(T/512) replays of a graph of K ~ T/ceil(T/512) sweeps
// (K even), then the few remaining sweeps launched one by one.  The result
// is in B if T is odd, else in A.
int run_inner(jacobi_plan_s *h, int dtype, int T, void *A, void *B, const void *G, cudaStream_t s)
{
    const int K = (T / ((T + 511) / 512)) & ~1;
    int done = 0;
    if (K >= 2) {
        const int st = ensure_inner(h, dtype, K, A, B, G);
        if (st != JACOBI_OK) return st;
        for (; done + K <= T; done += K)
            if (cudaGraphLaunch(h->inner_exec, s) != cudaSuccess) return JACOBI_ERR_CUDA;
    }
    bool x2 = false;
    const PlainArgs a = inner_args(h, dtype, G, &x2);
    for (int t = done; t < T; ++t)
        if (sweep_once(h, dtype, a, x2, (t % 2 == 0) ? A : B, (t % 2 == 0) ? B : A, s) != cudaSuccess)
            return JACOBI_ERR_CUDA;
    if (h->prof) h->prof_other += T;
    return JACOBI_OK;
}

// sqrt of the reduced sum of squares, read back to the host.
int read_norm(jacobi_plan_s *h, cudaStream_t s, double *out)
{
    reduce_partials_kernel<<<1, 32, 0, s>>>(h->partials, kRedBlocks, h->partials + kRedBlocks);
    if (h->prof) h->prof_other += 1;
    cudaError_t e = cudaMemcpyAsync(h->h_sum, h->partials + kRedBlocks, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return JACOBI_ERR_CUDA;
    *out = std::sqrt(*h->h_sum);
    return JACOBI_OK;
}

int residual_norm(jacobi_plan_s *h, const double *u, const double *f, float *g, double hgrid, cudaStream_t s,
                  double *rnorm)
{
    const double h2 = hgrid * hgrid;
    residual_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(u, f, g, h->nx, h->ny, h->nz, h2, 1.0 / h2, h->partials,
                                                       h->d_status, h->check_shrink);
    if (cudaGetLastError() != cudaSuccess) return JACOBI_ERR_CUDA;
    if (h->prof) h->prof_other += 1;
    return read_norm(h, s, rnorm);
}

int f_norm(jacobi_plan_s *h, const double *f, cudaStream_t s, double *fnorm)
{
    sumsq_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(f, h->nx, h->ny, h->nz, h->partials, h->d_status,
                                                    h->check_shrink);
    if (cudaGetLastError() != cudaSuccess) return JACOBI_ERR_CUDA;
    if (h->prof) h->prof_other += 1;
    return read_norm(h, s, fnorm);
}

}  // namespace

void free_poisson_scratch(jacobi_plan_s *h)
{
    if (h->g) cudaFree(h->g);
    if (h->e0) cudaFree(h->e0);
    if (h->e1) cudaFree(h->e1);
    if (h->partials) cudaFree(h->partials);
    if (h->h_sum) cudaFreeHost(h->h_sum);
    if (h->inner_exec) cudaGraphExecDestroy(h->inner_exec);
    h->g = h->e0 = h->e1 = nullptr;
    h->partials = nullptr;
    h->h_sum = nullptr;
    h->inner_exec = nullptr;
}

}  // namespace jac

using namespace jac;

extern "C" {

int jacobi_poisson_residual(jacobi_h h, const void *u, const void *f, double hgrid, jacobi_stream_t stream,
                            double *rel)
{
    if (!h || !u || !f || !rel || !(hgrid > 0.0)) return JACOBI_ERR_ARG;
    if (h->dtype != JACOBI_F64) return JACOBI_ERR_DTYPE;
    int st = ensure_common(h);
    if (st != JACOBI_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    double fn = 0.0, rn = 0.0;
    st = f_norm(h, static_cast<const double *>(f), s, &fn);
    if (st == JACOBI_OK) st = residual_norm(h, static_cast<const double *>(u), static_cast<const double *>(f), nullptr,
                                            hgrid, s, &rn);
    if (st != JACOBI_OK) return st;
    *rel = (fn > 0.0) ? rn / fn : 0.0;
    return JACOBI_OK;
}

int jacobi_poisson_jacobi(jacobi_h h, void *u, void *tmp, const void *f, double hgrid, int sweeps,
                          jacobi_stream_t stream)
{
    if (!h || !u || !tmp || !f || u == tmp || sweeps < 0 || !(hgrid > 0.0)) return JACOBI_ERR_ARG;
    if (h->dtype != JACOBI_F64) return JACOBI_ERR_DTYPE;
    if (sweeps == 0) return JACOBI_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (!h->g && cudaMalloc(&h->g, cells(h) * sizeof(double)) != cudaSuccess) return JACOBI_ERR_ALLOC;
    scale_kernel<<<608, 256, 0, s>>>(static_cast<const double *>(f), static_cast<double *>(h->g), hgrid * hgrid,
                                     h->nx, h->ny, h->nz, h->d_status, h->check_shrink);
    if (cudaGetLastError() != cudaSuccess) return JACOBI_ERR_CUDA;
    if (halo_copy_launch(JACOBI_F64, u, tmp, h->nx, h->ny, h->nz, s, h->d_status, h->check_shrink) != cudaSuccess)
        return JACOBI_ERR_CUDA;
    if (h->prof) h->prof_other += 2;  // scale, halo copy
    return run_inner(h, JACOBI_F64, sweeps, u, tmp, h->g, s);
}

int jacobi_refine(jacobi_h h, double *u, const double *f, double hgrid, double rel_tol, int inner_sweeps,
                  int max_outer, jacobi_stream_t stream, int *outer_done, double *final_rel_residual)
{
    if (!h || !u || !f || !(hgrid > 0.0) || !(rel_tol >= 0.0) || inner_sweeps < 1 || max_outer < 0)
        return JACOBI_ERR_ARG;
    if (h->dtype != JACOBI_F64) return JACOBI_ERR_DTYPE;
    cudaStream_t s = (cudaStream_t)stream;
    int st = ensure_common(h);
    if (st != JACOBI_OK) return st;
    const size_t n = cells(h);
    // h->g holds either FP32 h^2 r (here) or FP64 h^2 f (plain solver); it
    // is sized for FP64 and rewritten before every use
    if (!h->g && cudaMalloc(&h->g, n * sizeof(double)) != cudaSuccess) return JACOBI_ERR_ALLOC;
    if (!h->e0 && cudaMalloc(&h->e0, n * sizeof(float)) != cudaSuccess) return JACOBI_ERR_ALLOC;
    if (!h->e1 && cudaMalloc(&h->e1, n * sizeof(float)) != cudaSuccess) return JACOBI_ERR_ALLOC;

    double fn = 0.0;
    st = f_norm(h, f, s, &fn);
    if (st != JACOBI_OK) return st;
    int outer = 0;
    double rel = 0.0;
    for (;;) {
        double rn = 0.0;
        st = residual_norm(h, u, f, static_cast<float *>(h->g), hgrid, s, &rn);
        if (st != JACOBI_OK) return st;
        rel = (fn > 0.0) ? rn / fn : 0.0;
        if (rel <= rel_tol || outer >= max_outer) break;
        if (cudaMemsetAsync(h->e0, 0, n * sizeof(float), s) != cudaSuccess) return JACOBI_ERR_CUDA;
        if (cudaMemsetAsync(h->e1, 0, n * sizeof(float), s) != cudaSuccess) return JACOBI_ERR_CUDA;
        // zero correction and zero halo, then the FP32 sweeps on it
        st = run_inner(h, JACOBI_F32, inner_sweeps, h->e0, h->e1, h->g, s);
        if (st != JACOBI_OK) return st;
        const float *e = static_cast<const float *>((inner_sweeps % 2 == 0) ? h->e0 : h->e1);
        update_kernel<<<608, 256, 0, s>>>(u, e, h->nx, h->ny, h->nz, h->d_status, h->check_shrink);
        if (cudaGetLastError() != cudaSuccess) return JACOBI_ERR_CUDA;
        if (h->prof) h->prof_other += 1;  // update
        ++outer;
    }
    if (outer_done) *outer_done = outer;
    if (final_rel_residual) *final_rel_residual = rel;
    return rel <= rel_tol ? JACOBI_OK : JACOBI_ERR_NOT_CONVERGED;
}

}  // extern "C"
