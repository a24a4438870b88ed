// C ABI of libjacobi.so: handles, validation, pass planning, plan choice and
// the autotuner.  Every device step is a kernel of this library; there is no
// host or library fallback for any part of a sweep.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "checked.cuh"
#include "jacobi_internal.h"

using namespace jac;

namespace {

thread_local std::string g_last_cuda;

int cuda_fail(cudaError_t e)
{
    g_last_cuda = cudaGetErrorString(e);
    return JACOBI_ERR_CUDA;
}

size_t elem_size(int dtype) { return dtype == JACOBI_F64 ? 8 : 4; }

size_t grid_elems(const jacobi_plan_s *h)
{
    return (size_t)(h->nx + 2) * (size_t)(h->ny + 2) * (size_t)(h->nz + 2);
}

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, Plan> g_tune_cache;

// Plan of a handle that was neither tuned nor forced: the kernel families the
// tuner measured fastest on this GPU at large sizes.  FP64: the single-pass
// kernel (the FP64 sweep is bound by the FP64 pipe, so temporal blocking
// only adds redundant work); FP32: the register-blocked one-CTA kernel at
// depth 3 on 64 x 32 regions.  z chunks are clamped to the grid.
Plan default_plan(const jacobi_plan_s *h)
{
    Plan p;
    if (h->dtype == JACOBI_F64) {
        p.kernel = JACOBI_KERNEL_PLAIN;
        p.depth = 1;
        p.bx = 64;
        p.by = 4;
        p.bz = 4;
        return p;
    }
    p.kernel = JACOBI_KERNEL_TB_REG;
    p.depth = 3;
    p.bx = 64;
    p.by = 32;
    p.bz = std::min(128, h->nz);
    p.threads = 128;
    return p;
}

Plan active_plan(const jacobi_plan_s *h)
{
    if (h->forced) return h->plan;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(std::make_tuple(h->dtype, h->nx, h->ny, h->nz, h->sms));
        if (it != g_tune_cache.end()) return it->second;
    }
    return default_plan(h);
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Records a profiling event on s (when profiling is on); false on failure.
bool prof_event(jacobi_plan_s *h, cudaStream_t s)
{
    if (!h->prof) return true;
    if (h->ev_used == h->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return false;
        h->ev_pool.push_back(e);
    }
    return cudaEventRecord(h->ev_pool[h->ev_used++], s) == cudaSuccess;
}

// Replaces zero tile fields of a forced plan by the kernel family's defaults
// (PLAIN: 32 x 8 threads, 8 planes per thread; PLAIN_X2: 32 x 8 threads,
// 16 planes; TB: 64 x 16 tile, 64 planes; TB_CTA: 64 x 32 tile, 64 planes,
// 512 threads).
Plan resolve_plan(const jacobi_plan_s *h, Plan p)
{
    const bool plain = p.kernel == JACOBI_KERNEL_PLAIN || p.kernel == JACOBI_KERNEL_PLAIN_X2;
    if (p.kernel == JACOBI_KERNEL_TB_REG || p.kernel == JACOBI_KERNEL_TB_CHAIN) {
        const bool chain = p.kernel == JACOBI_KERNEL_TB_CHAIN;
        if (p.bx == 0) p.bx = 64;
        if (p.by == 0) p.by = chain ? 64 : 32;
        if (p.bz == 0) p.bz = std::min(64, h->nz);
        if (!chain) p.ring = 0;
        else if (p.ring == 0) p.ring = 2;
        p.threads = p.bx * p.by / 16;
        return p;
    }
    if (p.bx == 0) p.bx = plain ? 32 : std::min(64, h->nx);
    if (p.by == 0) p.by = plain ? 8 : std::min(p.kernel == JACOBI_KERNEL_TB_CTA ? 32 : 16, h->ny);
    if (p.bz == 0) p.bz = plain ? (p.kernel == JACOBI_KERNEL_PLAIN_X2 ? 16 : 8) : std::min(64, h->nz);
    if (p.kernel == JACOBI_KERNEL_TB_CTA && p.threads == 0) p.threads = 512;
    return p;
}

int check_plan(const jacobi_plan_s *h, const Plan &p)
{
    if (p.kernel == JACOBI_KERNEL_PLAIN_X2 && h->nx % 2 != 0)
        return JACOBI_ERR_UNSUPPORTED;
    if (p.kernel == JACOBI_KERNEL_PLAIN || p.kernel == JACOBI_KERNEL_PLAIN_X2) {
        if (p.bx < 32 || p.bx % 32 != 0 || p.by < 1 || (long long)p.bx * p.by > 1024 || p.bz < 1)
            return JACOBI_ERR_ARG;
        // (row block, z chunk) pairs must fit grid y * grid z
        const long long pairs = (long long)((h->ny + p.by - 1) / p.by) * ((h->nz + p.bz - 1) / p.bz);
        return pairs <= 65535ll * 65535ll ? JACOBI_OK : JACOBI_ERR_UNSUPPORTED;
    }
    if (p.kernel == JACOBI_KERNEL_TB_CHAIN) {
        if (p.depth < 2 || p.depth > 16 || p.bz < 1 || p.ring < 2 || p.ring > 4) return JACOBI_ERR_ARG;
        TbxArgs a;
        a.nx = h->nx;
        a.ny = h->ny;
        a.nz = h->nz;
        a.bz = p.bz;
        size_t smem = 0;
        const int st = tbx_configure(p.depth, p.ring, p.bx, p.by, &a, &smem);
        if (st != JACOBI_OK) return st;
        if (h->dtype != JACOBI_F32) return JACOBI_ERR_UNSUPPORTED;
        int clusters = 0;
        if (tbx_max_clusters(p.depth, p.ring, p.bx, p.by, h->nx, &clusters) != cudaSuccess) {
            cudaGetLastError();
            return JACOBI_ERR_UNSUPPORTED;
        }
        // passes of depth below the chain length run on the one-CTA kernel
        TbrArgs b;
        b.nx = h->nx;
        b.ny = h->ny;
        b.nz = h->nz;
        b.bz = p.bz;
        for (int d = 1; d < p.ring; ++d)
            if (tbr_configure(d, p.bx, p.by, &b, &smem, nullptr) != JACOBI_OK) return JACOBI_ERR_UNSUPPORTED;
        return clusters > 0 ? JACOBI_OK : JACOBI_ERR_UNSUPPORTED;
    }
    if (p.kernel == JACOBI_KERNEL_TB_REG) {
        if (p.depth < 1 || p.depth > 4 || p.bz < 1) return JACOBI_ERR_ARG;
        TbrArgs a;
        a.nx = h->nx;
        a.ny = h->ny;
        a.nz = h->nz;
        a.bz = p.bz;
        size_t smem = 0;
        const int st = tbr_configure(p.depth, p.bx, p.by, &a, &smem, nullptr);
        if (st != JACOBI_OK) return st;
        return h->dtype == JACOBI_F32 ? JACOBI_OK : JACOBI_ERR_UNSUPPORTED;
    }
    if (p.kernel == JACOBI_KERNEL_TB_CTA) {
        if (p.depth < 1 || p.depth > 4 || p.bx < 1 || p.by < 1 || p.bz < 1) return JACOBI_ERR_ARG;
        if (p.threads != 256 && p.threads != 512) return JACOBI_ERR_ARG;
        TbcArgs a;
        a.nx = h->nx;
        a.ny = h->ny;
        a.nz = h->nz;
        size_t smem = 0;
        const int st = tbc_configure(h->dtype, p.depth, p.bx, p.by, p.threads, &a, &smem);
        if (st != JACOBI_OK) return st;
        if ((h->ny + p.by - 1) / p.by > 65535 || (h->nz + p.bz - 1) / p.bz > 65535) return JACOBI_ERR_UNSUPPORTED;
        return JACOBI_OK;
    }
    if (p.kernel != JACOBI_KERNEL_TB) return JACOBI_ERR_ARG;
    if (p.depth < 1 || p.depth > 16 || p.bx < 1 || p.by < 1 || p.bz < 1) return JACOBI_ERR_ARG;
    if (p.ring != 0 && p.ring != 4 && p.ring != 8 && p.ring != 16) return JACOBI_ERR_ARG;
    if (p.threads != 0 && p.threads != 128 && p.threads != 256 && p.threads != 512) return JACOBI_ERR_ARG;
    TbLaunch L;
    if (tb_configure(h->dtype, p.depth, p.bx, p.by, p.ring, p.threads, &L) != cudaSuccess) return JACOBI_ERR_UNSUPPORTED;
    int clusters = 0;
    cudaError_t e = tb_max_clusters(h->dtype, L, p.depth, &clusters);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return JACOBI_ERR_UNSUPPORTED;
    }
    return clusters > 0 ? JACOBI_OK : JACOBI_ERR_UNSUPPORTED;
}

// Runs T sweeps with plan p; no argument checks.
int run_sweeps(jacobi_plan_s *h, const Plan &p, void *A, void *B, int T, cudaStream_t s)
{
    if (T == 0) return JACOBI_OK;
    cudaError_t e = halo_copy_launch(h->dtype, A, B, h->nx, h->ny, h->nz, s, h->d_status, h->check_shrink);
    if (e != cudaSuccess) return cuda_fail(e);
    if (h->prof) ++h->prof_other;
    if (p.kernel == JACOBI_KERNEL_PLAIN || p.kernel == JACOBI_KERNEL_PLAIN_X2) {
        PlainArgs a;
        a.nx = h->nx;
        a.ny = h->ny;
        a.nz = h->nz;
        a.kz = p.bz;
        a.tx = p.bx;
        a.ty = p.by;
        a.status = h->d_status;
        a.shrink = h->check_shrink;
        for (int t = 0; t < T; ++t) {
            a.src = (t % 2 == 0) ? A : B;
            a.dst = (t % 2 == 0) ? B : A;
            if (!prof_event(h, s)) return JACOBI_ERR_CUDA;
            e = (p.kernel == JACOBI_KERNEL_PLAIN_X2) ? plain_x2_launch(h->dtype, a, s) : plain_launch(h->dtype, a, s);
            if (e != cudaSuccess) return cuda_fail(e);
            if (!prof_event(h, s)) return JACOBI_ERR_CUDA;
            if (h->prof) ++h->prof_pass;
        }
        return JACOBI_OK;
    }
    std::vector<int> depths((size_t)T + 1);
    const int P = plan_passes(T, p.depth, depths.data(), T + 1);
    if (P < 0) return JACOBI_ERR_ARG;
    if (p.kernel == JACOBI_KERNEL_TB_REG || p.kernel == JACOBI_KERNEL_TB_CHAIN) {
        const bool chain = p.kernel == JACOBI_KERNEL_TB_CHAIN;
        TbrArgs a;
        a.nx = h->nx;
        a.ny = h->ny;
        a.nz = h->nz;
        a.bz = p.bz;
        a.status = h->d_status;
        a.shrink = h->check_shrink;
        TbxArgs c;
        c.nx = h->nx;
        c.ny = h->ny;
        c.nz = h->nz;
        c.bz = p.bz;
        c.status = h->d_status;
        c.shrink = h->check_shrink;
        c.limit_ns = h->limit_ns;
        for (int q = 0; q < P; ++q) {
            if (!prof_event(h, s)) return JACOBI_ERR_CUDA;
            a.src = c.src = (q % 2 == 0) ? A : B;
            a.dst = c.dst = (q % 2 == 0) ? B : A;
            if (chain && depths[q] >= p.ring) {
                c.fault_mode = h->fault_mode;
                h->fault_mode = 0;
                e = tbx_launch(depths[q], p.ring, p.bx, p.by, c, s);
            } else {
                e = tbr_launch(depths[q], p.bx, p.by, a, s);
            }
            if (e != cudaSuccess) return cuda_fail(e);
            if (!prof_event(h, s)) return JACOBI_ERR_CUDA;
            if (h->prof) ++h->prof_pass;
        }
        return JACOBI_OK;
    }
    if (p.kernel == JACOBI_KERNEL_TB_CTA) {
        TbcArgs a;
        a.nx = h->nx;
        a.ny = h->ny;
        a.nz = h->nz;
        a.bz = p.bz;
        a.status = h->d_status;
        a.shrink = h->check_shrink;
        for (int q = 0; q < P; ++q) {
            if (!prof_event(h, s)) return JACOBI_ERR_CUDA;
            size_t smem = 0;
            if (tbc_configure(h->dtype, depths[q], p.bx, p.by, p.threads, &a, &smem) != JACOBI_OK)
                return JACOBI_ERR_UNSUPPORTED;
            a.src = (q % 2 == 0) ? A : B;
            a.dst = (q % 2 == 0) ? B : A;
            e = tbc_launch(h->dtype, depths[q], p.threads, a, s);
            if (e != cudaSuccess) return cuda_fail(e);
            if (!prof_event(h, s)) return JACOBI_ERR_CUDA;
            if (h->prof) ++h->prof_pass;
        }
        return JACOBI_OK;
    }
    TbArgs a;
    a.nx = h->nx;
    a.ny = h->ny;
    a.nz = h->nz;
    a.bx = p.bx;
    a.by = p.by;
    a.bz = p.bz;
    a.ntx = (h->nx + p.bx - 1) / p.bx;
    a.status = h->d_status;
    a.limit_ns = h->limit_ns;
    a.shrink = h->check_shrink;
    TbLaunch L;
    int Ldepth = -1;
    for (int q = 0; q < P; ++q) {
        if (depths[q] != Ldepth) {
            if (tb_configure(h->dtype, depths[q], p.bx, p.by, p.ring, p.threads, &L) != cudaSuccess) return JACOBI_ERR_UNSUPPORTED;
            Ldepth = depths[q];
        }
        a.depth = depths[q];
        a.W = L.W;
        a.H = L.H;
        a.Wp = L.Wp;
        a.R = L.R;
        a.rshift = (L.R == 16) ? 4 : (L.R == 8 ? 3 : 2);
        a.src = (q % 2 == 0) ? A : B;
        a.dst = (q % 2 == 0) ? B : A;
        a.fault_mode = h->fault_mode;
        h->fault_mode = 0;
        if (!prof_event(h, s)) return JACOBI_ERR_CUDA;
        e = tb_launch(h->dtype, a, L, s);
        if (e != cudaSuccess) return cuda_fail(e);
        if (!prof_event(h, s)) return JACOBI_ERR_CUDA;
        if (h->prof) ++h->prof_pass;
    }
    return JACOBI_OK;
}

}  // namespace

namespace jac {
namespace {
std::mutex g_attr_mu;
std::map<std::pair<const void *, int>, size_t> g_smem_set;  // (kernel, device) -> limit set
std::map<std::pair<const void *, int>, int> g_cluster_set;   // (kernel, device) -> smem_max set
}  // namespace

cudaError_t ensure_smem_limit(const void *fn, size_t smem)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_attr_mu);
    size_t &cur = g_smem_set[std::make_pair(fn, dev)];
    if (smem <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) cur = smem;
    return e;
}

cudaError_t ensure_cluster_attrs(const void *fn, int smem_max)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_attr_mu);
    int &cur = g_cluster_set[std::make_pair(fn, dev)];
    if (cur >= smem_max) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) cur = smem_max;
    return e;
}
}  // namespace jac

extern "C" {

const char *jacobi_status_string(int status)
{
    switch (status) {
    case JACOBI_OK: return "ok";
    case JACOBI_ERR_ARG: return "invalid argument";
    case JACOBI_ERR_DTYPE: return "unsupported dtype";
    case JACOBI_ERR_ALLOC: return "allocation failed";
    case JACOBI_ERR_CUDA: return "CUDA error";
    case JACOBI_ERR_TIMEOUT: return "device-side wait timed out";
    case JACOBI_ERR_BOUNDS: return "device-side bounds check failed";
    case JACOBI_ERR_NOT_CONVERGED: return "not converged";
    case JACOBI_ERR_ALIGN: return "grid pointer not 16-byte aligned";
    case JACOBI_ERR_UNSUPPORTED: return "plan not launchable on this device";
    default: return "unknown status";
    }
}

int jacobi_version(void) { return 10000; }

const char *jacobi_last_cuda_error(void) { return g_last_cuda.c_str(); }

int jacobi_create(jacobi_h *out, int nx, int ny, int nz, int dtype)
{
    if (!out) return JACOBI_ERR_ARG;
    *out = nullptr;
    if (dtype != JACOBI_F64 && dtype != JACOBI_F32) return JACOBI_ERR_DTYPE;
    if (nx < 1 || ny < 1 || nz < 1) return JACOBI_ERR_ARG;
    const double cells = (double)(nx + 2) * (ny + 2) * (double)(nz + 2);
    if (cells >= 1099511627776.0 || (double)(nx + 2) * (ny + 2) >= 2147483647.0 || ny > 65535 * 8 ||
        nz > 65535 * 8)
        return JACOBI_ERR_ARG;
    jacobi_plan_s *h = new (std::nothrow) jacobi_plan_s;
    if (!h) return JACOBI_ERR_ALLOC;
    h->nx = nx;
    h->ny = ny;
    h->nz = nz;
    h->dtype = dtype;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e);
    }
    e = cudaMalloc(&h->d_status, sizeof(int));
    if (e != cudaSuccess) {
        delete h;
        g_last_cuda = cudaGetErrorString(e);
        return JACOBI_ERR_ALLOC;
    }
    e = cudaMemset(h->d_status, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(h->d_status);
        delete h;
        return cuda_fail(e);
    }
    h->plan = default_plan(h);
    *out = h;
    return JACOBI_OK;
}

int jacobi_destroy(jacobi_h h)
{
    if (!h) return JACOBI_OK;
    if (h->d_status) cudaFree(h->d_status);
    if (h->hostA) cudaFree(h->hostA);
    if (h->hostB) cudaFree(h->hostB);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    if (h->cg_ctl) cudaFree(h->cg_ctl);
    for (int *p : h->cg_old) cudaFree(p);
    free_poisson_scratch(h);
    delete h;
    return JACOBI_OK;
}

int jacobi_sweep(jacobi_h h, void *A, void *B, int T, jacobi_stream_t stream)
{
    if (!h || !A || !B || T < 0 || A == B) return JACOBI_ERR_ARG;
    if (!aligned16(A) || !aligned16(B)) return JACOBI_ERR_ALIGN;
    const size_t bytes = grid_elems(h) * elem_size(h->dtype);
    const char *a = (const char *)A, *b = (const char *)B;
    if (a < b + bytes && b < a + bytes) return JACOBI_ERR_ARG;
    return run_sweeps(h, active_plan(h), A, B, T, (cudaStream_t)stream);
}

int jacobi_sweep_host(jacobi_h h, const void *A_host, void *out_host, int T, jacobi_stream_t stream)
{
    if (!h || !A_host || !out_host || T < 0) return JACOBI_ERR_ARG;
    const size_t bytes = grid_elems(h) * elem_size(h->dtype);
    cudaError_t e;
    if (!h->hostA) {
        e = cudaMalloc(&h->hostA, bytes);
        if (e != cudaSuccess) return g_last_cuda = cudaGetErrorString(e), JACOBI_ERR_ALLOC;
        e = cudaMalloc(&h->hostB, bytes);
        if (e != cudaSuccess) {
            cudaFree(h->hostA);
            h->hostA = nullptr;
            g_last_cuda = cudaGetErrorString(e);
            return JACOBI_ERR_ALLOC;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemcpyAsync(h->hostA, A_host, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e);
    int st = run_sweeps(h, active_plan(h), h->hostA, h->hostB, T, s);
    if (st != JACOBI_OK) return st;
    e = cudaMemcpyAsync(out_host, (T % 2 == 0) ? h->hostA : h->hostB, bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    return JACOBI_OK;
}

int jacobi_set_plan(jacobi_h h, int kernel, int depth, int bx, int by, int bz, int ring, int threads)
{
    if (!h) return JACOBI_ERR_ARG;
    if (kernel == JACOBI_KERNEL_AUTO) {
        h->forced = false;
        return JACOBI_OK;
    }
    if (bx < 0 || by < 0 || bz < 0) return JACOBI_ERR_ARG;
    Plan p;
    p.kernel = kernel;
    const bool plain = kernel == JACOBI_KERNEL_PLAIN || kernel == JACOBI_KERNEL_PLAIN_X2;
    p.depth = plain ? 1 : depth;
    p.bx = bx;
    p.by = by;
    p.bz = bz;
    p.ring = (plain || kernel == JACOBI_KERNEL_TB_CTA || kernel == JACOBI_KERNEL_TB_REG) ? 0 : ring;
    p.threads = plain ? 0 : threads;
    p = resolve_plan(h, p);
    const int st = check_plan(h, p);
    if (st != JACOBI_OK) return st;
    h->plan = p;
    h->forced = true;
    return JACOBI_OK;
}

int jacobi_get_plan(jacobi_h h, int *kernel, int *depth, int *bx, int *by, int *bz, int *ring, int *threads)
{
    if (!h) return JACOBI_ERR_ARG;
    const Plan p = active_plan(h);
    if (kernel) *kernel = p.kernel;
    if (depth) *depth = p.depth;
    if (bx) *bx = p.bx;
    if (by) *by = p.by;
    if (bz) *bz = p.bz;
    if (ring) *ring = p.ring;
    if (threads) *threads = p.threads;
    return JACOBI_OK;
}

int jacobi_plan_passes(int T, int depth, int *depths, int max_passes)
{
    if (T < 0 || depth < 1 || max_passes < 0 || (T > 0 && !depths)) return -1;
    return plan_passes(T, depth, depths, max_passes);
}

int jacobi_get_status(jacobi_h h, int *device_status)
{
    if (!h || !device_status) return JACOBI_ERR_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e);
    int v = 0;
    e = cudaMemcpy(&v, h->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaMemset(h->d_status, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e);
    *device_status = v;
    return JACOBI_OK;
}

int jacobi_debug_set_fault(jacobi_h h, int mode, int limit_ms)
{
    if (!h || mode < 0 || mode > 2 || limit_ms < 1) return JACOBI_ERR_ARG;
    if (mode == 2 && !kChecked) return JACOBI_ERR_UNSUPPORTED;
    h->fault_mode = (mode == 1) ? 1 : 0;
    h->check_shrink = (mode == 2) ? 1 : 0;
    h->limit_ns = (unsigned long long)limit_ms * 1000000ull;
    return JACOBI_OK;
}

int jacobi_build_checked(void) { return kChecked ? 1 : 0; }

namespace {
// the compressed plan's defaults (measured on 1024^3 FP32 / 512^3 FP64)
void cg_resolve(jacobi_plan_s *h)
{
    const bool f64 = h->dtype == JACOBI_F64;
    if (h->cg_depth <= 0) h->cg_depth = f64 ? 1 : 3;
    if (h->cg_bz <= 0) h->cg_bz = f64 ? 64 : 128;
    if (h->cg_waves <= 0) h->cg_waves = 1;
}
}  // namespace

int jacobi_compressed_set_plan(jacobi_h h, int depth, int bz, int waves)
{
    if (!h || depth < 0 || bz < 0 || waves < 0) return JACOBI_ERR_ARG;
    const int d0 = h->cg_depth, b0 = h->cg_bz, w0 = h->cg_waves;
    h->cg_depth = depth;  // 0: the default, filled in below
    h->cg_bz = bz;
    h->cg_waves = waves;
    cg_resolve(h);
    const int st = cg_check(h, h->cg_depth, h->cg_bz, h->cg_waves);
    if (st != JACOBI_OK) {
        h->cg_depth = d0;
        h->cg_bz = b0;
        h->cg_waves = w0;
    }
    return st;
}

int jacobi_compressed_get_plan(jacobi_h h, int *depth, int *bz, int *waves, long long *shift_planes)
{
    if (!h) return JACOBI_ERR_ARG;
    cg_resolve(h);
    if (depth) *depth = h->cg_depth;
    if (bz) *bz = h->cg_bz;
    if (waves) *waves = h->cg_waves;
    if (shift_planes) *shift_planes = cg_shift_planes(h->cg_depth, h->cg_bz, h->cg_waves);
    return JACOBI_OK;
}

int jacobi_sweep_compressed(jacobi_h h, void *U, int T, int upper, int *upper_out, jacobi_stream_t stream)
{
    if (!h || !U || T < 0 || (upper != 0 && upper != 1)) return JACOBI_ERR_ARG;
    if (!aligned16(U)) return JACOBI_ERR_ALIGN;
    cg_resolve(h);
    const int st = cg_check(h, h->cg_depth, h->cg_bz, h->cg_waves);
    if (st != JACOBI_OK) return st;
    return cg_sweep(h, U, T, upper, upper_out, (cudaStream_t)stream);
}

int jacobi_profile_enable(jacobi_h h, int enable)
{
    if (!h) return JACOBI_ERR_ARG;
    h->prof = enable != 0;
    return JACOBI_OK;
}

int jacobi_profile_read(jacobi_h h, double *pass_ms, int *pass_launches, int *other_launches)
{
    if (!h) return JACOBI_ERR_ARG;
    double total = 0.0;
    for (size_t i = 0; i + 1 < h->ev_used; i += 2) {
        cudaError_t e = cudaEventSynchronize(h->ev_pool[i + 1]);
        if (e != cudaSuccess) return cuda_fail(e);
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, h->ev_pool[i], h->ev_pool[i + 1]);
        if (e != cudaSuccess) return cuda_fail(e);
        total += ms;
    }
    if (pass_ms) *pass_ms = total;
    if (pass_launches) *pass_launches = h->prof_pass;
    if (other_launches) *other_launches = h->prof_other;
    h->ev_used = 0;
    h->prof_pass = 0;
    h->prof_other = 0;
    return JACOBI_OK;
}

}  // extern "C"

namespace {

// Times plan p (T = max(8, 4*depth) sweeps, best of two after a warm-up) in
// GLUP/s.
int time_plan(jacobi_plan_s *h, const Plan &p, void *A, void *B, cudaStream_t s, cudaEvent_t e0,
              cudaEvent_t e1, double *glups)
{
    const int T = (4 * p.depth > 8) ? 4 * p.depth : 8;
    int st = run_sweeps(h, p, A, B, T, s);
    if (st != JACOBI_OK) return st;
    float best = 1e30f;
    for (int r = 0; r < 2; ++r) {
        cudaEventRecord(e0, s);
        st = run_sweeps(h, p, A, B, T, s);
        if (st != JACOBI_OK) return st;
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) return cuda_fail(e);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    *glups = (double)h->nx * h->ny * h->nz * T / (best * 1e-3) / 1e9;
    return JACOBI_OK;
}

Plan clamp_tile(const jacobi_plan_s *h, Plan p)
{
    if (p.bx > h->nx) p.bx = h->nx;
    if (p.by > h->ny) p.by = h->ny;
    if (p.bz > h->nz) p.bz = h->nz;
    return p;
}

// Stage-1 candidates of the autotuner (Sect. 2.4's parameter sweeps): the
// single-pass kernels over CTA shapes x planes per thread, temporal
// blocking inside one CTA over depth x tile x CTA width x z chunk, and the
// cluster pipeline over depth x tile.  Tiles are clamped to the grid;
// candidates the device cannot launch are filtered by the caller.
std::vector<Plan> tune_candidates(const jacobi_plan_s *h)
{
    std::vector<Plan> out;
    const bool f64 = h->dtype == JACOBI_F64;
    const int plain_shapes[][2] = {{32, 8}, {64, 4}, {128, 2}, {32, 16}, {64, 8}, {128, 4}, {256, 2}, {64, 16}};
    const int plain_kz[] = {4, 8, 16, 32};
    for (int kern : {JACOBI_KERNEL_PLAIN, JACOBI_KERNEL_PLAIN_X2})
        for (const auto &b : plain_shapes)
            for (int kz : plain_kz) {
                Plan p;
                p.kernel = kern;
                p.depth = 1;
                p.bx = b[0];
                p.by = b[1];
                p.bz = kz;
                out.push_back(p);
            }
    const int cta_tiles[][2] = {{32, 32}, {64, 24}, {64, 32}, {128, 16}};
    for (int d = 1; d <= 4; ++d)
        for (const auto &t : cta_tiles)
            for (int nt : {256, 512})
                for (int bz : {64, 128}) {
                    Plan p;
                    p.kernel = JACOBI_KERNEL_TB_CTA;
                    p.depth = d;
                    p.bx = t[0];
                    p.by = t[1];
                    p.bz = bz;
                    p.threads = nt;
                    out.push_back(clamp_tile(h, p));
                }
    if (!f64) {
        // register-blocked one-CTA kernel: depth x region x z chunk
        const int regions[][2] = {{64, 32}, {64, 64}, {128, 32}};
        for (int d = 1; d <= 4; ++d)
            for (const auto &r : regions)
                for (int bz : {64, 128}) {
                    Plan p;
                    p.kernel = JACOBI_KERNEL_TB_REG;
                    p.depth = d;
                    p.bx = r[0];
                    p.by = r[1];
                    p.bz = std::min(bz, h->nz);
                    p.threads = r[0] * r[1] / 16;
                    out.push_back(p);
                }
        // chains of CTAs: (depth, CTAs) x region, z chunk 128
        const int chains[][2] = {{4, 2}, {6, 2}, {6, 3}, {8, 2}, {8, 4}};
        for (const auto &c : chains)
            for (int by : {32, 64}) {
                Plan p;
                p.kernel = JACOBI_KERNEL_TB_CHAIN;
                p.depth = c[0];
                p.ring = c[1];
                p.bx = 64;
                p.by = by;
                p.bz = std::min(128, h->nz);
                p.threads = 64 * by / 16;
                out.push_back(p);
            }
    }
    const int depths64[] = {1, 2, 4};
    const int depths32[] = {1, 2, 4, 6, 8};
    const int tiles[][2] = {{32, 16}, {64, 8}, {64, 16}, {32, 32}, {64, 32}, {128, 16}, {128, 32}, {64, 64}};
    const int *dl = f64 ? depths64 : depths32;
    const int nd = f64 ? 3 : 5;
    for (int di = 0; di < nd; ++di)
        for (const auto &t : tiles) {
            Plan p;
            p.kernel = JACOBI_KERNEL_TB;
            p.depth = dl[di];
            p.bx = t[0];
            p.by = t[1];
            p.bz = 128;
            p.ring = 0;
            out.push_back(clamp_tile(h, p));
        }
    return out;
}

}  // namespace

extern "C" {

int jacobi_tune(jacobi_h h, void *scratchA, void *scratchB, jacobi_stream_t stream, double *glups)
{
    if (!h || !scratchA || !scratchB || scratchA == scratchB) return JACOBI_ERR_ARG;
    if (!aligned16(scratchA) || !aligned16(scratchB)) return JACOBI_ERR_ALIGN;
    cudaStream_t s = (cudaStream_t)stream;
    const int bzs[] = {32, 64, 128, 256};
    const int rings[] = {4, 8, 16};
    const int widths[] = {0, 128, 256, 512};
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(e);
    }
    // Benign, finite, normal values (uninitialised scratch could hold NaNs
    // or subnormals, which take slower arithmetic paths).
    e = fill_launch(h->dtype, scratchA, (long long)grid_elems(h), 0.5, s);
    if (e == cudaSuccess) e = fill_launch(h->dtype, scratchB, (long long)grid_elems(h), 0.5, s);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return cuda_fail(e);
    }
    double best = -1.0;
    Plan bestp;
    int st = JACOBI_OK;
    auto consider = [&](const Plan &p) {
        if (st != JACOBI_OK || check_plan(h, p) != JACOBI_OK) return;
        double g = 0.0;
        st = time_plan(h, p, scratchA, scratchB, s, e0, e1, &g);
        if (st == JACOBI_OK && g > best) {
            best = g;
            bestp = p;
        }
    };
    // Stage 1: every family over its shapes and depths.
    for (const Plan &p : tune_candidates(h)) consider(p);
    // Stage 2 (cluster pipeline only): z chunk, ring depth (pipeline
    // looseness) and CTA width around the winner.
    if (st == JACOBI_OK && best > 0 && bestp.kernel == JACOBI_KERNEL_TB) {
        const Plan base = bestp;
        for (int bz : bzs)
            for (int rg : rings) {
                Plan p = base;
                p.bz = bz;
                p.ring = rg;
                consider(clamp_tile(h, p));
            }
        const Plan base2 = bestp;
        for (int w : widths) {
            Plan p = base2;
            p.threads = w;
            consider(clamp_tile(h, p));
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != JACOBI_OK) return st;
    if (best <= 0) return JACOBI_ERR_UNSUPPORTED;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune_cache[std::make_tuple(h->dtype, h->nx, h->ny, h->nz, h->sms)] = bestp;
    }
    h->forced = false;
    if (glups) *glups = best;
    return JACOBI_OK;
}

int jacobi_tune_candidates(jacobi_h h, int *plans, int max_plans)
{
    if (!h || max_plans < 0 || (max_plans > 0 && !plans)) return JACOBI_ERR_ARG;
    std::vector<Plan> c;
    for (const Plan &p : tune_candidates(h))
        if (check_plan(h, p) == JACOBI_OK) c.push_back(p);
    const int n = (int)std::min<size_t>(c.size(), (size_t)max_plans);
    for (int i = 0; i < n; ++i) {
        int *o = plans + 7 * i;
        o[0] = c[i].kernel;
        o[1] = c[i].depth;
        o[2] = c[i].bx;
        o[3] = c[i].by;
        o[4] = c[i].bz;
        o[5] = c[i].ring;
        o[6] = c[i].threads;
    }
    return (int)c.size();
}

}  // extern "C"
