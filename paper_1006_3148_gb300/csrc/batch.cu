// Batched sweeps: many independent grids of different sizes and element
// types, all T_g sweeps of all grids in ONE persistent launch, replayed from
// a CUDA graph.
//
// Work items are (grid g, tile t of g, sweep p), numbered pass-major:
// item = p * total_tiles + (tile_base[g] + t).  Resident CTAs take items
// from a global atomic counter, so items are started in that order.  Item
// (g, t, p) reads grid buffer p%2 and writes buffer (p+1)%2 on the tile's
// cells (bx*by*bz; bz = nz unless z is split); it may start once tile t and
// its face neighbours
// (the only tiles whose cells the 7-point stencil reads) have finished
// sweep p-1: that covers the cells it reads (read after write) and the cells
// the neighbours' sweep p-1 still reads in the buffer it overwrites (write
// after read).  Every item waits only on items with smaller numbers, which
// were taken earlier by CTAs that are resident and never wait on later
// items, so the schedule cannot deadlock; each wait is also bounded.  The
// per-tile counters play the role of the per-thread counters c_i of the
// relaxed synchronisation of Sect. 2.2.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "arith.cuh"
#include "jacobi_internal.h"
#include "ptx.cuh"

namespace jac {

struct BatchGrid {
    void *A;
    void *B;
    const void *rhs;  // optional source term g (same dtype): update (sum + g)/6
    int nx, ny, nz, dtype, T;
    int ntx, nty, ntz;
    int tile_base;  // global index of this grid's tile 0
};

struct BatchArgs {
    const BatchGrid *grids;
    int ngrids;
    int total_tiles;
    long long total_items;
    int bx, by, bz;  // tile interior size
    int *head;   // next item
    int *progress;
    int *status;
    unsigned long long limit_ns;
    int fault_mode;
};

namespace {

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Waits until progress[i] >= want (bounded; aborts when the status word is
// set).  Returns false on timeout or abort.
__device__ bool wait_progress(const int *progress, int i, int want, unsigned long long limit_ns,
                              const volatile int *status)
{
    if (ld_acquire(progress + i) >= want) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        __nanosleep(64);
        if (ld_acquire(progress + i) >= want) return true;
        if ((it & 31u) == 0u) {
            if (*status != 0) return false;
            if (globaltimer_ns() - t0 > limit_ns) return false;
        }
    }
}

// One sweep of one tile: thread (lx, ly) walks z over the tile's planes with
// the values at k-1, k, k+1 of its column in registers; in-plane neighbours
// are read through L2 (.cg: other CTAs rewrote this buffer two sweeps ago).
template <typename T>
__device__ void sweep_tile(const BatchGrid &G, int tx, int ty, int tz, int p, int bx, int by, int bz)
{
    const T *src = static_cast<const T *>((p % 2 == 0) ? G.A : G.B);
    T *dst = static_cast<T *>((p % 2 == 0) ? G.B : G.A);
    const T *rhs = static_cast<const T *>(G.rhs);
    const long long NXP = G.nx + 2, plane = NXP * (G.ny + 2);
    const int nthreads = blockDim.x;
    const int x0 = 1 + tx * bx, y0 = 1 + ty * by, z0 = 1 + tz * bz;
    const int w = min(bx, G.nx + 1 - x0), hgt = min(by, G.ny + 1 - y0), z1 = min(z0 + bz, G.nz + 1);
    for (int c = threadIdx.x; c < w * hgt; c += nthreads) {
        const int x = x0 + c % w, y = y0 + c / w;
        const T *col = src + (long long)y * NXP + x;
        T *ocol = dst + (long long)y * NXP + x;
        T a = __ldcg(col + (long long)(z0 - 1) * plane), b = __ldcg(col + (long long)z0 * plane);
        for (int k = z0; k < z1; ++k) {
            const T *cp = col + k * plane;
            const T cnext = __ldcg(cp + plane);
            T v;
            if (rhs)
                v = Arith<T>::update_rhs(__ldcg(cp - 1), __ldcg(cp + 1), __ldcg(cp - NXP), __ldcg(cp + NXP), a, cnext,
                                         __ldg(rhs + (cp - src)));
            else
                v = Arith<T>::update(__ldcg(cp - 1), __ldcg(cp + 1), __ldcg(cp - NXP), __ldcg(cp + NXP), a, cnext);
            ocol[k * plane] = v;
            a = b;
            b = cnext;
        }
    }
}

__global__ void __launch_bounds__(256) batch_kernel(const BatchArgs a)
{
    __shared__ long long s_item;
    __shared__ int s_ok;
    const volatile int *vstatus = a.status;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(a.head, 1);
        __syncthreads();
        const long long item = s_item;
        __syncthreads();
        if (item >= a.total_items) break;
        const int p = (int)(item / a.total_tiles);
        const int tg = (int)(item % a.total_tiles);
        // grid of global tile tg: last g with tile_base <= tg
        int lo = 0, hi = a.ngrids - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.grids[mid].tile_base <= tg) lo = mid;
            else hi = mid - 1;
        }
        const BatchGrid G = a.grids[lo];
        const int t = tg - G.tile_base, txy = G.ntx * G.nty;
        const int tx = t % G.ntx, ty = (t / G.ntx) % G.nty, tz = t / txy;
        if (p >= G.T) continue;  // this grid is done; nothing waits on it
        if (threadIdx.x == 0) {
            bool ok = true;
            if (p > 0) {
                const int want = p;
                ok = ok && wait_progress(a.progress, tg, want, a.limit_ns, vstatus);
                if (tx > 0) ok = ok && wait_progress(a.progress, tg - 1, want, a.limit_ns, vstatus);
                if (tx + 1 < G.ntx) ok = ok && wait_progress(a.progress, tg + 1, want, a.limit_ns, vstatus);
                if (ty > 0) ok = ok && wait_progress(a.progress, tg - G.ntx, want, a.limit_ns, vstatus);
                if (ty + 1 < G.nty) ok = ok && wait_progress(a.progress, tg + G.ntx, want, a.limit_ns, vstatus);
                if (tz > 0) ok = ok && wait_progress(a.progress, tg - txy, want, a.limit_ns, vstatus);
                if (tz + 1 < G.ntz) ok = ok && wait_progress(a.progress, tg + txy, want, a.limit_ns, vstatus);
            }
            if (!ok) atomicCAS(a.status, 0, JACOBI_ERR_TIMEOUT);
            s_ok = ok;
        }
        __syncthreads();
        if (s_ok) {
            if (G.dtype == JACOBI_F64) sweep_tile<double>(G, tx, ty, tz, p, a.bx, a.by, a.bz);
            else sweep_tile<float>(G, tx, ty, tz, p, a.bx, a.by, a.bz);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            // test hook: never publish sweep 2 of global tile 0
            if (!(a.fault_mode == 1 && tg == 0 && p == 2)) st_release(a.progress + tg, p + 1);
        }
    }
}

// Copies the halo of A into B for every grid (blockIdx.y = grid).
__global__ void batch_halo_kernel(const BatchGrid *grids)
{
    const BatchGrid G = grids[blockIdx.y];
    if (G.T <= 0) return;
    const long long NXP = G.nx + 2, NYP = G.ny + 2, NZP = G.nz + 2;
    const long long total = NXP * NYP * NZP;
    const int es = G.dtype == JACOBI_F64 ? 8 : 4;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long x = i % NXP, y = (i / NXP) % NYP, z = i / (NXP * NYP);
        if (x != 0 && x != NXP - 1 && y != 0 && y != NYP - 1 && z != 0 && z != NZP - 1) continue;
        if (es == 8) static_cast<double *>(G.B)[i] = static_cast<const double *>(G.A)[i];
        else static_cast<float *>(G.B)[i] = static_cast<const float *>(G.A)[i];
    }
}

}  // namespace
}  // namespace jac

using namespace jac;

struct jacobi_batch_s {
    int n = 0;
    std::vector<BatchGrid> grids;  // host copy (pointers bound by jacobi_batch_run)
    int bx = 32, by = 8, bz = 0;  // bz 0: whole z column per item
    int total_tiles = 0, max_T = 0;
    long long total_items = 0;
    BatchGrid *d_grids = nullptr;
    int *d_ctl = nullptr;  // [0] head, [1] status, [2..] progress
    int persistent_blocks = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int fault_mode = 0;
    unsigned long long limit_ns = 2000000000ull;
    bool bound = false;
};

namespace {

thread_local std::string g_batch_err;

void layout(jacobi_batch_s *b)
{
    int base = 0;
    b->max_T = 0;
    for (BatchGrid &G : b->grids) {
        G.ntx = (G.nx + b->bx - 1) / b->bx;
        G.nty = (G.ny + b->by - 1) / b->by;
        G.ntz = (b->bz > 0) ? (G.nz + b->bz - 1) / b->bz : 1;
        G.tile_base = base;
        base += G.ntx * G.nty * G.ntz;
        b->max_T = std::max(b->max_T, G.T);
    }
    b->total_tiles = base;
    b->total_items = (long long)base * b->max_T;
}

void free_graph(jacobi_batch_s *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// (Re)allocates the control block for the current layout and captures the
// graph: reset of the item counter and progress counters, the halo copy of
// every grid, and the persistent launch.
int build_graph(jacobi_batch_s *b)
{
    free_graph(b);
    if (b->d_ctl) cudaFree(b->d_ctl);
    b->d_ctl = nullptr;
    cudaError_t e = cudaMalloc(&b->d_ctl, sizeof(int) * (2 + (size_t)b->total_tiles));
    if (e != cudaSuccess) return JACOBI_ERR_ALLOC;
    e = cudaMemset(b->d_ctl, 0, sizeof(int) * (2 + (size_t)b->total_tiles));
    if (e != cudaSuccess) return JACOBI_ERR_CUDA;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, 256, 0);
    if (e != cudaSuccess || per_sm < 1) return JACOBI_ERR_UNSUPPORTED;
    b->persistent_blocks = sms * per_sm;

    BatchArgs a;
    a.grids = b->d_grids;
    a.ngrids = b->n;
    a.total_tiles = b->total_tiles;
    a.total_items = b->total_items;
    a.bx = b->bx;
    a.by = b->by;
    a.bz = (b->bz > 0) ? b->bz : (1 << 30);
    a.head = b->d_ctl;
    a.status = b->d_ctl + 1;
    a.progress = b->d_ctl + 2;
    a.limit_ns = b->limit_ns;
    a.fault_mode = b->fault_mode;

    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return JACOBI_ERR_CUDA;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(b->d_ctl, 0, sizeof(int), cs);
        cudaMemsetAsync(b->d_ctl + 2, 0, sizeof(int) * (size_t)b->total_tiles, cs);
        batch_halo_kernel<<<dim3(64, (unsigned)b->n), 256, 0, cs>>>(b->d_grids);
        batch_kernel<<<b->persistent_blocks, 256, 0, cs>>>(a);
        e = cudaStreamEndCapture(cs, &b->graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        g_batch_err = cudaGetErrorString(e);
        free_graph(b);
        return JACOBI_ERR_CUDA;
    }
    return JACOBI_OK;
}

}  // namespace

extern "C" {

int jacobi_batch_create(jacobi_batch_h *out, int n, const int *nx, const int *ny, const int *nz,
                        const int *dtype, const int *T)
{
    if (!out) return JACOBI_ERR_ARG;
    *out = nullptr;
    if (n < 1 || n > 65535 || !nx || !ny || !nz || !dtype || !T) return JACOBI_ERR_ARG;
    for (int g = 0; g < n; ++g) {
        if (dtype[g] != JACOBI_F64 && dtype[g] != JACOBI_F32) return JACOBI_ERR_DTYPE;
        if (nx[g] < 1 || ny[g] < 1 || nz[g] < 1 || T[g] < 0) return JACOBI_ERR_ARG;
        if ((double)(nx[g] + 2) * (ny[g] + 2) * (double)(nz[g] + 2) >= 2147483647.0) return JACOBI_ERR_ARG;
    }
    jacobi_batch_s *b = new (std::nothrow) jacobi_batch_s;
    if (!b) return JACOBI_ERR_ALLOC;
    b->n = n;
    b->grids.resize((size_t)n);
    for (int g = 0; g < n; ++g) {
        BatchGrid &G = b->grids[(size_t)g];
        G.A = G.B = nullptr;
        G.rhs = nullptr;
        G.nx = nx[g];
        G.ny = ny[g];
        G.nz = nz[g];
        G.dtype = dtype[g];
        G.T = T[g];
    }
    layout(b);
    cudaError_t e = cudaMalloc(&b->d_grids, sizeof(BatchGrid) * (size_t)n);
    if (e != cudaSuccess) {
        delete b;
        return JACOBI_ERR_ALLOC;
    }
    const int st = build_graph(b);
    if (st != JACOBI_OK) {
        cudaFree(b->d_grids);
        if (b->d_ctl) cudaFree(b->d_ctl);
        delete b;
        return st;
    }
    *out = b;
    return JACOBI_OK;
}

int jacobi_batch_destroy(jacobi_batch_h b)
{
    if (!b) return JACOBI_OK;
    free_graph(b);
    if (b->d_grids) cudaFree(b->d_grids);
    if (b->d_ctl) cudaFree(b->d_ctl);
    delete b;
    return JACOBI_OK;
}

int jacobi_batch_run_rhs(jacobi_batch_h b, void *const *A, void *const *B, const void *const *RHS,
                         jacobi_stream_t stream)
{
    if (!b || !A || !B) return JACOBI_ERR_ARG;
    for (int g = 0; g < b->n; ++g) {
        if (!A[g] || !B[g] || A[g] == B[g]) return JACOBI_ERR_ARG;
        b->grids[(size_t)g].A = A[g];
        b->grids[(size_t)g].B = B[g];
        b->grids[(size_t)g].rhs = RHS ? RHS[g] : nullptr;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(b->d_grids, b->grids.data(), sizeof(BatchGrid) * (size_t)b->n,
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, s);
    if (e != cudaSuccess) {
        g_batch_err = cudaGetErrorString(e);
        return JACOBI_ERR_CUDA;
    }
    return JACOBI_OK;
}

int jacobi_batch_run(jacobi_batch_h b, void *const *A, void *const *B, jacobi_stream_t stream)
{
    return jacobi_batch_run_rhs(b, A, B, nullptr, stream);
}

int jacobi_batch_set_tile(jacobi_batch_h b, int bx, int by, int bz)
{
    if (!b || bx < 1 || by < 1 || bz < 0 || bx * by > 4096) return JACOBI_ERR_ARG;
    b->bx = bx;
    b->by = by;
    b->bz = bz;
    layout(b);
    return build_graph(b);
}

int jacobi_batch_get_info(jacobi_batch_h b, int *bx, int *by, int *bz, long long *items, int *blocks)
{
    if (!b) return JACOBI_ERR_ARG;
    if (bx) *bx = b->bx;
    if (by) *by = b->by;
    if (bz) *bz = b->bz;
    if (items) *items = b->total_items;
    if (blocks) *blocks = b->persistent_blocks;
    return JACOBI_OK;
}

int jacobi_batch_get_status(jacobi_batch_h b, int *device_status)
{
    if (!b || !device_status) return JACOBI_ERR_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    int v = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&v, b->d_ctl + 1, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(b->d_ctl + 1, 0, sizeof(int));
    if (e != cudaSuccess) return JACOBI_ERR_CUDA;
    *device_status = v;
    return JACOBI_OK;
}

int jacobi_batch_debug_set_fault(jacobi_batch_h b, int mode, int limit_ms)
{
    if (!b || mode < 0 || mode > 1 || limit_ms < 1) return JACOBI_ERR_ARG;
    b->fault_mode = mode;
    b->limit_ns = (unsigned long long)limit_ms * 1000000ull;
    return build_graph(b);
}

int jacobi_batch_tune(jacobi_batch_h b, void *const *scratchA, void *const *scratchB, jacobi_stream_t stream,
                      double *glups)
{
    if (!b || !scratchA || !scratchB) return JACOBI_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    for (int g = 0; g < b->n; ++g) {
        const BatchGrid &G = b->grids[(size_t)g];
        const long long n = (long long)(G.nx + 2) * (G.ny + 2) * (G.nz + 2);
        if (!scratchA[g] || !scratchB[g]) return JACOBI_ERR_ARG;
        if (fill_launch(G.dtype, scratchA[g], n, 0.5, s) != cudaSuccess) return JACOBI_ERR_CUDA;
        if (fill_launch(G.dtype, scratchB[g], n, 0.5, s) != cudaSuccess) return JACOBI_ERR_CUDA;
    }
    double lups = 0.0;
    for (const BatchGrid &G : b->grids) lups += (double)G.nx * G.ny * G.nz * G.T;
    const int tiles[][3] = {{32, 4, 0}, {32, 8, 0}, {32, 16, 0}, {64, 4, 0}, {64, 8, 0}, {128, 2, 0}, {32, 8, 64}};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return JACOBI_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return JACOBI_ERR_CUDA;
    }
    double best = -1.0;
    int bbx = b->bx, bby = b->by, bbz = b->bz, st = JACOBI_OK;
    for (const auto &t : tiles) {
        st = jacobi_batch_set_tile(b, t[0], t[1], t[2]);
        if (st != JACOBI_OK) break;
        st = jacobi_batch_run(b, scratchA, scratchB, stream);  // warm-up
        if (st != JACOBI_OK) break;
        cudaEventRecord(e0, s);
        st = jacobi_batch_run(b, scratchA, scratchB, stream);
        if (st != JACOBI_OK) break;
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = JACOBI_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double g = lups / (ms * 1e-3) / 1e9;
        if (g > best) {
            best = g;
            bbx = t[0];
            bby = t[1];
            bbz = t[2];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != JACOBI_OK) return st;
    if (glups) *glups = best;
    return jacobi_batch_set_tile(b, bbx, bby, bbz);
}

}  // extern "C"
