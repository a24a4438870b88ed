// Batched sweeps: many independent grids of different sizes and element
// types, replayed from a CUDA graph by one of two engines.
//
// Sweep engine (JACOBI_BATCH_SWEEPS): one launch per sweep p covers every
// grid, one CTA per (grid, run of 256 x-y cells, z chunk) unit running the
// single-pass column walk; kernel boundaries order the sweeps, so no CTA
// waits on another.  The runs follow the row-major order of the interior
// cells of a plane, so warps stay full whatever nx is (an FP64 warp
// instruction costs the same with idle lanes).  Units of FP64 and FP32 grids are dealt out alternately, so that
// FP64-pipe-bound and HBM-bound CTAs share the SMs.
//
// Persistent engine (JACOBI_BATCH_PERSISTENT): all T_g sweeps of all grids
// in ONE persistent launch.
//
// FP32 depth d > 1 (jacobi_batch_set_fp32_depth): the FP32 grids leave both
// engines and are swept by temporally blocked passes of depth <= d
// (batch_tbr.cu), on a branch of the graph that runs beside the FP64 work.
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
#include "batch_internal.h"
#include "checked.cuh"
#include "grid.cuh"
#include "jacobi_internal.h"
#include "ptx.cuh"

namespace jac {

// Sweep engine: grid g's units are numbered from unit_base within the list
// of grids of its dtype (FP64 list first in the table, then FP32).
struct SweepEntry {
    long long unit_base;
    int grid;
};

constexpr int kSweepThreads = 256;  // CTA of the sweep engine

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
    long long shrink;  // checked build: grids declared this many elements short
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
__device__ void sweep_tile(const BatchGrid &G, int tx, int ty, int tz, int p, int bx, int by, int bz, int *status,
                           long long shrink)
{
    const T *src = static_cast<const T *>((p % 2 == 0) ? G.A : G.B);
    T *dst = static_cast<T *>((p % 2 == 0) ? G.B : G.A);
    const T *rhs = static_cast<const T *>(G.rhs);
    const long long NXP = G.nx + 2, plane = NXP * (G.ny + 2);
    const int nthreads = blockDim.x;
    const int x0 = 1 + tx * bx, y0 = 1 + ty * by, z0 = 1 + tz * bz;
    const int w = min(bx, G.nx + 1 - x0), hgt = min(by, G.ny + 1 - y0), z1 = min(z0 + bz, G.nz + 1);
    const long long S = checked_grid_elems(G.nx, G.ny, G.nz, shrink);
    auto ld = [&](const T *q) { return in_bounds(q - src, 1, S, status) ? __ldcg(q) : T(0); };
    for (int c = threadIdx.x; c < w * hgt; c += nthreads) {
        const int x = x0 + c % w, y = y0 + c / w;
        const T *col = src + (long long)y * NXP + x;
        T *ocol = dst + (long long)y * NXP + x;
        T a = ld(col + (long long)(z0 - 1) * plane), b = ld(col + (long long)z0 * plane);
        for (int k = z0; k < z1; ++k) {
            const T *cp = col + k * plane;
            const T cnext = ld(cp + plane);
            T v;
            if (rhs)
                v = Arith<T>::update_rhs(ld(cp - 1), ld(cp + 1), ld(cp - NXP), ld(cp + NXP), a, cnext,
                                         in_bounds(cp - src, 1, S, status) ? __ldg(rhs + (cp - src)) : T(0));
            else
                v = Arith<T>::update(ld(cp - 1), ld(cp + 1), ld(cp - NXP), ld(cp + NXP), a, cnext);
            if (in_bounds(ocol + k * plane - dst, 1, S, status)) ocol[k * plane] = v;
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
        if (p >= G.Te) continue;  // this grid is done; nothing waits on it
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
            if (G.dtype == JACOBI_F64) sweep_tile<double>(G, tx, ty, tz, p, a.bx, a.by, a.bz, a.status, a.shrink);
            else sweep_tile<float>(G, tx, ty, tz, p, a.bx, a.by, a.bz, a.status, a.shrink);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            // test hook: never publish sweep 2 of global tile 0
            if (!(a.fault_mode == 1 && tg == 0 && p == 2)) st_release(a.progress + tg, p + 1);
        }
    }
}

// Sweep p of every grid with T_g > p.  Block b takes, while both lists have
// units left, alternately a unit of the FP64 list (even b) and of the FP32
// list (odd b); then the rest of the longer list.
template <typename T, bool RHS>
__device__ __forceinline__ void sweep_unit(const BatchGrid &G, int u, int p, int kz, int *status, long long shrink)
{
    const int r = u % G.nbxy, zc = u / G.nbxy;
    const int c = r * kSweepThreads + threadIdx.x;  // row-major interior cell of the plane
    if (c >= G.nx * G.ny) return;
    const int i = 1 + c % G.nx, j = 1 + c / G.nx;
    const long long NXP = G.nx + 2, plane = NXP * (G.ny + 2);
    const int kb = 1 + zc * kz;
    const int ke = (G.nz + 1 - kb < kz) ? G.nz + 1 : kb + kz;
    const long long c0 = kb * plane + j * NXP + i;
    const T *__restrict__ q0 = static_cast<const T *>((p % 2 == 0) ? G.A : G.B) + c0;
    T *__restrict__ q = static_cast<T *>((p % 2 == 0) ? G.B : G.A) + c0;
    const T *__restrict__ g = RHS ? static_cast<const T *>(G.rhs) + c0 : nullptr;
    const int nxp = G.nx + 2;
    // checked build: every element offset against the grid's extent
    const T *sb = static_cast<const T *>((p % 2 == 0) ? G.A : G.B), *gb = static_cast<const T *>(G.rhs);
    const T *db = static_cast<const T *>((p % 2 == 0) ? G.B : G.A);
    const long long S = checked_grid_elems(G.nx, G.ny, G.nz, shrink);
    auto ld = [&](const T *ptr, const T *base) { return in_bounds(ptr - base, 1, S, status) ? __ldg(ptr) : T(0); };
    T lo = ld(q0 - plane, sb), mid = ld(q0, sb);
#pragma unroll 4
    for (int k = kb; k < ke; ++k) {
        const T hi = ld(q0 + plane, sb);
        if (RHS) {
            const T v = Arith<T>::update_rhs(ld(q0 - 1, sb), ld(q0 + 1, sb), ld(q0 - nxp, sb), ld(q0 + nxp, sb), lo, hi,
                                             ld(g, gb));
            if (in_bounds(q - db, 1, S, status)) *q = v;
            g += plane;
        } else {
            const T v = Arith<T>::update(ld(q0 - 1, sb), ld(q0 + 1, sb), ld(q0 - nxp, sb), ld(q0 + nxp, sb), lo, hi);
            if (in_bounds(q - db, 1, S, status)) *q = v;
        }
        lo = mid;
        mid = hi;
        q0 += plane;
        q += plane;
    }
}

__global__ void __launch_bounds__(kSweepThreads) batch_sweep_kernel(const BatchGrid *grids,
                                                                         const SweepEntry *tab, int n64, int n32,
                                                                         long long u64, long long u32, int p, int kz,
                                                                         int *status, long long shrink)
{
    const long long b = blockIdx.x + (long long)gridDim.x * blockIdx.y;
    const long long m = u64 < u32 ? u64 : u32;
    int list;
    long long idx;
    if (b < 2 * m) {
        list = (int)(b & 1);
        idx = b >> 1;
    } else {
        list = (u64 > u32) ? 0 : 1;
        idx = b - m;
    }
    if (idx >= (list == 0 ? u64 : u32)) return;
    const SweepEntry *t = tab + (list == 0 ? 0 : n64);
    int lo = 0, hi = (list == 0 ? n64 : n32) - 1;  // last entry with unit_base <= idx
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t[mid].unit_base <= idx) lo = mid;
        else hi = mid - 1;
    }
    const BatchGrid &G = grids[t[lo].grid];
    if (p >= G.Te) return;
    const int u = (int)(idx - t[lo].unit_base);
    // element type and source term are uniform per block: the plane loop is
    // instantiated for each combination
    if (list == 0) {
        if (G.rhs) sweep_unit<double, true>(G, u, p, kz, status, shrink);
        else sweep_unit<double, false>(G, u, p, kz, status, shrink);
    } else {
        if (G.rhs) sweep_unit<float, true>(G, u, p, kz, status, shrink);
        else sweep_unit<float, false>(G, u, p, kz, status, shrink);
    }
}

// Copies the halo of A into B for every grid (blockIdx.y = grid).
__global__ void batch_halo_kernel(const BatchGrid *grids, int *status, long long shrink)
{
    const BatchGrid G = grids[blockIdx.y];
    if (G.T <= 0) return;
    const long long total = halo_count(G.nx, G.ny, G.nz);
    const long long S = checked_grid_elems(G.nx, G.ny, G.nz, shrink);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long i = halo_cell(t, G.nx, G.ny, G.nz);
        if (!in_bounds(i, 1, S, status)) continue;
        if (G.dtype == JACOBI_F64) static_cast<double *>(G.B)[i] = static_cast<const double *>(G.A)[i];
        else static_cast<float *>(G.B)[i] = static_cast<const float *>(G.A)[i];
    }
}

}  // namespace
}  // namespace jac

using namespace jac;

struct jacobi_batch_s {
    int n = 0;
    std::vector<BatchGrid> grids;  // host copy (pointers bound by jacobi_batch_run)
    int engine = JACOBI_BATCH_SWEEPS;
    int kz = 16;                   // sweep engine: planes per thread
    SweepEntry *d_tab = nullptr;   // sweep engine: FP64 list, then FP32 list
    int fp32_depth = 1;            // > 1: FP32 grids by blocked passes
    TbrBatchEntry *d_tbr = nullptr;
    std::vector<TbrBatchLaunch> tbr_launches;
    int n64 = 0, n32 = 0;
    long long u64 = 0, u32 = 0;    // units per list
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
    long long check_shrink = 0;  // checked build test hook (debug mode 2)
    bool bound = false;
};

namespace {

thread_local std::string g_batch_err;

// Whether grid G is swept by the sweep or persistent engine.
bool engine_grid(const jacobi_batch_s *b, const BatchGrid &G)
{
    return G.dtype == JACOBI_F64 || b->fp32_depth == 1;
}

void layout(jacobi_batch_s *b)
{
    int base = 0;
    b->max_T = 0;
    for (BatchGrid &G : b->grids) {
        G.Te = engine_grid(b, G) ? G.T : 0;
        G.ntx = (G.nx + b->bx - 1) / b->bx;
        G.nty = (G.ny + b->by - 1) / b->by;
        G.ntz = (b->bz > 0) ? (G.nz + b->bz - 1) / b->bz : 1;
        G.tile_base = base;
        base += G.ntx * G.nty * G.ntz;
        b->max_T = std::max(b->max_T, G.Te);
    }
    b->total_tiles = base;
    b->total_items = (long long)base * b->max_T;
    b->n64 = b->n32 = 0;
    b->u64 = b->u32 = 0;
    for (BatchGrid &G : b->grids) {
        if (!engine_grid(b, G)) continue;
        G.nbxy = (G.nx * G.ny + kSweepThreads - 1) / kSweepThreads;
        G.nbz = (G.nz + b->kz - 1) / b->kz;
        const long long units = (long long)G.nbxy * G.nbz;
        if (G.dtype == JACOBI_F64) {
            ++b->n64;
            b->u64 += units;
        } else {
            ++b->n32;
            b->u32 += units;
        }
    }
}

// Sweep-engine table: FP64 grids in order with their unit bases, then the
// FP32 grids.
std::vector<SweepEntry> sweep_table(const jacobi_batch_s *b)
{
    std::vector<SweepEntry> t;
    t.reserve((size_t)b->n);
    for (int pass = 0; pass < 2; ++pass) {
        long long base = 0;
        for (int g = 0; g < b->n; ++g) {
            const BatchGrid &G = b->grids[(size_t)g];
            if ((G.dtype == JACOBI_F64) != (pass == 0) || !engine_grid(b, G)) continue;
            t.push_back(SweepEntry{base, g});
            base += (long long)G.nbxy * G.nbz;
        }
    }
    return t;
}

void free_graph(jacobi_batch_s *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// (Re)allocates the control block for the current layout and captures the
// graph: (persistent engine) reset of the item counter and progress
// counters, the halo copy of every grid, then the engine's launches and,
// for an FP32 depth above 1, the blocked FP32 passes on a second branch.
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
    a.shrink = b->check_shrink;

    if (b->engine == JACOBI_BATCH_SWEEPS) {
        const std::vector<SweepEntry> tab = sweep_table(b);
        if (b->d_tab) cudaFree(b->d_tab);
        b->d_tab = nullptr;
        e = cudaMalloc(&b->d_tab, sizeof(SweepEntry) * std::max<size_t>(1, tab.size()));
        if (e != cudaSuccess) return JACOBI_ERR_ALLOC;
        if (!tab.empty())
            e = cudaMemcpy(b->d_tab, tab.data(), sizeof(SweepEntry) * tab.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return JACOBI_ERR_CUDA;
    }
    std::vector<TbrBatchEntry> ttab;
    b->tbr_launches.clear();
    if (b->fp32_depth > 1) batch_tbr_plan(b->grids, b->fp32_depth, ttab, b->tbr_launches);
    if (b->d_tbr) cudaFree(b->d_tbr);
    b->d_tbr = nullptr;
    if (!ttab.empty()) {
        e = cudaMalloc(&b->d_tbr, sizeof(TbrBatchEntry) * ttab.size());
        if (e != cudaSuccess) return JACOBI_ERR_ALLOC;
        e = cudaMemcpy(b->d_tbr, ttab.data(), sizeof(TbrBatchEntry) * ttab.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return JACOBI_ERR_CUDA;
    }
    for (const TbrBatchLaunch &L : b->tbr_launches)
        if (batch_tbr_configure(L) != cudaSuccess) return JACOBI_ERR_CUDA;
    const long long units = b->u64 + b->u32;
    const unsigned gx = (unsigned)std::max<long long>(1, std::min<long long>(units, 1ll << 30));
    const unsigned gy = (unsigned)((units + gx - 1) / gx);
    cudaStream_t cs, cs2;
    cudaEvent_t fork, join;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return JACOBI_ERR_CUDA;
    e = cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return JACOBI_ERR_CUDA;
    }
    cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
    const bool branch = !b->tbr_launches.empty();
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        if (b->engine == JACOBI_BATCH_PERSISTENT) {
            cudaMemsetAsync(b->d_ctl, 0, sizeof(int), cs);
            cudaMemsetAsync(b->d_ctl + 2, 0, sizeof(int) * (size_t)b->total_tiles, cs);
        }
        batch_halo_kernel<<<dim3(64, (unsigned)b->n), 256, 0, cs>>>(b->d_grids, a.status, a.shrink);
        cudaError_t eb = cudaSuccess;
        if (branch) {
            eb = cudaEventRecord(fork, cs);
            if (eb == cudaSuccess) eb = cudaStreamWaitEvent(cs2, fork, 0);
            for (const TbrBatchLaunch &L : b->tbr_launches)
                if (eb == cudaSuccess) eb = batch_tbr_launch(L, b->d_grids, b->d_tbr, a.status, a.shrink, cs2);
            if (eb == cudaSuccess) eb = cudaEventRecord(join, cs2);
        }
        if (b->engine == JACOBI_BATCH_SWEEPS) {
            for (int p = 0; p < b->max_T; ++p)
                batch_sweep_kernel<<<dim3(gx, gy), kSweepThreads, 0, cs>>>(
                    b->d_grids, b->d_tab, b->n64, b->n32, b->u64, b->u32, p, b->kz, a.status, a.shrink);
        } else {
            batch_kernel<<<b->persistent_blocks, 256, 0, cs>>>(a);
        }
        if (branch && eb == cudaSuccess) eb = cudaStreamWaitEvent(cs, join, 0);
        e = cudaStreamEndCapture(cs, &b->graph);
        if (e == cudaSuccess && eb != cudaSuccess) e = eb;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    cudaEventDestroy(fork);
    cudaEventDestroy(join);
    cudaStreamDestroy(cs2);
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
        if (b->d_tab) cudaFree(b->d_tab);
        if (b->d_tbr) cudaFree(b->d_tbr);
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
    if (b->d_tab) cudaFree(b->d_tab);
    if (b->d_tbr) cudaFree(b->d_tbr);
    delete b;
    return JACOBI_OK;
}

int jacobi_batch_run_rhs(jacobi_batch_h b, void *const *A, void *const *B, const void *const *RHS,
                         jacobi_stream_t stream)
{
    if (!b || !A || !B) return JACOBI_ERR_ARG;
    for (int g = 0; g < b->n; ++g) {
        if (!A[g] || !B[g] || A[g] == B[g]) return JACOBI_ERR_ARG;
        // the blocked FP32 passes have no source term
        if (RHS && RHS[g] && !engine_grid(b, b->grids[(size_t)g])) return JACOBI_ERR_UNSUPPORTED;
    }
    for (int g = 0; g < b->n; ++g) {
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
    b->engine = JACOBI_BATCH_PERSISTENT;
    b->bx = bx;
    b->by = by;
    b->bz = bz;
    layout(b);
    return build_graph(b);
}

int jacobi_batch_set_engine(jacobi_batch_h b, int engine, int kz)
{
    if (!b || (engine != JACOBI_BATCH_PERSISTENT && engine != JACOBI_BATCH_SWEEPS) || kz < 0) return JACOBI_ERR_ARG;
    b->engine = engine;
    if (kz > 0) b->kz = kz;
    layout(b);
    return build_graph(b);
}

int jacobi_batch_set_fp32_depth(jacobi_batch_h b, int depth)
{
    if (!b || depth < 1 || depth > 4) return JACOBI_ERR_ARG;
    b->fp32_depth = depth;
    layout(b);
    return build_graph(b);
}

int jacobi_batch_get_fp32_depth(jacobi_batch_h b, int *depth)
{
    if (!b || !depth) return JACOBI_ERR_ARG;
    *depth = b->fp32_depth;
    return JACOBI_OK;
}

int jacobi_batch_get_engine(jacobi_batch_h b, int *engine, int *kz)
{
    if (!b) return JACOBI_ERR_ARG;
    if (engine) *engine = b->engine;
    if (kz) *kz = b->kz;
    return JACOBI_OK;
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
    if (!b || mode < 0 || mode > 2 || limit_ms < 1) return JACOBI_ERR_ARG;
    if (mode == 1 && b->engine != JACOBI_BATCH_PERSISTENT) return JACOBI_ERR_UNSUPPORTED;
    if (mode == 2 && !kChecked) return JACOBI_ERR_UNSUPPORTED;
    b->fault_mode = (mode == 1) ? 1 : 0;
    b->check_shrink = (mode == 2) ? 1 : 0;
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
    bool any32 = false;
    for (const BatchGrid &G : b->grids) any32 = any32 || (G.dtype == JACOBI_F32 && G.T > 0);
    // candidates: {engine, bx, by, bz or kz, FP32 depth}; the blocked FP32
    // depths only where the batch has FP32 grids to sweep
    const int cands[][5] = {{JACOBI_BATCH_SWEEPS, 0, 0, 8, 1},       {JACOBI_BATCH_SWEEPS, 0, 0, 16, 1},
                            {JACOBI_BATCH_SWEEPS, 0, 0, 32, 1},      {JACOBI_BATCH_PERSISTENT, 32, 4, 0, 1},
                            {JACOBI_BATCH_PERSISTENT, 32, 8, 0, 1},  {JACOBI_BATCH_PERSISTENT, 32, 16, 0, 1},
                            {JACOBI_BATCH_PERSISTENT, 64, 4, 0, 1},  {JACOBI_BATCH_PERSISTENT, 64, 8, 0, 1},
                            {JACOBI_BATCH_PERSISTENT, 128, 2, 0, 1}, {JACOBI_BATCH_PERSISTENT, 32, 8, 64, 1},
                            {JACOBI_BATCH_SWEEPS, 0, 0, 16, 2},      {JACOBI_BATCH_SWEEPS, 0, 0, 16, 3},
                            {JACOBI_BATCH_SWEEPS, 0, 0, 32, 2},      {JACOBI_BATCH_SWEEPS, 0, 0, 32, 3}};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return JACOBI_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return JACOBI_ERR_CUDA;
    }
    double best = -1.0;
    int beng = b->engine, bkz = b->kz, bbx = b->bx, bby = b->by, bbz = b->bz, bdep = b->fp32_depth, st = JACOBI_OK;
    for (const auto &t : cands) {
        if (t[4] > 1 && !any32) continue;
        b->fp32_depth = t[4];
        if (t[0] == JACOBI_BATCH_SWEEPS) {
            b->bx = bbx;
            b->by = bby;
            b->bz = bbz;
            st = jacobi_batch_set_engine(b, t[0], t[3]);
        } else {
            b->engine = t[0];
            st = jacobi_batch_set_tile(b, t[1], t[2], t[3]);
        }
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
            beng = t[0];
            bdep = t[4];
            if (t[0] == JACOBI_BATCH_SWEEPS) {
                bkz = t[3];
            } else {
                bbx = t[1];
                bby = t[2];
                bbz = t[3];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != JACOBI_OK) return st;
    if (glups) *glups = best;
    b->engine = beng;
    b->fp32_depth = bdep;
    b->kz = bkz;
    b->bx = bbx;
    b->by = bby;
    b->bz = bbz;
    layout(b);
    return build_graph(b);
}

}  // extern "C"
