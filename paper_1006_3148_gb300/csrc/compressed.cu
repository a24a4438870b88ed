// Compressed grid (Sect. 2.1): Jacobi sweeps in ONE buffer, without the
// second grid of the ping-pong scheme.
//
// The paper writes each result shifted by (-1,-1,-1) in the first sweep and
// by (+1,+1,+1) in the next, with the loops reversed, so that a sequential
// sweep never overwrites a value it still has to read.  Here many CTAs run
// at once, so the shift is along z only and S planes long: the buffer holds
// nz + 2 + S planes, and the grid sits either in the upper position
// (logical plane k at buffer plane k + S) or in the lower one (at plane k).
// A pass of depth D (D sweeps, temporally blocked) reads the grid in one
// position and writes the result into the other: an upper-to-lower pass
// overwrites planes that held its own input S planes further down.
//
// Work items are (x-y tile, z chunk of bz planes), one CTA each.  Item
// (t, j) reads input planes [z0_j - D, z0_j + bz + D) and writes output
// planes [z0_j, z0_j + bz) (plus the boundary plane 0 or nz+1 for the first
// and last chunks), i.e. input planes [z0_j - S, z0_j - S + bz + 1) in an
// upper-to-lower pass.  With
// S = w*bz + D + 1 and bz >= 2D + 2 those are read only by the items of
// chunks j-w and j-w-1, and among them (the x-y regions reach D cells, less
// than a tile, past their tile) only by the items of tile t and its eight
// neighbours.  Items are handed out in chunk order (increasing z for an
// upper-to-lower pass, decreasing for the reverse, the counterpart of the
// paper's reversed loops) from an atomic ticket that each CTA takes when it
// starts, and item (t, j) starts only after those up to 18 items (chunks
// j+w, j+w+1 in reverse) have finished: no item overwrites a value another
// has yet to read, and a column of tiles runs up to w chunks ahead of its
// neighbours.  Every wait is on items with smaller tickets, taken by CTAs
// that started earlier and never wait on later ones, so the schedule cannot
// deadlock; each wait is also bounded in time.
//
// FP32 items run the register-blocked temporally blocked body of the
// one-CTA kernel (tbr_kernels.cuh; 64 x 32 regions, depth 1..4); FP64 items
// run a single-sweep column walk (FP64 sweeps are bound by the arithmetic
// pipes, where blocking does not pay).  Each item also moves the Dirichlet
// cells of its footprint (the x-y ring of its planes, and planes 0 / nz+1
// for the first / last chunk) to the new position.
#include <algorithm>

#include "arith.cuh"
#include "checked.cuh"
#include "jacobi_internal.h"
#include "ptx.cuh"
#include "tbr_kernels.cuh"

namespace jac {
namespace {

constexpr int kCgF64X = 32, kCgF64Y = 8;  // FP64 item: 32 x 8 columns, one thread each

struct CgArgs {
    TbrArgs t;          // FP32 body: src / dst at this pass's positions
    const void *src;    // grid at the read position (plane 0)
    void *dst;          // grid at the write position (plane 0)
    int nx, ny, nz;
    int bz, w, nch;     // z chunk, chunk waves, chunks
    int ntx, nty;       // x-y tiles
    int fx0, fbx;       // tile tix covers output columns fx0 + tix*fbx ...
    int fby;            // ... and rows 1 + tiy*fby ...
    int up;             // 1: read the upper position, write the lower one
    long long items;
    int *head, *done, *status;  // done[j * ntx * nty + t]: item (t, j) finished
    unsigned long long limit_ns;
    int fault_mode;
    long long shrink;
};

__device__ __forceinline__ int ld_acquire_gpu(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Waits until *p >= want (bounded; gives up early once the status word is
// set).  Returns false on timeout or abort.  Called by several lanes at once.
__device__ bool wait_count(const int *p, int want, unsigned long long limit_ns, const volatile int *status)
{
    if (ld_acquire_gpu(p) >= want) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        __nanosleep(128);
        if (ld_acquire_gpu(p) >= want) return true;
        if ((it & 31u) == 0u) {
            if (*status != 0) return false;
            if (globaltimer_ns() - t0 > limit_ns) return false;
        }
    }
}

// Takes this CTA's item (the next ticket); returns false when none is left.
// Warp 0 takes the ticket and does the waits; one barrier then hands the
// item, its column c, chunk j and whether the waits held to the whole CTA.
__device__ bool take_item(const CgArgs &a, long long &q, int &c, int &j, bool &ok)
{
    __shared__ long long s_item;
    __shared__ int s_ok;
    const int ncols = a.ntx * a.nty;
    if (threadIdx.x < 32) {
        const int l = threadIdx.x;
        long long item = 0;
        if (l == 0) item = (long long)atomicAdd(a.head, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        bool good = true;
        if (item < a.items) {
            // lane l < 18 waits for item (tile (tix + l%3 - 1, tiy + (l/3)%3 - 1),
            // chunk j -+ (w + l/9)), if it exists
            const long long qq = item / ncols;
            const int cc = (int)(item % ncols);
            const int jc = a.up ? (int)qq : a.nch - 1 - (int)qq;
            const int tix = cc % a.ntx, tiy = cc / a.ntx;
            const int nx_ = tix + l % 3 - 1, ny_ = tiy + (l / 3) % 3 - 1;
            const int jj = a.up ? jc - a.w - l / 9 : jc + a.w + l / 9;
            if (l < 18 && nx_ >= 0 && nx_ < a.ntx && ny_ >= 0 && ny_ < a.nty && jj >= 0 && jj < a.nch)
                good = wait_count(a.done + (long long)jj * ncols + ny_ * a.ntx + nx_, 1, a.limit_ns, a.status);
        }
        good = __all_sync(0xffffffffu, good);
        if (l == 0) {
            if (!good) atomicCAS(a.status, 0, JACOBI_ERR_TIMEOUT);
            s_item = item;
            s_ok = good;
        }
    }
    __syncthreads();
    const long long item = s_item;
    ok = s_ok != 0;
    if (item >= a.items) return false;
    q = item / ncols;
    c = (int)(item % ncols);
    j = a.up ? (int)q : a.nch - 1 - (int)q;
    return true;
}

// Publishes the end of an item: every thread's reads and writes of the item
// come before the flag (barrier, then a release store at device scope by
// one thread, cumulative over the writes the barrier ordered before it).
__device__ void finish_item(const CgArgs &a, long long q, int c, int j)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        // test hook: the first item never reports, so waits on it run out
        if (!(a.fault_mode == 1 && q == 0 && c == 0))
            asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(a.done + (long long)j * a.ntx * a.nty + c), "r"(1)
                         : "memory");
    }
}

// Copies the Dirichlet cells of a tile's footprint, columns [fx0, fx1) x
// rows [fy0, fy1), from the read position to the write position: the x-y
// ring cells of planes [z0, z1) and, for the first / last chunk, every
// footprint cell of plane 0 / nz+1.  Out of line, with its operands by
// value (a reference to the kernel's parameters would move them to local
// memory for the whole kernel).
template <typename T>
__device__ __noinline__ void move_boundary(const T *src, T *dst, int nx, int ny, int nz, int fx0, int fx1, int fy0,
                                           int fy1, int z0, int z1, bool first, bool last, int *status,
                                           long long shrink)
{
    const long long P = nx + 2, plane = P * (ny + 2);
    const long long SG = checked_grid_elems(nx, ny, nz, shrink);
    const int w = fx1 - fx0, h = fy1 - fy0;
    auto mv = [&](long long off) {
        if (in_bounds(off, 1, SG, status)) dst[off] = __ldcg(src + off);
    };
    for (int e = 0; e < 2; ++e) {
        if (!(e == 0 ? first : last)) continue;
        const long long pz = (e == 0 ? 0 : nz + 1) * plane;
        for (int i = threadIdx.x; i < w * h; i += blockDim.x) mv(pz + (long long)(fy0 + i / w) * P + fx0 + i % w);
    }
    const int yl = fy0 == 0, yr = fy1 == ny + 2, xl = fx0 == 0, xr = fx1 == nx + 2;
    const int nrow = (yl + yr) * w, ncol = (xl + xr) * (h - yl - yr);
    const int per = nrow + ncol;
    if (per == 0) return;
    const long long n = (long long)(z1 - z0) * per;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const int p = z0 + (int)(i / per), r = (int)(i % per);
        int x, y;
        if (r < nrow) {
            x = fx0 + r % w;
            y = (yl && r < w) ? 0 : ny + 1;
        } else {
            const int k = r - nrow, hh = h - yl - yr;
            y = fy0 + yl + k % hh;
            x = (xl && k < hh) ? 0 : nx + 1;
        }
        mv(p * plane + (long long)y * P + x);
    }
}

// The footprint of tile (tix, tiy) and the boundary move of item (tile, j).
template <typename T>
__device__ __forceinline__ void move_item_boundary(const CgArgs &a, int tix, int tiy, int j)
{
    const int fx0 = tix == 0 ? 0 : a.fx0 + tix * a.fbx;
    const int fx1 = tix == a.ntx - 1 ? a.nx + 2 : a.fx0 + (tix + 1) * a.fbx;
    const int fy0 = tiy == 0 ? 0 : 1 + tiy * a.fby;
    const int fy1 = tiy == a.nty - 1 ? a.ny + 2 : 1 + (tiy + 1) * a.fby;
    const int z0 = 1 + j * a.bz, z1 = min(z0 + a.bz, a.nz + 1);
    const bool first = j == 0, last = j == a.nch - 1;
    // only footprints on the grid's x-y boundary, and the first and last
    // chunks, hold Dirichlet cells
    if (!(first || last || fx0 == 0 || fy0 == 0 || fx1 == a.nx + 2 || fy1 == a.ny + 2)) return;
    move_boundary<T>(static_cast<const T *>(a.src), static_cast<T *>(a.dst), a.nx, a.ny, a.nz, fx0, fx1, fy0, fy1, z0,
                     z1, first, last, a.status, a.shrink);
}

template <int D, int A>
__global__ void __launch_bounds__(128, (TbrMinBlocks<D, 128, A>::value)) cg_f32_kernel(const CgArgs a)
{
    long long q;
    int c, j;
    bool ok;
    if (!take_item(a, q, c, j, ok)) return;
    if (ok) {
        const int tix = c % a.ntx, tiy = c / a.ntx;
        tbr_cta<D, 16, 8, A>(a.t, tix, tiy, j);
        move_item_boundary<float>(a, tix, tiy, j);
    }
    finish_item(a, q, c, j);
}

// FP64 item: one sweep of a 32 x 8 column tile over the chunk's planes, the
// values at k-1, k, k+1 of the thread's column in registers, the in-plane
// neighbours by ordinary (L1-cached, coherent) loads: within a pass an
// address is only read before it is overwritten, so no line is read stale.
__global__ void __launch_bounds__(kCgF64X *kCgF64Y) cg_f64_kernel(const CgArgs a)
{
    long long q;
    int c, j;
    bool ok;
    if (!take_item(a, q, c, j, ok)) return;
    const int tix = c % a.ntx, tiy = c / a.ntx;
    const int z0 = 1 + j * a.bz, z1 = min(z0 + a.bz, a.nz + 1);
    if (ok) {
        const int x = 1 + tix * kCgF64X + (int)threadIdx.x % kCgF64X;
        const int y = 1 + tiy * kCgF64Y + (int)threadIdx.x / kCgF64X;
        if (x <= a.nx && y <= a.ny) {
            const long long P = a.nx + 2, plane = P * (a.ny + 2);
            const long long c0 = (long long)z0 * plane + (long long)y * P + x;
            const double *sb = static_cast<const double *>(a.src);
            double *db = static_cast<double *>(a.dst);
            const double *p = sb + c0;
            double *o = db + c0;
            const int nxp = a.nx + 2;
            const long long SG = checked_grid_elems(a.nx, a.ny, a.nz, a.shrink);
            auto ld = [&](const double *ptr) { return in_bounds(ptr - sb, 1, SG, a.status) ? *ptr : 0.0; };
            double lo = ld(p - plane), mid = ld(p);
#pragma unroll 4
            for (int k = z0; k < z1; ++k) {
                const double hi = ld(p + plane);
                const double v = Arith<double>::update(ld(p - 1), ld(p + 1), ld(p - nxp), ld(p + nxp), lo, hi);
                if (in_bounds(o - db, 1, SG, a.status)) *o = v;
                lo = mid;
                mid = hi;
                p += plane;
                o += plane;
            }
        }
        move_item_boundary<double>(a, tix, tiy, j);
    }
    finish_item(a, q, c, j);
}

template <int D, int A>
cudaError_t launch_f32(const CgArgs &a, cudaStream_t s)
{
    auto fn = cg_f32_kernel<D, A>;
    const size_t smem = ((size_t)tbr_ring(D) * 64 * 32 + 2 * (size_t)D * (2 * 8 * 64 + 2 * 8 * 16 * kTbrVY)) * 4;
    cudaError_t e = ensure_smem_limit((const void *)fn, smem);
    if (e != cudaSuccess) return e;
    fn<<<(unsigned)a.items, 128, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_f32_depth(int D, const CgArgs &a, cudaStream_t s)
{
    const bool a2 = (a.nx + 2) % 2 == 0;
    switch (D) {
    case 1: return a2 ? launch_f32<1, 2>(a, s) : launch_f32<1, 1>(a, s);
    case 2: return a2 ? launch_f32<2, 2>(a, s) : launch_f32<2, 1>(a, s);
    case 3: return a2 ? launch_f32<3, 2>(a, s) : launch_f32<3, 1>(a, s);
    case 4: return a2 ? launch_f32<4, 2>(a, s) : launch_f32<4, 1>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_f64(const CgArgs &a, cudaStream_t s)
{
    cg_f64_kernel<<<(unsigned)a.items, kCgF64X * kCgF64Y, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

long long cg_shift_planes(int depth, int bz, int waves) { return (long long)waves * bz + depth + 1; }

int cg_check(const jacobi_plan_s *h, int depth, int bz, int waves)
{
    if (depth < 1 || waves < 1 || waves > 8 || bz < 2 * depth + 2) return JACOBI_ERR_ARG;
    if (h->dtype == JACOBI_F64 && depth != 1) return JACOBI_ERR_UNSUPPORTED;
    if (h->dtype == JACOBI_F32 && depth > 4) return JACOBI_ERR_ARG;
    return JACOBI_OK;
}

int cg_sweep(jacobi_plan_s *h, void *U, int T, int upper, int *upper_out, cudaStream_t s)
{
    const int depth = h->cg_depth, bz = h->cg_bz, waves = h->cg_waves;
    const long long S = cg_shift_planes(depth, bz, waves);
    const long long plane = (long long)(h->nx + 2) * (h->ny + 2);
    const size_t esz = h->dtype == JACOBI_F64 ? 8 : 4;
    const int nch = (h->nz + bz - 1) / bz;
    CgArgs a = {};
    a.nx = h->nx;
    a.ny = h->ny;
    a.nz = h->nz;
    a.bz = bz;
    a.w = waves;
    a.nch = nch;
    a.status = h->d_status;
    a.limit_ns = h->limit_ns;
    a.shrink = h->check_shrink;
    if (h->dtype == JACOBI_F32) {
        TbrArgs t;
        t.nx = h->nx;
        t.ny = h->ny;
        t.nz = h->nz;
        t.bz = bz;
        t.status = h->d_status;
        t.shrink = h->check_shrink;
        size_t smem = 0;
        const int st = tbr_configure(depth, 64, 32, &t, &smem, nullptr);
        if (st != JACOBI_OK) return st;
        a.ntx = (h->nx + t.bx - 1) / t.bx;
        a.nty = (h->ny + t.by - 1) / t.by;
        a.fx0 = t.x_first + t.off + depth;  // = 1
        a.fbx = t.bx;
        a.fby = t.by;
        a.t = t;
    } else {
        a.ntx = (h->nx + kCgF64X - 1) / kCgF64X;
        a.nty = (h->ny + kCgF64Y - 1) / kCgF64Y;
        a.fx0 = 1;
        a.fbx = kCgF64X;
        a.fby = kCgF64Y;
    }
    a.items = (long long)a.ntx * a.nty * nch;
    if (a.items >= (1ll << 31) || (long long)a.ntx * a.nty >= (1ll << 31)) return JACOBI_ERR_UNSUPPORTED;
    const size_t need = 1 + (size_t)nch * a.ntx * a.nty;
    if (h->cg_ctl_n < need) {
        // a CUDA graph captured from an earlier call may still use the old
        // array: it is kept until the handle is destroyed
        int *p = nullptr;
        if (cudaMalloc(&p, need * sizeof(int)) != cudaSuccess) return JACOBI_ERR_ALLOC;
        if (h->cg_ctl) h->cg_old.push_back(h->cg_ctl);
        h->cg_ctl = p;
        h->cg_ctl_n = need;
    }
    a.head = h->cg_ctl;
    a.done = h->cg_ctl + 1;
    char *lo = static_cast<char *>(U), *hi = lo + (size_t)S * plane * esz;
    const int P = T == 0 ? 0 : (T + depth - 1) / depth;
    for (int q = 0; q < P; ++q) {
        const int d = std::min(depth, T - q * depth);
        a.up = upper;
        a.src = upper ? hi : lo;
        a.dst = upper ? lo : hi;
        a.t.src = a.src;
        a.t.dst = a.dst;
        a.fault_mode = h->fault_mode;
        h->fault_mode = 0;
        if (cudaMemsetAsync(h->cg_ctl, 0, need * sizeof(int), s) != cudaSuccess) return JACOBI_ERR_CUDA;
        // a shorter last pass runs its own depth on the same tiles and shift
        cudaError_t e;
        if (h->dtype == JACOBI_F32) {
            TbrArgs t = a.t;
            size_t smem = 0;
            if (tbr_configure(d, 64, 32, &t, &smem, nullptr) != JACOBI_OK) return JACOBI_ERR_ARG;
            if (d != depth) {
                // tiles of the shallower pass: own geometry, same chunks
                CgArgs b = a;
                b.t = t;
                b.ntx = (h->nx + t.bx - 1) / t.bx;
                b.nty = (h->ny + t.by - 1) / t.by;
                b.fbx = t.bx;
                b.fby = t.by;
                b.items = (long long)b.ntx * b.nty * nch;
                e = launch_f32_depth(d, b, s);
            } else {
                e = launch_f32_depth(d, a, s);
            }
        } else {
            e = launch_f64(a, s);
        }
        if (e != cudaSuccess) return JACOBI_ERR_CUDA;
        upper = !upper;
    }
    if (upper_out) *upper_out = upper;
    return JACOBI_OK;
}

}  // namespace jac
