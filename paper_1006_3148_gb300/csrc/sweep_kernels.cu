// Sweep kernels of the library:
//   halo_copy_kernel   - boundary copy A -> B before the first pass
//   plain_pass_kernel  - one sweep per launch, operands from global memory
//                        (the single-pass baseline, code balance of Eq. 2)
//   tb_pass_kernel     - one pass of depth D: a z-streaming pipeline in which
//                        the D CTAs of a thread-block cluster each apply one
//                        time level and hand z-planes to the next CTA
//                        through distributed shared memory (tb_pass.cuh;
//                        its variants are instantiated in tb_inst_*.cu)
//
// The time-skewed pass is the GPU form of pipelined temporal blocking
// (Sect. 2.1): CTA s of the cluster plays thread s of a team that shares a
// cache, the cluster's distributed shared memory plays the shared L3, and
// z-planes play the blocks handed down the pipeline.  Level s works on
// plane k-s+1 while level 1 loads plane k+1 (the one-block shift of Fig. 1
// becomes a one-plane lag in z).  The ring of R plane slots between two
// levels enforces the two distance conditions of Eq. (3): a consumer waits
// until its producer is at least one plane ahead (the race bound d_l) and a
// producer waits until its consumer has released the slot it is about to
// overwrite (the looseness bound d_u = R).  In x and y every level works on
// the tile widened by D-s cells (the multi-layer halo of Sect. 3.1: update
// s covers a region h-s layers larger), so no level ever needs data from a
// neighbouring tile.
#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "arith.cuh"
#include "checked.cuh"
#include "grid.cuh"
#include "jacobi_internal.h"
#include "ptx.cuh"

namespace jac {

// ------------------------------------------------------------------ halo
template <typename T>
__global__ void halo_copy_kernel(const T *__restrict__ A, T *__restrict__ B, int nx, int ny, int nz, int *status,
                                 long long shrink)
{
    const long long total = halo_count(nx, ny, nz);
    const long long S = checked_grid_elems(nx, ny, nz, shrink);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long idx = halo_cell(t, nx, ny, nz);
        if (in_bounds(idx, 1, S, status)) B[idx] = A[idx];
    }
}

// ------------------------------------------------------------------ fill
template <typename T>
__global__ void fill_kernel(T *p, long long n, T v)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

// ----------------------------------------------------------------- plain
// One sweep per launch.  Thread (i, j) walks kz planes of its column with the
// values at k-1, k, k+1 in registers; the four in-plane neighbours come from
// global memory (mostly L1 hits: neighbouring threads load them too).  RHS:
// a source term g (same layout as the grid) is added to the neighbour sum
// before the division, (sum + g) / 6 (the Poisson sweeps).
template <typename T, bool RHS>
__global__ void __launch_bounds__(1024) plain_pass_kernel(const PlainArgs a)
{
    // (row block, z chunk) pairs are numbered t = yb + gy * zc and spread
    // over grid y and z (each at most 65535 blocks).  A loop over several
    // pairs per block would be simpler but costs a third of the bandwidth
    // (the compiler then schedules the plane loop's loads less well).
    const long long t = blockIdx.y + (long long)gridDim.y * blockIdx.z;
    if (t >= (long long)a.gy * a.gz) return;
    const int yb = (int)(t % a.gy), zc = (int)(t / a.gy);
    const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    const int j = 1 + yb * blockDim.y + threadIdx.y;
    if (i > a.nx || j > a.ny) return;
    const long long NXP = a.nx + 2, plane = NXP * (a.ny + 2);
    const int kb = 1 + zc * a.kz;
    const int ke = (a.nz + 1 - kb < a.kz) ? a.nz + 1 : kb + a.kz;
    const long long c0 = kb * plane + j * NXP + i;
    const T *__restrict__ p = static_cast<const T *>(a.src) + c0;
    T *__restrict__ q = static_cast<T *>(a.dst) + c0;
    const T *__restrict__ g = RHS ? static_cast<const T *>(a.rhs) + c0 : nullptr;
    const int nxp = a.nx + 2;
    // checked build: every element offset against the grid's extent
    const T *sb = static_cast<const T *>(a.src), *gb = static_cast<const T *>(a.rhs);
    const T *db = static_cast<const T *>(a.dst);
    const long long S = checked_grid_elems(a.nx, a.ny, a.nz, a.shrink);
    auto ld = [&](const T *ptr, const T *base) { return in_bounds(ptr - base, 1, S, a.status) ? __ldg(ptr) : T(0); };
    T lo = ld(p - plane, sb), mid = ld(p, sb);
#pragma unroll 4
    for (int k = kb; k < ke; ++k) {
        const T hi = ld(p + plane, sb);
        if (RHS) {
            const T v = Arith<T>::update_rhs(ld(p - 1, sb), ld(p + 1, sb), ld(p - nxp, sb), ld(p + nxp, sb), lo, hi,
                                             ld(g, gb));
            if (in_bounds(q - db, 1, S, a.status)) *q = v;
            g += plane;
        } else {
            const T v = Arith<T>::update(ld(p - 1, sb), ld(p + 1, sb), ld(p - nxp, sb), ld(p + nxp, sb), lo, hi);
            if (in_bounds(q - db, 1, S, a.status)) *q = v;
        }
        lo = mid;
        mid = hi;
        p += plane;
        q += plane;
    }
}

// Single-pass kernel with two x cells per thread (rows of even pitch, nx
// even).  Thread pair m of a row covers cells (2m, 2m+1), so the pairs tile
// the whole row, halo cells included; every value is one aligned 8-byte
// (FP32) or 16-byte (FP64) load.  The x-neighbours come from the adjacent
// lanes' centre values (shuffles; lanes 0 and 31 load the cell beyond their
// pair) and the y- and z-neighbours are vector loads, so a cell costs 1.5
// vector loads instead of the scalar kernel's five loads.  Both cells' Eq.
// (1) sums keep the scalar kernel's left-to-right order (FP32: packed
// additions).  Halo cells (x = 0, nx+1) are written back with their own
// value, which equals the destination's halo.
template <typename T>
struct Pair;
template <>
struct Pair<float> {
    using V = float2;
    static __device__ __forceinline__ V update(float w, V mid, float e, V ym, V yp, V lo, V hi)
    {
        V s = __fadd2_rn(make_float2(w, mid.x), make_float2(mid.y, e));
        s = __fadd2_rn(s, ym);
        s = __fadd2_rn(s, yp);
        s = __fadd2_rn(s, lo);
        s = __fadd2_rn(s, hi);
        return __fmul2_rn(s, make_float2(1.0f / 6.0f, 1.0f / 6.0f));
    }
    static __device__ __forceinline__ V update_rhs(float w, V mid, float e, V ym, V yp, V lo, V hi, V g)
    {
        V s = __fadd2_rn(make_float2(w, mid.x), make_float2(mid.y, e));
        s = __fadd2_rn(s, ym);
        s = __fadd2_rn(s, yp);
        s = __fadd2_rn(s, lo);
        s = __fadd2_rn(s, hi);
        s = __fadd2_rn(s, g);
        return __fmul2_rn(s, make_float2(1.0f / 6.0f, 1.0f / 6.0f));
    }
};
template <>
struct Pair<double> {
    using V = double2;
    static __device__ __forceinline__ V update(double w, V mid, double e, V ym, V yp, V lo, V hi)
    {
        V o;
        o.x = Arith<double>::update(w, mid.y, ym.x, yp.x, lo.x, hi.x);
        o.y = Arith<double>::update(mid.x, e, ym.y, yp.y, lo.y, hi.y);
        return o;
    }
    static __device__ __forceinline__ V update_rhs(double w, V mid, double e, V ym, V yp, V lo, V hi, V g)
    {
        V o;
        o.x = Arith<double>::update_rhs(w, mid.y, ym.x, yp.x, lo.x, hi.x, g.x);
        o.y = Arith<double>::update_rhs(mid.x, e, ym.y, yp.y, lo.y, hi.y, g.y);
        return o;
    }
};

template <typename T, bool RHS>
__global__ void __launch_bounds__(1024) plain_x2_kernel(const PlainArgs a)
{
    using V = typename Pair<T>::V;
    const long long t = blockIdx.y + (long long)gridDim.y * blockIdx.z;
    if (t >= (long long)a.gy * a.gz) return;  // uniform per block
    const int yb = (int)(t % a.gy), zc = (int)(t / a.gy);
    const int m = blockIdx.x * blockDim.x + threadIdx.x;  // pair index in the row
    const int j = 1 + yb * blockDim.y + threadIdx.y;
    const int npairs = (a.nx + 2) >> 1;
    // Whole warps stay together for the shuffles; lanes past the row or the
    // grid load nothing and store nothing.
    const bool live = (m < npairs) && (j <= a.ny);
    const int lane = threadIdx.x & 31;
    const long long NXP = a.nx + 2, plane = NXP * (a.ny + 2);
    const int kb = 1 + zc * a.kz;
    const int ke = (a.nz + 1 - kb < a.kz) ? a.nz + 1 : kb + a.kz;
    const long long c0 = kb * plane + (long long)(live ? j : 1) * NXP + 2 * (long long)(live ? m : 0);
    const T *__restrict__ p = static_cast<const T *>(a.src) + c0;
    const V *__restrict__ p2 = reinterpret_cast<const V *>(p);
    V *__restrict__ q2 = reinterpret_cast<V *>(static_cast<T *>(a.dst) + c0);
    const V *__restrict__ g2 = RHS ? reinterpret_cast<const V *>(static_cast<const T *>(a.rhs) + c0) : nullptr;
    const long long P2 = plane >> 1, R2 = NXP >> 1;  // plane and row in pairs
    V zero;
    zero.x = T(0);
    zero.y = T(0);
    // checked build: every element offset against the grid's extent
    const T *sb = static_cast<const T *>(a.src), *gb = static_cast<const T *>(a.rhs);
    const T *db = static_cast<const T *>(a.dst);
    const long long S = checked_grid_elems(a.nx, a.ny, a.nz, a.shrink);
    auto ld2 = [&](const V *ptr, const T *base) {
        return in_bounds(reinterpret_cast<const T *>(ptr) - base, 2, S, a.status) ? __ldg(ptr) : zero;
    };
    auto ld1 = [&](const T *ptr) { return in_bounds(ptr - sb, 1, S, a.status) ? __ldg(ptr) : T(0); };
    const bool left_halo = (m == 0), right_halo = (2 * m + 1 == a.nx + 1);
    V lo = live ? ld2(p2 - P2, sb) : zero, mid = live ? ld2(p2, sb) : zero;
#pragma unroll 4
    for (int k = kb; k < ke; ++k) {
        V hi = zero, ym = zero, yp = zero, gv = zero;
        T w = T(0), e = T(0);
        if (live) {
            hi = ld2(p2 + P2, sb);
            if (RHS) gv = ld2(g2, gb);
            ym = ld2(p2 - R2, sb);
            yp = ld2(p2 + R2, sb);
            // Cells beyond the pair at the warp's ends.  For pair 0 the cell
            // left of x = 0 is the previous row's last halo cell (in the
            // array, result unused); likewise right of x = nx+1.
            if (lane == 0) w = ld1(p - 1);
            if (lane == 31) e = ld1(p + 2);
        }
        const T wl = __shfl_up_sync(0xffffffffu, mid.y, 1);
        const T er = __shfl_down_sync(0xffffffffu, mid.x, 1);
        if (lane != 0) w = wl;
        if (lane != 31) e = er;
        V o = RHS ? Pair<T>::update_rhs(w, mid, e, ym, yp, lo, hi, gv) : Pair<T>::update(w, mid, e, ym, yp, lo, hi);
        if (left_halo) o.x = mid.x;
        if (right_halo) o.y = mid.y;
        if (live && in_bounds(reinterpret_cast<const T *>(q2) - db, 2, S, a.status)) *q2 = o;
        lo = mid;
        mid = hi;
        p2 += P2;
        q2 += P2;
        if (RHS) g2 += P2;
        p += plane;
    }
}

// ------------------------------------------------------------------- host
namespace {

struct Variant {
    int nc, maxc;
};
constexpr size_t kRingBudget = 100 * 1024;  // auto ring depth: fit 2 CTAs per SM
// Preferred order: the widest CTA whose threads cover the level-1 groups
// (more warps per SM hide the latency of the per-plane pipeline).
constexpr Variant kVariants[] = {{512, 1}, {512, 2}, {256, 1}, {256, 2}, {256, 4}, {256, 6}, {128, 2}, {128, 4}, {128, 6}, {128, 8}};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);
constexpr int kSmemMax = 232448;  // 227 KB per CTA on sm_100-class GPUs

// The variants' kernels are instantiated in tb_inst_0.cu .. tb_inst_3.cu.
const void *tb_kernel(int dtype, int nc, int maxc)
{
    const void *f = (dtype == JACOBI_F64) ? tb_kernel_part0(nc, maxc) : tb_kernel_part2(nc, maxc);
    if (!f) f = (dtype == JACOBI_F64) ? tb_kernel_part1(nc, maxc) : tb_kernel_part3(nc, maxc);
    return f;
}

cudaError_t prepare(const void *fn) { return ensure_cluster_attrs(fn, kSmemMax); }

}  // namespace

cudaError_t tb_configure(int dtype, int depth, int bx, int by, int ring, int threads, TbLaunch *out)
{
    const int es = dtype == JACOBI_F64 ? 8 : 4;
    const int V = 16 / es;
    TbLaunch L;
    L.W = bx + 2 * depth;
    L.H = by + 2 * depth;
    // columns from xs (a group left of x0-D, rounded down to VEC) to the right
    // neighbour of the last group of x1+D
    L.Wp = V * ((bx + 2 * depth + 3 * V + V - 1) / V);
    const size_t slot = (size_t)L.H * L.Wp * es;
    if (ring == 0) {
        ring = 4;
        if (16 * slot <= kRingBudget) ring = 16;
        else if (8 * slot <= kRingBudget) ring = 8;
    }
    if (ring != 4 && ring != 8 && ring != 16) return cudaErrorInvalidValue;
    L.R = ring;
    L.smem = (size_t)L.R * slot + 3 * 8 * (size_t)L.R;
    // groups of the widest output region (level 1): one extra group for the
    // alignment of its first column
    const long long groups = (long long)((bx + 2 * (depth - 1) + V - 1) / V + 1) * (by + 2 * (depth - 1));
    // Automatic width: the fewest threads (up to 2 groups each) that cover
    // the groups, else more groups per thread; a forced width takes the
    // smallest group count per thread that covers the tile.
    L.nc = 0;
    if (threads == 0) {
        for (int nc : {128, 256, 512})
            if ((long long)nc * 2 >= groups) {
                threads = nc;
                break;
            }
        if (threads == 0) threads = 512;
    }
    int best = 1 << 30;
    for (const Variant &v : kVariants)
        if (v.nc == threads && (long long)v.nc * v.maxc >= groups && v.maxc < best) {
            L.nc = v.nc;
            L.maxc = v.maxc;
            best = v.maxc;
        }
    if (L.nc == 0)  // forced width too narrow for this tile: widest that fits
        for (const Variant &v : kVariants)
            if ((long long)v.nc * v.maxc >= groups && (L.nc == 0 || v.nc * v.maxc < L.nc * L.maxc)) {
                L.nc = v.nc;
                L.maxc = v.maxc;
            }
    if (L.nc == 0 || L.smem > (size_t)kSmemMax) return cudaErrorInvalidConfiguration;
    *out = L;
    return cudaSuccess;
}

cudaError_t tb_launch(int dtype, const TbArgs &a, const TbLaunch &L, cudaStream_t s)
{
    const void *fn = tb_kernel(dtype, L.nc, L.maxc);
    if (!fn) return cudaErrorInvalidConfiguration;
    static bool prepared[2][kNumVariants] = {};
    int vi = 0;
    while (kVariants[vi].nc != L.nc || kVariants[vi].maxc != L.maxc) ++vi;
    if (!prepared[dtype][vi]) {
        cudaError_t e = prepare(fn);
        if (e != cudaSuccess) return e;
        prepared[dtype][vi] = true;
    }
    const int nty = (a.ny + a.by - 1) / a.by;
    const int ntz = (a.nz + a.bz - 1) / a.bz;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(a.depth * a.ntx), (unsigned)nty, (unsigned)ntz);
    cfg.blockDim = dim3((unsigned)L.nc, 1, 1);
    cfg.dynamicSmemBytes = L.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)a.depth;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {const_cast<TbArgs *>(&a)};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t tb_max_clusters(int dtype, const TbLaunch &L, int depth, int *clusters)
{
    const void *fn = tb_kernel(dtype, L.nc, L.maxc);
    if (!fn) return cudaErrorInvalidConfiguration;
    cudaError_t e = prepare(fn);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)depth, 1, 1);
    cfg.blockDim = dim3((unsigned)L.nc, 1, 1);
    cfg.dynamicSmemBytes = L.smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)depth;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(clusters, fn, &cfg);
}

cudaError_t plain_launch(int dtype, PlainArgs a, cudaStream_t s)
{
    a.gy = (a.ny + a.ty - 1) / a.ty;
    a.gz = (a.nz + a.kz - 1) / a.kz;
    const long long pairs = (long long)a.gy * a.gz;
    const long long by = std::min<long long>(pairs, 65535), bz = (pairs + by - 1) / by;
    if (bz > 65535) return cudaErrorInvalidConfiguration;
    dim3 block((unsigned)a.tx, (unsigned)a.ty, 1);
    dim3 grid((unsigned)((a.nx + a.tx - 1) / a.tx), (unsigned)by, (unsigned)bz);
    if (dtype == JACOBI_F64) {
        if (a.rhs) plain_pass_kernel<double, true><<<grid, block, 0, s>>>(a);
        else plain_pass_kernel<double, false><<<grid, block, 0, s>>>(a);
    } else {
        if (a.rhs) plain_pass_kernel<float, true><<<grid, block, 0, s>>>(a);
        else plain_pass_kernel<float, false><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t plain_x2_launch(int dtype, PlainArgs a, cudaStream_t s)
{
    a.gy = (a.ny + a.ty - 1) / a.ty;
    a.gz = (a.nz + a.kz - 1) / a.kz;
    const long long pairs = (long long)a.gy * a.gz;
    const long long by = std::min<long long>(pairs, 65535), bz = (pairs + by - 1) / by;
    if (bz > 65535) return cudaErrorInvalidConfiguration;
    const int npairs = (a.nx + 2) / 2;
    dim3 block((unsigned)a.tx, (unsigned)a.ty, 1);
    dim3 grid((unsigned)((npairs + a.tx - 1) / a.tx), (unsigned)by, (unsigned)bz);
    if (dtype == JACOBI_F64) {
        if (a.rhs) plain_x2_kernel<double, true><<<grid, block, 0, s>>>(a);
        else plain_x2_kernel<double, false><<<grid, block, 0, s>>>(a);
    } else {
        if (a.rhs) plain_x2_kernel<float, true><<<grid, block, 0, s>>>(a);
        else plain_x2_kernel<float, false><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t halo_copy_launch(int dtype, const void *A, void *B, int nx, int ny, int nz, cudaStream_t s, int *status,
                             long long shrink)
{
    const long long total = halo_count(nx, ny, nz);
    const int block = 256;
    const long long want = (total + block - 1) / block;
    const unsigned grid = (unsigned)std::min<long long>(want, 152 * 16);
    if (dtype == JACOBI_F64)
        halo_copy_kernel<double><<<grid, block, 0, s>>>(static_cast<const double *>(A), static_cast<double *>(B), nx,
                                                          ny, nz, status, shrink);
    else
        halo_copy_kernel<float><<<grid, block, 0, s>>>(static_cast<const float *>(A), static_cast<float *>(B), nx, ny,
                                                        nz, status, shrink);
    return cudaGetLastError();
}

cudaError_t fill_launch(int dtype, void *p, long long n, double v, cudaStream_t s)
{
    const unsigned grid = (unsigned)std::min<long long>((n + 255) / 256, 152 * 16);
    if (dtype == JACOBI_F64) fill_kernel<double><<<grid, 256, 0, s>>>(static_cast<double *>(p), n, v);
    else fill_kernel<float><<<grid, 256, 0, s>>>(static_cast<float *>(p), n, (float)v);
    return cudaGetLastError();
}

int plan_passes(int T, int d, int *depths, int max_passes)
{
    if (T <= 0) return 0;
    if (d < 1) d = 1;
    int P = (T + d - 1) / d;
    if ((P - T) % 2 != 0) ++P;  // P must have the parity of T
    if (P > max_passes) return -1;
    const int base = T / P, rem = T % P;
    for (int p = 0; p < P; ++p) depths[p] = base + (p < rem ? 1 : 0);
    return P;
}

}  // namespace jac
