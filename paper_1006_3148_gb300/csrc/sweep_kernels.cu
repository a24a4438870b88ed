// Sweep kernels of the library:
//   halo_copy_kernel   - boundary copy A -> B before the first pass
//   plain_pass_kernel  - one sweep per launch, operands from global memory
//                        (the single-pass baseline, code balance of Eq. 2)
//   tb_pass_kernel     - one pass of depth D: a z-streaming pipeline in which
//                        the D CTAs of a thread-block cluster each apply one
//                        time level and hand z-planes to the next CTA
//                        through distributed shared memory
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
#include "grid.cuh"
#include "jacobi_internal.h"
#include "ptx.cuh"

namespace jac {

__device__ __forceinline__ void record_error(int *status, int code)
{
    atomicCAS(status, 0, code);
}

// ------------------------------------------------------------------ halo
template <typename T>
__global__ void halo_copy_kernel(const T *__restrict__ A, T *__restrict__ B, int nx, int ny, int nz)
{
    const long long total = halo_count(nx, ny, nz);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long idx = halo_cell(t, nx, ny, nz);
        B[idx] = A[idx];
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
    T lo = __ldg(p - plane), mid = __ldg(p);
#pragma unroll 4
    for (int k = kb; k < ke; ++k) {
        const T hi = __ldg(p + plane);
        if (RHS) {
            *q = Arith<T>::update_rhs(__ldg(p - 1), __ldg(p + 1), __ldg(p - nxp), __ldg(p + nxp), lo, hi, __ldg(g));
            g += plane;
        } else {
            *q = Arith<T>::update(__ldg(p - 1), __ldg(p + 1), __ldg(p - nxp), __ldg(p + nxp), lo, hi);
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
    const bool left_halo = (m == 0), right_halo = (2 * m + 1 == a.nx + 1);
    V lo = live ? __ldg(p2 - P2) : zero, mid = live ? __ldg(p2) : zero;
#pragma unroll 4
    for (int k = kb; k < ke; ++k) {
        V hi = zero, ym = zero, yp = zero, gv = zero;
        T w = T(0), e = T(0);
        if (live) {
            hi = __ldg(p2 + P2);
            if (RHS) gv = __ldg(g2);
            ym = __ldg(p2 - R2);
            yp = __ldg(p2 + R2);
            // Cells beyond the pair at the warp's ends.  For pair 0 the cell
            // left of x = 0 is the previous row's last halo cell (in the
            // array, result unused); likewise right of x = nx+1.
            if (lane == 0) w = __ldg(p - 1);
            if (lane == 31) e = __ldg(p + 2);
        }
        const T wl = __shfl_up_sync(0xffffffffu, mid.y, 1);
        const T er = __shfl_down_sync(0xffffffffu, mid.x, 1);
        if (lane != 0) w = wl;
        if (lane != 31) e = er;
        V o = RHS ? Pair<T>::update_rhs(w, mid, e, ym, yp, lo, hi, gv) : Pair<T>::update(w, mid, e, ym, yp, lo, hi);
        if (left_halo) o.x = mid.x;
        if (right_halo) o.y = mid.y;
        if (live) *q2 = o;
        lo = mid;
        mid = hi;
        p2 += P2;
        q2 += P2;
        if (RHS) g2 += P2;
        p += plane;
    }
}

// -------------------------------------------------------- time-skewed pass
// Cells are handled in groups of VEC = 16/sizeof(T) consecutive x cells of
// one row (4 FP32 / 2 FP64), aligned so that a group starts at a global x
// that is a multiple of VEC.  Every thread owns up to MAXG groups of its
// level's output region, fixed for the whole z stream, and keeps per group
// the values at planes k-1 and k of its input level in registers (the z
// queue).  One step (output plane k) reads, per group, the rows y-1 and y+1
// of plane k and the group of plane k+1 with 16-byte shared loads, plus the
// two x-neighbours at the group's ends.
//
// Shared memory of every CTA: ring[R][H][Wp] of T.  Slot = one z-plane of
// the tile widened by D cells; element (x, y) sits at column x - xs and row
// y - (y0 - D), where xs is a multiple of VEC at least one group left of
// x0 - D (so every group's left neighbour is inside its row).  Then three
// arrays of R mbarriers:
//   in_full[s]   slot s holds its plane.  Level 1 streams its input from
//                global memory itself: each thread issues cp.async copies
//                for plane n+R-2 while computing plane n and arrives (on
//                completion of its copies) once per plane: expected count
//                NC.  Level >= 2: the producer CTA writes the plane with
//                st.async, each store completing its bytes on this barrier;
//                the barrier is armed with the plane's byte count (one
//                arrival) by warp 0 before the slot is released.
//   in_empty[s]  level 1: every warp released slot s (count NC/32), waited
//                on before copying the next plane into the slot.
//   out_empty[s] level < D: every warp of the next CTA released its slot s
//                (count NC/32, remote arrivals).
// No CTA-wide barrier runs per plane: warps advance independently, held
// together only by these slot barriers (the relaxed synchronisation of
// Sect. 2.2: a consumer waits for its producer to be one plane ahead, a
// producer waits until its consumer freed the slot, R planes of looseness).
//
// Lanes of a group outside this level's region or outside the grid compute
// values nobody reads; lanes on the grid's halo keep their own value.
__host__ __device__ __forceinline__ int floor_div(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }

template <typename T>
struct VecOf;
template <>
struct VecOf<float> {
    using V = float4;
};
template <>
struct VecOf<double> {
    using V = double2;
};

// Groups (VEC-aligned) covering [xa, xb) x [ya, yb): count per row and rows.
__device__ __forceinline__ void region_groups(int xa, int xb, int ya, int yb, int xs, int vec, int *jg0,
                                              int *gpr, int *rows)
{
    *jg0 = floor_div(xa - xs, vec);
    *gpr = floor_div(xb - xs + vec - 1, vec) - *jg0;
    *rows = yb - ya;
}

template <typename T, int NC, int MAXG, int MAXLD>
__global__ void __launch_bounds__(NC, (NC == 512 ? 2 : (NC == 128 ? 3 : 2))) tb_pass_kernel(const TbArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int VEC = 16 / (int)sizeof(T);
    constexpr int NW = NC / 32;
    using V = typename VecOf<T>::V;
    const int R = a.R, rsh = a.rshift, rmask = a.R - 1;
    const int L = R - 2;  // level-1 load lookahead (planes)
    const int D = a.depth;
    const int rank = (int)cluster_ctarank();
    const int lvl = rank + 1;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int NXP = nx + 2, NYP = ny + 2;
    const int x0 = 1 + (int)(blockIdx.x / D) * a.bx, x1 = min(x0 + a.bx, nx + 1);
    const int y0 = 1 + (int)blockIdx.y * a.by, y1 = min(y0 + a.by, ny + 1);
    const int z0 = 1 + (int)blockIdx.z * a.bz, z1 = min(z0 + a.bz, nz + 1);
    const int xs = VEC * floor_div(x0 - D, VEC) - VEC;  // global x of shared column 0
    const int ys = y0 - D;                              // global y of shared row 0
    const int Wp = a.Wp;
    const int slot_elems = a.H * Wp;
    T *ring = reinterpret_cast<T *>(smem);
    const uint32_t ring_s = smem_addr(ring);
    const uint32_t slot_bytes = (uint32_t)(slot_elems * (int)sizeof(T));
    const uint32_t in_full = ring_s + (uint32_t)R * slot_bytes;
    const uint32_t in_empty = in_full + 8u * R;
    const uint32_t out_empty = in_full + 16u * R;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const volatile int *vstatus = a.status;
    const long long plane = (long long)NYP * NXP;

    const int wl = D - lvl;  // this level's region is the tile widened by wl
    const int zo0 = max(z0 - wl, 0), zo1 = min(z1 + wl, nz + 2);
    const int zi0 = max(z0 - wl - 1, 0), zi1 = min(z1 + wl + 1, nz + 2);
    const int nin = zi1 - zi0;

    // bytes of one input plane written by the producer level (its groups)
    uint32_t in_bytes = 0;
    if (lvl > 1) {
        int jg, gp, rows;
        region_groups(max(x0 - wl - 1, 0), min(x1 + wl + 1, NXP), max(y0 - wl - 1, 0), min(y1 + wl + 1, NYP), xs, VEC,
                      &jg, &gp, &rows);
        in_bytes = (uint32_t)(gp * rows) * 16u;
    }
    if (tid == 0) {
        for (int s = 0; s < R; ++s) {
            mbar_init(in_full + 8u * s, lvl == 1 ? NC : 1);
            mbar_init(in_empty + 8u * s, NW);
            mbar_init(out_empty + 8u * s, NW);
        }
        fence_mbar_init_cluster();
        if (lvl > 1)
            for (int s = 0; s < R && s < nin; ++s) mbar_arrive_expect_tx(in_full + 8u * s, in_bytes);
    }
    cluster_sync_all();

    bool dead = false;
    auto wait = [&](uint32_t bar, int parity) {
        if (dead) return;
        if (!wait_parity_bounded(bar, (uint32_t)parity, a.limit_ns, vstatus)) {
            dead = true;
            record_error(a.status, JACOBI_ERR_TIMEOUT);
        }
    };

    // ---- level-1 input streaming.  Every row is copied in pieces of cs
    // elements, cs = the largest of VEC, 2, 1 that divides the row pitch, so
    // that a piece is naturally aligned in global memory in every row and
    // plane (the base pointer is 16-byte aligned); elements left of the first
    // or right of the last full piece of a row are copied one by one.  Every
    // row has the same piece layout, so each thread precomputes its pieces
    // (row and column inside the tile, size) once, packed in one register,
    // and re-issues them for every plane.
    const T *src = static_cast<const T *>(a.src);
    const int ix0 = max(x0 - D, 0), ix1 = min(x1 + D, NXP);
    const int iy0 = max(ys, 0), iy1 = min(y1 + D, NYP);
    const int cs = (NXP % VEC == 0) ? VEC : ((VEC == 4 && NXP % 2 == 0) ? 2 : 1);
    const int cxa = ((ix0 + cs - 1) / cs) * cs, cxb = (ix1 / cs) * cs;
    const int nl = (cxb > cxa) ? cxa - ix0 : ix1 - ix0;  // single elements on the left
    const int nf = (cxb > cxa) ? (cxb - cxa) / cs : 0;    // full pieces
    const int nr = (cxb > cxa) ? ix1 - cxb : 0;           // single elements on the right
    const int ppr = nl + nf + nr, npieces = ppr * (iy1 - iy0);
    uint32_t piece[MAXLD];  // bits 0..11 column - xs, 12..27 row - ys, 28..29 log2(bytes) - 2
    const bool use_pieces = (lvl == 1) && npieces <= NC * MAXLD;
#pragma unroll
    for (int q = 0; q < MAXLD; ++q) {
        const int i = tid + q * NC;
        uint32_t pc = 0xffffffffu;
        if (use_pieces && i < npieces) {
            const int r = i / ppr, pi = i % ppr;
            int x, bytes = (int)sizeof(T);
            if (pi < nl) x = ix0 + pi;
            else if (pi < nl + nf) {
                x = cxa + (pi - nl) * cs;
                bytes = cs * (int)sizeof(T);
            } else x = cxb + (pi - nl - nf);
            const int lg = (bytes == 16) ? 2 : (bytes == 8 ? 1 : 0);
            pc = (uint32_t)(x - xs) | ((uint32_t)(iy0 + r - ys) << 12) | ((uint32_t)lg << 28);
        }
        piece[q] = pc;
    }
    int issued = 0;
    auto issue_upto = [&](int last) {
        if (lvl != 1) return;
        for (; issued <= last && issued < nin; ++issued) {
            const int n = issued, slot = n & rmask;
            if (n >= R) wait(in_empty + 8u * slot, ((n >> rsh) - 1) & 1);
            const T *gp = src + (long long)(zi0 + n) * plane + (long long)ys * NXP + xs;
            const uint32_t sb = ring_s + (uint32_t)slot * slot_bytes;
            if (use_pieces) {
#pragma unroll
                for (int q = 0; q < MAXLD; ++q) {
                    const uint32_t pc = piece[q];
                    if (pc == 0xffffffffu) continue;
                    const int xl = (int)(pc & 0xfffu), yl = (int)((pc >> 12) & 0xffffu);
                    const uint32_t d = sb + (uint32_t)((yl * Wp + xl) * (int)sizeof(T));
                    const T *g = gp + (yl * NXP + xl);
                    const uint32_t lg = pc >> 28;
                    if (lg == 2) cp_async_16(d, g);
                    else if (lg == 1) cp_async_8(d, g);
                    else cp_async_4(d, g);
                }
            } else {
                // general layout: warp w copies rows w, w+NC/32, ... one element per lane
                for (int y = iy0 + warp; y < iy1; y += NW) {
                    const T *grow = gp + (long long)(y - ys) * NXP - xs;
                    const uint32_t srow = sb + (uint32_t)(((y - ys) * Wp - xs) * (int)sizeof(T));
                    for (int x = ix0 + lane; x < ix1; x += 32) {
                        if (sizeof(T) == 8) cp_async_8(srow + (uint32_t)x * 8u, grow + x);
                        else cp_async_4(srow + (uint32_t)x * 4u, grow + x);
                    }
                }
            }
            if (!(a.fault_mode == 1 && n == 2 && tid == 0)) cp_async_arrive_noinc(in_full + 8u * slot);
        }
    };
    issue_upto(L - 1);

    // ---- groups of this thread
    int jg0, gpr, orows;
    const int ox0 = max(x0 - wl, 0), ox1 = min(x1 + wl, NXP);
    const int oy0 = max(y0 - wl, 0), oy1 = min(y1 + wl, NYP);
    region_groups(ox0, ox1, oy0, oy1, xs, VEC, &jg0, &gpr, &orows);
    const int ngroups = gpr * orows;
    int goff[MAXG], gofs[MAXG];
    uint32_t flags[MAXG];  // bit 0 valid, bit 1 row interior, bits 2.. interior lanes, bits 8.. store lanes
#pragma unroll
    for (int q = 0; q < MAXG; ++q) {
        const int g = tid + q * NC;
        const int j = jg0 + (g % gpr), y = oy0 + g / gpr;
        const int xg = xs + VEC * j;
        goff[q] = (y - ys) * Wp + VEC * j;
        gofs[q] = y * NXP + xg;
        uint32_t f = 0;
        if (g < ngroups) {
            f |= 1u;
            if (y >= 1 && y <= ny) f |= 2u;
#pragma unroll
            for (int l = 0; l < VEC; ++l) {
                const int x = xg + l;
                if (x >= 1 && x <= nx) f |= 4u << l;
                if (x >= x0 && x < x1) f |= 256u << l;
            }
        }
        flags[q] = f;
    }

    const uint32_t next_ring = (lvl < D) ? mapa(ring_s, rank + 1) : 0u;
    const uint32_t next_full = (lvl < D) ? mapa(in_full, rank + 1) : 0u;
    const uint32_t prev_oe = (lvl > 1) ? mapa(out_empty, rank - 1) : 0u;
    T *dst = static_cast<T *>(a.dst);
    // Release of input seq by this warp (after its last read of the slot).
    // Warp 0 first re-arms the slot for the seq that will follow in it.
    auto release = [&](int seq) {
        __syncwarp();
        if (lane != 0) return;
        const uint32_t off = 8u * (uint32_t)(seq & rmask);
        if (lvl == 1) {
            mbar_arrive_local(in_empty + off);
        } else {
            if (warp == 0 && seq + R < nin) mbar_arrive_expect_tx(in_full + off, in_bytes);
            mbar_arrive_cluster(prev_oe + off);
        }
    };
    auto ldv = [&](const T *p, T (&v)[VEC]) {
        const V t = *reinterpret_cast<const V *>(p);
        if constexpr (VEC == 4) {
            v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
        } else {
            v[0] = t.x; v[1] = t.y;
        }
    };

    // z queue: three register sets that take the roles (plane k-1, plane k,
    // plane k+1) in rotation, so no values are moved between steps.
    T ra[MAXG][VEC], rb[MAXG][VEC], rc[MAXG][VEC];
#pragma unroll
    for (int q = 0; q < MAXG; ++q)
#pragma unroll
        for (int l = 0; l < VEC; ++l) ra[q][l] = rb[q][l] = rc[q][l] = T(0);
    if (zo0 > zi0) {
        wait(in_full, 0);
#pragma unroll
        for (int q = 0; q < MAXG; ++q)
            if (flags[q] & 1u) ldv(ring + goff[q], ra[q]);
    }
    {
        const int n = zo0 - zi0;
        wait(in_full + 8u * (n & rmask), (n >> rsh) & 1);
        const T *pl = ring + (n & rmask) * slot_elems;
#pragma unroll
        for (int q = 0; q < MAXG; ++q)
            if (flags[q] & 1u) ldv(pl + goff[q], rb[q]);
    }

    // One output plane k: A = values at k-1, B = at k (own cells), C is
    // loaded with k+1.  FAST: every cell of this level's region is an
    // interior cell of the grid and k is an interior plane, so no lane keeps
    // its own value (lanes of edge groups outside the region compute values
    // nobody reads).
    auto step = [&](const int k, T(&A)[MAXG][VEC], T(&B)[MAXG][VEC], T(&C)[MAXG][VEC], auto fast_tag) {
        constexpr bool FAST = decltype(fast_tag)::value;
        const int n = k - zi0, m = k - zo0;
        issue_upto(n + L);
        const bool has_next = FAST || (k + 1 < zi1);
        const bool interior_k = FAST || (k >= 1 && k <= nz);
        if (has_next) {
            wait(in_full + 8u * ((n + 1) & rmask), ((n + 1) >> rsh) & 1);
            const T *pl = ring + ((n + 1) & rmask) * slot_elems;
#pragma unroll
            for (int q = 0; q < MAXG; ++q)
                if (flags[q] & 1u) ldv(pl + goff[q], C[q]);
        }
        if (lvl < D && m >= R) wait(out_empty + 8u * (m & rmask), ((m >> rsh) - 1) & 1);

        const T *cen = ring + (n & rmask) * slot_elems;
        const uint32_t out_base = next_ring + (uint32_t)(m & rmask) * slot_bytes;
        const uint32_t out_bar = next_full + 8u * (uint32_t)(m & rmask);
        T *drow = dst + k * plane;
#pragma unroll
        for (int q = 0; q < MAXG; ++q) {
            const uint32_t f = flags[q];
            if (!(f & 1u)) continue;
            T v[VEC];
            if (FAST || (interior_k && (f & 2u))) {
                const T *c = cen + goff[q];
                T sv[VEC], nv[VEC];
                ldv(c - Wp, sv);
                ldv(c + Wp, nv);
                const T wv = c[-1], ev = c[VEC];
#pragma unroll
                for (int l = 0; l < VEC; ++l) {
                    const T left = (l == 0) ? wv : B[q][l - 1];
                    const T right = (l == VEC - 1) ? ev : B[q][l + 1];
                    const T u = Arith<T>::update(left, right, sv[l], nv[l], A[q][l], C[q][l]);
                    v[l] = (FAST || (f & (4u << l))) ? u : B[q][l];
                }
            } else {
#pragma unroll
                for (int l = 0; l < VEC; ++l) v[l] = B[q][l];
            }
            if (lvl < D) {
                st_async_v(out_base + (uint32_t)goff[q] * (uint32_t)sizeof(T), v, out_bar);
            } else {
                T *gpo = drow + gofs[q];
                const bool full = (f & (((1u << VEC) - 1u) << 8)) == (((1u << VEC) - 1u) << 8);
                if (full && cs == VEC) {
                    V t;
                    if constexpr (VEC == 4) t = make_float4(v[0], v[1], v[2], v[3]);
                    else t = make_double2(v[0], v[1]);
                    *reinterpret_cast<V *>(gpo) = t;
                } else if (VEC == 4 && full && cs == 2) {
                    reinterpret_cast<float2 *>(gpo)[0] = make_float2((float)v[0], (float)v[1]);
                    reinterpret_cast<float2 *>(gpo)[1] = make_float2((float)v[2], (float)v[3]);
                } else {
#pragma unroll
                    for (int l = 0; l < VEC; ++l)
                        if (f & (256u << l)) gpo[l] = v[l];
                }
            }
        }
        if (k == zo0 && zo0 > zi0) release(n - 1);
        release(n);
    };
    using Fast = std::integral_constant<bool, true>;
    using Slow = std::integral_constant<bool, false>;

    // Tiles whose widest region (level 1) avoids the grid's x/y halo take
    // the fast step on their interior planes; halo planes (k = 0, nz+1)
    // and boundary tiles take the general step.
    const bool fast_tile = (x0 - (D - 1) >= 1) && (x1 + (D - 1) <= nx + 1) && (y0 - (D - 1) >= 1) &&
                           (y1 + (D - 1) <= ny + 1);
    const int kf0 = fast_tile ? max(zo0, 1) : zo1;  // fast steps cover [kf0, kf1)
    const int kf1 = fast_tile ? min(zo1, nz + 1) : zo1;
    int k = zo0, rot = 0;  // rot: which register set holds plane k-1
    auto run = [&](int kk, auto tag) {
        if (rot == 0) step(kk, ra, rb, rc, tag);
        else if (rot == 1) step(kk, rb, rc, ra, tag);
        else step(kk, rc, ra, rb, tag);
        rot = (rot == 2) ? 0 : rot + 1;
    };
    for (; k < kf0; ++k) run(k, Slow());
    for (; k + 2 < kf1; k += 3) {  // three steps bring the roles back to rot
        if (rot == 0) {
            step(k, ra, rb, rc, Fast());
            step(k + 1, rb, rc, ra, Fast());
            step(k + 2, rc, ra, rb, Fast());
        } else if (rot == 1) {
            step(k, rb, rc, ra, Fast());
            step(k + 1, rc, ra, rb, Fast());
            step(k + 2, ra, rb, rc, Fast());
        } else {
            step(k, rc, ra, rb, Fast());
            step(k + 1, ra, rb, rc, Fast());
            step(k + 2, rb, rc, ra, Fast());
        }
    }
    for (; k < kf1; ++k) run(k, Fast());
    for (; k < zo1; ++k) run(k, Slow());
    cp_async_wait_all();
    cluster_sync_all();
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

// Load pieces per thread: enough for the level-1 plane of the largest tiles
// the tuner tries at each thread count (16 = 2048 pieces at 128 threads).
template <typename T>
const void *tb_kernel_ptr(int nc, int maxg)
{
    if (nc == 512 && maxg == 1) return (const void *)tb_pass_kernel<T, 512, 1, 4>;
    if (nc == 256 && maxg == 1) return (const void *)tb_pass_kernel<T, 256, 1, 8>;
    if (nc == 512 && maxg == 2) return (const void *)tb_pass_kernel<T, 512, 2, 4>;
    if (nc == 128 && maxg == 2) return (const void *)tb_pass_kernel<T, 128, 2, 16>;
    if (nc == 128 && maxg == 4) return (const void *)tb_pass_kernel<T, 128, 4, 16>;
    if (nc == 128 && maxg == 6) return (const void *)tb_pass_kernel<T, 128, 6, 16>;
    if (nc == 128 && maxg == 8) return (const void *)tb_pass_kernel<T, 128, 8, 16>;
    if (nc == 256 && maxg == 2) return (const void *)tb_pass_kernel<T, 256, 2, 8>;
    if (nc == 256 && maxg == 4) return (const void *)tb_pass_kernel<T, 256, 4, 8>;
    if (nc == 256 && maxg == 6) return (const void *)tb_pass_kernel<T, 256, 6, 8>;
    return nullptr;
}

const void *tb_kernel(int dtype, int nc, int maxc)
{
    return dtype == JACOBI_F64 ? tb_kernel_ptr<double>(nc, maxc) : tb_kernel_ptr<float>(nc, maxc);
}

cudaError_t prepare(const void *fn)
{
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

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

cudaError_t halo_copy_launch(int dtype, const void *A, void *B, int nx, int ny, int nz, cudaStream_t s)
{
    const long long total = halo_count(nx, ny, nz);
    const int block = 256;
    const long long want = (total + block - 1) / block;
    const unsigned grid = (unsigned)std::min<long long>(want, 152 * 16);
    if (dtype == JACOBI_F64)
        halo_copy_kernel<double><<<grid, block, 0, s>>>(static_cast<const double *>(A), static_cast<double *>(B), nx,
                                                          ny, nz);
    else
        halo_copy_kernel<float><<<grid, block, 0, s>>>(static_cast<const float *>(A), static_cast<float *>(B), nx, ny,
                                                        nz);
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
