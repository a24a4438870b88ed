// The time-skewed cluster pass kernel (tb_pass_kernel), shared by the
// translation units that instantiate its variants (tb_inst_*.cu) so that
// they compile in parallel.  See sweep_kernels.cu for the pass as a whole.
#pragma once

#include <type_traits>

#include "arith.cuh"
#include "checked.cuh"
#include "jacobi_internal.h"
#include "ptx.cuh"

namespace jac {

__device__ __forceinline__ void record_error(int *status, int code)
{
    atomicCAS(status, 0, code);
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
    // checked build: global offsets against the grid, ring indices (this
    // CTA's or, for the hand-off, the next CTA's) against the ring slots
    const long long SG = checked_grid_elems(nx, ny, nz, a.shrink);
    const long long SR = (long long)R * slot_elems;
    auto gok = [&](long long off, int cnt) { return in_bounds(off, cnt, SG, a.status); };
    auto rok = [&](long long idx, int cnt) { return in_bounds(idx, cnt, SR, a.status); };

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
                    if (kChecked) {
                        const int cnt = (4 << lg) / (int)sizeof(T);
                        if (!rok((long long)slot * slot_elems + yl * Wp + xl, cnt) ||
                            !gok((long long)(zi0 + n) * plane + (long long)(ys + yl) * NXP + xs + xl, cnt))
                            continue;
                    }
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
                        if (kChecked && (!rok((long long)slot * slot_elems + (y - ys) * Wp - xs + x, 1) ||
                                         !gok((long long)(zi0 + n) * plane + (long long)y * NXP + x, 1)))
                            continue;
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
        V t = V();
        if (rok(p - ring, VEC)) t = *reinterpret_cast<const V *>(p);
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
                const T wv = rok(c - 1 - ring, 1) ? c[-1] : T(0), ev = rok(c + VEC - ring, 1) ? c[VEC] : T(0);
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
                // in the checked build a skipped hand-off leaves the consumer
                // short of bytes: its bounded wait then ends with a timeout
                if (rok((long long)(m & rmask) * slot_elems + goff[q], VEC))
                    st_async_v(out_base + (uint32_t)goff[q] * (uint32_t)sizeof(T), v, out_bar);
            } else {
                T *gpo = drow + gofs[q];
                if (kChecked && !gok((long long)k * plane + gofs[q], VEC)) {
                    // a group partly outside the grid: store its lanes one by one
#pragma unroll
                    for (int l = 0; l < VEC; ++l)
                        if ((f & (256u << l)) && gok((long long)k * plane + gofs[q] + l, 1)) gpo[l] = v[l];
                    continue;
                }
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

}  // namespace jac
