// Temporal blocking inside one CTA with register-blocked cells (FP32), the
// T updates per thread of Sect. 2.1 with a whole CTA as the "thread":
// one CTA streams the z-planes of a W x H region (its output tile widened by
// the depth D on each side) and applies D time levels to each plane while it
// is on chip, so a pass reads the grid once and writes it once for D sweeps.
//
// Ownership: thread (tx, ty) owns a block of 4 x-cells x 4 rows of the
// region.  Per time level it keeps, in registers, the level's values of its
// block at three consecutive planes (a z-queue; the three arrays rotate
// with the step, so no values are moved).  In-plane neighbours outside the
// block come from the neighbouring threads' block boundaries: after level k
// produced a plane, each thread stores the top and bottom rows and the left
// and right columns of its block (four 16-byte shared-memory stores into
// row and column buffers laid out so that consecutive threads touch
// consecutive 16-byte words), and level k+1 reads its four neighbour
// vectors from there in the next step.  The buffers alternate with the
// step's parity, so one CTA barrier per step orders all writes and reads.
//
// Step s of the z stream: level 0 (the input) supplies plane s+1, level l
// computes plane s-l+1 (the one-plane skew between levels plays the
// one-block shift of Fig. 1).  Input planes stream into a 4-slot ring by
// cp.async, three planes ahead, each warp instruction copying a contiguous
// run of a row; the step's barrier makes a plane visible to all threads.
//
// x/y validity is the multi-layer halo of Sect. 3.1: level l is exact on
// the region minus l cells at each edge, so level D is exact on the output
// tile and no tile needs its neighbours.  Cells on the grid's halo keep
// their Dirichlet value at every level (they copy the previous level's
// value through); cells outside the array are never read by exact cells.
// A CTA whose region lies on the grid's interior in x and y (most of them)
// runs a copy of the loop without these per-cell cases.
// In z, a chunk [z0, z1) of output planes starts D planes early and ends
// D planes late; planes 0 and nz+1 are halo planes and are copied through.
//
// Copies and stores use pieces of A elements (A = 2: 8 bytes when the row
// pitch nx+2 is even, else A = 1), so every region starts on an A-element
// boundary: the output tile width bx is a multiple of A and the region
// starts `off` cells left of the tile's D-cell margin.
#pragma once

#include <cstdint>
#include <type_traits>

#include "checked.cuh"
#include "jacobi_internal.h"
#include "ptx.cuh"

namespace jac {

constexpr int kTbrVY = 4;  // rows per thread block

// Input ring slots (three planes in flight).  Eight slots at depth >= 3
// measured slower: the larger shared-memory carve-out leaves less L1 for the
// copies, which are staged through L1.
__host__ __device__ constexpr int tbr_ring(int) { return 4; }

// Asynchronous copy of A floats global -> shared; copies src_bytes of them
// (A*4 or 0) and zero-fills the rest, so the copy needs no branch (a zero
// count reads nothing; src is then any valid address).
template <int A>
__device__ __forceinline__ void tbr_copy(uint32_t dst, const float *src, uint32_t src_bytes)
{
    if (A == 2)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

// Predicated global stores (no branch).
__device__ __forceinline__ void tbr_st2_if(float *p, float a, float b, bool pred)
{
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %3, 0;\n\t@q st.global.v2.f32 [%0], {%1, %2};\n\t}" ::"l"(p), "f"(a),
        "f"(b), "r"((int)pred)
        : "memory");
}

__device__ __forceinline__ float4 tbr_ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void tbr_st4(float *p, float a, float b, float c, float d)
{
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}

// One time level of Eq. (1) on a thread's 4 x 4 block of cells: cur, below
// and above hold the previous level at the plane updated and at the planes
// below and above it (own cells); the row above the block, the row below,
// the column left and the column right come from the neighbouring blocks.
// Cells (0,1) and (2,3) of a row form packed pairs: the first addition
// (the x-neighbours) pairs cells unevenly and is done per cell, straight
// into a pair; the other four additions and the multiplication by RN(1/6)
// run on pairs.  Every cell keeps the left-to-right order of Eq. (1).
__device__ __forceinline__ void tbr_block_update(const float (&cur)[kTbrVY][4], const float (&below_pl)[kTbrVY][4],
                                                 const float (&above_pl)[kTbrVY][4], float4 above, float4 below,
                                                 float4 left, float4 right, float (&v)[kTbrVY][4])
{
    constexpr int VY = kTbrVY;
    const float sixth = 1.0f / 6.0f;
    const float le[4] = {left.x, left.y, left.z, left.w};
    const float ri[4] = {right.x, right.y, right.z, right.w};
    const float2 ab0 = make_float2(above.x, above.y), ab1 = make_float2(above.z, above.w);
    const float2 be0 = make_float2(below.x, below.y), be1 = make_float2(below.z, below.w);
    const float2 six2 = make_float2(sixth, sixth);
#pragma unroll
    for (int r = 0; r < VY; ++r) {
        const float c0 = cur[r][0], c1 = cur[r][1], c2 = cur[r][2], c3 = cur[r][3];
        float2 lo = make_float2(__fadd_rn(le[r], c1), __fadd_rn(c0, c2));
        float2 hi = make_float2(__fadd_rn(c1, c3), __fadd_rn(c2, ri[r]));
        const float2 s0 = r > 0 ? make_float2(cur[r - 1][0], cur[r - 1][1]) : ab0;
        const float2 s1 = r > 0 ? make_float2(cur[r - 1][2], cur[r - 1][3]) : ab1;
        const float2 n0 = r < VY - 1 ? make_float2(cur[r + 1][0], cur[r + 1][1]) : be0;
        const float2 n1 = r < VY - 1 ? make_float2(cur[r + 1][2], cur[r + 1][3]) : be1;
        lo = __fadd2_rn(lo, s0);
        hi = __fadd2_rn(hi, s1);
        lo = __fadd2_rn(lo, n0);
        hi = __fadd2_rn(hi, n1);
        lo = __fadd2_rn(lo, make_float2(below_pl[r][0], below_pl[r][1]));
        hi = __fadd2_rn(hi, make_float2(below_pl[r][2], below_pl[r][3]));
        lo = __fadd2_rn(lo, make_float2(above_pl[r][0], above_pl[r][1]));
        hi = __fadd2_rn(hi, make_float2(above_pl[r][2], above_pl[r][3]));
        lo = __fmul2_rn(lo, six2);
        hi = __fmul2_rn(hi, six2);
        v[r][0] = lo.x, v[r][1] = lo.y, v[r][2] = hi.x, v[r][3] = hi.y;
    }
}

// Resident CTAs requested per SM: three 128-thread CTAs at depth 1, and at
// depth 2 with copy pieces of two cells (at most 170 registers, which those
// fit without spilling); two at depth 2 with single-cell pieces (whose
// address arithmetic spills at 170); else one.
template <int D, int NT, int A>
struct TbrMinBlocks {
    static constexpr int value = (NT == 128 && (D == 1 || (D == 2 && A == 2))) ? 3 : (NT == 128 && D == 2) ? 2 : 1;
};

// The work of one CTA: tile (tix, tiy) in x and y, z chunk tiz.
template <int D, int TX, int TY, int A>
__device__ __forceinline__ void tbr_cta(const TbrArgs &a, int tix, int tiy, int tiz)
{
    constexpr int VY = kTbrVY, R = tbr_ring(D), NT = TX * TY;
    constexpr int W = 4 * TX, H = VY * TY;
    constexpr int RING = W * H;                // floats per ring slot
    constexpr int ROWS = 2 * TY * W;           // [top|bottom][ty][x]
    constexpr int COLS = 2 * TY * TX * VY;     // [left|right][ty][tx][row]
    constexpr int LEV = ROWS + COLS;           // one level, one parity
    extern __shared__ __align__(16) float tbr_smem[];
    float *ring = tbr_smem;
    float *bufs = tbr_smem + R * RING;         // [parity][level][LEV]

    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int xa = a.x_first + tix * a.bx;  // region origin (multiple of A)
    const int ya = 1 - D + tiy * a.by;
    const int z0 = 1 + tiz * a.bz;
    const int z1 = min(z0 + a.bz, a.nz + 1);
    const int xo = xa + a.off + D, yo = ya + D;         // output tile origin
    const int gx0 = xa + 4 * tx;
    const int P = a.nx + 2;
    const long long plane = (long long)P * (a.ny + 2);
    const float *__restrict__ src = static_cast<const float *>(a.src);
    float *__restrict__ dst = static_cast<float *>(a.dst);
    // checked build: global offsets against the grid, ring indices against
    // the ring, buffer indices against the level buffers
    const long long SG = checked_grid_elems(a.nx, a.ny, a.nz, a.shrink);
    auto gok = [&](long long off, int n) { return in_bounds(off, n, SG, a.status); };
    auto rok = [&](const float *ptr, int n) { return in_bounds(ptr - ring, n, (long long)R * RING, a.status); };
    auto bok = [&](const float *ptr) { return in_bounds(ptr - bufs, 4, 2LL * D * LEV, a.status); };

    // Per-cell masks (bit r*4+c): on the grid's interior (updated), in the
    // output tile (stored).
    unsigned upd = 0, st = 0;
    int rowoff[VY];
#pragma unroll
    for (int r = 0; r < VY; ++r) {
        const int gy = ya + VY * ty + r;
        const bool rin = gy >= 0 && gy <= a.ny + 1;
        rowoff[r] = rin ? gy * P + gx0 : 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int gx = gx0 + c;
            const unsigned bit = 1u << (r * 4 + c);
            const bool interior = gx >= 1 && gx <= a.nx && gy >= 1 && gy <= a.ny;
            if (interior) upd |= bit;
            if (interior && gx >= xo && gx < xo + a.bx && gy >= yo && gy < yo + a.by) st |= bit;
        }
    }
    const bool full = upd == 0xFFFFu;
    const float *ring_rd = ring + (VY * ty) * W + 4 * tx;
    // neighbour offsets inside one level buffer (clamped at the region edge:
    // those cells are outside every exact level)
    const int o_above = TY * W + max(ty - 1, 0) * W + 4 * tx;      // bottom row of (tx, ty-1)
    const int o_below = min(ty + 1, TY - 1) * W + 4 * tx;          // top row of (tx, ty+1)
    const int o_left = ROWS + (TY * TX + ty * TX + max(tx - 1, 0)) * VY;   // right column of (tx-1, ty)
    const int o_right = ROWS + (ty * TX + min(tx + 1, TX - 1)) * VY;       // left column of (tx+1, ty)
    const int o_top = ty * W + 4 * tx, o_bot = TY * W + ty * W + 4 * tx;
    const int o_lcol = ROWS + (ty * TX + tx) * VY, o_rcol = ROWS + (TY * TX + ty * TX + tx) * VY;

    // Input copies: the ring slot is filled row by row, piece i = tid + NT*j
    // of the W/A pieces per row, so each warp instruction copies a
    // contiguous run of a row.  A thread thus copies cells it does not own;
    // the reads come after every thread's copies completed and a barrier.
    constexpr int PPR = W / A;            // pieces per row
    constexpr int RPJ = NT / PPR;         // rows per copy instruction
    constexpr int NJ = H / RPJ;           // copy instructions per plane
    static_assert(NT % PPR == 0 && H % RPJ == 0, "copy layout");
    const int cp_row = tid / PPR, cp_col = (tid % PPR) * A;
    const int cp_gx = xa + cp_col;
    const bool cp_xin = cp_gx >= 0 && cp_gx <= a.nx + 1;  // whole piece (pieces never straddle the array edge)
    unsigned cp_rows = 0;                                    // bit j: row of copy j inside the array
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int gy = ya + cp_row + j * RPJ;
        if (cp_xin && gy >= 0 && gy <= a.ny + 1) cp_rows |= 1u << j;
    }
    const int cp_off0 = (ya + cp_row) * P + cp_gx;  // plane offset of copy 0 (used only if inside)
    const uint32_t cp_dst0 = smem_addr(ring + cp_row * W + cp_col);
    // FAST: the whole region lies inside the array, so every piece is copied.
    // planes beyond z1 - 1 + D feed only the steps past the chunk: not
    // loaded (their ring slots keep older planes, never stored)
    const int p_hi = min(a.nz + 1, z1 - 1 + D);
    auto load_plane = [&](int p, auto FAST) {
        if (p >= 0 && p <= p_hi) {
            const float *sp = src + (long long)p * plane;
            const uint32_t d0 = cp_dst0 + (uint32_t)((p & (R - 1)) * RING * 4);
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                const bool in = decltype(FAST)::value || ((cp_rows >> j) & 1u);
                if (kChecked) {
                    const float *dl = ring + (p & (R - 1)) * RING + cp_row * W + cp_col + j * RPJ * W;
                    if (!rok(dl, A) || (in && !gok((long long)p * plane + cp_off0 + j * RPJ * P, A))) continue;
                }
                if (decltype(FAST)::value) {
                    tbr_copy<A>(d0 + (uint32_t)(j * RPJ * W * 4), sp + cp_off0 + j * RPJ * P, 4u * A);
                } else {
                    tbr_copy<A>(d0 + (uint32_t)(j * RPJ * W * 4), in ? sp + cp_off0 + j * RPJ * P : sp,
                                in ? 4u * A : 0u);
                }
            }
        }
        cp_async_commit();
    };
    // The region lies on the grid's interior in x and y (every cell of every
    // thread is updated and copied): the CTA takes the fast path.
    const bool interior = xa >= 1 && xa + W - 1 <= a.nx && ya >= 1 && ya + H - 1 <= a.ny;
    const std::false_type slow_c;
    // Rows whose four cells are all stored take two predicated 8-byte
    // stores (A = 2); any other stored cell goes through the scalar path.
    unsigned rowfull = 0;
#pragma unroll
    for (int r = 0; r < VY; ++r)
        if (A == 2 && ((st >> (r * 4)) & 0xFu) == 0xFu) rowfull |= 1u << r;
    unsigned st_rest = st;
#pragma unroll
    for (int r = 0; r < VY; ++r)
        if ((rowfull >> r) & 1u) st_rest &= ~(0xFu << (r * 4));

    auto write_bounds = [&](float *b, const float (&v)[VY][4]) {
        if (bok(b + o_top)) tbr_st4(b + o_top, v[0][0], v[0][1], v[0][2], v[0][3]);
        if (bok(b + o_bot)) tbr_st4(b + o_bot, v[VY - 1][0], v[VY - 1][1], v[VY - 1][2], v[VY - 1][3]);
        if (bok(b + o_lcol)) tbr_st4(b + o_lcol, v[0][0], v[1][0], v[2][0], v[3][0]);
        if (bok(b + o_rcol)) tbr_st4(b + o_rcol, v[0][3], v[1][3], v[2][3], v[3][3]);
    };
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    auto ldb = [&](const float *ptr) { return bok(ptr) ? tbr_ld4(ptr) : zero4; };
    auto ldr = [&](const float *ptr) { return rok(ptr, 4) ? tbr_ld4(ptr) : zero4; };

    // z-queues: q[k][i] = level k (0 = input) at one of three consecutive
    // planes; at relative step t the new plane of every level goes to index
    // (t+1)%3, the centre plane of the next level's stencil is t%3 and the
    // plane below it (t+2)%3.
    float q[D][3][VY][4];
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int r = 0; r < VY; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) q[k][i][r][c] = 0.f;

    const int s_begin = z0 - D + 1;
    const int nsteps = z1 - z0 + 2 * D - 2;
    load_plane(s_begin - 1, slow_c);
    load_plane(s_begin, slow_c);
    cp_async_wait_group<0>();
    __syncthreads();  // every thread's copies of the two planes are complete
    {
        const float *r0 = ring_rd + ((s_begin - 1) & (R - 1)) * RING;
        const float *r1 = ring_rd + (s_begin & (R - 1)) * RING;
#pragma unroll
        for (int r = 0; r < VY; ++r) {
            const float4 u = ldr(r0 + r * W), v = ldr(r1 + r * W);
            q[0][2][r][0] = u.x, q[0][2][r][1] = u.y, q[0][2][r][2] = u.z, q[0][2][r][3] = u.w;
            q[0][0][r][0] = v.x, q[0][0][r][1] = v.y, q[0][0][r][2] = v.z, q[0][0][r][3] = v.w;
        }
    }
    write_bounds(bufs + 1 * D * LEV, q[0][0]);  // plane s_begin, read in step 0 (parity 1)
    __syncthreads();  // ring reads above are performed before their slots are refilled
#pragma unroll
    for (int i = 1; i < R; ++i) load_plane(s_begin + i, slow_c);

    auto step = [&](auto J, auto FAST, int t) {
        constexpr int j = decltype(J)::value;
        constexpr bool fast = decltype(FAST)::value;
        constexpr int iN = (j + 1) % 3, iC = j, iM = (j + 2) % 3;
        const int s = s_begin + t;
        cp_async_wait_group<R - 2>();  // this thread's copies of plane s+1 are complete
        __syncthreads();               // ... every thread's; level boundaries of step t-1 written
        {
            const float *rp = ring_rd + ((s + 1) & (R - 1)) * RING;
#pragma unroll
            for (int r = 0; r < VY; ++r) {
                const float4 u = ldr(rp + r * W);
                q[0][iN][r][0] = u.x, q[0][iN][r][1] = u.y, q[0][iN][r][2] = u.z, q[0][iN][r][3] = u.w;
            }
        }
        float *wb = bufs + (t & 1) * D * LEV;
        const float *rb = bufs + ((t + 1) & 1) * D * LEV;
        // neighbour vectors of level l are loaded one level ahead, before
        // the shared-memory stores of the level in between (the compiler
        // cannot move loads across stores it cannot prove disjoint)
        float4 nbv[4];
        nbv[0] = ldb(rb + o_above), nbv[1] = ldb(rb + o_below);
        nbv[2] = ldb(rb + o_left), nbv[3] = ldb(rb + o_right);
        load_plane(s + R, FAST);  // into the slot of plane s, read in step t-1
        write_bounds(wb, q[0][iN]);
#pragma unroll
        for (int l = 1; l <= D; ++l) {
            const int k = l - 1;
            const int p = s - l + 1;
            const bool zin = p >= 1 && p <= a.nz;
            const float4 above = nbv[0], below = nbv[1], left = nbv[2], right = nbv[3];
            if (l < D) {
                const float *nn = rb + l * LEV;
                nbv[0] = ldb(nn + o_above), nbv[1] = ldb(nn + o_below);
                nbv[2] = ldb(nn + o_left), nbv[3] = ldb(nn + o_right);
            }
            float v[VY][4];
            tbr_block_update(q[k][iC], q[k][iM], q[k][iN], above, below, left, right, v);
            if (fast) {
                if (!zin) {  // uniform: a halo plane (or one outside the array)
#pragma unroll
                    for (int r = 0; r < VY; ++r)
#pragma unroll
                        for (int c = 0; c < 4; ++c) v[r][c] = q[k][iC][r][c];
                }
            } else if (!(zin && full)) {
#pragma unroll
                for (int r = 0; r < VY; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (!zin || !(upd & (1u << (r * 4 + c)))) v[r][c] = q[k][iC][r][c];
            }
            if (l < D) {
#pragma unroll
                for (int r = 0; r < VY; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) q[l < D ? l : 0][iN][r][c] = v[r][c];
                write_bounds(wb + l * LEV, v);
            } else {
                const bool zst = p >= z0 && p < z1;
                float *dp = dst + (long long)p * plane;
                if (A == 2) {
#pragma unroll
                    for (int r = 0; r < VY; ++r) {
                        bool f = zst && ((rowfull >> r) & 1u);
                        if (kChecked && f) f = gok((long long)p * plane + rowoff[r], 4);
                        tbr_st2_if(dp + rowoff[r], v[r][0], v[r][1], f);
                        tbr_st2_if(dp + rowoff[r] + 2, v[r][2], v[r][3], f);
                    }
                }
                if (zst && st_rest) {
#pragma unroll
                    for (int r = 0; r < VY; ++r)
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            if (((st_rest >> (r * 4 + c)) & 1u) && gok((long long)p * plane + rowoff[r] + c, 1))
                                dp[rowoff[r] + c] = v[r][c];
                }
            }
        }
    };
    // Whole rotations of three steps; the up to two extra steps at the end
    // compute planes beyond the chunk (never stored; their loads are
    // skipped), so no step needs a guard.
    if (interior) {
        const std::true_type f;
        for (int t = 0; t < nsteps; t += 3) {
            step(std::integral_constant<int, 0>(), f, t);
            step(std::integral_constant<int, 1>(), f, t + 1);
            step(std::integral_constant<int, 2>(), f, t + 2);
        }
    } else {
        for (int t = 0; t < nsteps; t += 3) {
            step(std::integral_constant<int, 0>(), slow_c, t);
            step(std::integral_constant<int, 1>(), slow_c, t + 1);
            step(std::integral_constant<int, 2>(), slow_c, t + 2);
        }
    }
    cp_async_wait_group<0>();
}

template <int D, int TX, int TY, int A>
__global__ void __launch_bounds__(TX *TY, (TbrMinBlocks<D, TX * TY, A>::value)) tbr_pass_kernel(const TbrArgs a)
{
    tbr_cta<D, TX, TY, A>(a, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z);
}

}  // namespace jac
