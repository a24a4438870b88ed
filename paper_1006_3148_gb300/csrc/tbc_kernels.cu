// Temporal blocking inside one CTA (Sect. 2.1 with T updates per thread):
// one CTA streams the planes of a tile widened by D cells on each side and
// applies D time levels to them while they sit in shared memory, so each
// pass reads the grid once and writes it once for D sweeps.  D = 1 is the
// plain sweep with every input plane staged once in shared memory.
//
// Step s of the z stream: level 1 updates plane s, level l plane s-l+1 (the
// one-plane skew between consecutive levels plays the one-block shift of
// Fig. 1).  Level l needs level l-1 at planes p-1, p, p+1 (p = s-l+1):
//   p-1 and p   were produced in earlier steps and stay in registers (each
//               thread keeps, per owned cell and level, the last two values
//               of that level: a z-queue);
//   p+1         is produced by level l-1 in this same step, by this thread;
//   the four in-plane neighbours at plane p come from the level's shared-
//               memory plane, written at the end of the previous step.
// Level 0 is the input: planes stream through a 4-slot shared-memory ring
// filled by cp.async two planes ahead.  The level planes are double-
// buffered by step parity, so one CTA barrier per step orders everything:
// the writes of step s-1 before the reads of step s, and the reads of step
// s-1 before the overwrite in step s+1.  D levels of work share it.
//
// In x and y, level l is valid on the tile widened by D-l cells (the
// multi-layer halo of Sect. 3.1), so the level-D result is exact on the
// tile and no tile needs its neighbours.  In z a chunk [z0, z1) of output
// planes starts the stream D planes early and ends D planes late.  Cells on
// the grid's halo (x, y or z) and cells outside the array copy the previous
// level's value through, which keeps the halo's Dirichlet values; region-edge
// cells do the same (their later levels are never read by valid cells).
#include <algorithm>

#include "arith.cuh"
#include "checked.cuh"
#include "jacobi_internal.h"
#include "ptx.cuh"

namespace jac {
namespace {

constexpr int kRing = 4;  // input plane slots

template <typename T, int D, int NT, int CPT>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1) tbc_pass_kernel(const TbcArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *ring = reinterpret_cast<T *>(smem_raw);  // kRing planes of W*H
    T *lev = ring + kRing * a.WH;               // levels 1..D-1, two planes each (step parity)
    const int tid = threadIdx.x;
    const int W = a.W, WH = a.WH;
    const long long NXP = a.nx + 2, plane = NXP * (a.ny + 2);
    const int x0 = 1 + blockIdx.x * a.bx - D, y0 = 1 + blockIdx.y * a.by - D;
    const int z0 = 1 + blockIdx.z * a.bz, z1 = min(z0 + a.bz, a.nz + 1);
    const T *__restrict__ src = static_cast<const T *>(a.src);
    T *__restrict__ dst = static_cast<T *>(a.dst);
    // checked build: global offsets against the grid, shared indices against
    // the ring and level planes
    const long long SG = checked_grid_elems(a.nx, a.ny, a.nz, a.shrink);
    const long long SS = (long long)(kRing + 2 * (D - 1)) * WH;
    auto gok = [&](long long off) { return in_bounds(off, 1, SG, a.status); };
    auto sok = [&](const T *ptr) { return in_bounds(ptr - ring, 1, SS, a.status); };
    auto lds = [&](const T *ptr) { return sok(ptr) ? *ptr : T(0); };

    // Owned cells: c = tid + r*NT of the W x H region.
    int cell[CPT];
    int goff[CPT];        // offset of the cell's column within a plane
    unsigned flags = 0;   // per r: bit 4r: in array, 4r+1: computes, 4r+2: stores, 4r+3: owned
    for (int r = 0; r < CPT; ++r) {
        const int c = tid + r * NT;
        cell[r] = c < WH ? c : 0;
        const int cx = c % W, cy = c / W, gx = x0 + cx, gy = y0 + cy;
        const bool valid = c < WH;
        const bool inarr = valid && gx >= 0 && gx <= a.nx + 1 && gy >= 0 && gy <= a.ny + 1;
        const bool interior = inarr && gx >= 1 && gx <= a.nx && gy >= 1 && gy <= a.ny;
        const bool edge = cx == 0 || cx == W - 1 || cy == 0 || cy == a.H - 1;
        const bool store = interior && cx >= D && cx < D + a.bx && cy >= D && cy < D + a.by;
        goff[r] = inarr ? gy * (a.nx + 2) + gx : 0;
        flags |= (inarr ? 1u : 0u) << (4 * r);
        flags |= (interior && !edge ? 1u : 0u) << (4 * r + 1);
        flags |= (store ? 1u : 0u) << (4 * r + 2);
        flags |= (valid ? 1u : 0u) << (4 * r + 3);
    }
    for (int c = tid; c < 2 * (D - 1) * WH; c += NT)
        if (sok(lev + c)) lev[c] = T(0);

    // Input plane p (if inside the array's planes) into its ring slot.
    auto load_plane = [&](int p) {
        if (p >= 0 && p <= a.nz + 1) {
            T *slot = ring + (p & (kRing - 1)) * WH;
            const T *sp = src + (long long)p * plane;
            for (int r = 0; r < CPT; ++r) {
                if ((flags & (1u << (4 * r))) && sok(slot + cell[r]) && gok((long long)p * plane + goff[r])) {
                    const uint32_t d = smem_addr(slot + cell[r]);
                    if (sizeof(T) == 8) cp_async_8(d, sp + goff[r]);
                    else cp_async_4(d, sp + goff[r]);
                }
            }
        }
        cp_async_commit();
    };

    const int s_begin = z0 - D + 1, s_end = z1 + D - 2;
    // z-queues: q0[l][r] = level l at the older plane, q1[l][r] at the newer
    // one (level 0 = input; levels 1..D-1).
    T q0[D][CPT], q1[D][CPT];
    load_plane(s_begin - 1);
    load_plane(s_begin);
    load_plane(s_begin + 1);
    cp_async_wait_group<0>();
    __syncthreads();
    for (int r = 0; r < CPT; ++r) {
        q0[0][r] = lds(ring + ((s_begin - 1) & (kRing - 1)) * WH + cell[r]);
        q1[0][r] = lds(ring + (s_begin & (kRing - 1)) * WH + cell[r]);
#pragma unroll
        for (int l = 1; l < D; ++l) {
            q0[l][r] = T(0);
            q1[l][r] = T(0);
        }
    }
    load_plane(s_begin + 2);

    for (int s = s_begin; s <= s_end; ++s) {
        cp_async_wait_group<1>();  // plane s+1 is in its slot
        __syncthreads();           // ... for every thread; level planes of step s-1 written
        load_plane(s + 3);         // into the slot of plane s-1, read for the last time in step s-1
        T up[CPT];                 // level l-1 at plane p+1 (this step)
        const T *inb = ring + ((s + 1) & (kRing - 1)) * WH;
        for (int r = 0; r < CPT; ++r) up[r] = lds(inb + cell[r]);
#pragma unroll
        for (int l = 1; l <= D; ++l) {
            const int p = s - l + 1;
            const bool zin = p >= 1 && p <= a.nz;
            const T *nb = (l == 1) ? ring + (s & (kRing - 1)) * WH : lev + ((l - 2) * 2 + ((s - 1) & 1)) * WH;
            for (int r = 0; r < CPT; ++r) {
                const int c = cell[r];
                T v;
                if (zin && (flags & (2u << (4 * r))))
                    v = Arith<T>::update(lds(nb + c - 1), lds(nb + c + 1), lds(nb + c - W), lds(nb + c + W), q0[l - 1][r],
                                         up[r]);
                else
                    v = q1[l - 1][r];
                q0[l - 1][r] = q1[l - 1][r];
                q1[l - 1][r] = up[r];
                up[r] = v;
            }
            if (l == D && p >= z0 && p < z1) {
                T *dp = dst + (long long)p * plane;
                for (int r = 0; r < CPT; ++r)
                    if ((flags & (4u << (4 * r))) && gok((long long)p * plane + goff[r])) dp[goff[r]] = up[r];
            }
        }
#pragma unroll
        for (int l = 1; l < D; ++l)
            for (int r = 0; r < CPT; ++r)
                if ((flags & (8u << (4 * r))) && sok(lev + ((l - 1) * 2 + (s & 1)) * WH + cell[r]))
                    lev[((l - 1) * 2 + (s & 1)) * WH + cell[r]] = q1[l][r];
    }
    cp_async_wait_group<0>();
}

// FP32 form with quads: thread-owned groups of 4 x-consecutive cells of a
// row (the shared-memory row pitch W is a multiple of 4).  Per quad and
// level, the previous level's plane p is read back as one 16-byte load (the
// x-neighbours inside the quad come from it), the cells beyond the quad's
// two ends as two 4-byte loads and the rows above and below as two 16-byte
// loads; only the plane below (p-1) stays in registers.  Both cell pairs
// are summed with packed FP32 additions in Eq. (1)'s order, and a level's
// new values go to its next-parity plane as soon as they are computed.
// Same step structure and boundary rules as the scalar kernel above.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

template <int D, int NT, int QPT>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1) tbc4_pass_kernel(const TbcArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *ring = reinterpret_cast<float *>(smem_raw);  // kRing planes of W*H
    float *lev = ring + kRing * a.WH;                   // levels 1..D-1, two planes each
    const int tid = threadIdx.x;
    const int W = a.W, W4 = W >> 2, H = a.H, WH = a.WH, Wr = a.bx + 2 * D;
    const long long plane = (long long)(a.nx + 2) * (a.ny + 2);
    const int x0 = 1 + blockIdx.x * a.bx - D, y0 = 1 + blockIdx.y * a.by - D;
    const int z0 = 1 + blockIdx.z * a.bz, z1 = min(z0 + a.bz, a.nz + 1);
    const float *__restrict__ src = static_cast<const float *>(a.src);
    float *__restrict__ dst = static_cast<float *>(a.dst);
    // checked build: global offsets against the grid, shared indices against
    // the ring and level planes
    const long long SG = checked_grid_elems(a.nx, a.ny, a.nz, a.shrink);
    const long long SS = (long long)(kRing + 2 * (D - 1)) * WH;
    auto gok = [&](long long off) { return in_bounds(off, 1, SG, a.status); };
    auto sok = [&](const float *ptr, int n) { return in_bounds(ptr - ring, n, SS, a.status); };
    auto lds1 = [&](const float *ptr) { return sok(ptr, 1) ? *ptr : 0.f; };

    // flag bits of a quad: 0-3 load cell k, 4-7 cell k computes, 8-11 cell k
    // is stored, 12 owned, 13 has a left neighbour quad, 14 right, 15 row
    // above, 16 row below, 17 all four cells compute
    constexpr unsigned kOwned = 1u << 12, kLeft = 1u << 13, kRight = 1u << 14, kUp = 1u << 15, kDown = 1u << 16,
                       kFull = 1u << 17, kAny = 0xF0u;
    int qc[QPT], goff[QPT];
    unsigned qf[QPT];
    for (int r = 0; r < QPT; ++r) {
        const int q = tid + r * NT;
        const bool valid = q < W4 * H;
        const int qx = valid ? q % W4 : 0, cy = valid ? q / W4 : 0;
        const int gy = y0 + cy;
        unsigned f = valid ? kOwned : 0u;
        for (int k = 0; k < 4; ++k) {
            const int cx = 4 * qx + k, gx = x0 + cx;
            const bool inarr = valid && cx < Wr && gx >= 0 && gx <= a.nx + 1 && gy >= 0 && gy <= a.ny + 1;
            const bool interior = inarr && gx >= 1 && gx <= a.nx && gy >= 1 && gy <= a.ny;
            const bool edge = cx == 0 || cx >= Wr - 1 || cy == 0 || cy == H - 1;
            const bool store = interior && cx >= D && cx < D + a.bx && cy >= D && cy < D + a.by;
            f |= (inarr ? 1u : 0u) << k;
            f |= (interior && !edge ? 1u : 0u) << (4 + k);
            f |= (store ? 1u : 0u) << (8 + k);
        }
        if (qx > 0) f |= kLeft;
        if (qx < W4 - 1) f |= kRight;
        if (cy > 0) f |= kUp;
        if (cy < H - 1) f |= kDown;
        if ((f & kAny) == kAny) f |= kFull;
        qf[r] = f;
        qc[r] = cy * W + 4 * qx;
        goff[r] = gy * (a.nx + 2) + x0 + 4 * qx;  // offset of cell 0 in a plane (used only for cells in the array)
    }
    for (int c = tid; c < 2 * (D - 1) * WH; c += NT)
        if (sok(lev + c, 1)) lev[c] = 0.f;

    auto load_plane = [&](int p) {
        if (p >= 0 && p <= a.nz + 1) {
            float *slot = ring + (p & (kRing - 1)) * WH;
            const float *sp = src + (long long)p * plane;
            for (int r = 0; r < QPT; ++r)
                for (int k = 0; k < 4; ++k)
                    if ((qf[r] & (1u << k)) && sok(slot + qc[r] + k, 1) && gok((long long)p * plane + goff[r] + k))
                        cp_async_4(smem_addr(slot + qc[r] + k), sp + goff[r] + k);
        }
        cp_async_commit();
    };
    auto ld4 = [&](const float *p) {
        return sok(p, 4) ? *reinterpret_cast<const float4 *>(p) : make_float4(0.f, 0.f, 0.f, 0.f);
    };

    const int s_begin = z0 - D + 1, s_end = z1 + D - 2;
    // q0[l][r]: level l (0 = input) at the plane below the one level l+1
    // updates next; the plane itself is read back from shared memory.
    float4 q0[D][QPT];
    load_plane(s_begin - 1);
    load_plane(s_begin);
    load_plane(s_begin + 1);
    cp_async_wait_group<0>();
    __syncthreads();
    for (int r = 0; r < QPT; ++r) {
        q0[0][r] = ld4(ring + ((s_begin - 1) & (kRing - 1)) * WH + qc[r]);
#pragma unroll
        for (int l = 1; l < D; ++l) q0[l][r] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    load_plane(s_begin + 2);
    const float2 sixth = make_float2(1.0f / 6.0f, 1.0f / 6.0f);

    for (int s = s_begin; s <= s_end; ++s) {
        cp_async_wait_group<1>();
        __syncthreads();
        load_plane(s + 3);
        float4 up[QPT];
        const float *inb = ring + ((s + 1) & (kRing - 1)) * WH;
        for (int r = 0; r < QPT; ++r) up[r] = ld4(inb + qc[r]);
#pragma unroll
        for (int l = 1; l <= D; ++l) {
            const int p = s - l + 1;
            const bool zin = p >= 1 && p <= a.nz;
            const float *nb = (l == 1) ? ring + (s & (kRing - 1)) * WH : lev + ((l - 2) * 2 + ((s - 1) & 1)) * WH;
            float *out = lev + ((l - 1) * 2 + (s & 1)) * WH;  // level l's plane of this step (l < D)
            for (int r = 0; r < QPT; ++r) {
                const unsigned f = qf[r];
                const int i0 = qc[r];
                const float4 c = ld4(nb + i0);  // level l-1 at plane p
                float4 v = c;
                if (zin && (f & kAny)) {
                    const float w = (f & kLeft) ? lds1(nb + i0 - 1) : 0.f;
                    const float e = (f & kRight) ? lds1(nb + i0 + 4) : 0.f;
                    const float4 ym = (f & kUp) ? ld4(nb + i0 - W) : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 yp = (f & kDown) ? ld4(nb + i0 + W) : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 lo = q0[l - 1][r], hi = up[r];
                    float2 a01 = add2(make_float2(w, c.x), make_float2(c.y, c.z));
                    float2 a23 = add2(make_float2(c.y, c.z), make_float2(c.w, e));
                    a01 = add2(a01, make_float2(ym.x, ym.y));
                    a23 = add2(a23, make_float2(ym.z, ym.w));
                    a01 = add2(a01, make_float2(yp.x, yp.y));
                    a23 = add2(a23, make_float2(yp.z, yp.w));
                    a01 = add2(a01, make_float2(lo.x, lo.y));
                    a23 = add2(a23, make_float2(lo.z, lo.w));
                    a01 = add2(a01, make_float2(hi.x, hi.y));
                    a23 = add2(a23, make_float2(hi.z, hi.w));
                    a01 = __fmul2_rn(a01, sixth);
                    a23 = __fmul2_rn(a23, sixth);
                    if (f & kFull) {
                        v = make_float4(a01.x, a01.y, a23.x, a23.y);
                    } else {
                        v.x = (f & 0x10u) ? a01.x : c.x;
                        v.y = (f & 0x20u) ? a01.y : c.y;
                        v.z = (f & 0x40u) ? a23.x : c.z;
                        v.w = (f & 0x80u) ? a23.y : c.w;
                    }
                }
                q0[l - 1][r] = c;
                up[r] = v;
                // parity s&1 is read only in step s+1, after its barrier
                if (l < D && (f & kOwned) && sok(out + i0, 4)) *reinterpret_cast<float4 *>(out + i0) = v;
            }
            if (l == D && p >= z0 && p < z1) {
                float *dp = dst + (long long)p * plane;
                for (int r = 0; r < QPT; ++r) {
                    const unsigned f = qf[r];
                    const long long go = (long long)p * plane + goff[r];
                    if ((f & 0x100u) && gok(go)) dp[goff[r]] = up[r].x;
                    if ((f & 0x200u) && gok(go + 1)) dp[goff[r] + 1] = up[r].y;
                    if ((f & 0x400u) && gok(go + 2)) dp[goff[r] + 2] = up[r].z;
                    if ((f & 0x800u) && gok(go + 3)) dp[goff[r] + 3] = up[r].w;
                }
            }
        }
    }
    cp_async_wait_group<0>();
}

template <int D, int NT, int QPT>
cudaError_t launch_quad(const TbcArgs &a, cudaStream_t s)
{
    auto fn = tbc4_pass_kernel<D, NT, QPT>;
    const size_t smem = (size_t)(kRing + 2 * (D - 1)) * a.WH * sizeof(float);
    cudaError_t e = ensure_smem_limit((const void *)fn, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((a.nx + a.bx - 1) / a.bx), (unsigned)((a.ny + a.by - 1) / a.by),
              (unsigned)((a.nz + a.bz - 1) / a.bz));
    fn<<<grid, NT, smem, s>>>(a);
    return cudaGetLastError();
}

template <int D, int NT>
cudaError_t launch_qpt(const TbcArgs &a, cudaStream_t s)
{
    const int qpt = (a.WH / 4 + NT - 1) / NT;
    if (qpt <= 1) return launch_quad<D, NT, 1>(a, s);
    if (qpt <= 2) return launch_quad<D, NT, 2>(a, s);
    if (qpt <= 3) return launch_quad<D, NT, 3>(a, s);
    if (qpt <= 4) return launch_quad<D, NT, 4>(a, s);
    return cudaErrorInvalidValue;
}

template <int NT>
cudaError_t launch_quad_depth(const TbcArgs &a, int depth, cudaStream_t s)
{
    switch (depth) {
    case 1: return launch_qpt<1, NT>(a, s);
    case 2: return launch_qpt<2, NT>(a, s);
    case 3: return launch_qpt<3, NT>(a, s);
    case 4: return launch_qpt<4, NT>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T, int D, int NT, int CPT>
cudaError_t launch_one(const TbcArgs &a, cudaStream_t s)
{
    auto fn = tbc_pass_kernel<T, D, NT, CPT>;
    const size_t smem = (size_t)(kRing + 2 * (D - 1)) * a.WH * sizeof(T);
    cudaError_t e = ensure_smem_limit((const void *)fn, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((a.nx + a.bx - 1) / a.bx), (unsigned)((a.ny + a.by - 1) / a.by),
              (unsigned)((a.nz + a.bz - 1) / a.bz));
    fn<<<grid, NT, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int D, int NT>
cudaError_t launch_cpt(const TbcArgs &a, cudaStream_t s)
{
    const int cpt = (a.WH + NT - 1) / NT;
    if (cpt <= 2) return launch_one<T, D, NT, 2>(a, s);
    if (cpt <= 4) return launch_one<T, D, NT, 4>(a, s);
    if (cpt <= 6) return launch_one<T, D, NT, 6>(a, s);
    if (cpt <= 8) return launch_one<T, D, NT, 8>(a, s);
    return cudaErrorInvalidValue;
}

template <typename T, int NT>
cudaError_t launch_depth(const TbcArgs &a, int depth, cudaStream_t s)
{
    switch (depth) {
    case 1: return launch_cpt<T, 1, NT>(a, s);
    case 2: return launch_cpt<T, 2, NT>(a, s);
    case 3: return launch_cpt<T, 3, NT>(a, s);
    case 4: return launch_cpt<T, 4, NT>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int tbc_configure(int dtype, int depth, int bx, int by, int threads, TbcArgs *a, size_t *smem)
{
    if (depth < 1 || depth > 4 || bx < 1 || by < 1) return JACOBI_ERR_ARG;
    if ((long long)(a->nx + 2) * (a->ny + 2) >= (1ll << 31)) return JACOBI_ERR_UNSUPPORTED;  // 32-bit plane offsets
    if (threads != 256 && threads != 512) return JACOBI_ERR_ARG;
    a->bx = bx;
    a->by = by;
    a->W = bx + 2 * depth;
    if (dtype == JACOBI_F32) a->W = (a->W + 3) & ~3;  // quad rows
    a->H = by + 2 * depth;
    a->WH = a->W * a->H;
    if (dtype == JACOBI_F32 ? (a->WH / 4 + threads - 1) / threads > 4 : (a->WH + threads - 1) / threads > 8)
        return JACOBI_ERR_UNSUPPORTED;
    const size_t es = dtype == JACOBI_F64 ? 8 : 4;
    *smem = (size_t)(kRing + 2 * (depth - 1)) * a->WH * es;
    if (*smem > 227 * 1024) return JACOBI_ERR_UNSUPPORTED;
    return JACOBI_OK;
}

cudaError_t tbc_launch(int dtype, int depth, int threads, const TbcArgs &a, cudaStream_t s)
{
    if (dtype == JACOBI_F64)
        return threads == 512 ? launch_depth<double, 512>(a, depth, s) : launch_depth<double, 256>(a, depth, s);
    return threads == 512 ? launch_quad_depth<512>(a, depth, s) : launch_quad_depth<256>(a, depth, s);
}

}  // namespace jac
