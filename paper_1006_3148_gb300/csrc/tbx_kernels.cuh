// Temporal blocking by a chain of CTAs (FP32): the product of the two forms
// of Sect. 2.1, a team of threads (here the C CTAs of a thread-block cluster)
// each of which applies T updates to a block (here t_r time levels of the
// register-blocked step of tbr_kernels.cuh), so one pass over HBM applies
// d = t_0 + ... + t_{C-1} sweeps, up to 16.
//
// Every CTA of a cluster works on the same x-y tile and region and streams z
// like the one-CTA kernel.  CTA 0 reads the input grid through its cp.async
// ring.  CTA r > 0 reads the last level of CTA r-1 instead: CTA r-1 writes
// each plane of that level into CTA r's ring slot with st.async (distributed
// shared memory), every 16-byte store completing its bytes on the slot's
// mbarrier in CTA r (the GPU form of one thread handing a block to the next
// in the shared cache).  CTA C-1 stores the level-d values of its output
// planes to the grid.  The ring of R slots between two CTAs carries the two
// distance conditions of Eq. (3): a consumer waits until its producer has
// written the plane it reads next (at least one plane ahead), and a producer
// waits until its consumer has released the slot it is about to overwrite
// (at most R planes ahead).  A consumer releases a slot by re-arming its
// byte count and arriving on the producer's slot-free barrier.  Every wait is
// bounded: one that runs out records JACOBI_ERR_TIMEOUT and the CTA stops
// waiting (its results are then unspecified); a final cluster barrier keeps
// every CTA's shared memory alive until the hand-offs into it are done.
//
// The region's trapezoid is that of the whole depth d: CTA r's levels are
// the global levels L0+1 .. L0+t_r with L0 = t_0 + ... + t_{r-1}, valid on
// the region minus that many cells at each edge, and in z CTA r streams the
// planes its remaining depth d - L0 needs.
#pragma once

#include "tbr_kernels.cuh"

namespace jac {

constexpr int kTbxMaxCluster = 4;
constexpr int kTbxR = 4;  // ring slots between two CTAs (and of CTA 0's input)

__host__ __device__ constexpr size_t tbx_smem_floats(int TM, int W, int H)
{
    return (size_t)kTbxR * W * H + 2 * (size_t)TM * ((size_t)2 * (H / kTbrVY) * W + (size_t)2 * (H / kTbrVY) * (W / 4) * kTbrVY);
}

template <int TM, int TX, int TY, int A>
__global__ void __launch_bounds__(TX *TY, 1) tbx_pass_kernel(const TbxArgs a)
{
    constexpr int VY = kTbrVY, R = kTbxR, NT = TX * TY;
    constexpr int W = 4 * TX, H = VY * TY;
    constexpr int RING = W * H;
    constexpr int ROWS = 2 * TY * W;
    constexpr int COLS = 2 * TY * TX * VY;
    constexpr int LEV = ROWS + COLS;
    constexpr uint32_t PLANE_BYTES = (uint32_t)RING * 4u;
    extern __shared__ __align__(128) float tbx_smem[];
    float *ring = tbx_smem;
    float *bufs = tbx_smem + R * RING;  // [parity][level][LEV]
    const uint32_t in_full = smem_addr(bufs + 2 * TM * LEV);  // R mbarriers: slot holds its plane
    const uint32_t out_free = in_full + 8u * R;                // R mbarriers: next CTA released the slot

    const int C = a.cluster;
    const int rank = (int)cluster_ctarank();
    const int tr = a.levels[rank], L0 = a.lev_before[rank];
    const int Dd = a.depth, Dr = Dd - L0;  // total depth; depth left from this CTA's input
    const bool from_global = rank == 0, to_global = rank == C - 1;
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int tile = (int)blockIdx.x / C;
    const int xa = a.x_first + tile * a.bx;
    const int ya = 1 - Dd + (int)blockIdx.y * a.by;
    const int z0 = 1 + (int)blockIdx.z * a.bz;
    const int z1 = min(z0 + a.bz, a.nz + 1);
    const int xo = xa + a.off + Dd, yo = ya + Dd;
    const int gx0 = xa + 4 * tx;
    const int P = a.nx + 2;
    const long long plane = (long long)P * (a.ny + 2);
    const float *__restrict__ src = static_cast<const float *>(a.src);
    float *__restrict__ dst = static_cast<float *>(a.dst);
    int *status = a.status;
    const volatile int *vstatus = a.status;
    const long long SG = checked_grid_elems(a.nx, a.ny, a.nz, a.shrink);
    auto gok = [&](long long off, int n) { return in_bounds(off, n, SG, status); };
    auto rok = [&](const float *ptr, int n) { return in_bounds(ptr - ring, n, (long long)R * RING, status); };
    auto bok = [&](const float *ptr) { return in_bounds(ptr - bufs, 4, 2LL * TM * LEV, status); };

    // z range of this CTA: input planes q0 .. q0 + nin - 1, steps 0 .. nreal-1
    const int s_begin = z0 - Dr + 1, q0 = s_begin - 1;
    const int nreal = z1 - z0 + 2 * Dr - 2, nin = nreal + 2;
    // the next CTA's input planes
    const int Dn = Dr - tr, q0n = z0 - Dn, nin_next = (z1 - z0 + 2 * Dn - 2) + 2;

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
    const int o_above = TY * W + max(ty - 1, 0) * W + 4 * tx;
    const int o_below = min(ty + 1, TY - 1) * W + 4 * tx;
    const int o_left = ROWS + (TY * TX + ty * TX + max(tx - 1, 0)) * VY;
    const int o_right = ROWS + (ty * TX + min(tx + 1, TX - 1)) * VY;
    const int o_top = ty * W + 4 * tx, o_bot = TY * W + ty * W + 4 * tx;
    const int o_lcol = ROWS + (ty * TX + tx) * VY, o_rcol = ROWS + (TY * TX + ty * TX + tx) * VY;

    // ---- barriers (peer input, peer output)
    if (tid == 0) {
        for (int k = 0; k < R; ++k) {
            mbar_init(in_full + 8u * k, 1);
            mbar_init(out_free + 8u * k, 1);
        }
        fence_mbar_init_cluster();
        if (!from_global)
            for (int k = 0; k < R && k < nin; ++k) mbar_arrive_expect_tx(in_full + 8u * k, PLANE_BYTES);
    }
    cluster_sync_all();
    bool dead = false;
    auto wait = [&](uint32_t bar, int parity) {
        if (dead) return;
        if (!wait_parity_bounded(bar, (uint32_t)parity, a.limit_ns, vstatus)) {
            dead = true;
            atomicCAS(status, 0, JACOBI_ERR_TIMEOUT);
        }
    };
    const uint32_t next_ring = to_global ? 0u : mapa(smem_addr(ring), (uint32_t)(rank + 1));
    const uint32_t next_full = to_global ? 0u : mapa(in_full, (uint32_t)(rank + 1));
    const uint32_t prev_free = from_global ? 0u : mapa(out_free, (uint32_t)(rank - 1));
    // input index i (plane q0 + i) was read by every thread: re-arm its slot
    // for index i + R and tell the producer the slot is free
    auto release = [&](int i) {
        // (not after a timeout: the slot's phase may not have completed)
        if (from_global || tid != 0 || i >= nin || dead) return;
        const uint32_t k = (uint32_t)(i & (R - 1));
        if (i + R < nin) mbar_arrive_expect_tx(in_full + 8u * k, PLANE_BYTES);
        mbar_arrive_cluster(prev_free + 8u * k);
    };

    // ---- CTA 0: input planes through the cp.async ring (as the one-CTA kernel)
    constexpr int PPR = W / A, RPJ = NT / PPR, NJ = H / RPJ;
    const int cp_row = tid / PPR, cp_col = (tid % PPR) * A;
    const int cp_gx = xa + cp_col;
    const bool cp_xin = cp_gx >= 0 && cp_gx <= a.nx + 1;
    unsigned cp_rows = 0;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int gy = ya + cp_row + j * RPJ;
        if (cp_xin && gy >= 0 && gy <= a.ny + 1) cp_rows |= 1u << j;
    }
    const int cp_off0 = (ya + cp_row) * P + cp_gx;
    const uint32_t cp_dst0 = smem_addr(ring + cp_row * W + cp_col);
    auto load_plane = [&](int p) {
        const int i = p - q0;
        if (from_global && i < nin && p >= 0 && p <= a.nz + 1) {
            const float *sp = src + (long long)p * plane;
            const uint32_t d0 = cp_dst0 + (uint32_t)((i & (R - 1)) * RING * 4);
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                const bool in = (cp_rows >> j) & 1u;
                if (kChecked) {
                    const float *dl = ring + (i & (R - 1)) * RING + cp_row * W + cp_col + j * RPJ * W;
                    if (!rok(dl, A) || (in && !gok((long long)p * plane + cp_off0 + j * RPJ * P, A))) continue;
                }
                tbr_copy<A>(d0 + (uint32_t)(j * RPJ * W * 4), in ? sp + cp_off0 + j * RPJ * P : sp, in ? 4u * A : 0u);
            }
        }
        if (from_global) cp_async_commit();
    };
    auto write_bounds = [&](float *b, const float (&v)[VY][4]) {
        if (bok(b + o_top)) tbr_st4(b + o_top, v[0][0], v[0][1], v[0][2], v[0][3]);
        if (bok(b + o_bot)) tbr_st4(b + o_bot, v[VY - 1][0], v[VY - 1][1], v[VY - 1][2], v[VY - 1][3]);
        if (bok(b + o_lcol)) tbr_st4(b + o_lcol, v[0][0], v[1][0], v[2][0], v[3][0]);
        if (bok(b + o_rcol)) tbr_st4(b + o_rcol, v[0][3], v[1][3], v[2][3], v[3][3]);
    };
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    auto ldb = [&](const float *ptr) { return bok(ptr) ? tbr_ld4(ptr) : zero4; };
    auto ldr = [&](const float *ptr) { return rok(ptr, 4) ? tbr_ld4(ptr) : zero4; };

    float q[TM][3][VY][4];
#pragma unroll
    for (int k = 0; k < TM; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int r = 0; r < VY; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) q[k][i][r][c] = 0.f;

    // ---- prologue: input indices 0 and 1 (planes s_begin-1, s_begin)
    if (from_global) {
        load_plane(q0);
        load_plane(q0 + 1);
        cp_async_wait_group<0>();
    } else {
        wait(in_full, 0);
        wait(in_full + 8u, 0);
    }
    __syncthreads();
    {
        const float *r0 = ring_rd, *r1 = ring_rd + RING;
#pragma unroll
        for (int r = 0; r < VY; ++r) {
            const float4 u = ldr(r0 + r * W), v = ldr(r1 + r * W);
            q[0][2][r][0] = u.x, q[0][2][r][1] = u.y, q[0][2][r][2] = u.z, q[0][2][r][3] = u.w;
            q[0][0][r][0] = v.x, q[0][0][r][1] = v.y, q[0][0][r][2] = v.z, q[0][0][r][3] = v.w;
        }
    }
    write_bounds(bufs + 1 * TM * LEV, q[0][0]);
    __syncthreads();
    if (from_global)
        for (int i = 2; i < R + 1; ++i) load_plane(q0 + i);  // indices 2 .. R (R-1 groups in flight)

    auto step = [&](auto J, int t) {
        constexpr int j = decltype(J)::value;
        constexpr int iN = (j + 1) % 3, iC = j, iM = (j + 2) % 3;
        const int s = s_begin + t;
        const int iin = t + 2;  // input index of plane s+1
        if (from_global) cp_async_wait_group<R - 2>();
        else if (t < nreal) wait(in_full + 8u * (uint32_t)(iin & (R - 1)), (iin / R) & 1);
        __syncthreads();
        if (t == 0) release(0);
        release(t + 1);  // plane s: read in the previous step (or the prologue)
        {
            const float *rp = ring_rd + (iin & (R - 1)) * RING;
#pragma unroll
            for (int r = 0; r < VY; ++r) {
                const float4 u = ldr(rp + r * W);
                q[0][iN][r][0] = u.x, q[0][iN][r][1] = u.y, q[0][iN][r][2] = u.z, q[0][iN][r][3] = u.w;
            }
        }
        float *wb = bufs + (t & 1) * TM * LEV;
        const float *rb = bufs + ((t + 1) & 1) * TM * LEV;
        float4 nbv[4];
        nbv[0] = ldb(rb + o_above), nbv[1] = ldb(rb + o_below);
        nbv[2] = ldb(rb + o_left), nbv[3] = ldb(rb + o_right);
        load_plane(s + R);  // CTA 0: into the slot of plane s, read in the previous step
        write_bounds(wb, q[0][iN]);
#pragma unroll
        for (int l = 1; l <= TM; ++l) {
            if (l > tr) break;  // uniform
            const int k = l - 1;
            const int p = s - l + 1;
            const bool zin = p >= 1 && p <= a.nz;
            const float4 above = nbv[0], below = nbv[1], left = nbv[2], right = nbv[3];
            if (l < tr) {
                const float *nn = rb + l * LEV;
                nbv[0] = ldb(nn + o_above), nbv[1] = ldb(nn + o_below);
                nbv[2] = ldb(nn + o_left), nbv[3] = ldb(nn + o_right);
            }
            float v[VY][4];
            tbr_block_update(q[k][iC], q[k][iM], q[k][iN], above, below, left, right, v);
            if (!(zin && full)) {
#pragma unroll
                for (int r = 0; r < VY; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (!zin || !(upd & (1u << (r * 4 + c)))) v[r][c] = q[k][iC][r][c];
            }
            if (l < tr) {
#pragma unroll
                for (int r = 0; r < VY; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) q[l < TM ? l : 0][iN][r][c] = v[r][c];
                write_bounds(wb + l * LEV, v);
            } else if (to_global) {
                if (p >= z0 && p < z1 && st) {
                    float *dp = dst + (long long)p * plane;
#pragma unroll
                    for (int r = 0; r < VY; ++r)
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            if (((st >> (r * 4 + c)) & 1u) && gok((long long)p * plane + rowoff[r] + c, 1))
                                dp[rowoff[r] + c] = v[r][c];
                }
            } else {
                // hand plane p of global level L0 + tr to the next CTA
                const int jn = p - q0n;
                const bool drop = a.fault_mode == 1 && rank == 0 && jn == 2;  // test hook
                if (jn >= 0 && jn < nin_next && !drop && !dead) {
                    const uint32_t k2 = (uint32_t)(jn & (R - 1));
                    if (jn >= R) wait(out_free + 8u * k2, ((jn / R) - 1) & 1);
                    const uint32_t base = next_ring + k2 * PLANE_BYTES;
#pragma unroll
                    for (int r = 0; r < VY; ++r) {
                        const int e = (VY * ty + r) * W + 4 * tx;  // same cell in the next CTA's ring
                        if (in_bounds(e + (long long)k2 * RING, 4, (long long)R * RING, status)) {
                            const float vv[4] = {v[r][0], v[r][1], v[r][2], v[r][3]};
                            st_async_v(base + (uint32_t)e * 4u, vv, next_full + 8u * k2);
                        }
                    }
                }
            }
        }
    };
    for (int t = 0; t < nreal; t += 3) {
        step(std::integral_constant<int, 0>(), t);
        step(std::integral_constant<int, 1>(), t + 1);
        step(std::integral_constant<int, 2>(), t + 2);
    }
    if (from_global) cp_async_wait_group<0>();
    cluster_sync_all();
}

}  // namespace jac
