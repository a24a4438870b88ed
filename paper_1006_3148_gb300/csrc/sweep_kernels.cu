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

#include "arith.cuh"
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
    const long long NXP = nx + 2, NYP = ny + 2;
    const long long nzf = 2 * NXP * NYP;          // k = 0 and k = nz+1 planes
    const long long nyf = 2 * NXP * (long long)nz;  // j = 0 and j = ny+1 rows
    const long long nxf = 2 * (long long)ny * nz;   // i = 0 and i = nx+1 cells
    const long long total = nzf + nyf + nxf;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        long long i, j, k;
        if (t < nzf) {
            const long long p = t % (NXP * NYP);
            k = (t < NXP * NYP) ? 0 : nz + 1;
            j = p / NXP;
            i = p % NXP;
        } else if (t < nzf + nyf) {
            const long long u = t - nzf;
            const long long half = NXP * nz;
            j = (u < half) ? 0 : ny + 1;
            const long long p = u % half;
            k = 1 + p / NXP;
            i = p % NXP;
        } else {
            const long long u = t - nzf - nyf;
            const long long half = (long long)ny * nz;
            i = (u < half) ? 0 : nx + 1;
            const long long p = u % half;
            k = 1 + p / ny;
            j = 1 + p % ny;
        }
        const long long idx = (k * NYP + j) * NXP + i;
        B[idx] = A[idx];
    }
}

// ----------------------------------------------------------------- plain
template <typename T>
__global__ void __launch_bounds__(256) plain_pass_kernel(const PlainArgs a)
{
    const T *__restrict__ src = static_cast<const T *>(a.src);
    T *__restrict__ dst = static_cast<T *>(a.dst);
    const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    const int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;
    if (i > a.nx || j > a.ny) return;
    const long long NXP = a.nx + 2, plane = NXP * (a.ny + 2);
    const int kb = 1 + blockIdx.z * a.kz;
    const int ke = min(kb + a.kz, a.nz + 1);
    for (int k = kb; k < ke; ++k) {
        const long long c = k * plane + j * NXP + i;
        dst[c] = Arith<T>::update(__ldg(src + c - 1), __ldg(src + c + 1), __ldg(src + c - NXP),
                                  __ldg(src + c + NXP), __ldg(src + c - plane), __ldg(src + c + plane));
    }
}

// -------------------------------------------------------- time-skewed pass
// Thread roles: threads [0, NC) compute (each owns up to MAXC cells of the
// level's output region, fixed for the whole z stream, with a register queue
// of the values at planes k-1 and k); warp NC/32 of the level-1 CTA issues
// the bulk copies that stream input planes from HBM into its ring.
//
// Shared memory of every CTA: ring[R][H][Wp] of T (slot = one z-plane of
// the tile widened by D cells), then three arrays of R mbarriers:
//   in_full[s]   slot s holds its plane (level 1: byte count of the bulk
//                copies; level >= 2: one arrival from the producer CTA)
//   in_empty[s]  level 1 only: its compute threads released slot s
//   out_empty[s] the next CTA released its slot s (remote arrival)
// Element (x, y) of a slot sits at column (x - (x0-D)) + off, row y-(y0-D).
// off = 0 except in level 1's ring, whose rows are copied whole 16-byte
// units from global memory: there off = (global row start misalignment)/s.
template <typename T, int NC, int MAXC>
__global__ void __launch_bounds__(NC + kTbThreadsLoader, 1) tb_pass_kernel(const TbArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int V = 16 / (int)sizeof(T);
    const int D = a.depth;
    const int rank = (int)cluster_ctarank();
    const int lvl = rank + 1;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int NXP = nx + 2, NYP = ny + 2;
    const int x0 = 1 + (int)(blockIdx.x / D) * a.bx, x1 = min(x0 + a.bx, nx + 1);
    const int y0 = 1 + (int)blockIdx.y * a.by, y1 = min(y0 + a.by, ny + 1);
    const int z0 = 1 + (int)blockIdx.z * a.bz, z1 = min(z0 + a.bz, nz + 1);
    const int gx = x0 - D, gy = y0 - D;
    const int Wp = a.Wp, R = a.R;
    const int slot_elems = a.H * Wp;
    T *ring = reinterpret_cast<T *>(smem);
    const uint32_t ring_s = smem_addr(ring);
    const uint32_t in_full = ring_s + (uint32_t)(R * slot_elems * (int)sizeof(T));
    const uint32_t in_empty = in_full + 8u * R;
    const uint32_t out_empty = in_full + 16u * R;
    const int tid = threadIdx.x;
    const volatile int *vstatus = a.status;

    if (tid == 0) {
        for (int s = 0; s < R; ++s) {
            mbar_init(in_full + 8u * s, 1);
            mbar_init(in_empty + 8u * s, 1);
            mbar_init(out_empty + 8u * s, 1);
        }
        fence_mbar_init_cluster();
    }
    cluster_sync_all();

    const int wl = D - lvl;  // this level's region is the tile widened by wl
    const int zo0 = max(z0 - wl, 0), zo1 = min(z1 + wl, nz + 2);
    const int zi0 = max(z0 - wl - 1, 0), zi1 = min(z1 + wl + 1, nz + 2);

    if (tid >= NC) {
        // ------------------------------------------------ level-1 loader warp
        if (lvl == 1) {
            const int lane = tid - NC;
            const int ix0 = max(gx, 0), ix1 = min(x1 + D, NXP);
            const int iy0 = max(gy, 0), iy1 = min(y1 + D, NYP);
            const char *src = static_cast<const char *>(a.src);
            const long long es = sizeof(T);
            int n_issued = 0;
            for (int n = 0; n < zi1 - zi0; ++n) {
                const int k = zi0 + n, s = n % R;
                int ok = (*vstatus == 0);
                if (ok && n >= R && lane == 0)
                    ok = wait_parity_bounded(in_empty + 8u * s, ((n / R) - 1) & 1, a.limit_ns, vstatus);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) record_error(a.status, JACOBI_ERR_TIMEOUT);
                    break;
                }
                // Halo planes only feed z-neighbours of interior cells: rows 1..ny.
                const bool hz = (k == 0 || k == nz + 1);
                const int jr0 = hz ? max(iy0, 1) : iy0;
                const int jr1 = hz ? min(iy1, ny + 1) : iy1;
                uint32_t my_bytes = 0;
                for (int j = jr0 + lane; j < jr1; j += 32) {
                    const long long row = ((long long)k * NYP + j) * NXP;
                    const long long gs = ((row + ix0) * es) & ~15ll;
                    const long long ge = ((row + ix1) * es + 15) & ~15ll;
                    my_bytes += (uint32_t)(ge - gs);
                }
                if (my_bytes) mbar_expect_tx(in_full + 8u * s, my_bytes);
                __syncwarp();
                if (lane == 0 && !(a.fault_mode == 1 && n == 2)) mbar_arrive_local(in_full + 8u * s);
                for (int j = jr0 + lane; j < jr1; j += 32) {
                    const long long row = ((long long)k * NYP + j) * NXP;
                    const long long gs = ((row + ix0) * es) & ~15ll;
                    const long long ge = ((row + ix1) * es + 15) & ~15ll;
                    const long long vb = (row + gx) * es;
                    const long long vs = vb - (((vb % 16) + 16) % 16);  // floor to 16 bytes
                    const uint32_t dst = ring_s + (uint32_t)((s * slot_elems + (j - gy) * Wp) * (int)es) +
                                         (uint32_t)(gs - vs);
                    bulk_g2s(dst, src + gs, (uint32_t)(ge - gs), in_full + 8u * s);
                }
                n_issued = n + 1;
            }
            // Never leave with copies in flight into this CTA's shared memory.
            if (lane == 0)
                for (int n = max(0, n_issued - R); n < n_issued; ++n)
                    wait_parity_bounded(in_full + 8u * (n % R), (n / R) & 1, a.limit_ns, nullptr);
            __syncwarp();
        }
    } else {
        // ---------------------------------------------------- compute threads
        const int ox0 = max(x0 - wl, 0), ox1 = min(x1 + wl, NXP);
        const int oy0 = max(y0 - wl, 0), oy1 = min(y1 + wl, NYP);
        const int Wo = ox1 - ox0, Ho = oy1 - oy0, ncell = Wo * Ho;
        const int vmask = (lvl == 1) ? V - 1 : 0;
        const int NXV = NXP & (V - 1);
        const int PSV = (int)(((long long)NYP * NXP) & (V - 1));
        const int gxv = gx & (V - 1);

        int lofs[MAXC], yv[MAXC], gofs[MAXC];
        uint32_t valid = 0, comp = 0;
#pragma unroll
        for (int q = 0; q < MAXC; ++q) {
            const int idx = tid + q * NC;
            const int x = ox0 + (idx % Wo), y = oy0 + (idx / Wo);
            lofs[q] = (y - gy) * Wp + (x - gx);
            yv[q] = (y * NXV) & (V - 1);
            gofs[q] = y * NXP + x;
            if (idx < ncell) valid |= 1u << q;
            if (idx < ncell && x >= 1 && x <= nx && y >= 1 && y <= ny) comp |= 1u << q;
        }

        const uint32_t next_ring = (lvl < D) ? mapa(ring_s, rank + 1) : 0u;
        const uint32_t next_full = (lvl < D) ? mapa(in_full, rank + 1) : 0u;
        const uint32_t prev_oe = (lvl > 1) ? mapa(out_empty, rank - 1) : 0u;
        T *dst = static_cast<T *>(a.dst);
        const long long plane = (long long)NYP * NXP;
        bool dead = false;
        auto wait = [&](uint32_t bar, int parity) {
            if (dead) return;
            if (!wait_parity_bounded(bar, (uint32_t)parity, a.limit_ns, vstatus)) {
                dead = true;
                record_error(a.status, JACOBI_ERR_TIMEOUT);
            }
        };
        auto release = [&](int seq) {
            const uint32_t off = 8u * (uint32_t)(seq % R);
            if (lvl == 1) mbar_arrive_local(in_empty + off);
            else mbar_arrive_cluster(prev_oe + off);
        };
        auto own = [&](int p, int q) -> T {
            const int n = p - zi0;
            const int ok = (p * PSV + gxv + yv[q]) & vmask;
            return ring[(n % R) * slot_elems + lofs[q] + ok];
        };

        T av[MAXC], bv[MAXC];
#pragma unroll
        for (int q = 0; q < MAXC; ++q) av[q] = bv[q] = T(0);
        if (zo0 > zi0) {
            wait(in_full, 0);
#pragma unroll
            for (int q = 0; q < MAXC; ++q)
                if (valid & (1u << q)) av[q] = own(zo0 - 1, q);
        }
        {
            const int n = zo0 - zi0;
            wait(in_full + 8u * (n % R), (n / R) & 1);
#pragma unroll
            for (int q = 0; q < MAXC; ++q)
                if (valid & (1u << q)) bv[q] = own(zo0, q);
        }

        for (int k = zo0; k < zo1; ++k) {
            const int n = k - zi0, m = k - zo0;
            const bool has_next = (k + 1 < zi1);
            const bool interior_k = (k >= 1 && k <= nz);
            T cv[MAXC];
#pragma unroll
            for (int q = 0; q < MAXC; ++q) cv[q] = T(0);
            if (has_next) {
                wait(in_full + 8u * ((n + 1) % R), ((n + 1) / R) & 1);
#pragma unroll
                for (int q = 0; q < MAXC; ++q)
                    if (valid & (1u << q)) cv[q] = own(k + 1, q);
            }
            if (lvl < D && m >= R) wait(out_empty + 8u * (m % R), ((m / R) - 1) & 1);

            const T *cen = ring + (n % R) * slot_elems;
            const int okc = (k * PSV + gxv) & vmask;
#pragma unroll
            for (int q = 0; q < MAXC; ++q) {
                if (!(valid & (1u << q))) continue;
                T v = bv[q];
                if (interior_k && (comp & (1u << q))) {
                    const int oc = (okc + yv[q]) & vmask;
                    const int c = lofs[q] + oc;
                    const T wv = cen[c - 1];
                    const T ev = cen[c + 1];
                    const T sv = cen[lofs[q] - Wp + ((okc + yv[q] - NXV) & vmask)];
                    const T nv = cen[lofs[q] + Wp + ((okc + yv[q] + NXV) & vmask)];
                    v = Arith<T>::update(wv, ev, sv, nv, av[q], cv[q]);
                }
                if (lvl < D)
                    st_cluster(next_ring + (uint32_t)(((m % R) * slot_elems + lofs[q]) * (int)sizeof(T)), v);
                else
                    dst[k * plane + gofs[q]] = v;
                av[q] = bv[q];
                bv[q] = cv[q];
            }
            named_bar_sync(1, NC);
            if (tid == 0) {
                if (lvl < D) {
                    fence_acq_rel_cluster();
                    mbar_arrive_cluster(next_full + 8u * (uint32_t)(m % R));
                }
                if (k == zo0 && zo0 > zi0) release(n - 1);
                release(n);
            }
        }
    }
    cluster_sync_all();
}

// ------------------------------------------------------------------- host
namespace {

struct Variant {
    int nc, maxc;
};
constexpr Variant kVariants[] = {{128, 2}, {128, 4}, {256, 4}, {256, 8}, {512, 8}, {512, 16}};
constexpr int kSmemMax = 232448;  // 227 KB per CTA on sm_100-class GPUs

template <typename T>
const void *tb_kernel_ptr(int nc, int maxc)
{
    if (nc == 128 && maxc == 2) return (const void *)tb_pass_kernel<T, 128, 2>;
    if (nc == 128 && maxc == 4) return (const void *)tb_pass_kernel<T, 128, 4>;
    if (nc == 256 && maxc == 4) return (const void *)tb_pass_kernel<T, 256, 4>;
    if (nc == 256 && maxc == 8) return (const void *)tb_pass_kernel<T, 256, 8>;
    if (nc == 512 && maxc == 8) return (const void *)tb_pass_kernel<T, 512, 8>;
    if (nc == 512 && maxc == 16) return (const void *)tb_pass_kernel<T, 512, 16>;
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
    return cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

}  // namespace

cudaError_t tb_configure(int dtype, int depth, int bx, int by, TbLaunch *out)
{
    const int es = dtype == JACOBI_F64 ? 8 : 4;
    const int V = 16 / es;
    TbLaunch L;
    L.R = 4;
    L.W = bx + 2 * depth;
    L.H = by + 2 * depth;
    L.Wp = ((L.W + 2 * V + V - 1) / V) * V;
    L.smem = (size_t)L.R * L.H * L.Wp * es + 3 * 8 * (size_t)L.R;
    const long long cells = (long long)(bx + 2 * (depth - 1)) * (by + 2 * (depth - 1));
    L.nc = 0;
    for (const Variant &v : kVariants)
        if ((long long)v.nc * v.maxc >= cells) {
            L.nc = v.nc;
            L.maxc = v.maxc;
            break;
        }
    if (L.nc == 0 || L.smem > (size_t)kSmemMax) return cudaErrorInvalidConfiguration;
    *out = L;
    return cudaSuccess;
}

cudaError_t tb_launch(int dtype, const TbArgs &a, const TbLaunch &L, cudaStream_t s)
{
    const void *fn = tb_kernel(dtype, L.nc, L.maxc);
    if (!fn) return cudaErrorInvalidConfiguration;
    static bool prepared[2][6] = {};
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
    cfg.blockDim = dim3((unsigned)(L.nc + kTbThreadsLoader), 1, 1);
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
    cfg.blockDim = dim3((unsigned)(L.nc + kTbThreadsLoader), 1, 1);
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

cudaError_t plain_launch(int dtype, const PlainArgs &a, cudaStream_t s)
{
    dim3 block(32, 8, 1);
    dim3 grid((unsigned)((a.nx + 31) / 32), (unsigned)((a.ny + 7) / 8), (unsigned)((a.nz + a.kz - 1) / a.kz));
    if (dtype == JACOBI_F64) plain_pass_kernel<double><<<grid, block, 0, s>>>(a);
    else plain_pass_kernel<float><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t halo_copy_launch(int dtype, const void *A, void *B, int nx, int ny, int nz, cudaStream_t s)
{
    const long long NXP = nx + 2, NYP = ny + 2;
    const long long total = 2 * NXP * NYP + 2 * NXP * (long long)nz + 2 * (long long)ny * nz;
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
