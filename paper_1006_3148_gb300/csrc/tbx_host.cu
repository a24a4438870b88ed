// Host side and instances of the chained-cluster kernel (tbx_kernels.cuh):
// at most 2 or 4 levels per CTA (template), regions 64x32 and 64x64, copy
// pieces of one or two elements.
#include <algorithm>
#include <type_traits>

#include "jacobi_internal.h"
#include "tbx_kernels.cuh"

namespace jac {
namespace {

template <int TM, int TX, int TY, int A>
const void *kernel_ptr()
{
    return reinterpret_cast<const void *>(tbx_pass_kernel<TM, TX, TY, A>);
}

const void *pick(int tm, int W, int H, int A)
{
    if (W == 64 && H == 32) {
        if (tm == 2) return A == 2 ? kernel_ptr<2, 16, 8, 2>() : kernel_ptr<2, 16, 8, 1>();
        return A == 2 ? kernel_ptr<4, 16, 8, 2>() : kernel_ptr<4, 16, 8, 1>();
    }
    if (tm == 2) return A == 2 ? kernel_ptr<2, 16, 16, 2>() : kernel_ptr<2, 16, 16, 1>();
    return A == 2 ? kernel_ptr<4, 16, 16, 2>() : kernel_ptr<4, 16, 16, 1>();
}

cudaLaunchConfig_t config(const TbxArgs &a, int W, int H, size_t smem, cudaLaunchAttribute *attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(((a.nx + a.bx - 1) / a.bx) * a.cluster), (unsigned)((a.ny + a.by - 1) / a.by),
                       (unsigned)((a.nz + a.bz - 1) / a.bz));
    cfg.blockDim = dim3((unsigned)(W * H / 16));
    cfg.dynamicSmemBytes = smem;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)a.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

int max_levels(int depth, int cluster) { return (depth + cluster - 1) / cluster; }

}  // namespace

int tbx_configure(int depth, int cluster, int W, int H, TbxArgs *a, size_t *smem)
{
    if (cluster < 2 || cluster > kTbxMaxCluster || depth < cluster || depth > 4 * cluster) return JACOBI_ERR_ARG;
    if (!((W == 64 && H == 32) || (W == 64 && H == 64))) return JACOBI_ERR_ARG;
    if ((long long)(a->nx + 2) * (a->ny + 2) >= (1ll << 31)) return JACOBI_ERR_UNSUPPORTED;
    const int A = ((a->nx + 2) % 2 == 0) ? 2 : 1;
    const int off = ((1 - depth) % A + A) % A;
    const int bx = ((W - 2 * depth - off) / A) * A, by = H - 2 * depth;
    if (bx < 1 || by < 1 || a->bz < 1) return JACOBI_ERR_ARG;
    a->bx = bx;
    a->by = by;
    a->off = off;
    a->x_first = 1 - depth - off;
    a->depth = depth;
    a->cluster = cluster;
    int before = 0;
    for (int r = 0; r < 4; ++r) {
        a->levels[r] = (r < cluster) ? depth / cluster + (r < depth % cluster ? 1 : 0) : 0;
        a->lev_before[r] = before;
        before += a->levels[r];
    }
    const long long tiles_x = (a->nx + bx - 1) / bx;
    if (tiles_x * cluster > 0x7fffffffll || (a->ny + by - 1) / by > 65535 || (a->nz + a->bz - 1) / a->bz > 65535)
        return JACOBI_ERR_UNSUPPORTED;
    const int tm = max_levels(depth, cluster) <= 2 ? 2 : 4;
    *smem = tbx_smem_floats(tm, W, H) * sizeof(float) + 16 * (size_t)kTbxR;  // + 2R mbarriers
    if (*smem > 227 * 1024) return JACOBI_ERR_UNSUPPORTED;
    return JACOBI_OK;
}

cudaError_t tbx_launch(int depth, int cluster, int W, int H, const TbxArgs &a0, cudaStream_t s)
{
    TbxArgs a = a0;
    size_t smem = 0;
    if (tbx_configure(depth, cluster, W, H, &a, &smem) != JACOBI_OK) return cudaErrorInvalidValue;
    const int tm = max_levels(depth, cluster) <= 2 ? 2 : 4;
    const void *fn = pick(tm, W, H, (a.nx + 2) % 2 == 0 ? 2 : 1);
    cudaError_t e = ensure_smem_limit(fn, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = config(a, W, H, smem, attr);
    cfg.stream = s;
    void *args[] = {&a};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t tbx_max_clusters(int depth, int cluster, int W, int H, int nx, int *clusters)
{
    TbxArgs a;
    a.nx = nx;
    a.ny = H;
    a.nz = 1;
    a.bz = 1;
    size_t smem = 0;
    if (tbx_configure(depth, cluster, W, H, &a, &smem) != JACOBI_OK) return cudaErrorInvalidValue;
    const int tm = max_levels(depth, cluster) <= 2 ? 2 : 4;
    const void *fn = pick(tm, W, H, (nx + 2) % 2 == 0 ? 2 : 1);
    cudaError_t e = ensure_smem_limit(fn, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = config(a, W, H, smem, attr);
    return cudaOccupancyMaxActiveClusters(clusters, fn, &cfg);
}

}  // namespace jac
