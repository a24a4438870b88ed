// Batched temporally blocked FP32 passes: the register-blocked one-CTA
// kernel (tbr_kernels.cuh) over many grids in one launch, one block per
// (grid, tile, z chunk) unit, for the batch's FP32 grids (Sect. 2.1: several
// updates per cell per trip to memory, here for every grid of the batch).
#include <algorithm>
#include <vector>

#include "batch_internal.h"
#include "jacobi_internal.h"
#include "tbr_kernels.cuh"

namespace jac {
namespace {

template <int D, int A>
__global__ void __launch_bounds__(128, (TbrMinBlocks<D, 128, A>::value))
    tbr_batch_kernel(const BatchGrid *grids, const TbrBatchEntry *tab, int n, int pass, int *status, long long shrink)
{
    const long long b = blockIdx.x;
    int lo = 0, hi = n - 1;  // last entry with unit_base <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab[mid].unit_base <= b) lo = mid;
        else hi = mid - 1;
    }
    const TbrBatchEntry E = tab[lo];
    const long long u = b - E.unit_base;
    if (u >= (long long)E.ntx * E.nty * E.ntz) return;  // uniform per block
    const BatchGrid &G = grids[E.grid];
    TbrArgs a;
    a.src = (pass % 2 == 0) ? G.A : G.B;
    a.dst = (pass % 2 == 0) ? G.B : G.A;
    a.nx = G.nx;
    a.ny = G.ny;
    a.nz = G.nz;
    a.bx = E.bx;
    a.by = E.by;
    a.bz = kBatchTbrZ;
    a.x_first = E.x_first;
    a.off = E.off;
    a.status = status;
    a.shrink = shrink;
    const int txy = E.ntx * E.nty;
    tbr_cta<D, 16, 8, A>(a, (int)(u % E.ntx), (int)((u / E.ntx) % E.nty), (int)(u / txy));
}

template <int D>
constexpr size_t smem_bytes()
{
    // ring of 64 x 32 input planes and the two boundary buffers per level
    // (TX = 16, TY = 8 threads of 4 x 4 cells)
    return ((size_t)tbr_ring(D) * 64 * 32 + 2 * (size_t)D * (2 * 8 * 64 + 2 * 8 * 16 * kTbrVY)) * sizeof(float);
}

// configure: sets the kernel's shared memory limit only (outside capture)
template <int D, int A>
cudaError_t launch(const TbrBatchLaunch &L, const BatchGrid *d_grids, const TbrBatchEntry *d_tab, int *status,
                   long long shrink, cudaStream_t s, bool configure)
{
    auto fn = tbr_batch_kernel<D, A>;
    const size_t smem = smem_bytes<D>();
    if (configure) return ensure_smem_limit((const void *)fn, smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)L.units);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    return cudaLaunchKernelEx(&cfg, fn, d_grids, d_tab + L.tab_off, L.count, L.pass, status, shrink);
}

template <int A>
cudaError_t by_depth(const TbrBatchLaunch &L, const BatchGrid *g, const TbrBatchEntry *t, int *st, long long sh,
                     cudaStream_t s, bool configure)
{
    switch (L.depth) {
    case 1: return launch<1, A>(L, g, t, st, sh, s, configure);
    case 2: return launch<2, A>(L, g, t, st, sh, s, configure);
    case 3: return launch<3, A>(L, g, t, st, sh, s, configure);
    case 4: return launch<4, A>(L, g, t, st, sh, s, configure);
    default: return cudaErrorInvalidValue;
    }
}

static_assert(smem_bytes<4>() <= 227 * 1024, "shared memory of the deepest pass");

}  // namespace

void batch_tbr_plan(const std::vector<BatchGrid> &grids, int depth, std::vector<TbrBatchEntry> &tab,
                    std::vector<TbrBatchLaunch> &launches)
{
    tab.clear();
    launches.clear();
    std::vector<std::vector<int>> dep(grids.size());
    int maxp = 0;
    for (size_t g = 0; g < grids.size(); ++g) {
        const BatchGrid &G = grids[g];
        if (G.dtype != JACOBI_F32 || G.T <= 0) continue;
        dep[g].resize((size_t)G.T + 1);
        const int P = plan_passes(G.T, depth, dep[g].data(), G.T + 1);
        dep[g].resize((size_t)P);
        maxp = std::max(maxp, P);
    }
    for (int p = 0; p < maxp; ++p)
        for (int D = 1; D <= 4; ++D)
            for (int A = 1; A <= 2; ++A) {
                TbrBatchLaunch L;
                L.pass = p;
                L.depth = D;
                L.A = A;
                L.tab_off = (long long)tab.size();
                L.count = 0;
                L.units = 0;
                for (size_t g = 0; g < grids.size(); ++g) {
                    const BatchGrid &G = grids[g];
                    if ((int)dep[g].size() <= p || dep[g][(size_t)p] != D) continue;
                    if ((((G.nx + 2) % 2 == 0) ? 2 : 1) != A) continue;
                    TbrBatchEntry E;
                    E.off = ((1 - D) % A + A) % A;
                    E.bx = ((64 - 2 * D - E.off) / A) * A;
                    E.by = 32 - 2 * D;
                    E.x_first = 1 - D - E.off;
                    E.ntx = (G.nx + E.bx - 1) / E.bx;
                    E.nty = (G.ny + E.by - 1) / E.by;
                    E.ntz = (G.nz + kBatchTbrZ - 1) / kBatchTbrZ;
                    E.grid = (int)g;
                    E.unit_base = L.units;
                    L.units += (long long)E.ntx * E.nty * E.ntz;
                    tab.push_back(E);
                    ++L.count;
                }
                if (L.count > 0) launches.push_back(L);
            }
}

cudaError_t batch_tbr_configure(const TbrBatchLaunch &L)
{
    return L.A == 2 ? by_depth<2>(L, nullptr, nullptr, nullptr, 0, nullptr, true)
                    : by_depth<1>(L, nullptr, nullptr, nullptr, 0, nullptr, true);
}

cudaError_t batch_tbr_launch(const TbrBatchLaunch &L, const BatchGrid *d_grids, const TbrBatchEntry *d_tab,
                             int *status, long long shrink, cudaStream_t s)
{
    if (L.units <= 0 || L.units > 0x7fffffffll) return cudaErrorInvalidValue;
    return L.A == 2 ? by_depth<2>(L, d_grids, d_tab, status, shrink, s, false)
                    : by_depth<1>(L, d_grids, d_tab, status, shrink, s, false);
}

}  // namespace jac
