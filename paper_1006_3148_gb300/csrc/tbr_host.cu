// Host side of the register-blocked one-CTA kernel: plan checks, tile
// geometry and the launch dispatch (instances in tbr_inst_a1.cu, copy
// pieces of one element, and tbr_inst_a2.cu, pieces of two).
#include <algorithm>

#include "jacobi_internal.h"
#include "tbr_kernels.cuh"

namespace jac {

int tbr_configure(int depth, int W, int H, TbrArgs *a, size_t *smem, int *threads)
{
    if (depth < 1 || depth > 4) return JACOBI_ERR_ARG;
    if (!((W == 64 && H == 32) || (W == 64 && H == 64) || (W == 128 && H == 32))) return JACOBI_ERR_ARG;
    if ((long long)(a->nx + 2) * (a->ny + 2) >= (1ll << 31)) return JACOBI_ERR_UNSUPPORTED;  // 32-bit plane offsets
    const int A = ((a->nx + 2) % 2 == 0) ? 2 : 1;
    const int off = ((1 - depth) % A + A) % A;
    const int bx = ((W - 2 * depth - off) / A) * A;
    const int by = H - 2 * depth;
    if (bx < 1 || by < 1 || a->bz < 1) return JACOBI_ERR_ARG;
    a->bx = bx;
    a->by = by;
    a->off = off;
    a->x_first = 1 - depth - off;
    if ((a->ny + by - 1) / by > 65535 || (a->nz + a->bz - 1) / a->bz > 65535) return JACOBI_ERR_UNSUPPORTED;
    const int TX = W / 4, TY = H / kTbrVY;
    const size_t lev = (size_t)2 * TY * W + (size_t)2 * TY * TX * kTbrVY;
    *smem = ((size_t)tbr_ring(depth) * W * H + 2 * (size_t)depth * lev) * sizeof(float);
    if (*smem > 227 * 1024) return JACOBI_ERR_UNSUPPORTED;
    if (threads) *threads = TX * TY;
    return JACOBI_OK;
}

cudaError_t tbr_launch(int depth, int W, int H, const TbrArgs &a, cudaStream_t s)
{
    TbrArgs c = a;
    size_t smem = 0;
    if (tbr_configure(depth, W, H, &c, &smem, nullptr) != JACOBI_OK) return cudaErrorInvalidValue;
    return ((a.nx + 2) % 2 == 0) ? tbr_launch_a2(depth, W, H, c, smem, s) : tbr_launch_a1(depth, W, H, c, smem, s);
}

}  // namespace jac
