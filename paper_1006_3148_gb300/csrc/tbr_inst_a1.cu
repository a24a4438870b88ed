// Instances of the register-blocked one-CTA kernel with copy pieces of 1
// element(s) (row pitch nx+2 odd): depth 1..4 x regions 64x32, 64x64, 128x32.
#include <type_traits>

#include "tbr_kernels.cuh"

namespace jac {
namespace {

template <int D, int TX, int TY>
cudaError_t launch(const TbrArgs &a, size_t smem, cudaStream_t s)
{
    auto fn = tbr_pass_kernel<D, TX, TY, 1>;
    cudaError_t e = ensure_smem_limit((const void *)fn, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((a.nx + a.bx - 1) / a.bx), (unsigned)((a.ny + a.by - 1) / a.by),
                       (unsigned)((a.nz + a.bz - 1) / a.bz));
    cfg.blockDim = dim3(TX * TY);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    return cudaLaunchKernelEx(&cfg, fn, a);
}

template <int TX, int TY>
cudaError_t by_depth(int depth, const TbrArgs &a, size_t smem, cudaStream_t s)
{
    switch (depth) {
    case 1: return launch<1, TX, TY>(a, smem, s);
    case 2: return launch<2, TX, TY>(a, smem, s);
    case 3: return launch<3, TX, TY>(a, smem, s);
    case 4: return launch<4, TX, TY>(a, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t tbr_launch_a1(int depth, int W, int H, const TbrArgs &a, size_t smem, cudaStream_t s)
{
    if (W == 64 && H == 32) return by_depth<16, 8>(depth, a, smem, s);
    if (W == 64 && H == 64) return by_depth<16, 16>(depth, a, smem, s);
    if (W == 128 && H == 32) return by_depth<32, 8>(depth, a, smem, s);
    return cudaErrorInvalidValue;
}

}  // namespace jac
