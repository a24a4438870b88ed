// Instantiations of the cluster pass kernel (FP32, part 0 of the variant
// table of sweep_kernels.cu); one translation unit per part so that they
// compile in parallel.
#include "tb_pass.cuh"

namespace jac {

const void *tb_kernel_part2(int nc, int maxg)
{
    if (nc == 512 && maxg == 1) return (const void *)tb_pass_kernel<float, 512, 1, 4>;
    if (nc == 512 && maxg == 2) return (const void *)tb_pass_kernel<float, 512, 2, 4>;
    if (nc == 256 && maxg == 1) return (const void *)tb_pass_kernel<float, 256, 1, 8>;
    if (nc == 256 && maxg == 2) return (const void *)tb_pass_kernel<float, 256, 2, 8>;
    if (nc == 256 && maxg == 4) return (const void *)tb_pass_kernel<float, 256, 4, 8>;
    return nullptr;
}

}  // namespace jac
