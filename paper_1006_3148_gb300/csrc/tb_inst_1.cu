// Instantiations of the cluster pass kernel (FP64, part 1 of the variant
// table of sweep_kernels.cu); one translation unit per part so that they
// compile in parallel.
#include "tb_pass.cuh"

namespace jac {

const void *tb_kernel_part1(int nc, int maxg)
{
    if (nc == 256 && maxg == 6) return (const void *)tb_pass_kernel<double, 256, 6, 8>;
    if (nc == 128 && maxg == 2) return (const void *)tb_pass_kernel<double, 128, 2, 16>;
    if (nc == 128 && maxg == 4) return (const void *)tb_pass_kernel<double, 128, 4, 16>;
    if (nc == 128 && maxg == 6) return (const void *)tb_pass_kernel<double, 128, 6, 16>;
    if (nc == 128 && maxg == 8) return (const void *)tb_pass_kernel<double, 128, 8, 16>;
    return nullptr;
}

}  // namespace jac
