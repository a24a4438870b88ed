// Instantiations of the cluster pass kernel (FP32, part 1 of the variant
// table of sweep_kernels.cu); one translation unit per part so that they
// compile in parallel.
#include "tb_pass.cuh"

namespace jac {

const void *tb_kernel_part3(int nc, int maxg)
{
    if (nc == 256 && maxg == 6) return (const void *)tb_pass_kernel<float, 256, 6, 8>;
    if (nc == 128 && maxg == 2) return (const void *)tb_pass_kernel<float, 128, 2, 16>;
    if (nc == 128 && maxg == 4) return (const void *)tb_pass_kernel<float, 128, 4, 16>;
    if (nc == 128 && maxg == 6) return (const void *)tb_pass_kernel<float, 128, 6, 16>;
    if (nc == 128 && maxg == 8) return (const void *)tb_pass_kernel<float, 128, 8, 16>;
    return nullptr;
}

}  // namespace jac
