// Device self-test of the integer-pipe division used by the FP64 kernels.
#include <cuda_runtime.h>

#include "arith.cuh"
#include "jacobi_internal.h"

namespace jac {
namespace {

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ void check_one(unsigned long long bits, unsigned long long *bad, unsigned long long *first)
{
    const double x = __longlong_as_double((long long)bits);
    if (x != x) return;  // NaN: both sides return a NaN, payload not compared
    const double a = div6_rn(x), e = __ddiv_rn(x, 6.0);
    if (__double_as_longlong(a) != __double_as_longlong(e)) {
        if (atomicAdd(bad, 1ull) == 0ull) *first = bits;
    }
}

// Random bit patterns (counter-based SplitMix64) ...
__global__ void check_random(unsigned long long count, unsigned long long seed, unsigned long long *bad,
                             unsigned long long *first)
{
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < count;
         i += (unsigned long long)gridDim.x * blockDim.x)
        check_one(splitmix64(seed + i * 0x9E3779B97F4A7C15ull), bad, first);
}

// ... and, for every exponent and both signs, mantissas near the points
// where the algorithm changes branch or the result significand carries:
// 2^52, 3*2^51 and 2^53-1 (+-4096 each).
__global__ void check_structured(unsigned long long *bad, unsigned long long *first)
{
    const unsigned E = blockIdx.x;  // 0..2047
    const unsigned long long bases[3] = {0x10000000000000ull, 0x18000000000000ull, 0x1FFFFFFFFFFFFFull};
    for (int t = threadIdx.x; t < 3 * 8192; t += blockDim.x) {
        const long long d = (long long)(t % 8192) - 4096;
        const long long M = (long long)bases[t / 8192] + d;
        if (M < 0x10000000000000ll || M > 0x1FFFFFFFFFFFFFll) continue;
        const unsigned long long frac = (unsigned long long)M & 0xFFFFFFFFFFFFFull;
        const unsigned long long b = ((unsigned long long)E << 52) | frac;
        check_one(b, bad, first);
        check_one(b | 0x8000000000000000ull, bad, first);
    }
}

__device__ void check_add(unsigned long long ba, unsigned long long bb, unsigned long long *bad,
                          unsigned long long *first)
{
    const double x = __longlong_as_double((long long)ba), y = __longlong_as_double((long long)bb);
    const double r = add_rn_int(x, y), e = __dadd_rn(x, y);
    if (r != r && e != e) return;  // both NaN
    if (__double_as_longlong(r) != __double_as_longlong(e)) {
        if (atomicAdd(bad, 1ull) == 0ull) {
            first[0] = ba;
            first[1] = bb;
        }
    }
}

// Random pairs: independent bit patterns, pairs with the same sign and
// exponents a random distance 0..63 apart (the integer path's cases up to
// 31 apart: carries, sticky bits, ties) and a value plus a zero.
__global__ void check_add_random(unsigned long long count, unsigned long long seed, unsigned long long *bad,
                                 unsigned long long *first)
{
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < count;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long r1 = splitmix64(seed + 3 * i * 0x9E3779B97F4A7C15ull);
        const unsigned long long r2 = splitmix64(seed + (3 * i + 1) * 0x9E3779B97F4A7C15ull);
        const unsigned long long r3 = splitmix64(seed + (3 * i + 2) * 0x9E3779B97F4A7C15ull);
        check_add(r1, r2, bad, first);
        const unsigned e1 = 1u + (unsigned)((r3 >> 8) % 2045u);
        const unsigned d = (unsigned)(r3 & 63u);
        const unsigned e2 = (e1 > d) ? e1 - d : 1u;
        const unsigned long long s = (r3 >> 63) << 63;
        const unsigned long long a = s | ((unsigned long long)e1 << 52) | (r1 & 0xFFFFFFFFFFFFFull);
        unsigned long long b = s | ((unsigned long long)e2 << 52) | (r2 & 0xFFFFFFFFFFFFFull);
        if ((r3 >> 20) & 1ull) b = (b & ~0xFFFFFFFFFull) | (1ull << ((r3 >> 21) % 36));  // sparse low bits: ties
        check_add(a, b, bad, first);
        check_add(b, a, bad, first);
        // a zero of either sign against a random value
        check_add(a, (r3 & 2ull) ? 0x8000000000000000ull : 0ull, bad, first);
    }
}

}  // namespace
}  // namespace jac

extern "C" int jacobi_check_addition(unsigned long long count, unsigned long long seed,
                                     unsigned long long *mismatches, unsigned long long *first_bad)
{
    if (!mismatches) return JACOBI_ERR_ARG;
    unsigned long long *d = nullptr;
    if (cudaMalloc(&d, 3 * sizeof(unsigned long long)) != cudaSuccess) return JACOBI_ERR_ALLOC;
    cudaError_t e = cudaMemset(d, 0, 3 * sizeof(unsigned long long));
    if (e == cudaSuccess) {
        jac::check_add_random<<<152 * 16, 256>>>(count, seed, d, d + 1);
        e = cudaGetLastError();
    }
    unsigned long long h[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return JACOBI_ERR_CUDA;
    *mismatches = h[0];
    if (first_bad) {
        first_bad[0] = h[1];
        first_bad[1] = h[2];
    }
    return JACOBI_OK;
}

extern "C" int jacobi_check_division(unsigned long long count, unsigned long long seed,
                                     unsigned long long *mismatches, unsigned long long *first_bad)
{
    if (!mismatches) return JACOBI_ERR_ARG;
    unsigned long long *d = nullptr;
    if (cudaMalloc(&d, 2 * sizeof(unsigned long long)) != cudaSuccess) return JACOBI_ERR_ALLOC;
    cudaError_t e = cudaMemset(d, 0, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) {
        jac::check_structured<<<2048, 256>>>(d, d + 1);
        if (count) jac::check_random<<<152 * 16, 256>>>(count, seed, d, d + 1);
        e = cudaGetLastError();
    }
    unsigned long long h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return JACOBI_ERR_CUDA;
    *mismatches = h[0];
    if (first_bad) *first_bad = h[1];
    return JACOBI_OK;
}
