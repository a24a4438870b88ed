// The cell update of Eq. (1) in each precision.  Explicit round-to-nearest
// intrinsics keep the compiler from contracting or reassociating: the six
// neighbours are added left to right in the printed order (i-1, i+1, j-1,
// j+1, k-1, k+1).
//   FP64: the sum is divided by 6.0 (IEEE quotient, round to nearest), so
//         results are bit-identical to a plain CPU loop.
//   FP32: the sum is multiplied by RN_f32(1/6) (one multiplication and five
//         additions, the count of Sect. 2.3).
#pragma once

namespace jac {

template <typename T>
struct Arith;

template <>
struct Arith<double> {
    static __device__ __forceinline__ double update(double w, double e, double s, double n, double b,
                                                    double t)
    {
        double a = __dadd_rn(w, e);
        a = __dadd_rn(a, s);
        a = __dadd_rn(a, n);
        a = __dadd_rn(a, b);
        a = __dadd_rn(a, t);
        return __ddiv_rn(a, 6.0);
    }
};

template <>
struct Arith<float> {
    static __device__ __forceinline__ float update(float w, float e, float s, float n, float b, float t)
    {
        float a = __fadd_rn(w, e);
        a = __fadd_rn(a, s);
        a = __fadd_rn(a, n);
        a = __fadd_rn(a, b);
        a = __fadd_rn(a, t);
        return __fmul_rn(a, 1.0f / 6.0f);
    }
};

}  // namespace jac
