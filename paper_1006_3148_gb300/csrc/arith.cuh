// The cell update of Eq. (1) in each precision.  Explicit round-to-nearest
// intrinsics keep the compiler from contracting or reassociating: the six
// neighbours are added left to right in the printed order (i-1, i+1, j-1,
// j+1, k-1, k+1).
//   FP64: the sum is divided by 6.0 (IEEE quotient, round to nearest, via
//         div6_rn), so results are bit-identical to a plain CPU loop.
//   FP32: the sum is multiplied by RN_f32(1/6) (one multiplication and five
//         additions, the count of Sect. 2.3).
#pragma once

namespace jac {

// Correctly rounded s / 6 in binary64 (round to nearest even), computed on
// the integer pipe.  For a finite normal s = +-M * 2^(E-1075), M = 2^52 +
// mantissa, the quotient is (M/3) * 2^(E-1076).  Its 53-bit significand is
// N = RN(K*M/3) with K = 2 when M >= 3*2^51 (then K*M/3 lies in
// [2^52, 2^52.42)) and K = 4 otherwise (K*M/3 in [2^52.42, 2^53 - 4/3]);
// the result is N * 2^(E-1077) or N * 2^(E-1078), i.e. biased exponent
// E-2 or E-3.  X/3 for an integer X has remainder 0, 1 or 2, so it is never
// halfway between integers and RN(X/3) = floor((X + 1)/3): no tie rule is
// needed.  floor(Y/3) for 64-bit Y is the high half of Y * 0xAAAA...AAB
// shifted right by one (division by an invariant integer through a
// multiplication, Granlund and Montgomery, PLDI 1994).  Zero returns
// itself; subnormal and tiny sums (E < 4, whose quotient may be subnormal),
// infinities and NaNs take the IEEE division instead.  Exhaustively structured tests compare
// this with __ddiv_rn (jacobi_check_division).
__device__ __forceinline__ double div6_rn(double s)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(s);
    const unsigned E = (unsigned)(b >> 52) & 0x7FFu;
    if (E - 4u > 2042u) return ((b << 1) == 0ull) ? s : __ddiv_rn(s, 6.0);  // +-0 / 6 = +-0
    const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    const unsigned small = (M < 0x18000000000000ull) ? 1u : 0u;  // M < 3 * 2^51
    const unsigned long long X = (M << (1u + small)) + 1ull;
    const unsigned long long N = __umul64hi(X, 0xAAAAAAAAAAAAAAABull) >> 1;
    const unsigned long long r =
        (b & 0x8000000000000000ull) | ((((unsigned long long)(E - 3u - small)) << 52) + N);
    return __longlong_as_double((long long)r);
}

// x + y in binary64, round to nearest even, on the FP64 pipe.
__device__ __forceinline__ double add_rn(double x, double y) { return __dadd_rn(x, y); }

// x + y in binary64, round to nearest even, computed on the integer pipe
// (the FP64 pipe of this GPU retires at most 2 additions per SM per clock,
// so part of the additions of a sweep can run here instead).  Fast path: both
// operands finite and normal with biased exponent <= 2045, same sign; the
// magnitudes are added (no cancellation) and rounded once:
//   with |a| >= |b|, d = e_a - e_b: if d >= 54 then |b| < ulp(a)/2 and the
//   result is a.  Otherwise the 53-bit significands are placed at bits
//   62..10 of 64-bit words, b's shifted right by d with every bit shifted
//   out kept as a sticky bit, the two added (< 2^64); a carry into bit 63
//   shifts the sum right once (sticky kept) and raises the exponent; the
//   low 10 bits then decide the round to nearest, ties to the even
//   significand; a significand that rounds up to 2^53 carries into the
//   exponent through the final addition of the exponent field.
// Every other case (a zero, subnormal, huge, infinite or NaN operand, or
// operands of opposite sign) uses the FP64 addition.  Checked bit for bit
// against __dadd_rn by jacobi_check_addition.
__device__ __forceinline__ double add_rn_int(double x, double y)
{
    const unsigned long long a0 = (unsigned long long)__double_as_longlong(x);
    const unsigned long long b0 = (unsigned long long)__double_as_longlong(y);
    const unsigned ea0 = (unsigned)(a0 >> 52) & 0x7FFu, eb0 = (unsigned)(b0 >> 52) & 0x7FFu;
    if (((a0 ^ b0) >> 63) != 0ull || ea0 - 1u > 2044u || eb0 - 1u > 2044u) return __dadd_rn(x, y);
    const unsigned long long sign = a0 & 0x8000000000000000ull;
    unsigned long long ua = a0 & 0x7FFFFFFFFFFFFFFFull, ub = b0 & 0x7FFFFFFFFFFFFFFFull;
    if (ua < ub) {
        const unsigned long long t = ua;
        ua = ub;
        ub = t;
    }
    const unsigned ea = (unsigned)(ua >> 52), d = ea - (unsigned)(ub >> 52);
    if (d >= 54u) return __longlong_as_double((long long)(sign | ua));
    const unsigned long long ma = ((ua & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull) << 10;
    const unsigned long long mb = ((ub & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull) << 10;
    unsigned long long s = ma + ((mb >> d) | ((mb & ((1ull << d) - 1ull)) != 0ull ? 1ull : 0ull));
    unsigned e = ea;
    if (s >> 63) {
        s = (s >> 1) | (s & 1ull);
        e += 1u;
    }
    unsigned long long q = s >> 10;
    const unsigned r = (unsigned)s & 0x3FFu;
    q += (r > 0x200u || (r == 0x200u && (q & 1ull))) ? 1ull : 0ull;
    return __longlong_as_double((long long)(sign | ((((unsigned long long)(e - 1u)) << 52) + q)));
}

template <typename T>
struct Arith;

// Which of the additions of Eq. (1) (bit i = addition i+1, left to right)
// run on the integer pipe; the rest run on the FP64 pipe.  Both give the
// identical IEEE result, so the split only balances the two pipes.
#ifndef JACOBI_INT_ADDS
#define JACOBI_INT_ADDS 0x00u
#endif
template <unsigned I>
__device__ __forceinline__ double add_sel(double x, double y)
{
    return (JACOBI_INT_ADDS >> I) & 1u ? add_rn_int(x, y) : add_rn(x, y);
}

template <>
struct Arith<double> {
    static __device__ __forceinline__ double update(double w, double e, double s, double n, double b,
                                                    double t)
    {
        double a = add_sel<0>(w, e);
        a = add_sel<1>(a, s);
        a = add_sel<2>(a, n);
        a = add_sel<3>(a, b);
        a = add_sel<4>(a, t);
        return div6_rn(a);
    }
    // Jacobi for the Poisson problem: (neighbour sum + g) / 6, g = h^2 f.
    static __device__ __forceinline__ double update_rhs(double w, double e, double s, double n, double b,
                                                        double t, double g)
    {
        double a = add_rn(w, e);
        a = add_rn(a, s);
        a = add_rn(a, n);
        a = add_rn(a, b);
        a = add_rn(a, t);
        a = add_rn(a, g);
        return div6_rn(a);
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
    static __device__ __forceinline__ float update_rhs(float w, float e, float s, float n, float b, float t,
                                                       float g)
    {
        float a = __fadd_rn(w, e);
        a = __fadd_rn(a, s);
        a = __fadd_rn(a, n);
        a = __fadd_rn(a, b);
        a = __fadd_rn(a, t);
        a = __fadd_rn(a, g);
        return __fmul_rn(a, 1.0f / 6.0f);
    }
};

}  // namespace jac
