// The cell update of Eq. (1) in each precision.  Explicit round-to-nearest
// intrinsics keep the compiler from contracting or reassociating: the six
// neighbours are added left to right in the printed order (i-1, i+1, j-1,
// j+1, k-1, k+1).
//   FP64: the sum is divided by 6.0 (IEEE quotient, round to nearest, via
//         div6_rn), so results are bit-identical to a plain CPU loop.
//   FP32: the sum is multiplied by RN_f32(1/6) (one multiplication and five
//         additions, the count of Sect. 2.3).
#pragma once
#include <cstdint>

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
// so one of the five additions of a cell update can run here instead).
// Sets ok = false where this path does not apply; the caller then adds on
// the FP64 pipe.  It applies when both operands have the same sign, the
// larger magnitude is a normal number below 2^1023 (biased exponent
// 1..2045) and the smaller one is zero or normal with an exponent at most
// 31 below it.  With |a| >= |b|, d = e_a - e_b, and 53-bit significands
// M_a, M_b (hidden bit set), all in 32-bit words:
//   the exact sum is M_a + M_b / 2^d; M_b >> d is two funnel shifts and the
//   d bits shifted out form a 32-bit fraction F (left-aligned);
//   S = M_a + (M_b >> d) lies in [2^52, 2^54); c = S >> 53 is its carry;
//   the kept significand is S >> c, the guard bit the bit below it (bit 0
//   of S if c, else the top bit of F) and the sticky bit the OR of the bits
//   below the guard; round to nearest, ties to even, adds guard AND
//   (sticky OR lowest kept bit); the result is sign | ((e_a + c - 1) << 52)
//   plus the rounded significand, so a significand that rounds up to 2^53
//   carries into the exponent by the addition itself.
// A zero b gives a exactly (same sign).  Checked bit for bit against
// __dadd_rn by jacobi_check_addition.
__device__ __forceinline__ uint32_t shl_clamped(uint32_t v, uint32_t n)
{
    uint32_t r;  // PTX shl clamps shift counts above 32: 0 for n = 32
    asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(v), "r"(n));
    return r;
}

__device__ __forceinline__ double add_rn_int_path(double x, double y, bool &ok)
{
    // 32-bit words only: a sign mask on the 64-bit pattern of a computed
    // double would be turned into an FP64 absolute value by the compiler.
    const uint32_t xh = (uint32_t)__double2hiint(x), xl = (uint32_t)__double2loint(x);
    const uint32_t yh = (uint32_t)__double2hiint(y), yl = (uint32_t)__double2loint(y);
    const uint32_t mx = xh & 0x7FFFFFFFu, my = yh & 0x7FFFFFFFu;
    const bool sw = my > mx || (my == mx && yl > xl);
    const uint32_t ah = sw ? yh : xh, al = sw ? yl : xl, bh = sw ? xh : yh, bl = sw ? xl : yl;  // |A| >= |B|
    const uint32_t ea = (ah >> 20) & 0x7FFu, eb = (bh >> 20) & 0x7FFu, d = ea - eb;
    const bool bzero = ((bh & 0x7FFFFFFFu) | bl) == 0u;
    ok = ((ah ^ bh) >> 31) == 0u && ea - 1u < 2045u && (bzero || (eb != 0u && d < 32u));
    const uint32_t mah = (ah & 0xFFFFFu) | 0x100000u, mbh = (bh & 0xFFFFFu) | 0x100000u;
    const uint32_t dd = d & 31u;
    const uint32_t ql = __funnelshift_r(bl, mbh, dd), qh = mbh >> dd;
    const uint32_t F = shl_clamped(bl, 32u - dd);
    const unsigned long long S = (((unsigned long long)mah << 32) | al) + (((unsigned long long)qh << 32) | ql);
    const uint32_t sh = (uint32_t)(S >> 32), sl = (uint32_t)S;
    const uint32_t c = sh >> 21;
    const uint32_t Ml = __funnelshift_r(sl, sh, c), Mh = sh >> c;
    const uint32_t g = c ? (sl & 1u) : (F >> 31);
    const uint32_t sticky = (c ? F : (F << 1)) != 0u ? 1u : 0u;
    const uint32_t ru = g & (sticky | (Ml & 1u));
    const unsigned long long M = (((unsigned long long)Mh << 32) | Ml) + ru;
    const uint32_t rh = (uint32_t)(M >> 32) + ((ea + c - 1u) << 20) + (ah & 0x80000000u), rl = (uint32_t)M;
    return __hiloint2double((int)(bzero ? ah : rh), (int)(bzero ? al : rl));
}

// The same addition for one thread: the integer path, else the FP64 pipe.
__device__ __forceinline__ double add_rn_int(double x, double y)
{
    bool ok;
    const double r = add_rn_int_path(x, y, ok);
    return ok ? r : __dadd_rn(x, y);
}

// FP64-pipe addition kept out of line: inlined, the compiler computes it
// ahead of the branch that guards it.
static __device__ __noinline__ double add_rn_outlined(double x, double y) { return __dadd_rn(x, y); }

// In kernels: the integer path for every lane; the lanes it does not apply to
// add on the FP64 pipe behind a warp vote, so warps with no such lane never
// issue the FP64 instruction.
__device__ __forceinline__ double add_rn_int_warp(double x, double y)
{
    bool ok;
    double r = add_rn_int_path(x, y, ok);
    if (__any_sync(__activemask(), !ok)) {
        if (!ok) r = add_rn_outlined(x, y);
    }
    return r;
}

template <typename T>
struct Arith;

// Which of the additions of Eq. (1) (bit i = addition i+1, left to right)
// run on the integer pipe; the rest run on the FP64 pipe.  Both give the
// identical IEEE result, so the split only balances the two pipes.  The
// first and the last (0x11): measured on the 512^3 FP64 workload, no
// integer addition gives 104 GLUP/s (FP64 pipe 84 % busy, five additions
// per cell), one 130, two 139 (three FP64 additions left), three 101 (the
// integer ALU pipe then limits).
#ifndef JACOBI_INT_ADDS
#define JACOBI_INT_ADDS 0x11u
#endif
template <unsigned I>
__device__ __forceinline__ double add_sel(double x, double y)
{
    return (JACOBI_INT_ADDS >> I) & 1u ? add_rn_int_warp(x, y) : add_rn(x, y);
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
