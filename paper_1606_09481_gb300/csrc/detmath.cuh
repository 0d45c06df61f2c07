// detmath.cuh -- deterministic FP64 elementary functions for the device.
//
// The edge predicate of the method (Eq. 3 with the threshold rule of Alg. 1) is
// catastrophically cancelling near the threshold, so the edge set depends on
// every bit of cosh r, sinh r, cos(dphi), cosh R and of the sampled r.  These
// functions are therefore defined as fixed sequences of separately rounded IEEE
// binary64 operations (round to nearest even) over exact constants, so that any
// conforming implementation produces the same bits:
//   exp   Cody-Waite reduction with a two-part ln 2, Taylor polynomial to degree
//         13 (Horner), exact scaling by 2^k.
//   log   x = m 2^e with m in [sqrt(1/2), sqrt(2)), ln m = 2 atanh(s),
//         s = (m-1)/(m+1), odd series to s^23, then e ln2 added in two parts.
//   cos   quadrant j = floor(2d/pi + 1/2), three-part pi/2 reduction, Taylor
//         polynomials of cos (to r^16) and sin (to r^17).
//   cosh  (e + 1/e)/2;  sinh: odd Taylor series to x^15 below 0.5, else (e - 1/e)/2.
// Every multiply/add/subtract/divide below is an explicit __d*_rn intrinsic, which
// the compiler never contracts into an FMA.  Coefficients are 1/j! and 2/(2j+1)
// as correctly rounded quotients, folded at compile time (j! is exact for j <= 18).
#pragma once
#include <cstdint>

namespace rhg {
namespace dm {

// exact binary64 constants of the definition
constexpr double kPi = 0x1.921fb54442d18p+1;
constexpr double kTwoPi = 0x1.921fb54442d18p+2;
constexpr double kInvLn2 = 0x1.71547652b82fep+0;
constexpr double kLn2Hi = 0x1.62e42fee00000p-1;
constexpr double kLn2Lo = 0x1.a39ef35793c76p-33;
constexpr double kTwoOverPi = 0x1.45f306dc9c883p-1;
constexpr double kPio2A = 0x1.921fb54400000p+0;
constexpr double kPio2B = 0x1.0b4611a600000p-34;
constexpr double kPio2C = 0x1.3198a2e037073p-69;
constexpr double kSqrtHalf = 0x1.6a09e667f3bcdp-1;

__host__ __device__ constexpr double factorial(int j)
{
    double f = 1.0;
    for (int i = 2; i <= j; ++i) f = f * static_cast<double>(i);
    return f;
}
__host__ __device__ constexpr double inv_factorial(int j) { return 1.0 / factorial(j); }
__host__ __device__ constexpr double signed_inv_factorial(int j, int sign_index)
{
    return (sign_index & 1) ? -inv_factorial(j) : inv_factorial(j);
}
__host__ __device__ constexpr double atanh_coef(int j) { return 2.0 / static_cast<double>(2 * j + 1); }

__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }

// 2^k for -1022 <= k <= 1023, built from its bit pattern
__device__ __forceinline__ double pow2i(int k)
{
    return __longlong_as_double(static_cast<long long>(k + 1023) << 52);
}

__device__ __forceinline__ double exp(double x)
{
    if (x != x) return x;
    if (x > 708.0) return __longlong_as_double(0x7ff0000000000000LL);
    if (x < -708.0) return 0.0;
    const double kf = floor(add(mul(x, kInvLn2), 0.5));
    const double t = sub(sub(x, mul(kf, kLn2Hi)), mul(kf, kLn2Lo));
    double p = inv_factorial(13);
#pragma unroll
    for (int j = 12; j >= 0; --j) p = add(mul(p, t), inv_factorial(j));
    return mul(p, pow2i(static_cast<int>(kf)));
}

// positive, finite, normal x (the path only takes logs of values >= 1)
__device__ __forceinline__ double log(double x)
{
    if (!(x > 0.0)) return x == 0.0 ? __longlong_as_double(0xfff0000000000000LL)
                                    : __longlong_as_double(0x7ff8000000000000LL);
    const long long bits = __double_as_longlong(x);
    const int biased = static_cast<int>((bits >> 52) & 0x7ff);
    if (biased == 0x7ff) return x;
    // frexp: x = m0 2^e0 with m0 in [0.5, 1)
    int e = biased - 1022;
    double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | (1022LL << 52));
    if (m < kSqrtHalf) {
        m = mul(m, 2.0);
        e -= 1;
    }
    const double s = div(sub(m, 1.0), add(m, 1.0));
    const double z = mul(s, s);
    double q = atanh_coef(11);
#pragma unroll
    for (int j = 10; j >= 1; --j) q = add(mul(q, z), atanh_coef(j));
    const double lnm = add(mul(s, 2.0), mul(mul(s, z), q));
    const double ed = static_cast<double>(e);
    return add(mul(ed, kLn2Hi), add(mul(ed, kLn2Lo), lnm));
}

// cos d for 0 <= d < 2pi + 1
__device__ __forceinline__ double cos(double d)
{
    const double jf = floor(add(mul(d, kTwoOverPi), 0.5));
    double r = sub(d, mul(jf, kPio2A));
    r = sub(r, mul(jf, kPio2B));
    r = sub(r, mul(jf, kPio2C));
    const double z = mul(r, r);
    const int quadrant = static_cast<int>(jf) & 3;
    if (quadrant & 1) {
        double s = signed_inv_factorial(17, 8);
#pragma unroll
        for (int j = 7; j >= 0; --j) s = add(mul(s, z), signed_inv_factorial(2 * j + 1, j));
        const double sn = mul(r, s);
        return quadrant == 1 ? -sn : sn;
    }
    double c = signed_inv_factorial(16, 8);
#pragma unroll
    for (int j = 7; j >= 0; --j) c = add(mul(c, z), signed_inv_factorial(2 * j, j));
    return quadrant == 0 ? c : -c;
}

__device__ __forceinline__ double cosh(double x)
{
    const double e = exp(x);
    return mul(add(e, div(1.0, e)), 0.5);
}

__device__ __forceinline__ double sinh(double x)
{
    if (x < 0.5) {
        const double z = mul(x, x);
        double q = inv_factorial(15);
#pragma unroll
        for (int j = 13; j >= 1; j -= 2) q = add(mul(q, z), inv_factorial(j));
        return mul(x, q);
    }
    const double e = exp(x);
    return mul(sub(e, div(1.0, e)), 0.5);
}

// asinh(y) for y >= 0 (dynamic model, Algorithm 2): log(y + sqrt(y*y + 1)).
__device__ __forceinline__ double asinh(double y)
{
    const double t = add(mul(y, y), 1.0);
    return log(add(y, __dsqrt_rn(t)));
}

}  // namespace dm
}  // namespace rhg
