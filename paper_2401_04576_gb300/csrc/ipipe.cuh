// Correctly rounded FP64 square root, reciprocal and division, directed (rd / ru) and to
// nearest, computed on the integer and FP32 pipes.
//
// On this GPU the FP64 pipe retires about two lanes per clock per SM, while the integer
// and FP32 pipes are tens of times wider.  The library's directed square root and
// reciprocal are sequences of FP64 fused multiply-adds and compares; in the interval vote
// programs, where every other operation is a single FP64 add or multiply, they took about
// a quarter of the FP64 pipe.  Here the same correctly rounded results come from integer
// arithmetic on the 53-bit significands:
//
//   reciprocal of x = m 2^(e-1075), m in [2^52, 2^53):  q = floor(2^105 / m),
//       rem = 2^105 - q m;  1/x = (q + rem/m) 2^(970-e);
//   square root of x:  M2 = m or 2m so that the exponent is even, N = M2 2^52,
//       S = floor(sqrt(N)),  r = N - S^2;  sqrt(x) = sqrt(N) 2^(k/2-26);
//   quotient a / b:  q = floor(ma 2^k / mb) with k = 52 or 53, rem = ma 2^k - q mb.
//
// q (resp. S) is a 53-bit integer, so rd is q with the exponent, ru adds one unit in the
// last place when rem (resp. r) is nonzero (a carry into the exponent field gives the next
// power of two, as it should), and rn adds one when 2 rem >= m (resp. r > S; ties cannot
// occur for either operation).  q and S are estimated from the FP32 hardware
// approximations (rcp / rsqrt .approx) refined by two Newton steps in 64-bit fixed point
// (Q62), then corrected by their exact remainders, which are computed modulo 2^64 (they
// are small).  The corrected remainder is checked to lie in its range ([0, m) resp.
// [0, 2S]); if it does not, or the argument or the result is outside the normal range,
// the library operation is used instead.  The result is therefore the correctly rounded
// one for every argument, whatever the accuracy of the FP32 approximations.
#pragma once
#include <cstdint>

namespace apo {
namespace ipipe {

typedef unsigned long long u64;
typedef long long s64;

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// y in (0.25, 2) as a Q62 fixed-point number (exact: y has 24 significant bits)
__device__ __forceinline__ u64 q62(float y) {
    const unsigned b = __float_as_uint(y);
    const u64 m = (u64)((b & 0x7fffffu) | 0x800000u);
    return m << (((b >> 23) & 0xffu) - 88u);   // 62 - 23 + (e - 127)
}

// R ~ 2^114 / m (1 / g in Q62, g = m / 2^52 in [1, 2)) for a 53-bit significand m, to a
// few units of 2^-62: the FP32 approximation and two Newton steps.
__device__ __forceinline__ u64 recip_q62(u64 m) {
    const float g = __uint_as_float(0x3f800000u | (unsigned)((m >> 29) & 0x7fffffu));
    u64 R = q62(rcp_approx(g));
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const s64 e = (s64)((1ull << 61) - __umul64hi(m << 11, R));   // (1 - g r) 2^61
        R += (u64)__mul64hi((s64)R, (s64)((u64)e << 3));               // r (1 - g r) 2^62
    }
    return R;
}

// Reciprocal of x > 0 with biased exponent in [1, 2044] (normal argument and result).
// Returns the bits of rd(1/x) and sets *inexact and *up (rn rounds up); *ok is false when
// x is outside that range or the check failed (then the outputs are meaningless).
__device__ __forceinline__ u64 rcp_core(double x, bool *inexact, bool *up, bool *ok) {
    const u64 b = (u64)__double_as_longlong(x);
    const unsigned eb = (unsigned)(b >> 52);             // sign bit set -> eb >= 2048
    const u64 frac = b & 0xfffffffffffffull;
    const u64 m = frac | (1ull << 52);
    u64 q = recip_q62(m) >> 9;
    s64 rem = -(s64)(q * m);                             // 2^105 - q m  (mod 2^64)
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const bool lo = rem < 0;
        q = lo ? q - 1 : q;
        rem = lo ? rem + (s64)m : rem;
    }
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const bool hi = rem >= (s64)m;
        q = hi ? q + 1 : q;
        rem = hi ? rem - (s64)m : rem;
    }
    *ok = (eb - 1u < 2044u) && rem >= 0 && rem < (s64)m;
    *inexact = rem != 0;
    *up = 2 * (u64)rem >= m;
    return ((u64)(2045u - eb) << 52) + q - (1ull << 52);
}

// Square root of x > 0 with biased exponent in [1, 2046]; outputs as rcp_core.
__device__ __forceinline__ u64 sqrt_core(double x, bool *inexact, bool *up, bool *ok) {
    const u64 b = (u64)__double_as_longlong(x);
    const unsigned ex = (unsigned)(b >> 52);
    const u64 frac = b & 0xfffffffffffffull;
    const unsigned odd = (ex & 1u) ^ 1u;                 // x = M 2^k, k = ex - 1075 odd
    const u64 M2 = (frac | (1ull << 52)) << odd;
    const float f = __uint_as_float(((127u + odd) << 23) | (unsigned)(frac >> 29));
    u64 Y = q62(rsqrt_approx(f));                        // ~ 2^62 / sqrt(M2 / 2^52)
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const u64 yy = __umul64hi(Y, Y);                                   // y^2 2^60
        const s64 e = (s64)((1ull << 58) - __umul64hi(M2 << 10, yy));      // (1 - f y^2) 2^58
        Y += (u64)__mul64hi((s64)Y, (s64)((u64)e << 5));                         // y (1 - f y^2) / 2
    }
    u64 S = __umul64hi(M2 << 10, Y) >> 8;
    s64 r = (s64)((M2 << 52) - S * S);                   // N - S^2  (mod 2^64)
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const bool lo = r < 0;
        S = lo ? S - 1 : S;
        r = lo ? r + (s64)(2 * S + 1) : r;
    }
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const bool hi = r > (s64)(2 * S);
        r = hi ? r - (s64)(2 * S + 1) : r;
        S = hi ? S + 1 : S;
    }
    *ok = (ex - 1u < 2046u) && r >= 0 && r <= (s64)(2 * S);
    *inexact = r != 0;
    *up = r > (s64)S;
    // exponent field 1049 + (k - odd) / 2 with k - odd even
    const unsigned ef = (unsigned)(1049 + (((int)ex - 1075 - (int)odd) >> 1));
    return ((u64)ef << 52) + S - (1ull << 52);
}

// Quotient a / b of normal (or zero) a and normal b whose quotient is normal: returns the
// bits of the magnitude rounded down, with *inexact, *up (rn rounds the magnitude up),
// *neg (sign of the quotient) and *ok as rcp_core.  With ma, mb the significands and
// k = 52 (ma >= mb) or 53, q = floor(ma 2^k / mb) has 53 bits.
__device__ __forceinline__ u64 div_core(double a, double b, bool *inexact, bool *up, bool *neg, bool *ok) {
    const u64 A = (u64)__double_as_longlong(a), B = (u64)__double_as_longlong(b);
    const unsigned ea = (unsigned)(A >> 52) & 0x7ffu, eb = (unsigned)(B >> 52) & 0x7ffu;
    const u64 ma = (A & 0xfffffffffffffull) | (1ull << 52);
    const u64 mb = (B & 0xfffffffffffffull) | (1ull << 52);
    const bool zero = (A << 1) == 0;                     // a = +-0: the quotient is a signed 0
    const unsigned small = ma < mb ? 1u : 0u;            // k = 52 + small
    u64 q = __umul64hi(ma << 11, recip_q62(mb)) >> (9u - small);
    s64 rem = (s64)((ma << (52u + small)) - q * mb);     // ma 2^k - q mb  (mod 2^64)
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const bool lo = rem < 0;
        q = lo ? q - 1 : q;
        rem = lo ? rem + (s64)mb : rem;
    }
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const bool hi = rem >= (s64)mb;
        q = hi ? q + 1 : q;
        rem = hi ? rem - (s64)mb : rem;
    }
    const int be = (int)ea - (int)eb + 1023 - (int)small;   // biased exponent of the quotient
    *neg = ((A ^ B) >> 63) != 0;
    *ok = (eb - 1u < 2046u) &&
          (zero || ((ea - 1u < 2046u) && be >= 1 && be <= 2046 && rem >= 0 && rem < (s64)mb));
    *inexact = !zero && rem != 0;
    *up = !zero && 2 * (u64)rem > mb;
    return zero ? 0ull : ((u64)be << 52) + q - (1ull << 52);
}

__device__ __forceinline__ double from_bits(u64 b) { return __longlong_as_double((s64)b); }

__device__ __forceinline__ double rcp_rd(double x) {
    bool inex, up, ok;
    const u64 r = rcp_core(x, &inex, &up, &ok);
    double v = from_bits(r);
    if (__builtin_expect(!ok, 0)) v = __drcp_rd(x);                  // outside the fast path
    return v;
}
__device__ __forceinline__ double rcp_ru(double x) {
    bool inex, up, ok;
    const u64 r = rcp_core(x, &inex, &up, &ok);
    double v = from_bits(r + inex);
    if (__builtin_expect(!ok, 0)) v = __drcp_ru(x);                  // outside the fast path
    return v;
}
__device__ __forceinline__ double rcp_rn(double x) {
    bool inex, up, ok;
    const u64 r = rcp_core(x, &inex, &up, &ok);
    double v = from_bits(r + up);
    if (__builtin_expect(!ok, 0)) v = __drcp_rn(x);                  // outside the fast path
    return v;
}
__device__ __forceinline__ double sqrt_rd(double x) {
    bool inex, up, ok;
    const u64 r = sqrt_core(x, &inex, &up, &ok);
    double v = from_bits(r);
    if (__builtin_expect(!ok, 0)) v = __dsqrt_rd(x);                  // outside the fast path
    return v;
}
__device__ __forceinline__ double sqrt_ru(double x) {
    bool inex, up, ok;
    const u64 r = sqrt_core(x, &inex, &up, &ok);
    double v = from_bits(r + inex);
    if (__builtin_expect(!ok, 0)) v = __dsqrt_ru(x);                  // outside the fast path
    return v;
}
__device__ __forceinline__ double sqrt_rn(double x) {
    bool inex, up, ok;
    const u64 r = sqrt_core(x, &inex, &up, &ok);
    double v = from_bits(r + up);
    if (__builtin_expect(!ok, 0)) v = __dsqrt_rn(x);                  // outside the fast path
    return v;
}
__device__ __forceinline__ double div_rd(double a, double b) {
    bool inex, up, neg, ok;
    const u64 r = div_core(a, b, &inex, &up, &neg, &ok);
    double v = from_bits(neg ? (r + inex) | (1ull << 63) : r);
    if (__builtin_expect(!ok, 0)) v = __ddiv_rd(a, b);                   // outside the fast path
    return v;
}
__device__ __forceinline__ double div_ru(double a, double b) {
    bool inex, up, neg, ok;
    const u64 r = div_core(a, b, &inex, &up, &neg, &ok);
    double v = from_bits(neg ? r | (1ull << 63) : r + inex);
    if (__builtin_expect(!ok, 0)) v = __ddiv_ru(a, b);                   // outside the fast path
    return v;
}
__device__ __forceinline__ double div_rn(double a, double b) {
    bool inex, up, neg, ok;
    const u64 r = div_core(a, b, &inex, &up, &neg, &ok);
    double v = from_bits((r + up) | (neg ? 1ull << 63 : 0ull));
    if (__builtin_expect(!ok, 0)) v = __ddiv_rn(a, b);                   // outside the fast path
    return v;
}

}  // namespace ipipe
}  // namespace apo
