// Outward-rounded interval arithmetic on the GPU, FP64 and FP32.
//
// Each interval operation returns [rd(exact minimum), ru(exact maximum)] of the operation
// over its operand intervals, using the directed-rounding intrinsics (__dadd_rd, __fmul_ru,
// __dsqrt_rd, ...), which are never contracted into FMAs.  Products and quotients pick
// the end points by sign cases; since rd/ru are monotone this equals the min/max over all
// four end-point products or quotients.
#pragma once
#include <cstdint>

#include "ipipe.cuh"

namespace apo {

template <typename T> struct IV { T lo, hi; };

// ---- directed scalar operations, overloaded on the precision ----
__device__ __forceinline__ double rd_add(double a, double b) { return __dadd_rd(a, b); }
__device__ __forceinline__ double ru_add(double a, double b) { return __dadd_ru(a, b); }
__device__ __forceinline__ double rd_sub(double a, double b) { return __dsub_rd(a, b); }
__device__ __forceinline__ double ru_sub(double a, double b) { return __dsub_ru(a, b); }
__device__ __forceinline__ double rd_mul(double a, double b) { return __dmul_rd(a, b); }
__device__ __forceinline__ double ru_mul(double a, double b) { return __dmul_ru(a, b); }
__device__ __forceinline__ double rd_div(double a, double b) { return ipipe::div_rd(a, b); }
__device__ __forceinline__ double ru_div(double a, double b) { return ipipe::div_ru(a, b); }
// quotient (above), square root and reciprocal: correctly rounded on the integer pipe
// (ipipe.cuh)
__device__ __forceinline__ double rd_rcp(double a) { return ipipe::rcp_rd(a); }
__device__ __forceinline__ double ru_rcp(double a) { return ipipe::rcp_ru(a); }
__device__ __forceinline__ double rd_sqrt(double a) { return ipipe::sqrt_rd(a); }
__device__ __forceinline__ double ru_sqrt(double a) { return ipipe::sqrt_ru(a); }

__device__ __forceinline__ float rd_add(float a, float b) { return __fadd_rd(a, b); }
__device__ __forceinline__ float ru_add(float a, float b) { return __fadd_ru(a, b); }
__device__ __forceinline__ float rd_sub(float a, float b) { return __fsub_rd(a, b); }
__device__ __forceinline__ float ru_sub(float a, float b) { return __fsub_ru(a, b); }
__device__ __forceinline__ float rd_mul(float a, float b) { return __fmul_rd(a, b); }
__device__ __forceinline__ float ru_mul(float a, float b) { return __fmul_ru(a, b); }
__device__ __forceinline__ float rd_div(float a, float b) { return __fdiv_rd(a, b); }
__device__ __forceinline__ float ru_div(float a, float b) { return __fdiv_ru(a, b); }
__device__ __forceinline__ float rd_rcp(float a) { return __frcp_rd(a); }
__device__ __forceinline__ float ru_rcp(float a) { return __frcp_ru(a); }
__device__ __forceinline__ float rd_sqrt(float a) { return __fsqrt_rd(a); }
__device__ __forceinline__ float ru_sqrt(float a) { return __fsqrt_ru(a); }

// ---- value tests and min / max ----
// FP64 comparisons would run on the (narrow) FP64 pipe; they are done on the integer pipe
// through the bit pattern instead (operands are never NaN here).  For x != NaN the signed
// 64-bit pattern b satisfies: x > 0 <=> b > 0, x <= 0 <=> b <= 0, and the sign bit is set
// for every x in (-inf, -0].  okey() maps doubles to signed integers in value order.
// Sign-case selection (nonneg_lo / nonpos_hi) may route an end point of -0 through the
// mixed-sign formula; every formula used is valid for the intervals it is chosen for, so
// the end points equal the min / max over the end-point products in every case.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ long long okey(double x) {
    long long b = dbits(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ long long okey_inv(long long k) {   // okey is an involution
    return k ^ ((k >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool gt0(double x) { return dbits(x) > 0; }
__device__ __forceinline__ bool le0(double x) { return dbits(x) <= 0; }
__device__ __forceinline__ bool lt0(double x) { return okey(x) < -1; }     // -0 has key -1
__device__ __forceinline__ bool ge0(double x) { return okey(x) >= -1; }
__device__ __forceinline__ bool nonneg_lo(double x) { return dbits(x) >= 0; }   // in [+0, inf]
__device__ __forceinline__ bool nonpos_hi(double x) { return dbits(x) < 0; }    // in [-inf, -0]
__device__ __forceinline__ bool le(double a, double b) { return okey(a) <= okey(b); }
__device__ __forceinline__ double mn(double a, double b) { return okey(a) < okey(b) ? a : b; }
__device__ __forceinline__ double mx(double a, double b) { return okey(a) > okey(b) ? a : b; }

__device__ __forceinline__ bool gt0(float x) { return x > 0.f; }
__device__ __forceinline__ bool le0(float x) { return x <= 0.f; }
__device__ __forceinline__ bool lt0(float x) { return x < 0.f; }
__device__ __forceinline__ bool ge0(float x) { return x >= 0.f; }
__device__ __forceinline__ bool nonneg_lo(float x) { return x >= 0.f; }
__device__ __forceinline__ bool nonpos_hi(float x) { return x <= 0.f; }
__device__ __forceinline__ bool le(float a, float b) { return a <= b; }
__device__ __forceinline__ float mn(float a, float b) { return a < b ? a : b; }
__device__ __forceinline__ float mx(float a, float b) { return a > b ? a : b; }

template <typename T> __device__ __forceinline__ IV<T> mk(T lo, T hi) { return IV<T>{lo, hi}; }
template <typename T> __device__ __forceinline__ IV<T> add(IV<T> a, IV<T> b) {
    return {rd_add(a.lo, b.lo), ru_add(a.hi, b.hi)};
}
template <typename T> __device__ __forceinline__ IV<T> sub(IV<T> a, IV<T> b) {
    return {rd_sub(a.lo, b.hi), ru_sub(a.hi, b.lo)};
}
template <typename T> __device__ __forceinline__ IV<T> neg(IV<T> a) { return {-a.hi, -a.lo}; }

template <typename T> __device__ __forceinline__ IV<T> mul(IV<T> a, IV<T> b) {
    if (nonneg_lo(a.lo)) {
        if (nonneg_lo(b.lo)) return {rd_mul(a.lo, b.lo), ru_mul(a.hi, b.hi)};
        if (nonpos_hi(b.hi)) return {rd_mul(a.hi, b.lo), ru_mul(a.lo, b.hi)};
        return {rd_mul(a.hi, b.lo), ru_mul(a.hi, b.hi)};
    }
    if (nonpos_hi(a.hi)) {
        if (nonneg_lo(b.lo)) return {rd_mul(a.lo, b.hi), ru_mul(a.hi, b.lo)};
        if (nonpos_hi(b.hi)) return {rd_mul(a.hi, b.hi), ru_mul(a.lo, b.lo)};
        return {rd_mul(a.lo, b.hi), ru_mul(a.lo, b.lo)};
    }
    if (nonneg_lo(b.lo)) return {rd_mul(a.lo, b.hi), ru_mul(a.hi, b.hi)};
    if (nonpos_hi(b.hi)) return {rd_mul(a.hi, b.lo), ru_mul(a.lo, b.lo)};
    return {mn(rd_mul(a.lo, b.hi), rd_mul(a.hi, b.lo)), mx(ru_mul(a.lo, b.lo), ru_mul(a.hi, b.hi))};
}

// a / b with 0 not in b
template <typename T> __device__ __forceinline__ IV<T> divi(IV<T> a, IV<T> b) {
    if (gt0(b.lo)) {
        T l = nonneg_lo(a.lo) ? rd_div(a.lo, b.hi) : rd_div(a.lo, b.lo);
        T h = nonneg_lo(a.hi) ? ru_div(a.hi, b.lo) : ru_div(a.hi, b.hi);
        return {l, h};
    }
    T l = nonneg_lo(a.hi) ? rd_div(a.hi, b.hi) : rd_div(a.hi, b.lo);
    T h = nonneg_lo(a.lo) ? ru_div(a.lo, b.lo) : ru_div(a.lo, b.hi);
    return {l, h};
}

// 1 / b with 0 not in b
template <typename T> __device__ __forceinline__ IV<T> recip(IV<T> b) {
    return {rd_rcp(b.hi), ru_rcp(b.lo)};
}

template <typename T> __device__ __forceinline__ IV<T> sqr(IV<T> a) {
    if (nonneg_lo(a.lo)) return {rd_mul(a.lo, a.lo), ru_mul(a.hi, a.hi)};
    if (nonpos_hi(a.hi)) return {rd_mul(a.hi, a.hi), ru_mul(a.lo, a.lo)};
    return {T(0), mx(ru_mul(a.lo, a.lo), ru_mul(a.hi, a.hi))};
}

// FP32: branch-free forms.  The extremes of a b over the box are at a = a.lo or a.hi, each
// times the end of b chosen by that a's sign: two products per end point with selects (no
// branches, less code than sign cases).  Values equal the min / max over all four
// end-point products.
template <> __device__ __forceinline__ IV<float> mul<float>(IV<float> a, IV<float> b) {
    float l = fminf(fminf(__fmul_rd(a.lo, b.lo), __fmul_rd(a.lo, b.hi)),
                    fminf(__fmul_rd(a.hi, b.lo), __fmul_rd(a.hi, b.hi)));
    float h = fmaxf(fmaxf(__fmul_ru(a.lo, b.lo), __fmul_ru(a.lo, b.hi)),
                    fmaxf(__fmul_ru(a.hi, b.lo), __fmul_ru(a.hi, b.hi)));
    return {l, h};
}
// Square from the magnitudes: the upper end is ru(m^2) with m = max(-a.lo, a.hi), the
// larger |end|; the lower end is rd(n^2) with n = max(0, a.lo, -a.hi), which is a.lo for
// a >= 0, -a.hi for a <= 0 and 0 when a straddles 0.  Rounding is monotone, so these are
// the three sign cases' end points; two products and three min / max in all (the FP32
// kernels are issue-bound).
template <> __device__ __forceinline__ IV<float> sqr<float>(IV<float> a) {
    const float m = fmaxf(-a.lo, a.hi);
    const float n = fmaxf(0.f, fmaxf(a.lo, -a.hi));
    return {__fmul_rd(n, n), __fmul_ru(m, m)};
}
template <> __device__ __forceinline__ IV<float> divi<float>(IV<float> a, IV<float> b) {
    // b > 0: lo from a.lo, hi from a.hi; b < 0: lo from a.hi, hi from a.lo.  Either way the
    // numerator's sign picks the divisor end: lo uses b.hi if the numerator is >= 0.
    const bool bp = b.lo > 0.f;
    const float nl = bp ? a.lo : a.hi, nh = bp ? a.hi : a.lo;
    const float dl = nl >= 0.f ? b.hi : b.lo;
    const float dh = nh >= 0.f ? b.lo : b.hi;
    return {__fdiv_rd(nl, dl), __fdiv_ru(nh, dh)};
}

// a * b for b >= 0 (b.lo >= 0, known from the program's structure): a b is increasing in
// a, so the ends are a.lo and a.hi, each times the end of b chosen by its sign.
template <typename T> __device__ __forceinline__ IV<T> mul_nn(IV<T> a, IV<T> b) {
    return {rd_mul(a.lo, nonneg_lo(a.lo) ? b.lo : b.hi), ru_mul(a.hi, nonneg_lo(a.hi) ? b.hi : b.lo)};
}
// a * b for b <= 0 (b.hi <= 0): a b is decreasing in a, so the ends are a.hi and a.lo, each
// times the end of b chosen by its sign.
template <typename T> __device__ __forceinline__ IV<T> mul_np(IV<T> a, IV<T> b) {
    return {rd_mul(a.hi, nonneg_lo(a.hi) ? b.lo : b.hi), ru_mul(a.lo, nonneg_lo(a.lo) ? b.hi : b.lo)};
}
// FP32 forms of the two above with min / max instead of sign tests and selects: for
// b >= 0 the lower end is the smaller of a.lo b.lo and a.lo b.hi, the upper end the larger
// of a.hi b.lo and a.hi b.hi (mirrored for b <= 0); the same values, one ALU instruction
// per end instead of two.
template <> __device__ __forceinline__ IV<float> mul_nn<float>(IV<float> a, IV<float> b) {
    return {fminf(__fmul_rd(a.lo, b.lo), __fmul_rd(a.lo, b.hi)),
            fmaxf(__fmul_ru(a.hi, b.lo), __fmul_ru(a.hi, b.hi))};
}
template <> __device__ __forceinline__ IV<float> mul_np<float>(IV<float> a, IV<float> b) {
    return {fminf(__fmul_rd(a.hi, b.lo), __fmul_rd(a.hi, b.hi)),
            fmaxf(__fmul_ru(a.lo, b.lo), __fmul_ru(a.lo, b.hi))};
}
// a * b for a >= 0 and b >= 0
template <typename T> __device__ __forceinline__ IV<T> mul_pp(IV<T> a, IV<T> b) {
    return {rd_mul(a.lo, b.lo), ru_mul(a.hi, b.hi)};
}

// square root, lower end clamped at 0 (caller guarantees hi >= 0)
template <typename T> __device__ __forceinline__ IV<T> sqrti(IV<T> a) {
    return {gt0(a.lo) ? rd_sqrt(a.lo) : T(0), ru_sqrt(a.hi)};
}

// exact scalings by powers of two
template <typename T> __device__ __forceinline__ IV<T> scale2(IV<T> a) { return {a.lo * T(2), a.hi * T(2)}; }
template <typename T> __device__ __forceinline__ IV<T> scale4(IV<T> a) { return {a.lo * T(4), a.hi * T(4)}; }
template <typename T> __device__ __forceinline__ IV<T> half(IV<T> a) { return {a.lo * T(0.5), a.hi * T(0.5)}; }
template <typename T> __device__ __forceinline__ IV<T> clamp1(IV<T> a) {
    return {mx(a.lo, T(-1)), mn(a.hi, T(1))};
}
template <typename T> __device__ __forceinline__ IV<T> hull(IV<T> a, IV<T> b) {
    return {mn(a.lo, b.lo), mx(a.hi, b.hi)};
}
template <typename T> __device__ __forceinline__ T mag(IV<T> a) { return mx(-a.lo, a.hi); }
template <typename T> __device__ __forceinline__ bool contains0(IV<T> a) {
    return le0(a.lo) && ge0(a.hi);
}
template <typename T> __device__ __forceinline__ IV<T> pm(T r) { return {-r, r}; }

// [rd(1/k), ru(1/k)] for an integer k > 0
template <typename T> __device__ __forceinline__ IV<T> inv_int(int k) {
    return {rd_rcp(T(k)), ru_rcp(T(k))};
}

}  // namespace apo
