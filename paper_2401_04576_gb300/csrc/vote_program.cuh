// The interval vote program of one (cell, hit) pair, Eq. (ApoVote) of arXiv:2401.04576,
// split for reuse: `prefix` holds everything that does not depend on tan(lambda), `tail`
// the rest.  The split only shares common sub-expressions: every interval operation and
// its operands are the same as in the unsplit program, so votes are bit-identical.
//
// The condition is 0 in the interval extension of G = rho F, where
//   F = (x^Ax - x_c)^2 + (y^Ax - y_c)^2 - (R + d^Ax)^2          (Eqs. ApoEQ3D, defdiAX_a,b)
// with the reference plane z_ref = z0, Phi from the second-order expansion
// (Eqs. ApproxPhi_a-d), and the whole expression written in the frame of the helix at
// its point of closest approach (POCA) to the origin, where the curvature rho = 1/R
// appears linearly (the paper's rule of few interval occurrences, Section 3.1).  Both
// drift signs are tried (Section 3.1); either passing gives one vote.
#pragma once
#include "interval.cuh"

namespace apo {

// Reciprocals of the series' integer divisors, [rd(1/k), ru(1/k)], computed on the device
// once per geometry (1/k for k = 1, 3, ..., 17 and 6, 120, 24; the last entries unused).
struct SeriesConsts {
    double d_lo[16], d_hi[16];
    float f_lo[16], f_hi[16];
};
enum { C_ATAN0 = 0 /* 1/(2k+1), k = 0..8 */, C_SIN3 = 9, C_SIN5 = 10, C_SIN7 = 11,
       C_COS4 = 12, C_COS6 = 13, C_REM9 = 14, C_REM8 = 15 };
__host__ __device__ inline int series_divisor(int i) {
    const int k[16] = {1, 3, 5, 7, 9, 11, 13, 15, 17, 6, 120, 5040, 24, 720, 362880, 40320};
    return k[i];
}

template <typename T> __device__ __forceinline__ IV<T> cst(const SeriesConsts &c, int i);
template <> __device__ __forceinline__ IV<double> cst<double>(const SeriesConsts &c, int i) {
    return {c.d_lo[i], c.d_hi[i]};
}
template <> __device__ __forceinline__ IV<float> cst<float>(const SeriesConsts &c, int i) {
    return {c.f_lo[i], c.f_hi[i]};
}

template <typename T> struct Cell { IV<T> D, S0, C0, W, Z, L; };
template <typename T> struct Hit { IV<T> x0, y0, sph, cph, t, spt, cpt, t2, d; };

// omega < 0: exact reflection y -> -y (d0, phi0, omega change sign; the wire keeps its line
// written with (sin phi_s, -cos phi_s)); afterwards omega > 0 and the R > 0 formulas of the
// paper's appendix apply.  The drift sign is tried both ways, so it needs no flip.
template <typename T> __device__ __forceinline__ bool mirror_cell(Cell<T> &c) {
    if (lt0(c.W.hi)) {
        c.D = neg(c.D); c.S0 = neg(c.S0); c.W = neg(c.W);
        return true;
    }
    return false;
}
template <typename T> __device__ __forceinline__ void mirror_hit(Hit<T> &h) {
    h.y0 = neg(h.y0); h.cph = neg(h.cph); h.cpt = neg(h.cpt);
}

// ru(m^17) for m >= 0 by repeated squaring: m^2, m^4, m^8, m^16, then m^16 m.
template <typename T> __device__ __forceinline__ T ru_pow17(T m) {
    T m2 = ru_mul(m, m), m4 = ru_mul(m2, m2), m8 = ru_mul(m4, m4), m16 = ru_mul(m8, m8);
    return ru_mul(m16, m);
}

// atan over an interval: two half-angle reductions atan(x) = 2 atan(x/(1 + sqrt(1 + x^2))),
// the alternating series through x^15 in Horner form on x^2, remainder |x|^17/17, times 4.
template <typename T> __device__ __forceinline__ IV<T> atan_iv(IV<T> x, const SeriesConsts &k) {
    const IV<T> one{T(1), T(1)};
#pragma unroll
    for (int i = 0; i < 2; i++) x = divi(x, add(one, sqrti(add(one, sqr(x)))));
    IV<T> y = sqr(x);
    IV<T> h = cst<T>(k, C_ATAN0 + 7);
#pragma unroll
    for (int j = 6; j >= 0; j--) h = sub(cst<T>(k, C_ATAN0 + j), mul_nn(h, y));   // y >= 0
    IV<T> a = mul(x, h);
    T rem = ru_mul(ru_pow17(mag(x)), cst<T>(k, C_ATAN0 + 8).hi);
    a = add(a, pm(rem));
    return {a.lo * T(4), a.hi * T(4)};
}

// sin and cos over an interval d with |d| <= 1 (d is the small stereo correction of the
// phase): sin d = d (1 - d^2/6) + [-1, 1] |d|^5/5!, cos d = 1 - d^2/2 + [-1, 1] |d|^4/4!
// (Taylor with Lagrange remainders); [-1, 1] when |d| > 1.
template <typename T>
__device__ __forceinline__ void sincos_iv(IV<T> d, IV<T> &s, IV<T> &c, const SeriesConsts &k) {
    const IV<T> one{T(1), T(1)};
    T m = mag(d);
    if (!le(m, T(1))) { s = {T(-1), T(1)}; c = {T(-1), T(1)}; return; }
    IV<T> y = sqr(d);
    IV<T> S = sub(one, mul_pp(y, cst<T>(k, C_SIN3)));
    T m2 = ru_mul(m, m), m4 = ru_mul(m2, m2);
    IV<T> sv = add(mul_nn(d, S), pm(ru_mul(ru_mul(m4, m), cst<T>(k, C_SIN5).hi)));
    IV<T> cv = add(sub(one, half(y)), pm(ru_mul(m4, cst<T>(k, C_COS4).hi)));
    s = clamp1(sv);
    c = clamp1(cv);
}

// Products use mul_nn (second operand >= 0) or mul_pp (both >= 0) where the program's
// structure guarantees the sign: rho > 0 after the mirror and its guard, 1/N > 0, squares,
// the drift d, Q, R, tan^2(tau), 1 - cos(2 Phi^Ax), 1 - d^2/6 for |d| <= 1.  They return
// the same end points as the general product.

// Everything of the program that does not depend on tan(lambda).
template <typename T> struct Pre {
    bool guard;                       // a divisor reached 0: the pair votes (sound)
    IV<T> G0, psi, N, Ninv, sPA, cPA, rsA, rcA, sin2, Nh, dW, psi_sPA, dW_cPA, inner_e,
          psi_cos2, onepN;
};

// c: a mirrored cell (W > 0); h: a mirrored hit when the cell was mirrored.
template <typename T>
__device__ __forceinline__ Pre<T> prefix(const Cell<T> &c, const Hit<T> &h, const SeriesConsts &k) {
    const IV<T> one{T(1), T(1)};
    Pre<T> p;
    p.guard = false;
    // wire point in the reference plane z_ref = z0 (Eqs. EQSinter_d,e)
    IV<T> Xw = add(h.x0, mul(c.Z, h.spt));
    IV<T> Yw = sub(h.y0, mul(c.Z, h.cpt));
    // coordinates along the tangent / left normal of the helix at the POCA
    IV<T> wt = add(mul(Xw, c.C0), mul(Yw, c.S0));
    IV<T> wn = sub(mul(Yw, c.C0), mul(Xw, c.S0));
    IV<T> V = sub(wn, c.D);
    // xi = rho (x^Ax - x_c, y^Ax - y_c); |xi| = rho R_i^Ax
    IV<T> Xt = mul_nn(wt, c.W);
    IV<T> Xn = sub(mul_nn(V, c.W), one);
    p.N = sqrti(add(sqr(Xt), sqr(Xn)));
    if (le0(p.N.lo)) { p.guard = true; return p; }
    // rho ((R_i^Ax)^2 - R^2)
    p.G0 = add(mul_pp(c.W, sqr(wt)), mul(V, sub(Xn, one)));
    // turning angle psi = phi_i^Ax - phi0 from tan(psi/2) = Xt / (N - Xn)
    IV<T> den = sub(p.N, Xn);
    if (le0(den.lo)) { p.guard = true; return p; }
    p.psi = scale2(atan_iv(divi(Xt, den), k));
    // rho s_i^Ax, rho c_i^Ax (Eq. defEQApo1)
    IV<T> E1 = add(mul(c.C0, h.cph), mul(c.S0, h.sph));
    IV<T> E2 = sub(mul(c.C0, h.sph), mul(c.S0, h.cph));
    p.rsA = add(mul(Xt, E1), mul(Xn, E2));
    p.rcA = sub(mul(Xt, E2), mul(Xn, E1));
    p.Ninv = recip(p.N);
    // sin / cos of Phi^Ax and of its double
    p.sPA = clamp1(mul_nn(p.rsA, p.Ninv));
    p.cPA = clamp1(mul_nn(p.rcA, p.Ninv));
    IV<T> cos2 = clamp1(sub(sqr(p.cPA), sqr(p.sPA)));
    p.sin2 = clamp1(scale2(mul(p.sPA, p.cPA)));
    // tan(lambda)-free factors of Eqs. (ApproxPhi_b,c), numerator and denominator divided
    // by R^2: Phi1 = -lambda (psi sin Phi^Ax + (d rho) cos Phi^Ax) / N and
    // Phi2 = [lambda^2 (psi (1 - cos 2Phi^Ax) + psi^2 sin 2Phi^Ax - (d rho)^2 sin 2Phi^Ax)
    //         + (d rho) (2 lambda^2 psi cos 2Phi^Ax + (N + lambda^2 (1 + N)) sin 2Phi^Ax)] / (2 N^2)
    p.dW = mul_pp(h.d, c.W);
    p.Nh = half(sqr(p.Ninv));
    p.psi_sPA = mul(p.psi, p.sPA);
    p.dW_cPA = mul_nn(p.cPA, p.dW);
    p.inner_e = sub(add(mul_nn(p.psi, sub(one, cos2)), mul_nn(p.sin2, sqr(p.psi))),
                    mul_nn(p.sin2, sqr(p.dW)));
    p.psi_cos2 = mul(p.psi, cos2);
    p.onepN = add(one, p.N);
    return p;
}

// The tan(lambda)-dependent rest: Phi (ApproxPhi_a), u_d (normudi), z^St (EQSinter_c),
// c^tau and the radicand of Eq. (defdiAX_b); returns the vote (either drift sign).
template <typename T>
__device__ __forceinline__ bool tail(const Pre<T> &p, IV<T> L, const Hit<T> &h, IV<T> R, IV<T> W,
                                     const SeriesConsts &k) {
    const IV<T> one{T(1), T(1)};
    IV<T> L2 = sqr(L);
    IV<T> P1e = neg(mul_nn(mul(L, p.psi_sPA), p.Ninv));
    IV<T> P1o = neg(mul_nn(mul(L, p.dW_cPA), p.Ninv));
    IV<T> P2e = mul_nn(mul_nn(p.inner_e, L2), p.Nh);
    IV<T> P2o = mul_nn(mul_nn(add(scale2(mul_nn(p.psi_cos2, L2)), mul_nn(p.sin2, add(p.N, mul_pp(L2, p.onepN)))),
                              p.dW),
                       p.Nh);
    // delta = Phi - Phi^Ax, parts even / odd in the drift sign
    IV<T> de = add(mul(P1e, h.t), mul_nn(P2e, h.t2));
    IV<T> dod = add(mul(P1o, h.t), mul_nn(P2o, h.t2));
    IV<T> dP = add(de, dod);
    IV<T> dM = sub(de, dod);
    IV<T> sd, cd;
    sincos_iv(hull(dP, dM), sd, cd, k);
    IV<T> sP = clamp1(add(mul(p.sPA, cd), mul(p.cPA, sd)));
    IV<T> cP = clamp1(sub(mul(p.cPA, cd), mul(p.sPA, sd)));
    // u_d^2 (Eq. normudi)
    IV<T> u2 = add(add(add(one, mul(scale2(h.t), mul(L, sP))), mul_pp(L2, h.t2)), mul_pp(sqr(cP), h.t2));
    if (le0(u2.lo)) return true;
    IV<T> Q = mul_pp(h.d, recip(sqrti(u2)));
    IV<T> Qct = mul_nn(mul(cP, h.t), Q);
    IV<T> LQ = mul_nn(L, Q);
    IV<T> LQrsA = mul(LQ, p.rsA);
    IV<T> a2 = mul_pp(W, sqr(Q));
    IV<T> a5 = mul_pp(W, sqr(mul(LQ, h.t)));
    IV<T> t2x = scale2(h.t);
    bool vote = false;
#pragma unroll
    for (int sg = 0; sg < 2; sg++) {
        IV<T> dl = sg == 0 ? dP : dM;
        IV<T> sp = mul_nn(add(p.psi, dl), R);                                  // s_perp
        IV<T> zS = sg == 0 ? sub(mul(L, sp), Qct) : add(mul(L, sp), Qct);   // z^St - z_ref
        IV<T> rct = sg == 0 ? sub(mul(zS, p.rcA), LQrsA) : add(mul(zS, p.rcA), LQrsA);
        IV<T> a1 = sg == 0 ? scale2(Q) : neg(scale2(Q));
        IV<T> a3 = mul(t2x, rct);
        IV<T> a4 = mul_pp(W, sqr(mul(zS, h.t)));
        IV<T> Arad = sub(sub(sub(add(a1, a2), a3), a4), a5);
        IV<T> G = sub(p.G0, Arad);
        vote = vote || contains0(G);
    }
    return vote;
}

// Whole program for one (cell, hit); the cell is given unmirrored.
template <typename T>
__device__ __forceinline__ bool vote_pair(Cell<T> c, Hit<T> h, const SeriesConsts &k) {
    if (mirror_cell(c)) mirror_hit(h);
    if (le0(c.W.lo)) return true;
    IV<T> R = recip(c.W);
    Pre<T> p = prefix(c, h, k);
    if (p.guard) return true;
    return tail(p, c.L, h, R, c.W, k);
}

}  // namespace apo
