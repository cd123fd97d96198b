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
    // Not a series constant: 1 applies the direction condition of the program (a hit votes
    // only where it can lie on the track's outgoing arc); set per call by the host.
    int outgoing;
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
    if (sizeof(T) == 8) {   // FP64: one copy of the reduction (its root and quotient are
                            // long integer-pipe sequences), less instruction fetch
#pragma unroll 1
        for (int i = 0; i < 2; i++) x = divi(x, add(one, sqrti(add(one, sqr(x)))));
    } else {
#pragma unroll
        for (int i = 0; i < 2; i++) x = divi(x, add(one, sqrti(add(one, sqr(x)))));
    }
    IV<T> y = sqr(x);
    IV<T> h = cst<T>(k, C_ATAN0 + 7);
#pragma unroll
    for (int j = 6; j >= 0; j--) h = sub(cst<T>(k, C_ATAN0 + j), mul_nn(h, y));   // y >= 0
    IV<T> a = mul(x, h);
    T rem = ru_mul(ru_pow17(mag(x)), cst<T>(k, C_ATAN0 + 8).hi);
    a = add(a, pm(rem));
    return scale4(a);
}

// sin and cos over an interval d with |d| <= 1 (d is the small stereo correction of the
// phase): sin d = d (1 - d^2/6) + [-1, 1] |d|^5/5!, cos d = 1 - d^2/2 + [-1, 1] |d|^4/4!
// (Taylor with Lagrange remainders); [-1, 1] when |d| > 1.  Returns whether |d| <= 1, in
// which case c >= 1 - 1/2 - 1/24 > 0.
template <typename T>
__device__ __forceinline__ bool sincos_iv(IV<T> d, IV<T> &s, IV<T> &c, const SeriesConsts &k) {
    const IV<T> one{T(1), T(1)};
    T m = mag(d);
    if (!le(m, T(1))) { s = {T(-1), T(1)}; c = {T(-1), T(1)}; return false; }
    IV<T> y = sqr(d);
    IV<T> S = sub(one, mul_pp(y, cst<T>(k, C_SIN3)));
    T m2 = ru_mul(m, m), m4 = ru_mul(m2, m2);
    IV<T> sv = add(mul_nn(d, S), pm(ru_mul(ru_mul(m4, m), cst<T>(k, C_SIN5).hi)));
    IV<T> cv = add(sub(one, half(y)), pm(ru_mul(m4, cst<T>(k, C_COS4).hi)));
    s = clamp1(sv);
    c = clamp1(cv);
    return true;
}

// Products use mul_nn (second operand >= 0) or mul_pp (both >= 0) where the program's
// structure guarantees the sign: rho > 0 after the mirror and its guard, 1/N > 0, squares,
// the drift d, Q, R, tan^2(tau), 1 - cos(2 Phi^Ax), 1 - d^2/6 for |d| <= 1.  They return
// the same end points as the general product.

// Everything of the program that does not depend on tan(lambda).
template <typename T> struct Pre {
    bool guard;                       // a divisor reached 0: the pair votes (sound)
    bool novote;                      // direction condition: the hit is upstream everywhere
    IV<T> G0, psi, N, Ninv, sPA, cPA, rsA, rcA, sin2, Nh, dW, psi_sPA, dW_cPA, inner_e,
          psi_cos2, onepN;
};

// c: a mirrored cell (W > 0); h: a mirrored hit when the cell was mirrored.
template <typename T>
__device__ __forceinline__ Pre<T> prefix(const Cell<T> &c, const Hit<T> &h, const SeriesConsts &k) {
    const IV<T> one{T(1), T(1)};
    Pre<T> p;
    p.guard = false;
    p.novote = false;
    // wire point in the reference plane z_ref = z0 (Eqs. EQSinter_d,e)
    IV<T> Xw = add(h.x0, mul(c.Z, h.spt));
    IV<T> Yw = sub(h.y0, mul(c.Z, h.cpt));
    // coordinates along the tangent / left normal of the helix at the POCA
    IV<T> wt = add(mul(Xw, c.C0), mul(Yw, c.S0));
    IV<T> wn = sub(mul(Yw, c.C0), mul(Xw, c.S0));
    // direction: the turning angle psi from the POCA to the hit has the sign of w_t (rho > 0);
    // a hit with w_t < 0 over the whole cell lies upstream of every helix in it
    if (k.outgoing && lt0(wt.hi)) { p.novote = true; return p; }
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

// Products and square of tan(lambda) L when the caller knows its sign: LS = 1 for L >= 0,
// -1 for L <= 0, 0 when unknown.  Each returns the same end points as the general form.
template <int LS, typename T> __device__ __forceinline__ IV<T> lmul(IV<T> a, IV<T> L) {
    if (LS > 0) return mul_nn(a, L);
    if (LS < 0) return mul_np(a, L);
    return mul(L, a);
}
template <int LS, typename T> __device__ __forceinline__ IV<T> lsqr(IV<T> L) {
    if (LS > 0) return mul_pp(L, L);
    if (LS < 0) return {rd_mul(L.hi, L.hi), ru_mul(L.lo, L.lo)};
    return sqr(L);
}
// a b when both signs are known (SA, SB = 1 for >= 0, -1 for <= 0): one product per end
// point, the one the sign cases of the general product pick.
template <int SA, int SB, typename T> __device__ __forceinline__ IV<T> mul_ss(IV<T> a, IV<T> b) {
    static_assert(SA != 0 && SB != 0, "signs must be known");
    if (SA > 0 && SB > 0) return {rd_mul(a.lo, b.lo), ru_mul(a.hi, b.hi)};
    if (SA > 0 && SB < 0) return {rd_mul(a.hi, b.lo), ru_mul(a.lo, b.hi)};
    if (SA < 0 && SB > 0) return {rd_mul(a.lo, b.hi), ru_mul(a.hi, b.lo)};
    return {rd_mul(a.hi, b.hi), ru_mul(a.lo, b.lo)};
}
// a t for the stereo tangent t of the hit's wire when its sign is known (TS as LS)
template <int TS, typename T> __device__ __forceinline__ IV<T> tmul(IV<T> a, IV<T> t) {
    if (TS > 0) return mul_nn(a, t);
    if (TS < 0) return mul_np(a, t);
    return mul(a, t);
}
// square of an interval whose sign is known (S as LS)
template <int S, typename T> __device__ __forceinline__ IV<T> sqr_s(IV<T> a) {
    if (S > 0) return {rd_mul(a.lo, a.lo), ru_mul(a.hi, a.hi)};
    if (S < 0) return {rd_mul(a.hi, a.hi), ru_mul(a.lo, a.lo)};
    return sqr(a);
}

// The tan(lambda)-dependent rest: Phi (ApproxPhi_a), u_d (normudi), z^St (EQSinter_c),
// c^tau and the radicand of Eq. (defdiAX_b); returns the vote (either drift sign).  LS: the
// sign of L when the caller knows it (see lmul); TS: that of the wire's stereo tangent h.t
// (see tmul), which needs LS known too.  OUT: also store the evaluated intervals in ends
// (see vote_pair_ends); the voting kernels use OUT = false.
//
// Sign-known forms give the same end points as the general ones, so every instantiation
// returns the same vote.  The program is also unchanged, bit for bit, under the reflection
// z -> -z of the cell and the wire ((L, t) -> (-L, -t); z^St and c^tau change sign, every
// other quantity keeps its end points, because an interval product with both operands
// negated has the same four end-point products and one with a single operand negated is
// the exact negation): a caller may evaluate (-L, -t) in place of (L, t) to reach a known
// sign of L.
template <typename T, int LS = 0, bool OUT = false, int TS = 0>
__device__ __forceinline__ bool tail(const Pre<T> &p, IV<T> L, const Hit<T> &h, IV<T> R, IV<T> W,
                                     const SeriesConsts &k, double *ends = nullptr) {
    static_assert(TS == 0 || LS != 0, "a known sign of t needs a known sign of L");
    constexpr int LT = LS * TS;   // the sign of L t when both are known
    const IV<T> one{T(1), T(1)};
    IV<T> L2 = lsqr<LS>(L);
    IV<T> P1e = neg(mul_nn(lmul<LS>(p.psi_sPA, L), p.Ninv));
    IV<T> P1o = neg(mul_nn(lmul<LS>(p.dW_cPA, L), p.Ninv));
    IV<T> P2e = mul_nn(mul_nn(p.inner_e, L2), p.Nh);
    IV<T> P2o = mul_nn(mul_nn(add(scale2(mul_nn(p.psi_cos2, L2)), mul_nn(p.sin2, add(p.N, mul_pp(L2, p.onepN)))),
                              p.dW),
                       p.Nh);
    // delta = Phi - Phi^Ax, parts even / odd in the drift sign
    IV<T> de = add(tmul<TS>(P1e, h.t), mul_nn(P2e, h.t2));
    IV<T> dod = add(tmul<TS>(P1o, h.t), mul_nn(P2o, h.t2));
    IV<T> dP = add(de, dod);
    IV<T> dM = sub(de, dod);
    if (OUT) { ends[5] = dP.lo; ends[6] = dP.hi; ends[7] = dM.lo; ends[8] = dM.hi; }
    IV<T> sd, cd, sP, cP;
    const bool small = sincos_iv(hull(dP, dM), sd, cd, k);
    if (sizeof(T) == 4 && small) {   // FP32: cos(delta) > 0 (FP64 keeps its sign cases)
        sP = clamp1(add(mul_nn(p.sPA, cd), mul(p.cPA, sd)));
        cP = clamp1(sub(mul_nn(p.cPA, cd), mul(p.sPA, sd)));
    } else {
        sP = clamp1(add(mul(p.sPA, cd), mul(p.cPA, sd)));
        cP = clamp1(sub(mul(p.cPA, cd), mul(p.sPA, sd)));
    }
    // u_d^2 (Eq. normudi)
    IV<T> tLsP = TS != 0 ? tmul<TS>(lmul<LS>(sP, L), scale2(h.t)) : mul(scale2(h.t), lmul<LS>(sP, L));
    IV<T> u2 = add(add(add(one, tLsP), mul_pp(L2, h.t2)), mul_pp(sqr(cP), h.t2));
    if (le0(u2.lo)) {
        if (OUT) ends[4] = 1;
        return true;
    }
    IV<T> Q = mul_pp(h.d, recip(sqrti(u2)));
    IV<T> Qct = mul_nn(tmul<TS>(cP, h.t), Q);
    IV<T> LQ = LS > 0 ? mul_pp(L, Q) : mul_nn(L, Q);                  // Q >= 0
    IV<T> LQrsA = LS > 0 ? mul_nn(p.rsA, LQ) : LS < 0 ? mul_np(p.rsA, LQ) : mul(LQ, p.rsA);
    IV<T> a2 = mul_pp(W, sqr_s<1>(Q));
    IV<T> LQt;
    if constexpr (LT != 0) LQt = mul_ss<LS, TS>(LQ, h.t);
    else LQt = mul(LQ, h.t);
    IV<T> a5 = mul_pp(W, sqr_s<LT>(LQt));
    IV<T> t2x = scale2(h.t);
    bool vote = false;
#pragma unroll
    for (int sg = 0; sg < 2; sg++) {
        IV<T> dl = sg == 0 ? dP : dM;
        IV<T> sp = mul_nn(add(p.psi, dl), R);                                  // s_perp
        IV<T> zS = sg == 0 ? sub(lmul<LS>(sp, L), Qct) : add(lmul<LS>(sp, L), Qct);   // z^St - z_ref
        IV<T> rct = sg == 0 ? sub(mul(zS, p.rcA), LQrsA) : add(mul(zS, p.rcA), LQrsA);
        IV<T> a1 = sg == 0 ? scale2(Q) : neg(scale2(Q));
        IV<T> a3 = TS != 0 ? tmul<TS>(rct, t2x) : mul(t2x, rct);
        IV<T> a4 = mul_pp(W, sqr(tmul<TS>(zS, h.t)));
        IV<T> Arad = sub(sub(sub(add(a1, a2), a3), a4), a5);
        IV<T> G = sub(p.G0, Arad);
        if (OUT) { ends[2 * sg] = G.lo; ends[2 * sg + 1] = G.hi; }
        vote = vote || contains0(G);
    }
    return vote;
}

// Whole program for one (cell, hit), cell unmirrored, with the evaluated intervals in
// ends[9]: G+ lo / hi, G- lo / hi, a guard flag (1 when a divisor reached 0 and the pair
// votes unevaluated), then delta = Phi - Phi^Ax of the drift signs + and - (lo / hi each);
// zeros where the program stopped before computing them.  Used to compare end points
// with the oracle.
template <typename T>
__device__ __forceinline__ bool vote_pair_ends(Cell<T> c, Hit<T> h, const SeriesConsts &k, double *ends) {
    for (int i = 0; i < 9; i++) ends[i] = 0.0;
    if (mirror_cell(c)) mirror_hit(h);
    if (le0(c.W.lo)) { ends[4] = 1; return true; }
    IV<T> R = recip(c.W);
    Pre<T> p = prefix(c, h, k);
    if (p.novote) { ends[4] = 2; return false; }
    if (p.guard) { ends[4] = 1; return true; }
    return tail<T, 0, true>(p, c.L, h, R, c.W, k, ends);
}

// Whole program for one (cell, hit); the cell is given unmirrored.
template <typename T>
__device__ __forceinline__ bool vote_pair(Cell<T> c, Hit<T> h, const SeriesConsts &k) {
    if (mirror_cell(c)) mirror_hit(h);
    if (le0(c.W.lo)) return true;
    IV<T> R = recip(c.W);
    Pre<T> p = prefix(c, h, k);
    if (p.novote) return false;
    if (p.guard) return true;
    return tail(p, c.L, h, R, c.W, k);
}

// ---------------------------------------------------------------------------------------
// Exact phase, FP64 only: Eq. CSAXtoPHI_a solved for delta = Phi - Phi^Ax instead of its
// expansion.  In the frame of the program (times rho, N = rho R^Ax) delta solves
//   delta = g(delta) = atan( rho (rho s^tau) t / (N^2 + rho (rho c^tau) t) ),
//   rho c^tau = -lambda q rho s^Ax + z^St rho c^Ax,  rho s^tau = -lambda q rho c^Ax - z^St rho s^Ax,
// with q, u_d, z^St and s_perp = R (psi + delta) at that delta.  Per drift sign: X0 = the
// expansion's delta + [-2^-8, 2^-8]; if g(X0) lies in X0 every point of the cell has a
// solution in X0, and X <- g(X) meet X twice more keeps every solution; otherwise (or a
// zero divisor) the pair votes.  The rest of the program then uses delta = X per sign.
// ---------------------------------------------------------------------------------------
constexpr double kExactEps = 0.00390625;

__device__ __forceinline__ IV<double> exact_g(IV<double> dl, int sg, const Pre<double> &p, IV<double> R,
                                              IV<double> W, IV<double> N2, IV<double> L, IV<double> L2,
                                              const Hit<double> &h, const SeriesConsts &k, bool &ok) {
    const IV<double> one{1.0, 1.0};
    IV<double> sd, cd;
    sincos_iv(dl, sd, cd, k);
    const IV<double> sP = clamp1(add(mul(p.sPA, cd), mul(p.cPA, sd)));
    const IV<double> cP = clamp1(sub(mul(p.cPA, cd), mul(p.sPA, sd)));
    const IV<double> u2 = add(add(add(one, mul(scale2(h.t), mul(L, sP))), mul(L2, h.t2)), mul(sqr(cP), h.t2));
    if (le0(u2.lo)) { ok = false; return {-1.0, 1.0}; }
    const IV<double> Q = mul(h.d, recip(sqrti(u2)));
    const IV<double> Qct = mul(Q, mul(cP, h.t));
    const IV<double> LQ = mul(L, Q);
    const IV<double> sp = mul(add(p.psi, dl), R);
    const IV<double> zS = sg == 0 ? sub(mul(L, sp), Qct) : add(mul(L, sp), Qct);
    const IV<double> rct = sg == 0 ? sub(mul(zS, p.rcA), mul(LQ, p.rsA)) : add(mul(zS, p.rcA), mul(LQ, p.rsA));
    const IV<double> rst = sg == 0 ? sub(neg(mul(LQ, p.rcA)), mul(zS, p.rsA)) : sub(mul(LQ, p.rcA), mul(zS, p.rsA));
    const IV<double> den = add(N2, mul(mul(W, rct), h.t));
    if (le0(den.lo)) { ok = false; return {-1.0, 1.0}; }
    return atan_iv(divi(mul(mul(W, rst), h.t), den), k);
}

// The tan(lambda)-dependent rest with the exact phase; returns the vote.
__device__ __forceinline__ bool tail_exact(const Pre<double> &p, IV<double> L, const Hit<double> &h,
                                           IV<double> R, IV<double> W, const SeriesConsts &k) {
    const IV<double> one{1.0, 1.0};
    const IV<double> L2 = sqr(L);
    const IV<double> N2 = sqr(p.N);
    // the expansion's delta per sign (as in tail), the starting point
    const IV<double> P1e = neg(mul(mul(L, p.psi_sPA), p.Ninv));
    const IV<double> P1o = neg(mul(mul(L, p.dW_cPA), p.Ninv));
    const IV<double> P2e = mul(mul(L2, p.inner_e), p.Nh);
    const IV<double> P2o = mul(mul(p.dW, add(scale2(mul(L2, p.psi_cos2)), mul(add(p.N, mul(L2, p.onepN)), p.sin2))),
                               p.Nh);
    const IV<double> de = add(mul(P1e, h.t), mul(P2e, h.t2));
    const IV<double> dod = add(mul(P1o, h.t), mul(P2o, h.t2));
    bool vote = false;
#pragma unroll 1
    for (int sg = 0; sg < 2; sg++) {
        const IV<double> dl = sg == 0 ? add(de, dod) : sub(de, dod);
        IV<double> X = add(dl, IV<double>{-kExactEps, kExactEps});
        bool ok = true;
        const IV<double> Y = exact_g(X, sg, p, R, W, N2, L, L2, h, k, ok);
        if (!ok || !(Y.lo >= X.lo && Y.hi <= X.hi)) { vote = true; continue; }
        X = Y;
#pragma unroll 1
        for (int it = 0; it < 2 && ok; it++) {
            const IV<double> Z = exact_g(X, sg, p, R, W, N2, L, L2, h, k, ok);
            X = {X.lo > Z.lo ? X.lo : Z.lo, X.hi < Z.hi ? X.hi : Z.hi};
        }
        if (!ok || X.lo > X.hi) { vote = true; continue; }
        IV<double> sd, cd;
        sincos_iv(X, sd, cd, k);
        const IV<double> sP = clamp1(add(mul(p.sPA, cd), mul(p.cPA, sd)));
        const IV<double> cP = clamp1(sub(mul(p.cPA, cd), mul(p.sPA, sd)));
        const IV<double> u2 = add(add(add(one, mul(scale2(h.t), mul(L, sP))), mul(L2, h.t2)), mul(sqr(cP), h.t2));
        if (le0(u2.lo)) { vote = true; continue; }
        const IV<double> Q = mul(h.d, recip(sqrti(u2)));
        const IV<double> Qct = mul(Q, mul(cP, h.t));
        const IV<double> LQ = mul(L, Q);
        const IV<double> LQrsA = mul(LQ, p.rsA);
        const IV<double> a2 = mul(W, sqr(Q));
        const IV<double> a5 = mul(W, sqr(mul(LQ, h.t)));
        const IV<double> sp = mul(add(p.psi, X), R);
        const IV<double> zS = sg == 0 ? sub(mul(L, sp), Qct) : add(mul(L, sp), Qct);
        const IV<double> rct = sg == 0 ? sub(mul(zS, p.rcA), LQrsA) : add(mul(zS, p.rcA), LQrsA);
        const IV<double> a1 = sg == 0 ? scale2(Q) : neg(scale2(Q));
        const IV<double> a3 = mul(scale2(h.t), rct);
        const IV<double> a4 = mul(W, sqr(mul(zS, h.t)));
        const IV<double> Arad = sub(sub(sub(add(a1, a2), a3), a4), a5);
        const IV<double> G = sub(p.G0, Arad);
        vote = vote || contains0(G);
    }
    return vote;
}

// Whole exact-phase program for one (cell, hit); the cell is given unmirrored.
__device__ __forceinline__ bool vote_pair_exact(Cell<double> c, Hit<double> h, const SeriesConsts &k) {
    if (mirror_cell(c)) mirror_hit(h);
    if (le0(c.W.lo)) return true;
    const IV<double> R = recip(c.W);
    const Pre<double> p = prefix(c, h, k);
    if (p.novote) return false;
    if (p.guard) return true;
    return tail_exact(p, c.L, h, R, c.W, k);
}

// ---------------------------------------------------------------------------------------
// Midpoint form, FP64 only: the faster, approximate variant of Section 3.1, where the
// quantities that build d^Ax (Eq. defdiAX_b) are taken at the middle of the voxel.  The
// point part runs the steps of the interval program on the voxel centre, per drift sign,
// with plain round-to-nearest numbers, giving A = rho ((R + d^Ax)^2 - R^2) and
// d^Ax = A / (sqrt(1 + rho A) + 1); the interval part tests 0 in
// G = G0 - (2 d^Ax + rho d^Ax^2) with G0 = rho ((R^Ax)^2 - R^2) and rho over the voxel.
// Not sound: a voxel holding the solution can lose the vote.  A point divisor or root
// argument that is not positive makes the pair vote.  Every point step is an explicit
// round-to-nearest intrinsic, never contracted into an FMA.
// ---------------------------------------------------------------------------------------
namespace pt {
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double div(double a, double b) { return ipipe::div_rn(a, b); }
__device__ __forceinline__ double sqrt(double a) { return ipipe::sqrt_rn(a); }
__device__ __forceinline__ double clamp1(double x) { return x < -1.0 ? -1.0 : (x > 1.0 ? 1.0 : x); }
__device__ __forceinline__ double centre(IV<double> a) { return mul(add(a.lo, a.hi), 0.5); }

// atan with the steps of atan_iv and no remainder: two half-angle reductions, the
// alternating series through x^15 in Horner form on x^2, times 4.
__device__ __forceinline__ double atan(double x) {
#pragma unroll
    for (int i = 0; i < 2; i++) x = div(x, add(1.0, sqrt(add(1.0, mul(x, x)))));
    const double y = mul(x, x);
    double h = 1.0 / 15.0;
    h = sub(1.0 / 13.0, mul(h, y));
    h = sub(1.0 / 11.0, mul(h, y));
    h = sub(1.0 / 9.0, mul(h, y));
    h = sub(1.0 / 7.0, mul(h, y));
    h = sub(1.0 / 5.0, mul(h, y));
    h = sub(1.0 / 3.0, mul(h, y));
    h = sub(1.0, mul(h, y));
    return mul(mul(x, h), 4.0);
}

// sin / cos of the small phase correction: Taylor through d^9 / d^10 in nested Horner
// form on y = d^2 with round-to-nearest 1/k constants.
__device__ __forceinline__ void sincos(double d, double &s, double &c) {
    const double y = mul(d, d);
    double ps = sub(1.0, mul(y, 1.0 / 72.0));
    ps = sub(1.0, mul(mul(y, 1.0 / 42.0), ps));
    ps = sub(1.0, mul(mul(y, 1.0 / 20.0), ps));
    ps = sub(1.0, mul(mul(y, 1.0 / 6.0), ps));
    s = mul(d, ps);
    double pc = sub(1.0, mul(y, 1.0 / 90.0));
    pc = sub(1.0, mul(mul(y, 1.0 / 56.0), pc));
    pc = sub(1.0, mul(mul(y, 1.0 / 30.0), pc));
    pc = sub(1.0, mul(mul(y, 1.0 / 12.0), pc));
    c = sub(1.0, mul(mul(y, 0.5), pc));
}
}  // namespace pt

// Voxel centre (after the mirror): d0, sin / cos phi0, omega, z0 (tan(lambda) per tail).
struct MidCentre { double D, S0, C0, W, Z; };

// tan(lambda)-free part: point quantities at the centre and the interval G0 over the voxel.
struct MidPre {
    bool guard;   // a point divisor reached 0: both drift signs vote
    IV<double> G0;
    double R, W, psi, N, Ninv, sPA, cPA, rsA, rcA, sin2, Nh, dW, psi_sPA, dW_cPA, inner_e,
        psi_cos2, onepN;
};

// c: the mirrored voxel (W > 0); m: its mirrored centre; h: the (mirrored) hit.
__device__ __forceinline__ MidPre mid_prefix(const Cell<double> &c, const MidCentre &m,
                                             const Hit<double> &h) {
    using namespace pt;
    const IV<double> one{1.0, 1.0};
    MidPre p;
    p.guard = false;
    // interval part: G0 = rho ((R^Ax)^2 - R^2) over the voxel
    {
        IV<double> Xw = apo::add(h.x0, apo::mul(c.Z, h.spt));
        IV<double> Yw = apo::sub(h.y0, apo::mul(c.Z, h.cpt));
        IV<double> wt = apo::add(apo::mul(Xw, c.C0), apo::mul(Yw, c.S0));
        IV<double> wn = apo::sub(apo::mul(Yw, c.C0), apo::mul(Xw, c.S0));
        IV<double> V = apo::sub(wn, c.D);
        IV<double> Xn = apo::sub(mul_nn(V, c.W), one);
        p.G0 = apo::add(mul_pp(c.W, sqr(wt)), apo::mul(V, apo::sub(Xn, one)));
    }
    // point part at the centre
    const double x0 = h.x0.lo, y0 = h.y0.lo, sph = h.sph.lo, cph = h.cph.lo, spt = h.spt.lo,
                 cpt = h.cpt.lo, d = h.d.lo;
    p.W = m.W;
    p.R = div(1.0, m.W);
    const double Xw = add(x0, mul(m.Z, spt));
    const double Yw = sub(y0, mul(m.Z, cpt));
    const double wt = add(mul(Xw, m.C0), mul(Yw, m.S0));
    const double wn = sub(mul(Yw, m.C0), mul(Xw, m.S0));
    const double V = sub(wn, m.D);
    const double Xt = mul(wt, m.W);
    const double Xn = sub(mul(V, m.W), 1.0);
    p.N = sqrt(add(mul(Xt, Xt), mul(Xn, Xn)));
    if (!(p.N > 0.0)) { p.guard = true; return p; }
    const double den = sub(p.N, Xn);
    if (!(den > 0.0)) { p.guard = true; return p; }
    p.psi = mul(2.0, pt::atan(div(Xt, den)));
    const double E1 = add(mul(m.C0, cph), mul(m.S0, sph));
    const double E2 = sub(mul(m.C0, sph), mul(m.S0, cph));
    p.rsA = add(mul(Xt, E1), mul(Xn, E2));
    p.rcA = sub(mul(Xt, E2), mul(Xn, E1));
    p.Ninv = div(1.0, p.N);
    p.sPA = clamp1(mul(p.rsA, p.Ninv));
    p.cPA = clamp1(mul(p.rcA, p.Ninv));
    const double cos2 = clamp1(sub(mul(p.cPA, p.cPA), mul(p.sPA, p.sPA)));
    p.sin2 = clamp1(mul(2.0, mul(p.sPA, p.cPA)));
    p.dW = mul(d, m.W);
    p.Nh = mul(0.5, mul(p.Ninv, p.Ninv));
    p.psi_sPA = mul(p.psi, p.sPA);
    p.dW_cPA = mul(p.cPA, p.dW);
    p.inner_e = sub(add(mul(p.psi, sub(1.0, cos2)), mul(p.sin2, mul(p.psi, p.psi))),
                    mul(p.sin2, mul(p.dW, p.dW)));
    p.psi_cos2 = mul(p.psi, cos2);
    p.onepN = add(1.0, p.N);
    return p;
}

// The vote at the centre's tan(lambda) L (either drift sign), W the voxel's interval.
__device__ __forceinline__ bool mid_tail(const MidPre &p, double L, const Hit<double> &h,
                                         IV<double> W) {
    using namespace pt;
    const double t = h.t.lo, t2 = h.t2.lo, d = h.d.lo;
    const double L2 = mul(L, L);
    const double P1e = -mul(mul(L, p.psi_sPA), p.Ninv);
    const double P1o = -mul(mul(L, p.dW_cPA), p.Ninv);
    const double P2e = mul(mul(p.inner_e, L2), p.Nh);
    const double P2o = mul(mul(add(mul(2.0, mul(p.psi_cos2, L2)), mul(p.sin2, add(p.N, mul(L2, p.onepN)))),
                               p.dW),
                           p.Nh);
    const double de = add(mul(P1e, t), mul(P2e, t2));
    const double dod = add(mul(P1o, t), mul(P2o, t2));
    const double t2x = mul(2.0, t);
    bool vote = false;
#pragma unroll
    for (int sg = 0; sg < 2; sg++) {
        const double dl = sg == 0 ? add(de, dod) : sub(de, dod);
        double sd, cd;
        pt::sincos(dl, sd, cd);
        const double sP = clamp1(add(mul(p.sPA, cd), mul(p.cPA, sd)));
        const double cP = clamp1(sub(mul(p.cPA, cd), mul(p.sPA, sd)));
        const double u2 = add(add(add(1.0, mul(t2x, mul(L, sP))), mul(L2, t2)), mul(mul(cP, cP), t2));
        if (!(u2 > 0.0)) { vote = true; continue; }
        const double Q = mul(d, div(1.0, sqrt(u2)));
        const double Qct = mul(mul(cP, t), Q);
        const double LQ = mul(L, Q);
        const double LQrsA = mul(LQ, p.rsA);
        const double a2 = mul(p.W, mul(Q, Q));
        const double LQt = mul(LQ, t);
        const double a5 = mul(p.W, mul(LQt, LQt));
        const double sp = mul(add(p.psi, dl), p.R);
        const double zS = sg == 0 ? sub(mul(L, sp), Qct) : add(mul(L, sp), Qct);
        const double rct = sg == 0 ? sub(mul(zS, p.rcA), LQrsA) : add(mul(zS, p.rcA), LQrsA);
        const double a1 = sg == 0 ? mul(2.0, Q) : -mul(2.0, Q);
        const double a3 = mul(t2x, rct);
        const double zSt = mul(zS, t);
        const double a4 = mul(p.W, mul(zSt, zSt));
        const double A = sub(sub(sub(add(a1, a2), a3), a4), a5);
        const double r = add(1.0, mul(p.W, A));
        if (!(r >= 0.0)) { vote = true; continue; }
        const double dax = div(A, add(sqrt(r), 1.0));
        const IV<double> x{dax, dax};
        const IV<double> G = apo::sub(p.G0, apo::add(scale2(x), mul_pp(W, sqr(x))));
        vote = vote || contains0(G);
    }
    return vote;
}

// Whole midpoint-form program for one (voxel, hit); voxel, centre and hit unmirrored.
// m.L-less centre plus L = tan(lambda) centre.
__device__ __forceinline__ bool mid_vote_pair(Cell<double> c, MidCentre m, double L, Hit<double> h) {
    if (mirror_cell(c)) {
        mirror_hit(h);
        m.D = -m.D; m.S0 = -m.S0; m.W = -m.W;
    }
    if (le0(c.W.lo)) return true;
    MidPre p = mid_prefix(c, m, h);
    if (p.guard) return true;
    return mid_tail(p, L, h, c.W);
}

}  // namespace apo
