// The midpoint-form vote of the paper's own 4-D search (Sections 3.1-3.3): voxels
// x_c x y_c x R x z0 with tan(lambda) fixed by the momentum, one accumulator per sign.
// Eq. ApoVote, 0 in (x^Ax - x_c)^2 + (y^Ax - y_c)^2 - (R + d^Ax)^2, keeps the voxel's
// intervals for x_c, y_c and R; d^Ax (Eq. defdiAX_b) is a point value at the voxel centre,
// from the printed Eqs. defEQApo1, ApproxPhi_a-d, normudi and EQSinter_c with the
// transverse reference plane z_ref = z0 (the wire point x^Ax(z0) of Eqs. EQSinter_d,e is on
// the interval side, over the voxel's z0; the point side uses it at the centre's z0, and
// z0 - z_ref = 0 in z^Ax and z^St) and psi = phi^Ax - phi0 taken along the track: every phase is measured counter-clockwise from the
// direction of the origin seen from the centre, in [0, 2 pi), and psi is the wire point's
// phase minus the reference point's.  Point steps round to nearest through explicit
// intrinsics (never fused), interval steps are directed; T = double or float.
#pragma once
#include "interval.cuh"

namespace apo {
namespace p4 {

__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double div(double a, double b) { return ipipe::div_rn(a, b); }
__device__ __forceinline__ double sqrt(double a) { return ipipe::sqrt_rn(a); }
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float sqrt(float a) { return __fsqrt_rn(a); }

// atan for |x| <= 1 (phase4 only asks for half angles up to pi/4): two half-angle
// reductions (|x| below tan(pi/16)), the alternating series through x^15 (Horner on x^2),
// times 4; no remainder term.  1/(2k+1) are round-to-nearest constants of T.
template <typename T> __device__ __forceinline__ T atan(T x) {
    if (sizeof(T) == 8) {   // FP64: one copy of the reduction (see atan_iv)
#pragma unroll 1
        for (int i = 0; i < 2; i++) x = div(x, add(T(1), sqrt(add(T(1), mul(x, x)))));
    } else {
#pragma unroll
        for (int i = 0; i < 2; i++) x = div(x, add(T(1), sqrt(add(T(1), mul(x, x)))));
    }
    const T y = mul(x, x);
    T h = T(1) / T(15);
    h = sub(T(1) / T(13), mul(h, y));
    h = sub(T(1) / T(11), mul(h, y));
    h = sub(T(1) / T(9), mul(h, y));
    h = sub(T(1) / T(7), mul(h, y));
    h = sub(T(1) / T(5), mul(h, y));
    h = sub(T(1) / T(3), mul(h, y));
    h = sub(T(1), mul(h, y));
    return mul(mul(x, h), T(4));
}

// sin / cos of the small phase correction: Taylor through d^9 / d^10, nested Horner on d^2.
template <typename T> __device__ __forceinline__ void sincos(T d, T &s, T &c) {
    const T y = mul(d, d);
    T ps = sub(T(1), mul(y, T(1) / T(72)));
    ps = sub(T(1), mul(mul(y, T(1) / T(42)), ps));
    ps = sub(T(1), mul(mul(y, T(1) / T(20)), ps));
    ps = sub(T(1), mul(mul(y, T(1) / T(6)), ps));
    s = mul(d, ps);
    T pc = sub(T(1), mul(y, T(1) / T(90)));
    pc = sub(T(1), mul(mul(y, T(1) / T(56)), pc));
    pc = sub(T(1), mul(mul(y, T(1) / T(30)), pc));
    pc = sub(T(1), mul(mul(y, T(1) / T(12)), pc));
    c = sub(T(1), mul(mul(y, T(0.5)), pc));
}

}  // namespace p4

// Voxel centre (x_c, y_c, R), |tan(lambda)| there, the direction of the origin seen from
// it and the reference point's phase.
template <typename T> struct Ctr4 { T xc, yc, R, aL, ox, oy, on, psi_ref; bool valid, guard; };

// Phase of the point (dx, dy) = |d| (cos, sin) from the centre, counter-clockwise from
// the direction (ox, oy) of norm on, in [0, 2 pi).  With r = on |d|, r sin = o x d, r cos =
// o . d: for cos >= 0 the angle is 2 atan(sin / (1 + cos)), otherwise +-pi - 2 atan(sin /
// (1 - cos)) (the complementary half angle), so neither denominator cancels.  dn = |d|,
// from the caller; bad when r = 0.
template <typename T>
__device__ __forceinline__ T phase4(T ox, T oy, T on, T dx, T dy, T dn, bool &bad) {
    using namespace p4;
    const T sn = sub(mul(ox, dy), mul(oy, dx));
    const T cs = add(mul(ox, dx), mul(oy, dy));
    const T r = mul(on, dn);
    if (!(r > T(0))) { bad = true; return T(0); }
    T ph;
    if (cs >= T(0)) ph = mul(T(2), p4::atan(div(sn, add(r, cs))));
    else ph = sub(sn < T(0) ? -T(3.141592653589793) : T(3.141592653589793), mul(T(2), p4::atan(div(sn, sub(r, cs)))));
    if (ph < T(0)) ph = add(ph, T(6.283185307179586));
    return ph;
}

// p_gev, b_t: momentum and field in T; (xr, yr): reference point.
template <typename T>
__device__ __forceinline__ Ctr4<T> centre4(T xc, T yc, T R, T p_gev, T b_t, T xr, T yr) {
    using namespace p4;
    Ctr4<T> m;
    m.xc = xc; m.yc = yc; m.R = R;
    const T pt = mul(mul(T(0.3), b_t), R);
    const T ratio = div(p_gev, pt);
    m.valid = ratio > T(1);
    m.aL = m.valid ? sqrt(sub(mul(ratio, ratio), T(1))) : T(0);
    m.ox = -xc;
    m.oy = -yc;
    m.on = sqrt(add(mul(m.ox, m.ox), mul(m.oy, m.oy)));
    m.guard = false;
    m.psi_ref = T(0);
    if (!(m.on > T(0))) m.guard = true;
    else {
        const T ex = sub(xr, xc), ey = sub(yr, yc);
        m.psi_ref = phase4<T>(m.ox, m.oy, m.on, ex, ey, sqrt(add(mul(ex, ex), mul(ey, ey))), m.guard);
    }
    return m;
}

// z0- and sign-free point quantities of one (voxel centre, hit).
template <typename T> struct Pre4 { bool guard; T R, RA, A2, sA, cA, sPA, cPA, cos2, sin2, psi, Rpsi; };

// Hit constants as point values of T: x0, y0, sin phi_s, cos phi_s, tan tau,
// sin phi_s tan tau, cos phi_s tan tau, tan^2 tau, d.
template <typename T> struct HitP { T x0, y0, sph, cph, t, spt, cpt, t2, d; };

// z0: the centre's z0, the reference plane of the wire point
template <typename T>
__device__ __forceinline__ Pre4<T> prefix4(const Ctr4<T> &m, T z0, const HitP<T> &h) {
    using namespace p4;
    Pre4<T> p;
    p.guard = false;
    p.R = m.R;
    const T xw = add(h.x0, mul(z0, h.spt)), yw = sub(h.y0, mul(z0, h.cpt));   // EQSinter_d,e
    const T dx = sub(xw, m.xc), dy = sub(yw, m.yc);
    p.A2 = add(mul(dx, dx), mul(dy, dy));
    p.RA = sqrt(p.A2);
    if (!(p.RA > T(0)) || m.guard) { p.guard = true; return p; }
    // c^Ax, s^Ax of Eq. defEQApo1
    p.cA = sub(mul(dx, h.sph), mul(dy, h.cph));
    p.sA = add(mul(dx, h.cph), mul(dy, h.sph));
    p.sPA = div(p.sA, p.RA);
    p.cPA = div(p.cA, p.RA);
    p.cos2 = div(sub(mul(p.cA, p.cA), mul(p.sA, p.sA)), p.A2);
    p.sin2 = div(mul(mul(T(2), p.sA), p.cA), p.A2);
    // psi: the wire point's phase minus the reference point's
    bool bad = false;
    const T ph = phase4<T>(m.ox, m.oy, m.on, dx, dy, p.RA, bad);
    if (bad) { p.guard = true; return p; }
    p.psi = sub(ph, m.psi_ref);
    p.Rpsi = mul(p.R, p.psi);
    return p;
}

// d^Ax for the drift signs + (dax[0]) and - (dax[1]); bit s of the result: guard of sign s.
template <typename T>
__device__ __forceinline__ int dax4(const Pre4<T> &p, T L, const HitP<T> &h, T dax[2]) {
    using namespace p4;
    const T R = p.R, RA = p.RA, t = h.t, t2 = h.t2;
    const T zA = mul(L, p.Rpsi);                                       // ApproxPhi_d, z_ref = z0
    int guard = 0;
#pragma unroll
    for (int sg = 0; sg < 2; sg++) {
        const T ds = sg == 0 ? h.d : -h.d;
        const T Phi1 = div(-add(mul(zA, p.sPA), mul(mul(L, ds), p.cPA)), RA);      // ApproxPhi_b
        const T Phi2 = div(add(sub(mul(mul(L, R), zA), mul(mul(mul(L, zA), sub(R, mul(T(2), ds))), p.cos2)),
                               mul(add(mul(zA, zA), mul(ds, add(RA, mul(mul(L, L), sub(add(R, RA), ds))))),
                                   p.sin2)),
                           mul(T(2), p.A2));                                        // ApproxPhi_c
        const T dl = add(mul(Phi1, t), mul(Phi2, t2));                             // ApproxPhi_a
        T sd, cd;
        p4::sincos(dl, sd, cd);
        const T sP = add(mul(p.sPA, cd), mul(p.cPA, sd));
        const T cP = sub(mul(p.cPA, cd), mul(p.sPA, sd));
        const T u2 = add(add(add(T(1), mul(mul(T(2), t), mul(L, sP))), mul(mul(L, L), t2)),
                         mul(mul(cP, cP), t2));                                     // normudi
        dax[sg] = T(0);
        if (!(u2 > T(0))) { guard |= 1 << sg; continue; }
        const T q = div(ds, sqrt(u2));
        const T sperp = mul(R, add(p.psi, dl));
        const T zS = sub(mul(L, sperp), mul(mul(q, cP), t));                        // EQSinter_c
        const T ctau = sub(mul(zS, p.cA), mul(mul(L, q), p.sA));
        const T Rq = add(R, q), zSt = mul(zS, t), Lqt = mul(mul(L, q), t);
        const T rad = sub(sub(sub(mul(Rq, Rq), mul(mul(T(2), ctau), t)), mul(zSt, zSt)), mul(Lqt, Lqt));
        if (!(rad >= T(0))) { guard |= 1 << sg; continue; }
        dax[sg] = sub(sqrt(rad), R);                                                // defdiAX_b
    }
    return guard;
}

// (x^Ax - X)^2 + (y^Ax - Y)^2, directed, with the wire point x^Ax = x0 + Z spt,
// y^Ax = y0 - Z cpt over the voxel's z0 interval Z (shared by both signs of tan(lambda)
// and both drift signs).
template <typename T> struct HitI { IV<T> x0, y0, spt, cpt; };

template <typename T>
__device__ __forceinline__ IV<T> a2_4(IV<T> X, IV<T> Y, IV<T> Z, const HitI<T> &w) {
    const IV<T> xw = add(w.x0, mul(Z, w.spt)), yw = sub(w.y0, mul(Z, w.cpt));
    return add(sqr(sub(xw, X)), sqr(sub(yw, Y)));
}

// 0 in A2 - (Rv + dax)^2
template <typename T> __device__ __forceinline__ bool test4(IV<T> A2, IV<T> Rv, T dax) {
    return contains0(sub(A2, sqr(add(Rv, IV<T>{dax, dax}))));
}

// Disk pre-filter, Eq. ApoVoteDisk: 0 in X^2 + Y^2 - (Rv + [-rd, rd])^2.
template <typename T>
__device__ __forceinline__ bool disk4(IV<T> X, IV<T> Y, IV<T> Rv, T rd) {
    const IV<T> G = sub(add(sqr(X), sqr(Y)), sqr(add(Rv, IV<T>{-rd, rd})));
    return contains0(G);
}

// The vote of one hit at one centre (prefix at its z0) and sign over the voxel (A2 of its
// x_c, y_c, z0 and the wire; Rv): either drift sign (a guard votes).
template <typename T>
__device__ __forceinline__ bool pair4(const Ctr4<T> &m, const Pre4<T> &pre, int sign, const HitP<T> &h,
                                      IV<T> A2, IV<T> Rv) {
    T dax[2];
    const int g = dax4(pre, sign > 0 ? m.aL : -m.aL, h, dax);
    if (g & 1) return true;
    if (test4(A2, Rv, dax[0])) return true;
    if (g & 2) return true;
    return test4(A2, Rv, dax[1]);
}

}  // namespace apo
