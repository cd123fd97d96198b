"""Point (non-interval) evaluation of the paper's stereo drift-distance equations, in plain
float64 NumPy/libm, written in the paper's notation.

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg
use anything under oracle/.

This file is the independent reference against which the interval vote program is pinned:
it uses atan2/sin/cos from libm and the paper's variables (x_c, y_c, R, R_i^Ax, c_i^Ax,
s_i^Ax, Phi_i^Ax, ...) directly, not the rescaled track-frame form the interval program
evaluates.

Sections / equations cited are those of the paper (arXiv:2401.04576):
  HelixEq_a-d (Section 2.2), wirePar_a,b, defSignedDriftDist, normudi, EQSinter_a-e,
  defdiAX_a,b, CSAXtoPHI_a, defEQApo1 and ApproxPhi_a-d (Appendix A).
"""
from __future__ import annotations

import numpy as np


def helix_centre(d0, phi0, omega):
    """Centre (x_c, y_c) and signed R of the helix whose POCA to the origin is at signed
    distance d0 along (-sin phi0, cos phi0); Eq. (HelixEq_d) with (x_ref, y_ref) = 0."""
    R = 1.0 / omega
    return -(R + d0) * np.sin(phi0), (R + d0) * np.cos(phi0), R


def mirror(params, wire, d_st=0.0):
    """Exact reflection y -> -y of a helix (d0, phi0, omega, z0, tanl), a wire
    (x0, y0, sin phis, cos phis, tan tau) and a signed drift distance.  Maps a clockwise
    helix (omega < 0) to a counter-clockwise one, for which the appendix's angular formulas
    (R > 0) hold.  The reflected wire is the same line written with (sin phis, -cos phis)
    and the same tan tau; the drift-line direction D x T is a cross product, so the signed
    drift distance changes sign."""
    d0, phi0, omega, z0, tanl = params
    x0, y0, sphi, cphi, t = wire
    return (-d0, -phi0, -omega, z0, tanl), (x0, -y0, sphi, -cphi, t), -d_st


def wire_point(wire, z):
    """Eq. (wirePar_a,b) / (EQSinter_d,e): the stereo wire's point at height z."""
    x0, y0, sphi, cphi, t = wire
    return x0 + z * sphi * t, y0 - z * cphi * t


def u_norm(Phi, lam, t):
    """Eq. (normudi)."""
    return np.sqrt(1.0 + 2.0 * lam * np.sin(Phi) * t + lam * lam * t * t
                   + np.cos(Phi) ** 2 * t * t)


def ax_quantities(params, wire, z_ref):
    """R_i^Ax, c_i^Ax, s_i^Ax, phi_i^Ax, Phi_i^Ax of Eq. (defEQApo1) for R > 0."""
    d0, phi0, omega, z0, lam = params
    x0, y0, sphi, cphi, t = wire
    xc, yc, R = helix_centre(d0, phi0, omega)
    xa, ya = wire_point(wire, z_ref)
    RA = np.hypot(xa - xc, ya - yc)
    cA = -(xc - xa) * sphi + (yc - ya) * cphi
    sA = -(xc - xa) * cphi - (yc - ya) * sphi
    phiA = np.arctan2(xa - xc, yc - ya)
    phis = np.arctan2(sphi, cphi)
    return dict(xc=xc, yc=yc, R=R, xa=xa, ya=ya, RA=RA, cA=cA, sA=sA, phiA=phiA,
                PhiA=phiA - phis, phis=phis)


def F_given_phi(params, wire, d_st, Phi, s_perp, z_ref):
    """Left-hand side of Eq. (defdiAX_a) with d_i^Ax from Eq. (defdiAX_b), written as
    (x^Ax - x_c)^2 + (y^Ax - y_c)^2 - [radicand of defdiAX_b]; the helix phase at the
    closest point enters through Phi (Eq. normudi) and s_perp (Eq. EQSinter_c).
    Valid for either sign of R."""
    d0, phi0, omega, z0, lam = params
    x0, y0, sphi, cphi, t = wire
    xc, yc, R = helix_centre(d0, phi0, omega)
    xa, ya = wire_point(wire, z_ref)
    u = u_norm(Phi, lam, t)
    q = d_st / u
    zS = z0 + lam * s_perp - z_ref - q * np.cos(Phi) * t          # EQSinter_c
    cA = -(xc - xa) * sphi + (yc - ya) * cphi
    sA = -(xc - xa) * cphi - (yc - ya) * sphi
    c_tau = -lam * q * sA + zS * cA
    rad = (R + q) ** 2 - 2.0 * c_tau * t - (zS * t) ** 2 - (lam * q * t) ** 2
    return (xa - xc) ** 2 + (ya - yc) ** 2 - rad


def phi_approx(params, wire, d_st, z_ref):
    """Eq. (ApproxPhi_a-d): second-order expansion of Phi_i in tan(tau); R > 0.
    Returns (Phi, Phi1, Phi2, z^Ax, s_perp) with s_perp = (Phi + phi_s - phi0) / rho,
    phi^Ax - phi0 taken in (-pi, pi]."""
    d0, phi0, omega, z0, lam = params
    t = wire[4]
    a = ax_quantities(params, wire, z_ref)
    R, RA, PhiA = a["R"], a["RA"], a["PhiA"]
    psi = np.angle(np.exp(1j * (a["phiA"] - phi0)))
    zA = z0 - z_ref + lam * R * psi                                   # ApproxPhi_d
    Phi1 = -(zA * np.sin(PhiA) + lam * d_st * np.cos(PhiA)) / RA      # ApproxPhi_b
    Phi2 = (lam * R * zA - lam * zA * (R - 2.0 * d_st) * np.cos(2 * PhiA)
            + (zA * zA + d_st * (RA + lam * lam * (R + RA - d_st))) * np.sin(2 * PhiA)
            ) / (2.0 * RA * RA)                                       # ApproxPhi_c
    Phi = PhiA + Phi1 * t + Phi2 * t * t                              # ApproxPhi_a
    s_perp = (psi + Phi1 * t + Phi2 * t * t) * R
    return Phi, Phi1, Phi2, zA, s_perp


def phi_solve(params, wire, d_st, z_ref, iters=200):
    """Numerical solution of the angular equation, Eq. (CSAXtoPHI_a), by fixed-point
    iteration started at Phi^Ax; R > 0.  Returns (Phi, s_perp)."""
    d0, phi0, omega, z0, lam = params
    t = wire[4]
    a = ax_quantities(params, wire, z_ref)
    R, RA, cA, sA = a["R"], a["RA"], a["cA"], a["sA"]
    psi0 = np.angle(np.exp(1j * (a["phiA"] - phi0)))
    Phi = a["PhiA"]
    for _ in range(iters):
        s_perp = (Phi - a["PhiA"] + psi0) * R
        u = u_norm(Phi, lam, t)
        q = d_st / u
        zS = z0 + lam * s_perp - z_ref - q * np.cos(Phi) * t
        c_tau = -lam * q * sA + zS * cA
        s_tau = -lam * q * cA - zS * sA
        Phi = a["PhiA"] + np.arctan2(s_tau * t, RA * RA + c_tau * t)
    s_perp = (Phi - a["PhiA"] + psi0) * R
    return Phi, s_perp


def F_approx(params, wire, d_st, z_ref=None):
    """The vote function of Eq. (ApoVote) at a point: Eq. (defdiAX_a,b) with Phi from the
    second-order expansion (ApproxPhi) and z_ref = z0 by default.  Helices with omega < 0
    are reflected first (`mirror`); F is unchanged by the reflection."""
    if params[2] < 0:
        params, wire, d_st = mirror(params, wire, d_st)
    z_ref = params[3] if z_ref is None else z_ref
    Phi, _, _, _, s_perp = phi_approx(params, wire, d_st, z_ref)
    return F_given_phi(params, wire, d_st, Phi, s_perp, z_ref)
