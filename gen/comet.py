"""COMET-like full-stereo drift chamber and electron tracks from the origin: the toy of the
paper's own performance study (Section 3.2), rebuilt from its description (detector
simulation only; none of the voting arithmetic is here).

The paper's toy: 20 sensitive layers, 4,986 wires, inner / outer radius about 496 / 837
mm, length about 1,536 mm, stereo angles of about 100 mrad, a uniform 1 T field along the
chamber axis; electrons of 105 MeV/c emitted isotropically from the origin (the middle of
the chamber axis) with the transverse momentum constrained so that the helix makes less
than one turn inside the chamber and reaches the first three layers; the drift distance is
the smallest wire-helix distance, at most 8 mm; 25-62 hits per track.

Readings (the paper gives no more detail):
  * layer radii evenly spaced from 0.496 to 0.837 m; wires per layer proportional to the
    radius, rounded, summing to 4,986; waist points evenly spaced in azimuth, projection
    angle phi_s = the wire's azimuth, stereo angle +0.1 / -0.1 rad alternating by layer;
  * electrons turn counter-clockwise seen from +z (omega > 0 in the helix convention of
    gen/chamber.py, d0 = z0 = 0 at the origin);
  * "less than one turn inside the chamber": 2 pi R |tan(lambda)| exceeds the chamber
    half length, so the helix leaves |z| <= L/2 before completing a turn; "reaches the
    first three layers": 2 R exceeds the third layer's radius;
  * drift distances are the true distances (the paper adds no smearing);
  * the paper's sample has 25-62 hits per track: tracks with fewer than 25 hits (the
    steepest ones, which leave the chamber soonest) are redrawn;
  * the simulated arc is one full turn; a wire gets one hit, at its global closest
    approach, when that distance is under 8 mm and under half a cell.
"""
from __future__ import annotations

import numpy as np

from . import chamber

N_LAYERS = 20
N_WIRES = 4986
R_INNER = 0.496
R_OUTER = 0.837
Z_HALF_LEN = 0.768
STEREO_RAD = 0.1
B_TESLA = 1.0
P_GEV = 0.105
MAX_DRIFT = 0.008


def make_wires() -> chamber.Wires:
    radii = R_INNER + np.arange(N_LAYERS) * ((R_OUTER - R_INNER) / (N_LAYERS - 1))
    n = np.round(N_WIRES * radii / radii.sum()).astype(int)
    n[-1] += N_WIRES - int(n.sum())
    layer, x0, y0, phis, tant, half = [], [], [], [], [], []
    for i in range(N_LAYERS):
        a = 2.0 * np.pi * np.arange(n[i]) / n[i]
        layer.append(np.full(n[i], i, np.int32))
        x0.append(radii[i] * np.cos(a))
        y0.append(radii[i] * np.sin(a))
        phis.append(a)
        tau = STEREO_RAD if i % 2 == 0 else -STEREO_RAD
        tant.append(np.full(n[i], np.tan(tau)))
        half.append(np.full(n[i], np.pi * radii[i] / n[i]))
    phis_a = np.concatenate(phis)
    tan_tau = np.concatenate(tant)
    s, c = np.sin(phis_a), np.cos(phis_a)
    return chamber.Wires(layer=np.concatenate(layer), x0=np.concatenate(x0),
                         y0=np.concatenate(y0), phis=phis_a, sin_phis=s, cos_phis=c,
                         tan_tau=tan_tau, sphi_t=s * tan_tau, cphi_t=c * tan_tau,
                         t2=tan_tau * tan_tau, half_cell=np.concatenate(half),
                         z_half_len=Z_HALF_LEN)


def pt_range():
    """Transverse momenta [GeV] allowed by the two constraints for p = 105 MeV/c."""
    r3 = R_INNER + 2 * ((R_OUTER - R_INNER) / (N_LAYERS - 1))
    pt_min = 0.3 * B_TESLA * (r3 / 2.0)
    # 2 pi R |tanl| > L/2 with R = pt / (0.3 B), tanl = sqrt(p^2 - pt^2) / pt:
    # 2 pi sqrt(p^2 - pt^2) / (0.3 B) > L/2
    pt_max = np.sqrt(P_GEV ** 2 - (Z_HALF_LEN * 0.3 * B_TESLA / (2 * np.pi)) ** 2)
    return pt_min, pt_max


def draw_electron(rng: np.random.Generator) -> chamber.Track:
    """Isotropic direction from the origin, kept when the transverse momentum is in
    pt_range()."""
    lo, hi = pt_range()
    while True:
        cos_t = rng.uniform(-1.0, 1.0)
        pt = P_GEV * np.sqrt(1.0 - cos_t * cos_t)
        if lo <= pt <= hi:
            break
    phi0 = rng.uniform(0.0, 2.0 * np.pi)
    tanl = P_GEV * cos_t / pt
    return chamber.Track(d0=0.0, phi0=phi0, omega=0.3 * B_TESLA / pt, z0=0.0, tanl=tanl)


def events(n_events: int, seed: int, w: chamber.Wires | None = None,
           min_hits: int = 25) -> chamber.Events:
    """n_events single-electron events (noiseless drifts); tracks with fewer than
    min_hits hits are redrawn (25: the lower end of the paper's 25-62)."""
    w = make_wires() if w is None else w
    rng = np.random.default_rng(seed)
    per, tracks, truths = [], [], []
    while len(per) < n_events:
        tr = draw_electron(rng)
        R = 1.0 / tr.omega
        hs = chamber.simulate_track(tr, w, None, s_max=2.0 * np.pi * R, max_drift=MAX_DRIFT,
                                    ns=601)
        if len(hs) < min_hits:
            continue
        hs.sort(key=lambda h: h.wire)
        per.append([(h.wire, h.drift) for h in hs])
        tracks.append([tr])
        truths.append(hs)
    return chamber._pack(per, tracks, truths)


def helix_centre(tr: chamber.Track):
    """(x_c, y_c, R) of a generated track (R > 0)."""
    R = 1.0 / tr.omega
    return -(R + tr.d0) * np.sin(tr.phi0), (R + tr.d0) * np.cos(tr.phi0), R


def z_at_point(tr: chamber.Track, x: float, y: float) -> float:
    """z of the helix where its phase around the centre equals that of (x, y), on the
    simulated arc (one turn from the origin)."""
    xc, yc, R = helix_centre(tr)
    ph = np.arctan2(x - xc, yc - y)          # phase with P = C + R (sin ph, -cos ph)
    s = ((ph - tr.phi0) % (2.0 * np.pi)) * R
    return tr.z0 + tr.tanl * s
