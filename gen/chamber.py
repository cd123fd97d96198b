"""Seeded toy full-stereo cylindrical drift chamber (detector simulation only).

The paper evaluates its method on drift distances generated from helices crossing a
home-made full-stereo chamber (Section 3.2).  This module builds a chamber of the same kind
and produces events: a wire table, helix tracks drawn from fixed distributions, and for
every wire the smallest 3-D distance between the wire and the helix (the drift distance,
Section 3.2), smeared by the drift resolution.

It holds none of the voting arithmetic: it only simulates the detector.  The helix is
Eq. (HelixEq_a-d) and the stereo wire is Eq. (wirePar_a,b); the signed drift distance
follows Eq. (defSignedDriftDist) with the drift-line direction u_d = D x T (D the wire
direction, T the helix tangent), which is the sign convention under which Eqs.
(EQSinter_a-c) hold.

Conventions (metres, radians, GeV, tesla):
  * helix centre C = (-(R + d0) sin(phi0), (R + d0) cos(phi0)) with signed R = 1/omega,
    omega = q * 0.3 * B / pT; the point of closest approach (POCA) to the origin sits at
    signed distance d0 along the left normal (-sin(phi0), cos(phi0));
  * helix point at transverse arc length s >= 0:
      x = xc + R sin(omega s + phi0),  y = yc - R cos(omega s + phi0),  z = z0 + tanl * s;
  * only the outgoing arc 0 <= s < pi |R| is simulated;
  * wire j of layer i: waist point (r_i cos a, r_i sin a, 0), a = 2 pi j / n_i, projection
    angle phi_s = a, stereo angle +-0.1 rad alternating with the layer.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

B_TESLA = 1.0
N_LAYERS = 10
R_FIRST = 0.20
R_LAST = 0.70
Z_HALF_LEN = 0.75
STEREO_RAD = 0.1
SIGMA_DRIFT = 150e-6
HIT_CAP = 256


@dataclass
class Wires:
    """Structure-of-arrays wire table.  All products are rounded once here (host side) and
    then used as given by every consumer."""
    layer: np.ndarray       # int32
    x0: np.ndarray          # waist point (z = 0)
    y0: np.ndarray
    phis: np.ndarray        # projection angle phi_s
    sin_phis: np.ndarray
    cos_phis: np.ndarray
    tan_tau: np.ndarray     # tan of the stereo angle
    sphi_t: np.ndarray      # sin(phi_s) * tan(tau), rounded once
    cphi_t: np.ndarray      # cos(phi_s) * tan(tau), rounded once
    t2: np.ndarray          # tan(tau)^2, rounded once
    half_cell: np.ndarray   # pi r_i / n_i
    z_half_len: float = Z_HALF_LEN

    @property
    def n(self) -> int:
        return int(self.x0.shape[0])


def make_wires() -> Wires:
    """Ten all-stereo layers at radii 0.20..0.70 m, 64 + 8 i wires in layer i (1000 wires)."""
    layer, x0, y0, phis, tant, half = [], [], [], [], [], []
    for i in range(N_LAYERS):
        r = R_FIRST + i * ((R_LAST - R_FIRST) / (N_LAYERS - 1))
        n = 64 + 8 * i
        a = 2.0 * np.pi * np.arange(n) / n
        layer.append(np.full(n, i, np.int32))
        x0.append(r * np.cos(a))
        y0.append(r * np.sin(a))
        phis.append(a)
        tau = STEREO_RAD if i % 2 == 0 else -STEREO_RAD
        tant.append(np.full(n, np.tan(tau)))
        half.append(np.full(n, np.pi * r / n))
    phis_a = np.concatenate(phis)
    tan_tau = np.concatenate(tant)
    s, c = np.sin(phis_a), np.cos(phis_a)
    return Wires(layer=np.concatenate(layer), x0=np.concatenate(x0), y0=np.concatenate(y0),
                 phis=phis_a, sin_phis=s, cos_phis=c, tan_tau=tan_tau,
                 sphi_t=s * tan_tau, cphi_t=c * tan_tau, t2=tan_tau * tan_tau,
                 half_cell=np.concatenate(half))


@dataclass
class Track:
    d0: float
    phi0: float
    omega: float
    z0: float
    tanl: float

    @property
    def params(self) -> np.ndarray:
        return np.array([self.d0, self.phi0, self.omega, self.z0, self.tanl])


def draw_track(rng: np.random.Generator) -> Track:
    """pT ~ U[0.3, 2] GeV, random charge, phi0 ~ U[0, 2pi), d0 ~ U[-1, 1] cm,
    z0 ~ U[-10, 10] cm, tan(lambda) ~ U[-0.8, 0.8], B = 1 T."""
    pt = rng.uniform(0.3, 2.0)
    q = 1.0 if rng.random() < 0.5 else -1.0
    phi0 = rng.uniform(0.0, 2.0 * np.pi)
    d0 = rng.uniform(-0.01, 0.01)
    z0 = rng.uniform(-0.10, 0.10)
    tanl = rng.uniform(-0.8, 0.8)
    return Track(d0=d0, phi0=phi0, omega=q * 0.3 * B_TESLA / pt, z0=z0, tanl=tanl)


def _helix(tr: Track, s):
    R = 1.0 / tr.omega
    xc = -(R + tr.d0) * np.sin(tr.phi0)
    yc = (R + tr.d0) * np.cos(tr.phi0)
    ph = tr.omega * s + tr.phi0
    P = np.stack([xc + R * np.sin(ph), yc - R * np.cos(ph), tr.z0 + tr.tanl * s], axis=-1)
    T = np.stack([np.cos(ph), np.sin(ph), np.full_like(ph, tr.tanl)], axis=-1)
    Tp = np.stack([-tr.omega * np.sin(ph), tr.omega * np.cos(ph), np.zeros_like(ph)], axis=-1)
    return P, T, Tp


def _wire_dirs(w: Wires, idx):
    D = np.stack([w.sphi_t[idx], -w.cphi_t[idx], np.ones(len(idx))], axis=-1)
    W0 = np.stack([w.x0[idx], w.y0[idx], np.zeros(len(idx))], axis=-1)
    return W0, D


@dataclass
class Hit:
    wire: int
    drift: float        # measured, >= 0
    dist: float         # true closest distance
    d_signed: float     # signed drift distance d^St of Eq. (defSignedDriftDist)
    s: float            # transverse arc length of the helix point M
    z_wire: float       # z of the wire point M^St
    Phi: float          # omega s + phi0 - phi_s (helix phase at M minus wire angle)


def simulate_track(tr: Track, w: Wires, rng: np.random.Generator | None,
                   sigma: float = SIGMA_DRIFT, s_max: float | None = None,
                   max_drift: float | None = None, ns: int = 301) -> list[Hit]:
    """All wires whose closest approach to the helix (over the arc 0 <= s < s_max, by
    default the outgoing half turn, with the wire point inside the chamber length) is under
    half a cell (and under max_drift when given); drift = distance + N(0, sigma), clipped
    at 0.  rng=None gives noiseless drifts."""
    s_max = min(np.pi / abs(tr.omega), 1.5) if s_max is None else s_max
    s_grid = np.linspace(0.0, s_max, ns)
    P, _, _ = _helix(tr, s_grid)
    # A wire can only be hit if its waist point lies within half a cell plus its largest
    # transverse stereo shift (|z| <= z_half_len) of the helix's circle: the 3-D distance
    # is at least the transverse one.  The rest need no distance computation.
    R = 1.0 / tr.omega
    xc, yc = -(R + tr.d0) * np.sin(tr.phi0), (R + tr.d0) * np.cos(tr.phi0)
    d_circ = np.abs(np.hypot(w.x0 - xc, w.y0 - yc) - abs(R))
    near = np.nonzero(d_circ <= w.half_cell + w.z_half_len * np.abs(w.tan_tau) + 1e-3)[0]
    # squared distance of every sample to every remaining wire line
    W0 = np.stack([w.x0[near], w.y0[near], np.zeros(near.size)], axis=-1)
    D = np.stack([w.sphi_t[near], -w.cphi_t[near], np.ones(near.size)], axis=-1)
    D2 = 1.0 + w.t2[near]
    v = P[None, :, :] - W0[:, None, :]
    vd = np.einsum('wsk,wk->ws', v, D)
    dist2 = np.einsum('wsk,wsk->ws', v, v) - vd * vd / D2[:, None]
    kmin = np.argmin(dist2, axis=1)
    dmin = np.sqrt(np.maximum(dist2[np.arange(near.size), kmin], 0.0))
    step = s_grid[1] - s_grid[0]
    sel = np.nonzero(dmin < w.half_cell[near] + step)[0]
    cand = near[sel]
    kmin = kmin[sel]
    hits: list[Hit] = []
    if cand.size == 0:
        return hits
    k = kmin
    lo = s_grid[np.maximum(k - 1, 0)]
    hi = s_grid[np.minimum(k + 1, ns - 1)]
    W0c, Dc = _wire_dirs(w, cand)
    D2c = (1.0 + w.t2[cand])[:, None]

    def f(s):
        Ps, _, _ = _helix(tr, s)
        vv = Ps - W0c
        a = np.sum(vv * Dc, axis=-1)
        return np.sum(vv * vv, axis=-1) - a * a / D2c[:, 0]

    # golden-section bracket refinement, then Newton on the stationarity condition
    g = (np.sqrt(5.0) - 1.0) / 2.0
    a_, b_ = lo.copy(), hi.copy()
    c_ = b_ - g * (b_ - a_)
    d_ = a_ + g * (b_ - a_)
    fc, fd = f(c_), f(d_)
    for _ in range(24):
        left = fc < fd
        b_ = np.where(left, d_, b_)
        a_ = np.where(left, a_, c_)
        d_new = np.where(left, c_, a_ + g * (b_ - a_))
        c_new = np.where(left, b_ - g * (b_ - a_), d_)
        fd_new = np.where(left, fc, np.nan)
        fc_new = np.where(left, np.nan, fd)
        c_, d_ = c_new, d_new
        need_c = np.isnan(fc_new)
        need_d = np.isnan(fd_new)
        fc = np.where(need_c, f(c_), fc_new)
        fd = np.where(need_d, f(d_), fd_new)
    s = 0.5 * (a_ + b_)
    for _ in range(6):
        Ps, T, Tp = _helix(tr, s)
        vv = Ps - W0c
        a = np.sum(vv * Dc, axis=-1)
        zc = a / D2c[:, 0]
        M_st = W0c + zc[:, None] * Dc
        r = Ps - M_st
        gval = np.sum(r * T, axis=-1)
        Tperp = T - (np.sum(T * Dc, axis=-1) / D2c[:, 0])[:, None] * Dc
        gder = np.sum(Tperp * T, axis=-1) + np.sum(r * Tp, axis=-1)
        s = s - gval / gder
    Ps, T, _ = _helix(tr, s)
    vv = Ps - W0c
    zc = np.sum(vv * Dc, axis=-1) / D2c[:, 0]
    M_st = W0c + zc[:, None] * Dc
    r = Ps - M_st
    dist = np.sqrt(np.sum(r * r, axis=-1))
    u = np.cross(Dc, T)
    u /= np.linalg.norm(u, axis=-1)[:, None]
    dsg = np.sum(r * u, axis=-1)
    for j, wid in enumerate(cand):
        if not (0.0 < s[j] < s_max and lo[j] - step <= s[j] <= hi[j] + step):
            continue  # closest approach at the end of the arc: no perpendicular crossing
        if abs(zc[j]) > w.z_half_len or dist[j] >= w.half_cell[wid]:
            continue
        if max_drift is not None and dist[j] >= max_drift:
            continue
        drift = dist[j] if rng is None else max(dist[j] + rng.normal(0.0, sigma), 0.0)
        Phi = tr.omega * s[j] + tr.phi0 - w.phis[wid]
        hits.append(Hit(wire=int(wid), drift=float(drift), dist=float(dist[j]),
                        d_signed=float(dsg[j]), s=float(s[j]), z_wire=float(zc[j]),
                        Phi=float(Phi)))
    return hits


@dataclass
class Events:
    """CSR batch of events: hits of event e are offsets[e]:offsets[e+1]."""
    offsets: np.ndarray      # int32 [n_events + 1]
    wire_id: np.ndarray      # int32 [n_hits]
    drift: np.ndarray        # float64 [n_hits]
    tracks: list = field(default_factory=list)       # per event: list[Track]
    hit_truth: list = field(default_factory=list)    # per event: list[Hit | None] (None = noise)

    @property
    def n_events(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def n_hits(self, e: int) -> int:
        return int(self.offsets[e + 1] - self.offsets[e])

    def subset(self, idx) -> "Events":
        idx = list(idx)
        offs, wid, dr = [0], [], []
        for e in idx:
            a, b = self.offsets[e], self.offsets[e + 1]
            wid.append(self.wire_id[a:b])
            dr.append(self.drift[a:b])
            offs.append(offs[-1] + (b - a))
        return Events(offsets=np.asarray(offs, np.int32),
                      wire_id=np.concatenate(wid).astype(np.int32) if wid else np.zeros(0, np.int32),
                      drift=np.concatenate(dr) if dr else np.zeros(0),
                      tracks=[self.tracks[e] for e in idx] if self.tracks else [],
                      hit_truth=[self.hit_truth[e] for e in idx] if self.hit_truth else [])


def _pack(per_event_hits, tracks, truths) -> Events:
    offs = [0]
    wid, dr = [], []
    for hs in per_event_hits:
        wid.extend(h[0] for h in hs)
        dr.extend(h[1] for h in hs)
        offs.append(len(wid))
    return Events(offsets=np.asarray(offs, np.int32), wire_id=np.asarray(wid, np.int32),
                  drift=np.asarray(dr, np.float64), tracks=tracks, hit_truth=truths)


def single_track_events(n_events: int, seed: int, w: Wires | None = None,
                        min_hits: int = 6, noiseless: bool = False) -> Events:
    """n_events events with one helix each (no noise hits).  Tracks leaving fewer than
    min_hits hits are redrawn so every event is usable."""
    w = make_wires() if w is None else w
    rng = np.random.default_rng(seed)
    per, tracks, truths = [], [], []
    while len(per) < n_events:
        tr = draw_track(rng)
        hs = simulate_track(tr, w, None if noiseless else rng)
        if len(hs) < min_hits:
            continue
        hs.sort(key=lambda h: h.wire)
        per.append([(h.wire, h.drift) for h in hs])
        tracks.append([tr])
        truths.append(hs)
    return _pack(per, tracks, truths)


def multi_track_events(n_events: int, seed: int, w: Wires | None = None,
                       hit_cap: int = 200) -> Events:
    """Uneven events: 1-5 helices each plus uniform noise hits.  Noise occupancy occ is
    drawn U[0.1, 0.3] and read as the fraction of the event's hits that are noise, i.e.
    n_noise = round(occ / (1 - occ) * n_track_hits); noise drifts are U[0, half-cell].
    Totals are capped at hit_cap."""
    w = make_wires() if w is None else w
    rng = np.random.default_rng(seed)
    per, tracks, truths = [], [], []
    while len(per) < n_events:
        nt = int(rng.integers(1, 6))
        trs, hs_all = [], {}
        for _ in range(nt):
            tr = draw_track(rng)
            hs = simulate_track(tr, w, rng)
            trs.append(tr)
            for h in hs:
                if h.wire not in hs_all or h.drift < hs_all[h.wire].drift:
                    hs_all[h.wire] = h
        n_trk = len(hs_all)
        if n_trk < 6:
            continue
        occ = rng.uniform(0.1, 0.3)
        n_noise = int(round(occ / (1.0 - occ) * n_trk))
        n_noise = max(0, min(n_noise, hit_cap - n_trk))
        free = np.setdiff1d(np.arange(w.n), np.fromiter(hs_all.keys(), int))
        noise_w = rng.choice(free, size=n_noise, replace=False)
        items = [(h.wire, h.drift, h) for h in hs_all.values()]
        for nw in noise_w:
            items.append((int(nw), float(rng.uniform(0.0, w.half_cell[nw])), None))
        items = items[:hit_cap]
        items.sort(key=lambda it: it[0])
        per.append([(it[0], it[1]) for it in items])
        tracks.append(trs)
        truths.append([it[2] for it in items])
    return _pack(per, tracks, truths)
