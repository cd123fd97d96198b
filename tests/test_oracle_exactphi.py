"""Pins of the oracle's exact-phase vote program (Eq. CSAXtoPHI_a solved by an interval
fixed point instead of the expansion of Eqs. ApproxPhi_a-d), without a GPU.

  * on a cell shrunk to a point, the per-sign enclosure of delta = Phi - Phi^Ax contains
    the numerical solution of Eq. CSAXtoPHI_a from the libm point model (fixed-point
    iteration in the paper's notation) and is tight;
  * there, G+- contain rho F of Eqs. defdiAX_a,b evaluated with that exact phase;
  * a tiny cell around the true helix gets every noiseless hit's vote (the exact phase
    makes F vanish at the truth, with no truncation left);
  * soundness: a cell over which the exact F changes sign (dense sampling) votes.
"""
import numpy as np
import pytest

from gen import chamber
from oracle import oracle as O, point_model as pm

EXACT = 4


@pytest.fixture(scope="module")
def wires():
    return chamber.make_wires()


@pytest.fixture(scope="module")
def events(wires):
    return chamber.single_track_events(8, seed=81, w=wires)


@pytest.fixture(scope="module")
def events_noiseless(wires):
    return chamber.single_track_events(6, seed=82, w=wires, noiseless=True)


def _wire5(w, i):
    return (w.x0[i], w.y0[i], w.sin_phis[i], w.cos_phis[i], w.tan_tau[i])


def _point_cell(pt):
    s0, c0 = np.sin(pt[1]), np.cos(pt[1])
    return np.array([pt[0], pt[0], s0, s0, c0, c0, pt[2], pt[2], pt[3], pt[3], pt[4], pt[4]])


def _exact(pt, wire5, d_st):
    """(delta, rho F) of the exact phase at a point, in the frame where omega > 0."""
    prm, wm, dm = (tuple(pt), wire5, d_st) if pt[2] > 0 else pm.mirror(tuple(pt), wire5, d_st)
    a = pm.ax_quantities(prm, wm, prm[3])
    Phi, sperp = pm.phi_solve(prm, wm, dm, prm[3])
    F = pm.F_given_phi(prm, wm, dm, Phi, sperp, prm[3])
    return Phi - a["PhiA"], F * abs(pt[2])


def test_exact_delta_and_G_enclose_the_solution(wires, events):
    rng = np.random.default_rng(1)
    n = 0
    for e in range(events.n_events):
        p = np.array(events.tracks[e][0].params)
        for h in events.hit_truth[e]:
            pt = p + rng.normal(0, 1, 5) * np.array([1e-3, 1e-2, 1e-2, 1e-2, 1e-2])
            _, out = O.vote_pair(_point_cell(pt), O.hit9(wires, h.wire, h.drift), EXACT)
            if out[4]:
                continue
            for sg in (0, 1):
                d_st = (1 - 2 * sg) * h.drift * (1 if pt[2] > 0 else -1)
                delta, G = _exact(pt, _wire5(wires, h.wire), d_st)
                lo, hi = out[5 + 2 * sg], out[6 + 2 * sg]
                assert lo - 1e-15 <= delta <= hi + 1e-15, (e, h.wire, sg, lo, delta, hi)
                assert hi - lo < 1e-7, (lo, hi)     # three contractions from +-2^-8
                glo, ghi = out[2 * sg], out[2 * sg + 1]
                tol = 1e-13 * (1 + abs(G))
                assert glo - tol <= G <= ghi + tol, (e, h.wire, sg, glo, G, ghi)
                n += 1
    assert n > 150


def test_exact_true_cell_gets_every_noiseless_hit(wires, events_noiseless):
    rng = np.random.default_rng(2)
    for e in range(events_noiseless.n_events):
        p = np.array(events_noiseless.tracks[e][0].params)
        lo = p - 1e-7 * rng.uniform(0.1, 1, 5)
        hi = p + 1e-7 * rng.uniform(0.1, 1, 5)
        s0, c0 = np.sin([lo[1], hi[1]]), np.cos([lo[1], hi[1]])
        cell = np.array([lo[0], hi[0], np.nextafter(s0.min(), -9), np.nextafter(s0.max(), 9),
                         np.nextafter(c0.min(), -9), np.nextafter(c0.max(), 9), lo[2], hi[2],
                         lo[3], hi[3], lo[4], hi[4]])
        for h in events_noiseless.hit_truth[e]:
            v, out = O.vote_pair(cell, O.hit9(wires, h.wire, h.drift), EXACT)
            assert v == 1, (e, h.wire, out)


def test_exact_soundness_sign_change(wires, events):
    """Cells of a few hundred micrometres around points near the track: wherever the
    exact rho F of one drift sign changes sign over sampled points, the cell votes."""
    rng = np.random.default_rng(3)
    checked = 0
    for e in range(events.n_events):
        p = np.array(events.tracks[e][0].params)
        for h in events.hit_truth[e][:5]:
            c = p + rng.normal(0, 1, 5) * np.array([3e-4, 3e-3, 3e-3, 3e-3, 3e-3])
            half = np.array([2e-4, 2e-3, 2e-3, 2e-3, 2e-3]) * rng.uniform(0.3, 1, 5)
            lo, hi = c - half, c + half
            s = np.sin(np.linspace(lo[1], hi[1], 64))
            co = np.cos(np.linspace(lo[1], hi[1], 64))
            cell = np.array([lo[0], hi[0], np.nextafter(s.min(), -9), np.nextafter(s.max(), 9),
                             np.nextafter(co.min(), -9), np.nextafter(co.max(), 9), lo[2], hi[2],
                             lo[3], hi[3], lo[4], hi[4]])
            v, _ = O.vote_pair(cell, O.hit9(wires, h.wire, h.drift), EXACT)
            for sg in (1, -1):
                vals = []
                for _ in range(40):
                    pt = lo + (hi - lo) * rng.uniform(0, 1, 5)
                    d_st = sg * h.drift if pt[2] > 0 else -sg * h.drift
                    vals.append(_exact(pt, _wire5(wires, h.wire), d_st)[1])
                if min(vals) < 0 < max(vals):
                    assert v == 1
                    checked += 1
    assert checked > 5
