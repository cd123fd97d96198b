"""Pins of the oracle's midpoint form of the vote (Section 3.1: the quantities of d^Ax in
Eq. defdiAX_b taken at the voxel centre), without a GPU.

  * tan tau = 0: d^Ax is the drift itself and G is the exact axial tangency value of the
    golden rationals (Section 2.1);
  * a voxel shrunk to a point: the midpoint form and the interval program evaluate the
    same expression, so the point result lies in the interval program's enclosure;
  * d^Ax against the independent libm point model written in the paper's notation
    (Eqs. ApproxPhi_a-d, normudi, EQSinter_c, defdiAX_b), at random points near the
    generated tracks, for both drift signs and both curvature signs;
  * grid plumbing: cell votes over a small grid equal the pair-by-pair evaluation with
    the centre table's sin/cos.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from gen import chamber, grid as G
from oracle import oracle as O, point_model as pm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def wires():
    return chamber.make_wires()


@pytest.fixture(scope="module")
def events(wires):
    return chamber.single_track_events(10, seed=31, w=wires)


def _wire5(w, i):
    return (w.x0[i], w.y0[i], w.sin_phis[i], w.cos_phis[i], w.tan_tau[i])


def test_mid_axial_tangency_golden():
    """tan tau = 0: u_d = 1, the stereo terms vanish and d^Ax = +-d; G+- equal the exact
    rationals to rounding, and the vote follows wherever |G| is above rounding."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "axial_tangency.txt"))
            if not l.startswith("#")]
    n = 0
    for r in rows:
        s0, c0, om, d0, x0, y0, d, gp, gm = (float(Fraction(v)) for v in r[:9])
        vote = int(r[9])
        cell = np.array([d0, d0, s0, s0, c0, c0, om, om, 0.0, 0.0, 0.37, 0.37])
        a = np.arctan2(y0, x0)
        hit = np.array([x0, y0, np.sin(a), np.cos(a), 0.0, 0.0, 0.0, 0.0, d])
        v, out = O.vote_pair_mid(cell, np.array([s0, c0]), hit)
        assert out[4] == 0, r
        # in the frame where omega > 0 (rows with omega < 0 are mirrored): R + d^Ax =
        # |R + d| for the sign + and |R - d| for the sign - (the positive root of Eq.
        # defdiAX_b)
        R = 1.0 / abs(om)
        tol = 8e-16 * (R + d)
        assert abs(out[5] - d) <= tol, (r, out[5])
        assert abs(out[6] - (abs(R - d) - R)) <= tol, (r, out[6])
        scale = 64 * np.finfo(float).eps * (1.0 + abs(gp) + abs(gm) + d * d * abs(om) + 2 * d)
        assert out[0] <= out[1] and out[2] <= out[3]
        assert abs(0.5 * (out[0] + out[1]) - gp) <= scale, (r, out)
        assert abs(0.5 * (out[2] + out[3]) - gm) <= scale, (r, out)
        if min(abs(gp), abs(gm)) > 2 * scale:
            assert v == vote, r
        n += 1
    assert n > 500


def test_mid_point_voxel_matches_interval_program(wires, events):
    """A voxel shrunk to one point (thin intervals, sin/cos of phi0 thin): the midpoint
    form's G+- must lie inside the interval program's G+- (up to rounding), since both
    evaluate the same expression there; a wrong step in either breaks it."""
    rng = np.random.default_rng(11)
    n = 0
    for e in range(events.n_events):
        p = np.array(events.tracks[e][0].params)
        for h in events.hit_truth[e]:
            for _k in range(2):
                pt = p + rng.normal(0, 1, 5) * np.array([1e-3, 1e-2, 1e-2, 1e-2, 1e-2])
                s0, c0 = np.sin(pt[1]), np.cos(pt[1])
                cell = np.array([pt[0], pt[0], s0, s0, c0, c0, pt[2], pt[2], pt[3], pt[3],
                                 pt[4], pt[4]])
                hv = O.hit9(wires, h.wire, h.drift)
                vs, so = O.vote_pair(cell, hv, 0)
                vm, mo = O.vote_pair_mid(cell, np.array([s0, c0]), hv)
                if so[4] or mo[4]:
                    continue
                for sg in (0, 1):
                    glo, ghi = so[2 * sg], so[2 * sg + 1]
                    tol = 1e-13 * (1.0 + abs(glo) + abs(ghi))
                    assert glo - tol <= mo[2 * sg] <= mo[2 * sg + 1] <= ghi + tol, (
                        e, h.wire, sg, so, mo)
                    n += 1
    assert n > 300


def test_mid_dax_matches_point_model(wires, events):
    """d^Ax of the midpoint form at a voxel centre equals sqrt(A2 - F) - R of the libm
    point model (F of Eq. defdiAX_a with d^Ax from Eq. defdiAX_b and the second-order Phi)
    at the same point, for both drift signs and both curvature signs."""
    rng = np.random.default_rng(12)
    n = 0
    worst = 0.0
    for e in range(events.n_events):
        p = np.array(events.tracks[e][0].params)
        for h in events.hit_truth[e]:
            pt = p + rng.normal(0, 1, 5) * np.array([1e-3, 3e-2, 1e-2, 1e-2, 3e-2])
            half = rng.uniform(1e-6, 1e-3, 5)
            lo, hi = pt - half, pt + half
            c = (lo + hi) * 0.5                # the centre the oracle computes
            s0, c0 = np.sin(c[1]), np.cos(c[1])
            cell = np.array([lo[0], hi[0], np.sin(lo[1]) - 1, np.sin(lo[1]) + 1,
                             np.cos(lo[1]) - 1, np.cos(lo[1]) + 1, lo[2], hi[2], lo[3], hi[3],
                             lo[4], hi[4]])
            hv = O.hit9(wires, h.wire, h.drift)
            _, mo = O.vote_pair_mid(cell, np.array([s0, c0]), hv)
            if mo[4]:
                continue
            cpt = (c[0], c[1], c[2], c[3], c[4])
            wv = _wire5(wires, h.wire)
            for sg in (0, 1):
                # the program tries +d and -d in the frame where omega > 0
                d_st = (1 - 2 * sg) * h.drift * (1 if c[2] > 0 else -1)
                prm, wm, dm = (cpt, wv, d_st) if c[2] > 0 else pm.mirror(cpt, wv, d_st)
                a = pm.ax_quantities(prm, wm, prm[3])
                F = pm.F_approx(cpt, wv, d_st)
                dax = np.sqrt(a["RA"] ** 2 - F) - a["R"]
                err = abs(mo[5 + sg] - dax)
                worst = max(worst, err)
                assert err <= 1e-9 + 1e-7 * h.drift, (e, h.wire, sg, mo[5 + sg], dax)
                n += 1
    assert n > 150
    assert worst < 1e-9


def test_mid_grid_votes_use_centre_table(wires, events):
    """Cell votes on a small grid (any level) equal the pair-by-pair midpoint votes with
    cell12 and the centre table's sin/cos."""
    g = G.make_grid([4, 6, 4, 4, 4], 2, 8)
    tab = O.Tables(g, wires)
    rng = np.random.default_rng(13)
    e = 0
    a, b = events.offsets[e], events.offsets[e + 1]
    wid, dr = events.wire_id[a:b], events.drift[a:b]
    for level in (0, 2):
        n = [int(g.bins[k]) << level for k in range(5)]
        idx = np.stack([rng.integers(0, n[k], 60) for k in range(5)], axis=1)
        keys = G.cell_key(idx)
        votes = O.vote_cells(tab, wid, dr, level, keys, prec=3)
        for j in range(idx.shape[0]):
            c12 = O.cell12(g, level, idx[j])
            sc = O.scm2(g, level, idx[j])
            v = sum(O.vote_pair_mid(c12, sc, O.hit9(wires, int(w), float(d)))[0]
                    for w, d in zip(wid, dr))
            assert v == votes[j], (level, idx[j])
