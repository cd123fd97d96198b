"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test ties the oracle to something other than itself:
  * exact axial Apollonius tangency (Section 2.1), golden rationals;
  * the exact-phase identity of Eqs. (EQSinter_a-c) -> (defdiAX_a,b) on generated hits;
  * the O(tan^3 tau) accuracy of the paper's Phi^(1), Phi^(2) (ApproxPhi) against a
    numerical solution of the angular equation (CSAXtoPHI_a);
  * interval enclosure of the independent point model (libm, paper notation);
  * soundness by sign changes (Section 3.1: no vote => no solution in the voxel);
  * the true cell receiving every noiseless hit at every level;
  * inclusion isotonicity, FP32 superset, transcendental enclosures vs libm;
  * top-K / bisection / estimate against brute force, and an exhaustive tiny grid.
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
    return chamber.single_track_events(12, seed=21, w=wires)


@pytest.fixture(scope="module")
def events_noiseless(wires):
    return chamber.single_track_events(6, seed=22, w=wires, noiseless=True)


def _wire5(w, i):
    return (w.x0[i], w.y0[i], w.sin_phis[i], w.cos_phis[i], w.tan_tau[i])


def _fr(s):
    return float(Fraction(s))


# ------------------------------------------------------------------------------------ #
def test_axial_tangency_golden():
    """tan tau = 0: G = rho(|W-C|^2 - (R +- d)^2) exactly, vote iff tangent."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "axial_tangency.txt"))
            if not l.startswith("#")]
    assert len(rows) > 500
    for r in rows:
        s0, c0, om, d0, x0, y0, d, gp, gm = (_fr(v) for v in r[:9])
        vote = int(r[9])
        cell = np.array([d0, d0, s0, s0, c0, c0, om, om, 0.0, 0.0, 0.37, 0.37])
        a = np.arctan2(y0, x0)
        hit = np.array([x0, y0, np.sin(a), np.cos(a), 0.0, 0.0, 0.0, 0.0, d])
        for prec in (0, 1):
            v, out = O.vote_pair(cell, hit, prec)
            if prec == 0:
                assert out[0] == gp and out[1] == gp, r
                assert out[2] == gm and out[3] == gm, r
                assert v == vote, r
            else:   # FP32: encloses the exact value (inputs rounded outward)
                assert out[0] <= gp <= out[1] and out[2] <= gm <= out[3], r
                assert v >= vote


def test_exact_phase_identity(wires, events_noiseless):
    """At the generator's exact closest point, Eq. (defdiAX_a,b) holds to rounding: the
    derivation EQSinter_a,b -> defdiAX and the generator agree (both signs of omega, any
    z_ref)."""
    n = 0
    for e in range(events_noiseless.n_events):
        tr = events_noiseless.tracks[e][0]
        for h in events_noiseless.hit_truth[e]:
            for zr in (0.0, tr.z0, 0.3):
                F = pm.F_given_phi(tuple(tr.params), _wire5(wires, h.wire), h.d_signed,
                                   h.Phi, h.s, zr)
                assert abs(F) < 1e-12
                n += 1
    assert n > 100


def test_mirror_invariance(wires, events_noiseless):
    """The y -> -y reflection maps F to itself (exact phase used on both sides)."""
    for e in range(events_noiseless.n_events):
        tr = events_noiseless.tracks[e][0]
        p = tuple(tr.params)
        for h in events_noiseless.hit_truth[e][:4]:
            wv = _wire5(wires, h.wire)
            pm_, wm, dm = pm.mirror(p, wv, h.d_signed)
            phis_m = np.arctan2(wm[2], wm[3])
            Phi_m = -tr.omega * h.s - tr.phi0 - phis_m
            F1 = pm.F_given_phi(p, wv, h.d_signed, h.Phi, h.s, tr.z0)
            F2 = pm.F_given_phi(pm_, wm, dm, Phi_m, h.s, tr.z0)
            assert abs(F1 - F2) < 1e-12


def test_phi_expansion_cubic_residual():
    """Phi - (Phi^Ax + Phi1 t + Phi2 t^2) = O(t^3): halving tan(tau) divides the residual
    by ~8, with the angular equation solved by fixed-point iteration.  This checks the
    paper's Mathematica-derived Phi^(2) (Eq. ApproxPhi_c)."""
    rng = np.random.default_rng(3)
    for _ in range(6):
        params = (rng.uniform(-.01, .01), rng.uniform(0, 2 * np.pi), rng.uniform(0.15, 1.0),
                  0.0, rng.uniform(-.8, .8))
        d0, phi0, om, z0, lam = params
        R = 1 / om
        xc, yc, _ = pm.helix_centre(d0, phi0, om)
        ang = phi0 - np.pi / 2 + rng.uniform(0.05, 0.5)
        r = R + rng.uniform(-0.01, 0.01)
        x0, y0 = xc + r * np.cos(ang), yc + r * np.sin(ang)
        phis = np.arctan2(y0, x0)
        d = rng.uniform(-0.01, 0.01)
        res = []
        for t in (0.04, 0.02, 0.01):
            wire = (x0, y0, np.sin(phis), np.cos(phis), t)
            Phs, _ = pm.phi_solve(params, wire, d, 0.0, iters=400)
            Ph = pm.phi_approx(params, wire, d, 0.0)[0]
            res.append(Phs - Ph)
        for i in range(2):
            assert 6.5 < res[i] / res[i + 1] < 9.5, res


def test_truncation_residual_small(wires, events_noiseless):
    """With noiseless drifts, F at the true helix with the second-order phase is tiny
    (the O(tan^3) truncation): |F| / (2R) below 20 micrometres."""
    worst = 0.0
    for e in range(events_noiseless.n_events):
        tr = events_noiseless.tracks[e][0]
        for h in events_noiseless.hit_truth[e]:
            F = pm.F_approx(tuple(tr.params), _wire5(wires, h.wire), h.d_signed)
            worst = max(worst, abs(F) * abs(tr.omega) / 2)
    assert worst < 2e-5


def _tiny_cell(p, rng, eps=1e-7):
    lo = p - eps * rng.uniform(0.1, 1, 5)
    hi = p + eps * rng.uniform(0.1, 1, 5)
    s0 = np.sin([lo[1], hi[1]])
    c0 = np.cos([lo[1], hi[1]])
    cell = np.array([lo[0], hi[0], np.nextafter(s0.min(), -9), np.nextafter(s0.max(), 9),
                     np.nextafter(c0.min(), -9), np.nextafter(c0.max(), 9), lo[2], hi[2],
                     lo[3], hi[3], lo[4], hi[4]])
    return cell, lo, hi


def _point_G(pt, wire, d_st):
    """rho * F at a point, from the point model (paper notation, libm)."""
    return pm.F_approx(tuple(pt), wire, d_st) * abs(pt[2])


def test_interval_encloses_point_model(wires, events):
    """For tiny cells around each true helix, the interval G+/G- of the vote program
    contain rho*F of the point model at points sampled inside the cell.  A dropped term,
    a wrong sign or a transposed operand in the interval program breaks this."""
    rng = np.random.default_rng(5)
    n = 0
    for e in range(events.n_events):
        p = np.array(events.tracks[e][0].params)
        for h in events.hit_truth[e]:
            cell, lo, hi = _tiny_cell(p, rng)
            hv = O.hit9(wires, h.wire, h.drift)
            wv = _wire5(wires, h.wire)
            for prec in (0, 1):
                _, out = O.vote_pair(cell, hv, prec)
                for _k in range(2):
                    pt = lo + (hi - lo) * rng.uniform(0, 1, 5)
                    for sg, (glo, ghi) in ((1, out[0:2]), (-1, out[2:4])):
                        # the vote program tries +d and -d in the frame where omega > 0
                        d_st = sg * h.drift if pt[2] > 0 else -sg * h.drift
                        g = _point_G(pt, wv, d_st)
                        tol = 1e-13
                        assert glo - tol <= g <= ghi + tol, (e, h.wire, prec, sg, glo, g, ghi)
                        n += 1
    assert n > 400


def test_phase_expansion_matches_paper_form(wires, events):
    """On a voxel shrunk to a point, the interval program's phase corrections
    delta+- = Phi - Phi^Ax (its rescaled form of Eqs. ApproxPhi_b,c) are thin and contain
    Phi1 tan(tau) + Phi2 tan^2(tau) of the point model, which writes Eq. (ApproxPhi_c) as
    printed, for each drift sign.  The G enclosure tests above cannot see an error in a
    small term here: the vote program joins both signs' phases before sin/cos."""
    rng = np.random.default_rng(15)
    n = 0
    for e in range(events.n_events):
        p = np.array(events.tracks[e][0].params)
        for h in events.hit_truth[e]:
            pt = p + rng.normal(0, 1, 5) * np.array([1e-3, 3e-2, 1e-2, 1e-2, 3e-2])
            s0, c0 = np.sin(pt[1]), np.cos(pt[1])
            cell = np.array([pt[0], pt[0], s0, s0, c0, c0, pt[2], pt[2], pt[3], pt[3],
                             pt[4], pt[4]])
            _, out = O.vote_pair(cell, O.hit9(wires, h.wire, h.drift), 0)
            if out[4]:
                continue
            wv = _wire5(wires, h.wire)
            for sg in (0, 1):
                d_st = (1 - 2 * sg) * h.drift * (1 if pt[2] > 0 else -1)
                prm, wm, dm = (tuple(pt), wv, d_st) if pt[2] > 0 else pm.mirror(tuple(pt), wv, d_st)
                a = pm.ax_quantities(prm, wm, prm[3])
                Phi = pm.phi_approx(prm, wm, dm, prm[3])[0]
                delta = Phi - a["PhiA"]
                lo, hi = out[5 + 2 * sg], out[6 + 2 * sg]
                tol = 1e-14 + 1e-12 * abs(delta)
                assert lo - tol <= delta <= hi + tol, (e, h.wire, sg, lo, delta, hi)
                assert hi - lo <= 1e-12 * (1 + abs(delta)), (lo, hi)
                n += 1
    assert n > 150


def test_interval_encloses_point_model_wide_cells(wires, events):
    """Same enclosure on coarse-size cells (random points inside a level-2 cell)."""
    rng = np.random.default_rng(6)
    g = G.make_grid([16] * 5, 6, 64)
    for e in range(4):
        p = np.array(events.tracks[e][0].params)
        idx = [int(np.searchsorted(g.lo_edge[a][::1 << (g.levels - 2)], p[a], side="right") - 1)
               for a in range(5)]
        cell = O.cell12(g, 2, idx)
        lo = np.array([cell[0], g.cell_edges(2, 1, idx[1])[0], cell[6], cell[8], cell[10]])
        hi = np.array([cell[1], g.cell_edges(2, 1, idx[1])[1], cell[7], cell[9], cell[11]])
        for h in events.hit_truth[e][:6]:
            _, out = O.vote_pair(cell, O.hit9(wires, h.wire, h.drift), 0)
            for _k in range(20):
                pt = lo + (hi - lo) * rng.uniform(0, 1, 5)
                for sg, (glo, ghi) in ((1, out[0:2]), (-1, out[2:4])):
                    d_st = sg * h.drift if pt[2] > 0 else -sg * h.drift
                    gv = _point_G(pt, _wire5(wires, h.wire), d_st)
                    assert glo <= gv <= ghi


def test_soundness_sign_change(wires, events):
    """Section 3.1: when the condition is false the solution is not in the voxel.  If the
    point function changes sign inside a cell, a zero lies in it (continuity on a box), so
    the cell must vote.  Cells are placed across the zero set by shifting the drift."""
    rng = np.random.default_rng(7)
    checked = 0
    for e in range(events.n_events):
        p = np.array(events.tracks[e][0].params)
        for h in events.hit_truth[e][:5]:
            wv = _wire5(wires, h.wire)
            for _ in range(3):
                cell, lo, hi = _tiny_cell(p + rng.normal(0, 3e-6, 5), rng, eps=1e-5)
                for d in (h.dist, h.dist + 3e-6, max(h.dist - 3e-6, 0)):
                    v, _ = O.vote_pair(cell, O.hit9(wires, h.wire, d), 0)
                    vals = []
                    for _k in range(24):
                        pt = lo + (hi - lo) * rng.uniform(0, 1, 5)
                        for sg in (1, -1):
                            d_st = sg * d if pt[2] > 0 else -sg * d
                            vals.append((sg, _point_G(pt, wv, d_st)))
                    for sg in (1, -1):
                        gs = [g for s, g in vals if s == sg]
                        if min(gs) < -1e-12 and max(gs) > 1e-12:
                            assert v == 1
                            checked += 1
    assert checked > 20


@pytest.mark.parametrize("prec", [0, 1])
def test_true_cell_gets_every_noiseless_hit(wires, events_noiseless, prec):
    """At every level of the config-1 grid the cell holding the true helix receives a vote
    from every noiseless hit (soundness + exact-phase identity + small truncation)."""
    g = G.make_grid([10] * 5, 4, 16)
    for e in range(events_noiseless.n_events):
        p = np.array(events_noiseless.tracks[e][0].params)
        a, b = events_noiseless.offsets[e], events_noiseless.offsets[e + 1]
        for L in range(g.levels + 1):
            idx = [int(np.searchsorted(g.lo_edge[ax][::1 << (g.levels - L)], p[ax],
                                       side="right") - 1) for ax in range(5)]
            cell = O.cell12(g, L, idx)
            votes = sum(O.vote_pair(cell, O.hit9(wires, events_noiseless.wire_id[i],
                                                 events_noiseless.drift[i]), prec)[0]
                        for i in range(a, b))
            assert votes == b - a, (e, L)


def test_child_votes_never_exceed_parent(wires, events):
    """Inclusion isotonicity: a child cell's vote count is at most its parent's."""
    g = G.make_grid([16] * 5, 6, 64)
    tab = O.Tables(g, wires)
    rng = np.random.default_rng(8)
    for e in range(3):
        a, b = events.offsets[e], events.offsets[e + 1]
        wid, dr = events.wire_id[a:b], events.drift[a:b]
        p = np.array(events.tracks[e][0].params)
        for L in range(0, g.levels):
            # parents near the track and random ones
            near = [int(np.searchsorted(g.lo_edge[ax][::1 << (g.levels - L)], p[ax],
                                        side="right") - 1) for ax in range(5)]
            par = [near] + [[int(rng.integers(0, int(g.bins[ax]) << L)) for ax in range(5)]
                            for _ in range(3)]
            pk = G.cell_key(np.array(par))
            pv = O.vote_cells(tab, wid, dr, L, pk)
            ck = O.children(pk)
            cv = O.vote_cells(tab, wid, dr, L + 1, ck)
            assert np.all(cv.reshape(-1, 32) <= pv[:, None])


def test_fp32_superset_of_fp64(wires, events):
    """FP32 intervals (same program, inputs rounded outward) contain the FP64 intervals,
    so every FP64 vote is also an FP32 vote."""
    g = G.make_grid([16] * 5, 6, 64)
    rng = np.random.default_rng(9)
    for e in range(events.n_events):
        p = np.array(events.tracks[e][0].params)
        for h in events.hit_truth[e][:4]:
            hv = O.hit9(wires, h.wire, h.drift)
            for L in (0, 3, 6):
                idx = [int(np.searchsorted(g.lo_edge[ax][::1 << (g.levels - L)], p[ax],
                                           side="right") - 1) for ax in range(5)]
                idx = [min(max(i + int(rng.integers(-1, 2)), 0), (int(g.bins[ax]) << L) - 1)
                       for ax, i in enumerate(idx)]
                cell = O.cell12(g, L, idx)
                v64, o64 = O.vote_pair(cell, hv, 0)
                v32, o32 = O.vote_pair(cell, hv, 1)
                assert v32 >= v64
                if o64[4] == 0 and o32[4] == 0:
                    assert o32[0] <= o64[0] and o64[1] <= o32[1]
                    assert o32[2] <= o64[2] and o64[3] <= o32[3]


def test_transcendental_enclosures():
    """atan / sin / cos enclosures (+ - * / sqrt only) contain libm's values, are tight for
    thin arguments in FP64, and contain the exact range over wide arguments."""
    rng = np.random.default_rng(10)
    for x in np.concatenate([rng.uniform(-3, 3, 200), [0.0, 1e-9, 2.6, -2.6]]):
        for prec in (0, 1):
            a = O.atan_iv(x, x, prec)
            ref = np.arctan(x)
            assert a[0] <= ref <= a[1]
            if prec == 0:   # width: twice 4 |r|^17/17 (r = tan(atan(x)/4)) plus rounding
                r = abs(np.tan(ref / 4))
                assert a[1] - a[0] <= 8 * r ** 17 / 17 * 1.01 + 1e-14
    for lo, hi in [(-2.0, 0.5), (0.1, 0.3), (-0.3, -0.29)]:
        a = O.atan_iv(lo, hi, 0)
        assert a[0] <= np.arctan(lo) and np.arctan(hi) <= a[1]
    for x in np.concatenate([rng.uniform(-1, 1, 200), [0.0, 1.0, -1.0]]):
        for prec in (0, 1):
            s = O.sincos_iv(x, x, prec)
            assert s[0] <= np.sin(x) <= s[1] and s[2] <= np.cos(x) <= s[3]
            if prec == 0:   # width: twice the Lagrange remainder plus rounding
                m = abs(x)
                assert s[1] - s[0] <= 2 * m ** 5 / 120 * 1.000001 + 1e-15
                assert s[3] - s[2] <= 2 * m ** 4 / 24 * 1.000001 + 1e-15
    s = O.sincos_iv(-0.5, 0.7, 0)
    xs = np.linspace(-0.5, 0.7, 1001)
    assert s[0] <= np.sin(xs).min() and np.sin(xs).max() <= s[1]
    assert s[2] <= np.cos(xs).min() and np.cos(xs).max() <= s[3]
    assert np.all(O.sincos_iv(-1.5, 2.0, 0) == [-1, 1, -1, 1])


def test_rounding_is_directed():
    """An inexact thin evaluation gives lo < hi (outward rounding really happens)."""
    cell = np.array([0.001, 0.001, 0.3, 0.3, np.sqrt(1 - 0.09), np.sqrt(1 - 0.09), 0.3, 0.3,
                     0.01, 0.01, 0.2, 0.2])
    hit = np.array([0.25, 0.1, 0.37, 0.93, 0.1003, 0.037, 0.093, 0.01006, 0.004])
    _, out = O.vote_pair(cell, hit, 0)
    assert out[0] < out[1] and out[2] < out[3]
    # the drift-sign hull in u_d widens even a thin cell slightly (micro-metre scale)
    assert out[1] - out[0] < 1e-7
    # axial wire, inexact operands: only rounding separates the ends
    hit_ax = np.array([0.25, 0.1, 0.37, 0.93, 0.0, 0.0, 0.0, 0.0, 0.004])
    _, out = O.vote_pair(cell, hit_ax, 0)
    assert 0 < out[1] - out[0] < 1e-14 and 0 < out[3] - out[2] < 1e-14


def test_topk_children_estimate_brute_force():
    rng = np.random.default_rng(11)
    keys = np.unique(G.cell_key(rng.integers(0, 512, size=(3000, 5))))[:3000]
    rng.shuffle(keys)
    votes = rng.integers(0, 6, size=keys.shape[0]).astype(np.int32)
    k, v = O.topk(keys, votes, 64)
    ref = sorted(zip(votes.tolist(), keys.tolist()), key=lambda t: (-t[0], t[1]))[:64]
    assert [int(x) for x in k] == [t[1] for t in ref]
    assert [int(x) for x in v] == [t[0] for t in ref]
    idx = G.key_indices(k[:3])
    ch = G.key_indices(O.children(k[:3])).reshape(3, 32, 5)
    for j in range(3):
        for b in range(32):
            np.testing.assert_array_equal(ch[j, b], 2 * idx[j] + [(b >> a) & 1 for a in range(5)])


def test_exhaustive_tiny_grid(wires, events):
    """With K >= every cell count, the coarse-to-fine search visits every finest cell and
    its last-level votes equal direct votes of those cells; the estimate is the mean centre
    of the maximum-vote finest cells."""
    g = G.make_grid([2, 2, 2, 2, 2], 2, 32 * 32)
    tab = O.Tables(g, wires)
    a, b = events.offsets[0], events.offsets[1]
    wid, dr = events.wire_id[a:b], events.drift[a:b]
    r = O.solve_event(tab, wid, dr)
    allk = G.cell_key(np.stack(np.meshgrid(*[np.arange(8)] * 5, indexing="ij"), -1).reshape(-1, 5))
    direct = O.vote_cells(tab, wid, dr, 2, allk)
    got = dict(zip(r["last_keys"].tolist(), r["last_votes"].tolist()))
    assert len(got) == 8 ** 5
    for k, v in zip(allk.tolist(), direct.tolist()):
        assert got[k] == v
    m = direct.max()
    idx = G.key_indices(allk[direct == m])
    for ax in range(5):
        lo, hi = g.cell_edges(2, ax, idx[:, ax])
        assert np.isclose(r["p"][ax], ((lo + hi) / 2).mean(), rtol=1e-12, atol=1e-15)
        assert r["w"][ax] == (hi.max() - lo.min()) / 2
    assert r["votes"] == m
