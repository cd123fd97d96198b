"""Pins of the oracle's multi-track extraction (CPU): the hit finding of Section 3.3
applied to several tracks, checked against the generator's truth and the stop rules.

* A hit is taken by a found track when it votes (FP64) for one of the track's final cells
  with its drift widened by 3 sigma.  Given the cell that holds the generated helix, every
  hit whose true distance lies within 3 sigma of its measured drift must be taken (the
  interval program is sound), and hits on wires far from the helix must not be.
* The extraction stops at max_tracks, when no hit is left, or when the best final vote
  count is below min_votes; each rule is made to fire on its own.
"""
import numpy as np
import pytest

from gen import chamber, grid as G
from oracle import oracle as O

SIGMA = 150e-6


def _true_key(g, level, params):
    idx = []
    for a in range(5):
        n = int(g.bins[a]) << level
        lo, hi = g.cell_edges(level, a, np.arange(n))
        j = np.nonzero((lo <= params[a]) & (params[a] <= hi))[0]
        assert j.size, (a, params[a])
        idx.append(int(j[0]))
    return G.cell_key(np.array(idx))


@pytest.fixture(scope="module")
def setup():
    w = chamber.make_wires()
    g = G.make_grid([10] * 5, 6, 16)
    return w, g, O.Tables(g, w)


@pytest.mark.parametrize("level", [2, 4, 6])
def test_true_cell_takes_every_hit_within_three_sigma(setup, level):
    w, g, tab = setup
    rng = np.random.default_rng(71)
    n_taken = n_within = 0
    for _ in range(6):
        tr = chamber.draw_track(rng)
        hs = chamber.simulate_track(tr, w, rng)
        if len(hs) < 3:
            continue
        wid = np.array([h.wire for h in hs], np.int32)
        dr = np.array([h.drift for h in hs])
        within = np.array([abs(h.drift - h.dist) <= 3 * SIGMA for h in hs])
        key = _true_key(g, level, tr.params)
        taken = O.mask_hits(tab, wid, dr, level, [key], 3 * SIGMA)
        assert np.all(taken[within]), (level, np.nonzero(within & ~taken))
        n_taken += int(taken.sum())
        n_within += int(within.sum())
    assert n_within > 20 and n_taken >= n_within


def test_far_hits_are_not_taken(setup):
    """Noise hits on wires whose waist lies more than 0.2 m from the helix's circle (so the
    wire passes at least 0.2 - 0.075 m from it anywhere along its length) are not taken by
    the true cell at levels 2-6, even with drifts up to half a cell."""
    w, g, tab = setup
    rng = np.random.default_rng(72)
    for _ in range(6):
        tr = chamber.draw_track(rng)
        hs = chamber.simulate_track(tr, w, None)
        R = 1.0 / tr.omega
        xc, yc = -(R + tr.d0) * np.sin(tr.phi0), (R + tr.d0) * np.cos(tr.phi0)
        far = np.nonzero(np.abs(np.hypot(w.x0 - xc, w.y0 - yc) - abs(R)) > 0.2)[0]
        noise = rng.choice(far, size=40, replace=False)
        wid = np.concatenate([[h.wire for h in hs], noise]).astype(np.int32)
        dr = np.concatenate([[h.drift for h in hs], rng.uniform(0, w.half_cell[noise])])
        for level in (2, 4, 6):
            taken = O.mask_hits(tab, wid, dr, level, [_true_key(g, level, tr.params)], 3 * SIGMA)
            assert taken[:len(hs)].all()          # noiseless: every track hit
            assert not taken[len(hs):].any()


def test_active_flags_and_cell_union(setup):
    """Inactive hits are never taken, and a set of cells takes exactly the union of what
    each cell takes on its own."""
    w, g, tab = setup
    ev = chamber.multi_track_events(2, seed=73, w=w)
    for e in range(ev.n_events):
        a, b = ev.offsets[e], ev.offsets[e + 1]
        wid, dr = ev.wire_id[a:b], ev.drift[a:b]
        keys = [_true_key(g, 4, tr.params) for tr in ev.tracks[e]]
        union = np.zeros(b - a, bool)
        for k in keys:
            union |= O.mask_hits(tab, wid, dr, 4, [k], 3 * SIGMA)
        assert np.array_equal(O.mask_hits(tab, wid, dr, 4, keys, 3 * SIGMA), union)
        act = np.arange(b - a) % 2 == 0
        got = O.mask_hits(tab, wid, dr, 4, keys, 3 * SIGMA, active=act)
        assert np.array_equal(got, union & act)


def test_stop_rules():
    w = chamber.make_wires()
    g = G.make_grid([6] * 5, 2, 8)
    tab = O.Tables(g, w)
    ev = chamber.single_track_events(4, seed=74, w=w, noiseless=True)
    fired = {"all_taken": 0, "below_min": 0}
    # no hits: no track
    r = O.solve_event_multi(tab, np.zeros(0, np.int32), np.zeros(0), 5, 0)
    assert r["n_tracks"] == 0
    for e in range(ev.n_events):
        a, b = ev.offsets[e], ev.offsets[e + 1]
        wid, dr = ev.wire_id[a:b], ev.drift[a:b]
        n = b - a
        # min_votes above the hit count: the first search already gives no track
        r = O.solve_event_multi(tab, wid, dr, 5, n + 1)
        assert r["n_tracks"] == 0 and np.all(r["hit_track"] == -1)
        # max_tracks = 1 stops after one track
        r1 = O.solve_event_multi(tab, wid, dr, 1, 0)
        assert r1["n_tracks"] == 1
        single = O.solve_event(tab, wid, dr)
        assert r1["votes"][0] == single["votes"]
        assert np.array_equal(r1["p"][0], single["p"]) and np.array_equal(r1["w"][0], single["w"])
        # a first track that takes every hit ends the extraction (no hit left), whatever
        # max_tracks allows; a final cell with every hit's vote takes every hit
        r5 = O.solve_event_multi(tab, wid, dr, 5, 0)
        if single["votes"] == n:
            assert r5["n_tracks"] == 1 and np.all(r5["hit_track"] == 0)
            fired["all_taken"] += 1
        # every recorded track meets min_votes; when the extraction stopped with hits left
        # and tracks to spare, a search on the remaining hits falls below min_votes
        mv = 3
        rm = O.solve_event_multi(tab, wid, dr, 5, mv)
        assert np.all(rm["votes"] >= mv)
        left = rm["hit_track"] < 0
        if rm["n_tracks"] < 5 and left.any():
            assert O.solve_event(tab, wid[left], dr[left])["votes"] < mv
            fired["below_min"] += 1
    assert fired["all_taken"] and fired["below_min"], fired
