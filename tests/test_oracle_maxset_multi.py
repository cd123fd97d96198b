"""Pins of the oracle's multi-track max-set extraction (CPU).

Each round runs the single-track max-set search on the hits no earlier track took, then
takes one track out of the final maximum-vote group: the cells whose voting hits are
exactly those of the group's lowest-key cell.  Tracks with the same number of hits tie in
the group, so without that step one round would swallow several tracks.  Checked against
the generator's truth (two tied, noiseless tracks come out as two tracks, each with its
own hits), against the single-track search round by round, and against the stop rules.
"""
import numpy as np
import pytest

from gen import chamber, grid as G
from oracle import oracle as O

OUT = O.OUTGOING
PREC = [1 | OUT, 1 | OUT, 0 | OUT, 0 | OUT]


@pytest.fixture(scope="module")
def setup():
    w = chamber.make_wires()
    g = G.make_grid([2, 64, 8, 2, 4], 3, 64)
    return w, g, O.Tables(g, w)


def _tied_pair(w, rng):
    """Two noiseless tracks with the same number of hits on disjoint wires, their phi0 at
    least 1 rad apart."""
    while True:
        a, b = chamber.draw_track(rng), chamber.draw_track(rng)
        ha, hb = chamber.simulate_track(a, w, None), chamber.simulate_track(b, w, None)
        dphi = abs((a.params[1] - b.params[1] + np.pi) % (2 * np.pi) - np.pi)
        wa, wb = {h.wire for h in ha}, {h.wire for h in hb}
        if len(ha) == len(hb) >= 8 and dphi > 1.0 and not (wa & wb):
            items = sorted([(h.wire, h.drift, 0) for h in ha] + [(h.wire, h.drift, 1) for h in hb])
            wid = np.array([i[0] for i in items], np.int32)
            dr = np.array([i[1] for i in items])
            lab = np.array([i[2] for i in items])
            return (a, b), wid, dr, lab


def test_two_tied_tracks_are_separated(setup):
    w, g, tab = setup
    rng = np.random.default_rng(201)
    for _ in range(3):
        (ta, tb), wid, dr, lab = _tied_pair(w, rng)
        n_each = int((lab == 0).sum())
        # the single search's final maximum-vote group holds both tracks
        single = O.solve_event_maxset(tab, wid, dr, 3000, 1, PREC)
        assert single["votes"] == n_each
        r = O.solve_event_maxset_multi(tab, wid, dr, 3000, 5, 6, slack=1, prec_per_level=PREC)
        assert r["n_tracks"] == 2 and list(r["votes"]) == [n_each, n_each]
        assert r["n_final"][0] < single["n_final"]
        truths = np.array([ta.params, tb.params])
        owner = []
        for k in range(2):
            inside = np.all(np.abs(r["p"][k] - truths) <= r["w"][k], axis=1)
            assert inside.sum() == 1, (k, r["p"][k], truths, r["w"][k])
            owner.append(int(np.nonzero(inside)[0][0]))
            # the track takes exactly the hits of the helix it holds
            np.testing.assert_array_equal(r["hit_track"] == k, lab == owner[-1])
        assert sorted(owner) == [0, 1]


def test_rounds_are_single_searches_on_the_hits_left(setup):
    """Round t's vote count and final level are those of the single-track search on the
    hits that rounds 0..t-1 did not take; its cells are part of that search's final group;
    it takes at least its vote count of hits."""
    w, g, tab = setup
    ev = chamber.multi_track_events(3, seed=202, w=w)
    n_rounds = 0
    for e in range(ev.n_events):
        a, b = ev.offsets[e], ev.offsets[e + 1]
        wid, dr = ev.wire_id[a:b], ev.drift[a:b]
        r = O.solve_event_maxset_multi(tab, wid, dr, 3000, 4, 6, slack=2, prec_per_level=PREC)
        ht = r["hit_track"]
        for t in range(r["n_tracks"]):
            left = (ht < 0) | (ht >= t)
            s = O.solve_event_maxset(tab, wid[left], dr[left], 3000, 2, PREC)
            assert s["votes"] == r["votes"][t] and s["final_level"] == r["final_level"][t]
            assert 1 <= r["n_final"][t] <= s["n_final"]
            assert int((ht == t).sum()) >= r["votes"][t]
            n_rounds += 1
        if r["n_tracks"] < 4 and np.any(ht < 0):   # stopped by min_votes
            left = ht < 0
            assert O.solve_event_maxset(tab, wid[left], dr[left], 3000, 2, PREC)["votes"] < 6
    assert n_rounds >= 4


def test_one_hit_set_gives_the_single_search(setup):
    """Noiseless single tracks where every hit votes in the final group: the group has one
    hit set, so the first round is the single search itself."""
    w, g, tab = setup
    ev = chamber.single_track_events(3, seed=203, w=w, noiseless=True)
    for e in range(ev.n_events):
        a, b = ev.offsets[e], ev.offsets[e + 1]
        wid, dr = ev.wire_id[a:b], ev.drift[a:b]
        s = O.solve_event_maxset(tab, wid, dr, 3000, 1, PREC)
        assert s["votes"] == b - a
        r = O.solve_event_maxset_multi(tab, wid, dr, 3000, 1, 0, slack=1, prec_per_level=PREC)
        assert r["n_tracks"] == 1 and r["votes"][0] == s["votes"] and r["n_final"][0] == s["n_final"]
        np.testing.assert_array_equal(r["p"][0], s["p"])
        np.testing.assert_array_equal(r["w"][0], s["w"])
        assert np.all(r["hit_track"] == 0)


def test_stop_rules(setup):
    w, g, tab = setup
    r = O.solve_event_maxset_multi(tab, np.zeros(0, np.int32), np.zeros(0), 3000, 5, 0,
                                   prec_per_level=PREC)
    assert r["n_tracks"] == 0
    ev = chamber.single_track_events(2, seed=204, w=w, noiseless=True)
    for e in range(ev.n_events):
        a, b = ev.offsets[e], ev.offsets[e + 1]
        wid, dr = ev.wire_id[a:b], ev.drift[a:b]
        r = O.solve_event_maxset_multi(tab, wid, dr, 3000, 5, b - a + 1, prec_per_level=PREC)
        assert r["n_tracks"] == 0 and np.all(r["hit_track"] == -1)
        # every hit taken by the first track: the extraction ends there
        r = O.solve_event_maxset_multi(tab, wid, dr, 3000, 5, 0, slack=1, prec_per_level=PREC)
        assert r["n_tracks"] == 1 and np.all(r["hit_track"] == 0)
