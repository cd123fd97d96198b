"""Pins of the max-set schedule and of the direction condition (CPU).

Direction condition: the generator's hits lie on the outgoing arc (turning angle psi >= 0
from the point of closest approach, POCA).  The same helix run backwards, (-d0, phi0 + pi,
-omega, z0, -tan(lambda)), passes through the same hits, so without the condition the votes
cannot tell the two apart (the exact two-fold tie).  With it a hit votes only where psi can
be >= 0.  sin psi has the sign of the wire point's coordinate w_t along the helix tangent
at the POCA, so the program refuses a vote when w_t < 0 over the whole cell.

Max-set schedule (Section 3.3: the result is the set of maximum-vote voxels): every level
keeps whole vote groups {votes >= T} (T >= vmax - slack, at most max_keep cells), bisects
them, and the last level's maximum-vote group gives the estimate.
"""
import numpy as np
import pytest

from gen import chamber, grid as G
from oracle import oracle as O, point_model as PM

OUT = O.OUTGOING


def _true_idx(g, level, params):
    idx = []
    for a in range(5):
        n = int(g.bins[a]) << level
        lo, hi = g.cell_edges(level, a, np.arange(n))
        j = np.nonzero((lo <= params[a]) & (params[a] <= hi))[0]
        idx.append(int(j[0]) if j.size else -1)
    return idx


def _reversed(p):
    d0, phi0, om, z0, tl = p
    return np.array([-d0, (phi0 + np.pi) % (2 * np.pi), -om, z0, -tl])


@pytest.fixture(scope="module")
def wires():
    return chamber.make_wires()


def test_direction_breaks_the_reversal_degeneracy(wires):
    g = G.make_grid([10] * 5, 4, 16)
    tab = O.Tables(g, wires)
    ev = chamber.single_track_events(6, seed=81, w=wires, noiseless=True)
    for e in range(ev.n_events):
        a, b = ev.offsets[e], ev.offsets[e + 1]
        wid, dr, n = ev.wire_id[a:b], ev.drift[a:b], b - a
        tp = ev.tracks[e][0].params
        for level in range(5):
            kt = G.cell_key(np.array(_true_idx(g, level, tp)))
            kr = G.cell_key(np.array(_true_idx(g, level, _reversed(tp))))
            k = np.array([kt, kr], np.uint64)
            plain = O.vote_cells(tab, wid, dr, level, k, 0)
            out = O.vote_cells(tab, wid, dr, level, k, 0 | OUT)
            assert plain[0] == n and plain[1] == n          # the degeneracy is exact
            assert out[0] == n                               # the true direction keeps every vote
            if level >= 2:
                assert out[1] == 0, (e, level, out)          # the reversed one loses them all
            out32 = O.vote_cells(tab, wid, dr, level, k, 1 | OUT)
            assert out32[0] == n and out32[1] >= out[1]      # FP32 contains FP64


def test_direction_refusal_holds_at_every_point(wires):
    """Wherever the program refuses a (cell, hit) vote by the direction condition, the
    point model puts the hit's turning angle psi = phi^Ax - phi0 below 0 at every sampled
    point of the cell."""
    rng = np.random.default_rng(82)
    g = G.make_grid([10] * 5, 4, 16)
    ev = chamber.single_track_events(4, seed=82, w=wires)
    n_refused = 0
    for e in range(ev.n_events):
        tp = ev.tracks[e][0].params
        for level in (1, 2, 3):
            ti = _true_idx(g, level, _reversed(tp) if level % 2 else tp)
            for _ in range(8):
                idx = [int(np.clip(ti[a] + rng.integers(-2, 3), 0, (g.bins[a] << level) - 1))
                       for a in range(5)]
                cell = O.cell12(g, level, idx)
                for wid in ev.wire_id[ev.offsets[e]:ev.offsets[e + 1]]:
                    v, outv = O.vote_pair(cell, O.hit9(wires, wid, 0.0), 0 | OUT)
                    if outv[4] != 2:
                        continue
                    assert v == 0
                    n_refused += 1
                    wire = (wires.x0[wid], wires.y0[wid], wires.sin_phis[wid],
                            wires.cos_phis[wid], wires.tan_tau[wid])
                    for _ in range(30):
                        pt = [rng.uniform(*g.cell_edges(level, a, idx[a])) for a in range(5)]
                        if pt[2] < 0:
                            pt, wire_m, _ = PM.mirror(pt, wire)
                        else:
                            wire_m = wire
                        q = PM.ax_quantities(pt, wire_m, pt[3])
                        psi = (q["phiA"] - pt[1] + np.pi) % (2 * np.pi) - np.pi
                        assert psi < 0, (e, level, idx, wid, psi)
    assert n_refused > 50


def test_key_layout_of_a_wide_axis(wires):
    g = G.make_grid([2, 256, 16, 2, 8], 5, 64)
    assert g.key_bits() == [10, 13, 10, 10, 10]
    tab = O.Tables(g, wires)
    rng = np.random.default_rng(83)
    idx = np.stack([rng.integers(0, int(g.bins[a]) << 4, 200) for a in range(5)], -1)
    keys = G.cell_key(idx, g)
    np.testing.assert_array_equal(G.key_indices(keys, g), idx)
    ch = G.key_indices(O.children(keys, tab), g).reshape(200, 32, 5)
    for b in range(32):
        np.testing.assert_array_equal(ch[:, b], 2 * idx + [(b >> a) & 1 for a in range(5)])
    # coarse keys in linear order are increasing (the key order is the linear order)
    ck = O.coarse_keys(tab)
    assert np.all(np.diff(ck.astype(np.float64)) > 0)
    np.testing.assert_array_equal(G.key_indices(ck, g),
                                  G.coarse_index_to_idx5(np.arange(g.n_coarse()), g.bins))


def _centres(g, level, keys):
    idx = G.key_indices(keys, g)
    lo = np.stack([g.cell_edges(level, a, idx[:, a])[0] for a in range(5)], -1)
    hi = np.stack([g.cell_edges(level, a, idx[:, a])[1] for a in range(5)], -1)
    return lo, hi


def test_maxset_matches_exhaustive_finest_votes(wires):
    """Tiny grid, every finest cell voted directly.  Keeping every group down to one vote
    loses nothing (a child never has more votes than its parent), so the final maximum
    group is exactly the exhaustive one; with slack 0 the final group is a subset of it
    whenever it reaches the same count."""
    g = G.make_grid([3, 4, 4, 3, 3], 2, 8)
    tab = O.Tables(g, wires)
    ev = chamber.single_track_events(3, seed=84, w=wires)
    fine = G.cell_key(np.stack(np.meshgrid(*[np.arange(int(b) << 2) for b in g.bins],
                                           indexing="ij"), -1).reshape(-1, 5), g)
    for e in range(ev.n_events):
        a, b = ev.offsets[e], ev.offsets[e + 1]
        wid, dr = ev.wire_id[a:b], ev.drift[a:b]
        direct = O.vote_cells(tab, wid, dr, 2, fine, OUT)
        vstar = int(direct.max())
        group = np.sort(fine[direct == vstar])
        prec = [OUT] * 3
        r = O.solve_event_maxset(tab, wid, dr, 10 ** 7, 300, prec, trace=True)
        assert r["final_level"] == 2 and r["votes"] == vstar and r["n_final"] == group.size
        lo, hi = _centres(g, 2, group)
        np.testing.assert_allclose(r["p"], lo.mean(0) * 0.5 + hi.mean(0) * 0.5, rtol=1e-11, atol=1e-15)
        np.testing.assert_array_equal(r["w"], (hi.max(0) - lo.min(0)) / 2)
        r0 = O.solve_event_maxset(tab, wid, dr, 10 ** 7, 0, prec, trace=True)
        assert r0["votes"] <= vstar
        if r0["votes"] == vstar:
            lo0, hi0 = _centres(g, 2, group)
            assert r0["n_final"] <= group.size


def test_maxset_whole_groups_and_true_cell(wires):
    """Every kept set is a union of whole vote groups, the largest allowed by max_keep and
    the slack; on noiseless events the true cell is kept at every level and the estimate's
    box holds the generated helix."""
    g = G.make_grid([2, 64, 8, 2, 4], 3, 64)
    tab = O.Tables(g, wires)
    ev = chamber.single_track_events(4, seed=85, w=wires, noiseless=True)
    keep, slack = 3000, 1
    for e in range(ev.n_events):
        a, b = ev.offsets[e], ev.offsets[e + 1]
        wid, dr = ev.wire_id[a:b], ev.drift[a:b]
        tp = ev.tracks[e][0].params
        prec = [1 | OUT, 1 | OUT, 0 | OUT, 0 | OUT]
        r = O.solve_event_maxset(tab, wid, dr, keep, slack, prec, trace=True)
        keys = O.coarse_keys(tab)
        for L in range(r["final_level"]):
            votes = O.vote_cells(tab, wid, dr, L, keys, prec[L])
            kk, kv = r["trace"][L]
            vmax = int(votes.max())
            T = int(kv.min())
            assert np.array_equal(np.sort(keys[votes >= T]), kk)
            assert len(kk) <= keep and T >= max(vmax - slack, 1)
            below = int(np.sum(votes == T - 1))
            assert T - 1 < max(vmax - slack, 1) or len(kk) + below > keep
            assert int(G.cell_key(np.array(_true_idx(g, L, tp)), g)) in set(kk.tolist())
            keys = O.children(kk, tab)
        assert np.all(np.abs(r["p"] - tp) <= r["w"]), (e, r["p"] - tp, r["w"])
        assert r["votes"] == b - a
