"""Seeded input generator: wire table, grid tables, events (host only)."""
import numpy as np

from gen import chamber, grid as G


def test_wire_table():
    w = chamber.make_wires()
    assert w.n == 1000
    radii = np.hypot(w.x0, w.y0)
    for i in range(10):
        sel = w.layer == i
        assert sel.sum() == 64 + 8 * i
        np.testing.assert_allclose(radii[sel], 0.20 + i * 0.5 / 9, rtol=0, atol=1e-15)
        assert np.all(np.sign(w.tan_tau[sel]) == (1 if i % 2 == 0 else -1))
    np.testing.assert_array_equal(w.sphi_t, w.sin_phis * w.tan_tau)
    np.testing.assert_array_equal(w.cphi_t, w.cos_phis * w.tan_tau)
    np.testing.assert_array_equal(w.t2, w.tan_tau * w.tan_tau)


def test_events_deterministic_and_in_range():
    w = chamber.make_wires()
    a = chamber.single_track_events(8, seed=3, w=w)
    b = chamber.single_track_events(8, seed=3, w=w)
    np.testing.assert_array_equal(a.wire_id, b.wire_id)
    np.testing.assert_array_equal(a.drift, b.drift)
    nh = np.diff(a.offsets)
    assert nh.min() >= 6 and nh.max() <= 30
    assert np.all(a.drift >= 0)
    for e in range(a.n_events):
        tr = a.tracks[e][0]
        assert 0.15 <= abs(tr.omega) <= 1.0 and abs(tr.d0) <= 0.01 and abs(tr.z0) <= 0.1
        for h in a.hit_truth[e]:
            assert h.dist < w.half_cell[h.wire]
            assert abs(h.z_wire) <= w.z_half_len
            assert abs(abs(h.d_signed) - h.dist) < 1e-12


def test_multitrack_events():
    w = chamber.make_wires()
    ev = chamber.multi_track_events(6, seed=4, w=w)
    nh = np.diff(ev.offsets)
    assert nh.min() >= 6 and nh.max() <= 200
    for e in range(ev.n_events):
        ids = ev.wire_id[ev.offsets[e]:ev.offsets[e + 1]]
        assert len(set(ids.tolist())) == len(ids)
        assert 1 <= len(ev.tracks[e]) <= 5


def test_grid_edges_and_nesting():
    g = G.make_grid([16] * 5, 6, 64)
    for a in range(5):
        lo, hi = g.lo_edge[a], g.hi_edge[a]
        assert np.all(hi > lo)
        if a != 2:
            np.testing.assert_array_equal(lo[1:], hi[:-1])
    # omega: no cell straddles 0
    assert np.all((g.hi_edge[2] < 0) | (g.lo_edge[2] > 0))
    # a cell's children tile it exactly
    for L in range(g.levels):
        for a in range(5):
            n = int(g.bins[a]) << L
            idx = np.arange(n)
            plo, phi = g.cell_edges(L, a, idx)
            c0lo, c0hi = g.cell_edges(L + 1, a, 2 * idx)
            c1lo, c1hi = g.cell_edges(L + 1, a, 2 * idx + 1)
            np.testing.assert_array_equal(plo, c0lo)
            np.testing.assert_array_equal(phi, c1hi)
            np.testing.assert_array_equal(c0hi, c1lo)


def test_sincos_table_encloses_and_nests():
    g = G.make_grid([16] * 5, 6, 64)
    for L in range(g.levels + 1):
        n = int(g.bins[1]) << L
        tab = g.sincos[g.sincos_offset[L]:g.sincos_offset[L] + n]
        a, b = g.cell_edges(L, 1, np.arange(n))
        x = a[:, None] + (b - a)[:, None] * np.linspace(0, 1, 33)[None, :]
        s, c = np.sin(x), np.cos(x)
        assert np.all(tab[:, 0:1] <= s) and np.all(s <= tab[:, 1:2])
        assert np.all(tab[:, 2:3] <= c) and np.all(c <= tab[:, 3:4])
        if L > 0:
            par = g.sincos[g.sincos_offset[L - 1] + (np.arange(n) >> 1)]
            assert np.all(tab[:, 0] >= par[:, 0]) and np.all(tab[:, 1] <= par[:, 1])
            assert np.all(tab[:, 2] >= par[:, 2]) and np.all(tab[:, 3] <= par[:, 3])


def test_key_round_trip_and_order():
    bins = np.array([16] * 5)
    lin = np.arange(16 ** 5, dtype=np.int64)[::997]
    idx = G.coarse_index_to_idx5(lin, bins)
    keys = G.cell_key(idx)
    np.testing.assert_array_equal(G.key_indices(keys), idx)
    assert np.all(np.diff(keys.astype(np.float64)) > 0)   # linear order == key order


def test_comet_toy_matches_the_paper_description():
    """The 20-layer toy (4,986 wires, 496-837 mm, +-0.1 rad stereo) and its electrons: from
    the origin, p = 105 MeV/c, less than one turn inside the chamber, reaching the third
    layer, 25 or more hits, drifts under 8 mm and equal to the true distance."""
    import numpy as np
    from gen import comet
    w = comet.make_wires()
    assert w.n == 4986 and len(set(w.layer.tolist())) == 20
    r = np.hypot(w.x0, w.y0)
    assert abs(r.min() - 0.496) < 1e-12 and abs(r.max() - 0.837) < 1e-12
    assert np.allclose(np.abs(np.arctan(w.tan_tau)), 0.1)
    ev = comet.events(40, seed=9, w=w)
    nh = np.diff(ev.offsets)
    assert nh.min() >= 25 and nh.max() <= 62
    lo, hi = comet.pt_range()
    for e in range(ev.n_events):
        tr = ev.tracks[e][0]
        pt = 0.3 * comet.B_TESLA / tr.omega
        assert lo - 1e-12 <= pt <= hi + 1e-12
        assert abs(np.hypot(pt, pt * tr.tanl) - comet.P_GEV) < 1e-12
        xc, yc, R = comet.helix_centre(tr)
        assert abs(np.hypot(xc, yc) - R) < 1e-12                  # the circle passes the origin
        assert 2 * np.pi * R * abs(tr.tanl) > comet.Z_HALF_LEN    # leaves within a turn
        for h in ev.hit_truth[e]:
            assert h.drift == h.dist < comet.MAX_DRIFT
