"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element by
element on the same seeded inputs.  Vote counts are integers and must be bit-exact; the
estimate is computed in the same order and rounding on both sides and must match exactly.
"""
import numpy as np
import pytest

from gen import chamber, grid as G
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2401_04576_gb300 import apo  # noqa: E402


@pytest.fixture(scope="module")
def wires():
    return chamber.make_wires()


@pytest.fixture(scope="module")
def grid1():
    return G.make_grid([10] * 5, 4, 16)        # 10^5 coarse cells, K = 16, 4 levels


@pytest.fixture(scope="module")
def grid2():
    return G.make_grid([16] * 5, 6, 64)        # 16^5 coarse cells, K = 64, 6 levels


@pytest.fixture(scope="module")
def ev1(wires):
    return chamber.single_track_events(6, seed=1, w=wires)


@pytest.fixture(scope="module")
def ev2(wires):
    return chamber.single_track_events(1024, seed=2, w=wires)


def _hits(ev):
    return apo.DeviceHits.from_events(ev)


@pytest.mark.parametrize("prec", [apo.F64, apo.F32, apo.F64_FILTERED])
def test_coarse_votes_bit_exact(wires, grid1, ev1, prec):
    geom = apo.Geometry(grid1, wires)
    sub = ev1.subset(range(3))
    got = apo.vote(geom, _hits(sub), precision=prec).cpu().numpy()
    tab = O.Tables(grid1, wires)
    oprec = 1 if prec == apo.F32 else 0
    for e in range(sub.n_events):
        a, b = sub.offsets[e], sub.offsets[e + 1]
        ref = O.vote_coarse(tab, sub.wire_id[a:b], sub.drift[a:b], oprec)
        np.testing.assert_array_equal(got[e], ref)


@pytest.mark.parametrize("prec", [apo.F64, apo.F32, apo.F64_FILTERED, apo.F64_EXACT])
def test_coarse_votes_ragged_grid(wires, prec):
    """Uneven bins (7 x 6 x 8 x 5 x 9): an odd number of (d0, z0) cells per tile, so the
    FP64 kernels' split of a tile over two blocks leaves one thread without a cell."""
    grid = G.make_grid([7, 6, 8, 5, 9], 3, 16)
    ev = chamber.single_track_events(3, seed=44, w=wires)
    geom = apo.Geometry(grid, wires)
    got = apo.vote(geom, _hits(ev), precision=prec).cpu().numpy()
    tab = O.Tables(grid, wires)
    oprec = {apo.F64: 0, apo.F64_FILTERED: 0, apo.F32: 1, apo.F64_EXACT: 4}[prec]
    for e in range(ev.n_events):
        a, b = ev.offsets[e], ev.offsets[e + 1]
        np.testing.assert_array_equal(got[e], O.vote_coarse(tab, ev.wire_id[a:b], ev.drift[a:b], oprec))


@pytest.mark.parametrize("prec", [apo.F64, apo.F32, apo.F64_FILTERED])
def test_cell_votes_every_level_bit_exact(wires, grid2, ev2, prec):
    """Random cells and cells around the true helix at every level 0..6."""
    geom = apo.Geometry(grid2, wires)
    sub = ev2.subset([0, 1, 2, 3])
    tab = O.Tables(grid2, wires)
    rng = np.random.default_rng(12)
    for L in range(grid2.levels + 1):
        keys = np.zeros((sub.n_events, 256), np.uint64)
        for e in range(sub.n_events):
            p = sub.tracks[e][0].params
            near = [int(np.searchsorted(grid2.lo_edge[a][::1 << (grid2.levels - L)], p[a],
                                        side="right") - 1) for a in range(5)]
            n = [int(grid2.bins[a]) << L for a in range(5)]
            idx = np.array([[min(max(near[a] + int(rng.integers(-2, 3)), 0), n[a] - 1)
                             for a in range(5)] for _ in range(128)] +
                           [[int(rng.integers(0, n[a])) for a in range(5)] for _ in range(128)])
            keys[e] = G.cell_key(idx)
        kt = torch.as_tensor(keys.view(np.int64), device="cuda")
        got = apo.vote(geom, _hits(sub), keys=kt, level=L, precision=prec).cpu().numpy()
        for e in range(sub.n_events):
            a, b = sub.offsets[e], sub.offsets[e + 1]
            ref = O.vote_cells(tab, sub.wire_id[a:b], sub.drift[a:b], L, keys[e],
                               1 if prec == apo.F32 else 0)
            np.testing.assert_array_equal(got[e], ref, err_msg=f"level {L} event {e}")


def _trace(geom, hits, grid, precision):
    ne, K, lv = hits.n_events, grid.topk, grid.levels
    tk = torch.zeros((ne, lv + 1, K), dtype=torch.int64, device="cuda")
    tv = torch.zeros((ne, lv + 1, K), dtype=torch.int32, device="cuda")
    o = apo.solve_opts(precision=precision, trace_keys=tk, trace_votes=tv)
    tracks, nt = apo.solve_batch(geom, hits, o)
    torch.cuda.synchronize()
    return (apo.tracks_to_numpy(tracks, ne), nt.cpu().numpy(), tk.cpu().numpy().view(np.uint64),
            tv.cpu().numpy())


def _compare_event(r, tr, tk, tv, grid):
    # level 0: same kept set (GPU keeps selection order, oracle sorts)
    ref0 = sorted(zip(r["trace_keys"][0].tolist(), r["trace_votes"][0].tolist()))
    got0 = sorted(zip(tk[0].tolist(), tv[0].tolist()))
    assert got0 == ref0
    for L in range(1, grid.levels):
        assert tk[L].tolist() == r["trace_keys"][L].tolist(), L
        assert tv[L].tolist() == r["trace_votes"][L].tolist(), L
    assert tr["votes"] == r["votes"]
    assert np.array_equal(tr["p"], r["p"]) and np.array_equal(tr["w"], r["w"])


@pytest.mark.parametrize("prec", [apo.F64, apo.F32])
def test_solve_small_grid_bit_exact(wires, grid1, ev1, prec):
    geom = apo.Geometry(grid1, wires)
    precision = [prec] * (grid1.levels + 1)
    tracks, nt, tk, tv = _trace(geom, _hits(ev1), grid1, precision)
    tab = O.Tables(grid1, wires)
    for e in range(ev1.n_events):
        a, b = ev1.offsets[e], ev1.offsets[e + 1]
        r = O.solve_event(tab, ev1.wire_id[a:b], ev1.drift[a:b], precision)
        _compare_event(r, tracks[e, 0], tk[e], tv[e], grid1)
        assert nt[e] == 1 and tracks[e, 0]["n_hits"] == b - a


def test_full_size_batch_sampled_events(wires, grid2, ev2):
    """The 1024-event, 16^5-cell, K = 64, 6-level FP64 batch in the launch configuration the
    benchmark times; three sampled events are recomputed whole by the oracle (coarse votes,
    every kept set, the estimate)."""
    geom = apo.Geometry(grid2, wires)
    hits = _hits(ev2)
    precision = [apo.F64] * (grid2.levels + 1)
    tracks, nt, tk, tv = _trace(geom, hits, grid2, precision)
    tab = O.Tables(grid2, wires)
    for e in (0, 511, 1023):
        a, b = ev2.offsets[e], ev2.offsets[e + 1]
        r = O.solve_event(tab, ev2.wire_id[a:b], ev2.drift[a:b], precision)
        _compare_event(r, tracks[e, 0], tk[e], tv[e], grid2)
    assert np.all(nt == 1)
    # full-grid votes of the same batch: sampled cells against the oracle one by one
    votes = apo.vote(geom, hits)
    rng = np.random.default_rng(13)
    evs = rng.integers(0, ev2.n_events, 24)
    for e in evs:
        lin = rng.integers(0, geom.n_coarse, 64)
        keys = G.cell_key(G.coarse_index_to_idx5(lin, grid2.bins))
        a, b = ev2.offsets[e], ev2.offsets[e + 1]
        ref = O.vote_cells(tab, ev2.wire_id[a:b], ev2.drift[a:b], 0, keys)
        got = votes[int(e)][torch.as_tensor(lin, device="cuda")].cpu().numpy()
        np.testing.assert_array_equal(got, ref)


def test_full_size_fp32_bulk_batch_sampled_events(wires, grid2, ev2):
    """The precision form at full size (1024 events, 16^5, K = 64, 6 levels; FP32 intervals
    on the coarse grid and levels 1-4, FP64 on levels 5-6) in the benchmark's launch
    configuration; three sampled events recomputed whole by the oracle in the same
    precisions (every kept set and the estimate)."""
    geom = apo.Geometry(grid2, wires)
    precision = [apo.F32] * 5 + [apo.F64] * 2
    tracks, nt, tk, tv = _trace(geom, _hits(ev2), grid2, precision)
    tab = O.Tables(grid2, wires)
    for e in (3, 600, 1020):
        a, b = ev2.offsets[e], ev2.offsets[e + 1]
        r = O.solve_event(tab, ev2.wire_id[a:b], ev2.drift[a:b], [1] * 5 + [0] * 2)
        _compare_event(r, tracks[e, 0], tk[e], tv[e], grid2)
    assert np.all(nt == 1)


def test_fp32_votes_contain_fp64_votes(wires, grid2, ev2):
    """Full-grid votes of 8 config-2 events: FP32 >= FP64 cell by cell, and the filtered
    and unfiltered FP64 kernels agree exactly."""
    geom = apo.Geometry(grid2, wires)
    sub = ev2.subset(range(8))
    h = _hits(sub)
    v64 = apo.vote(geom, h, precision=apo.F64)
    v64u = apo.vote(geom, h, precision=apo.F64_FILTERED)
    v32 = apo.vote(geom, h, precision=apo.F32)
    assert bool(torch.all(v32 >= v64))
    assert bool(torch.equal(v64, v64u))


def test_edge_cases(wires, grid1):
    geom = apo.Geometry(grid1, wires)
    tab = O.Tables(grid1, wires)
    rng = np.random.default_rng(14)
    # empty batch
    empty = apo.DeviceHits(torch.zeros(1, dtype=torch.int32, device="cuda"),
                           torch.zeros(0, dtype=torch.int32, device="cuda"),
                           torch.zeros(0, dtype=torch.float64, device="cuda"))
    apo.solve_batch(geom, empty)
    # events: 0 hits, 256 hits (the cap), 257 hits, bad wire id, negative drift, NaN drift, ok
    sizes = [0, 256, 257, 5, 5, 5, 7]
    wid, dr, offs = [], [], [0]
    for i, n in enumerate(sizes):
        w_ = rng.choice(wires.n, size=n, replace=n > wires.n).astype(np.int32)
        d_ = rng.uniform(0, 0.008, n)
        if i == 3:
            w_[2] = wires.n + 5
        if i == 4:
            d_[1] = -1e-3
        if i == 5:
            d_[0] = np.nan
        wid.append(w_)
        dr.append(d_)
        offs.append(offs[-1] + n)
    ev = chamber.Events(offsets=np.array(offs, np.int32), wire_id=np.concatenate(wid),
                        drift=np.concatenate(dr))
    tracks, nt = apo.solve_batch(geom, _hits(ev))
    t = apo.tracks_to_numpy(tracks, ev.n_events)[:, 0]
    nt = nt.cpu().numpy()
    for i in (2, 3, 4, 5):
        assert t[i]["votes"] == apo.APO_EINVAL and nt[i] == 0, i
    assert nt[0] == 0 and t[0]["votes"] == 0            # no hit: no track
    for i in (1, 6):
        a, b = offs[i], offs[i + 1]
        r = O.solve_event(tab, ev.wire_id[a:b], ev.drift[a:b])
        assert t[i]["votes"] == r["votes"] and nt[i] == 1, i
        assert np.array_equal(t[i]["p"], r["p"]) and np.array_equal(t[i]["w"], r["w"]), i


def test_host_entry_matches_device_entry(wires, grid1, ev1):
    geom = apo.Geometry(grid1, wires)
    tr_d, _ = apo.solve_batch(geom, _hits(ev1))
    t_d = apo.tracks_to_numpy(tr_d, ev1.n_events)
    t_h, nt = apo.solve_batch_host(geom, ev1.offsets, ev1.wire_id, ev1.drift)
    assert np.array_equal(t_d.view(np.uint8), t_h.view(np.uint8))
    assert np.all(nt == 1)


def test_refine_matches_oracle(wires, grid1, ev1):
    geom = apo.Geometry(grid1, wires)
    sub = ev1.subset(range(2))
    h = _hits(sub)
    votes = apo.vote(geom, h)
    kk, kv, ch = apo.refine(geom, h, votes)
    tab = O.Tables(grid1, wires)
    kk, kv, ch = (x.cpu().numpy() for x in (kk, kv, ch))
    for e in range(sub.n_events):
        a, b = sub.offsets[e], sub.offsets[e + 1]
        keys = O.coarse_keys(tab)
        ref_v = O.vote_cells(tab, sub.wire_id[a:b], sub.drift[a:b], 0, keys)
        rk, rv = O.topk(keys, ref_v, grid1.topk)
        assert sorted(zip(kk[e].view(np.uint64).tolist(), kv[e].tolist())) == \
            sorted(zip(rk.tolist(), rv.tolist()))
        np.testing.assert_array_equal(np.sort(ch[e].view(np.uint64)), np.sort(O.children(rk)))


def _multi(geom, ev, grid, precision, max_tracks, min_votes):
    ht = torch.full((int(ev.offsets[-1]),), 7, dtype=torch.int32, device="cuda")
    o = apo.solve_opts(precision=precision, max_tracks=max_tracks, min_votes=min_votes,
                       hit_track=ht)
    tracks, nt = apo.solve_batch(geom, _hits(ev), o)
    torch.cuda.synchronize()
    return apo.tracks_to_numpy(tracks, ev.n_events, max_tracks), nt.cpu().numpy(), ht.cpu().numpy()


def _compare_multi(tab, ev, e, t, nt, ht, precision, max_tracks, min_votes):
    a, b = ev.offsets[e], ev.offsets[e + 1]
    r = O.solve_event_multi(tab, ev.wire_id[a:b], ev.drift[a:b], max_tracks, min_votes,
                            prec_per_level=precision)
    assert nt[e] == r["n_tracks"], (e, nt[e], r["n_tracks"])
    for k in range(r["n_tracks"]):
        assert t[e, k]["votes"] == r["votes"][k], (e, k)
        assert np.array_equal(t[e, k]["p"], r["p"][k]) and np.array_equal(t[e, k]["w"], r["w"][k])
    # which track took each hit (the hit finding of Section 3.3), -1 for none
    np.testing.assert_array_equal(ht[a:b], r["hit_track"], err_msg=f"event {e}")


@pytest.mark.parametrize("mixed", [False, True])
def test_multi_track_small_grid_bit_exact(wires, mixed):
    """Multi-track extraction with hit masking (1-5 helices + noise per event): number of
    tracks, every track's estimate and votes against the oracle."""
    g = G.make_grid([8] * 5, 3, 16)
    geom = apo.Geometry(g, wires)
    ev = chamber.multi_track_events(6, seed=41, w=wires)
    precision = ([apo.F32] * 2 + [apo.F64] * 2) if mixed else [apo.F64] * 4
    t, nt, ht = _multi(geom, ev, g, precision, 5, 6)
    tab = O.Tables(g, wires)
    for e in range(ev.n_events):
        _compare_multi(tab, ev, e, t, nt, ht, precision, 5, 6)
    assert nt.sum() > ev.n_events
    assert (ht >= 0).any() and (ht < 0).any()


def test_multi_track_full_size_sampled(wires):
    """4096 uneven events (1-5 tracks + 10-30 % noise, up to 200 hits), 10^5 coarse cells,
    top-64, 6 levels, FP32 levels 0-4 and FP64 levels 5-6, at most 5 tracks: two sampled
    events recomputed whole by the oracle."""
    g = G.make_grid([10] * 5, 6, 64)
    geom = apo.Geometry(g, wires)
    ev = chamber.multi_track_events(4096, seed=4, w=wires)
    precision = [apo.F32] * 5 + [apo.F64] * 2
    t, nt, ht = _multi(geom, ev, g, precision, 5, 6)
    tab = O.Tables(g, wires)
    for e in (7, 3000):
        _compare_multi(tab, ev, e, t, nt, ht, precision, 5, 6)
    assert np.all((nt >= 0) & (nt <= 5))


def test_graph_replay_and_tuning_knobs_do_not_change_results(wires):
    """Recording the search as a CUDA graph and replaying it, and every execution knob the
    autotuner chooses from, give the same tracks bit for bit; a replay sees new contents
    of the same input buffers."""
    g = G.make_grid([8] * 5, 3, 16)
    geom = apo.Geometry(g, wires)
    ev = chamber.multi_track_events(40, seed=43, w=wires)
    hits = _hits(ev)
    ws = geom.workspace(ev.n_events)
    prec = [apo.F32, apo.F32, apo.F64, apo.F64]

    def run(**kw):
        o = apo.solve_opts(precision=prec, max_tracks=4, min_votes=6, **kw)
        tr, nt = apo.solve_batch(geom, hits, o, workspace=ws)
        torch.cuda.synchronize()
        return tr.cpu().numpy().copy(), nt.cpu().numpy().copy()

    ref_t, ref_n = run()
    assert ref_n.sum() > ev.n_events
    for cf in (0, 1):
        for lf in (0, 1):
            for bs in (128, 256):
                for ch in (0, 7):
                    for full in (0, 1):   # level 0: block candidates or every vote
                        t, n = run(tune=apo.ApoTune(cf, lf, bs, ch, full))
                        assert np.array_equal(t, ref_t) and np.array_equal(n, ref_n), (cf, lf, bs, ch, full)
    o = apo.solve_opts(precision=prec, max_tracks=4, min_votes=6, use_graph=True)
    tracks = torch.zeros(ev.n_events * 4 * apo.TRACK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    ntr = torch.zeros(ev.n_events, dtype=torch.int32, device="cuda")
    for _ in range(2):                        # first call records, second replays
        tracks.zero_()
        apo.solve_batch(geom, hits, o, tracks=tracks, n_tracks=ntr, workspace=ws)
        torch.cuda.synchronize()
        assert np.array_equal(tracks.cpu().numpy(), ref_t) and np.array_equal(ntr.cpu().numpy(), ref_n)
    # new drift values in the same buffer: the replay must follow them
    hits.drift.mul_(0.5)
    apo.solve_batch(geom, hits, o, tracks=tracks, n_tracks=ntr, workspace=ws)
    t_g = tracks.cpu().numpy().copy()
    apo.solve_batch(geom, hits, apo.solve_opts(precision=prec, max_tracks=4, min_votes=6),
                    tracks=tracks, n_tracks=ntr, workspace=ws)
    torch.cuda.synchronize()
    assert np.array_equal(t_g, tracks.cpu().numpy())
    best, ms = apo.autotune(geom, hits, apo.solve_opts(precision=prec, max_tracks=4, min_votes=6),
                            workspace=ws)
    assert ms > 0 and best.cells_block in (128, 256)
