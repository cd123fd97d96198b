"""GPU parity of the direction condition (APO_OUTGOING) and the max-set schedule
(APO_SCHED_MAXSET) against the CPU oracle, through the C ABI.  Votes, kept sets, counts and
levels are integers and must be bit-exact; the estimate is summed in the same order and
rounding on both sides and must match exactly."""
import numpy as np
import pytest

from gen import chamber, grid as G
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2401_04576_gb300 import apo  # noqa: E402

OUT = apo.OUTGOING


@pytest.fixture(scope="module")
def wires():
    return chamber.make_wires()


def _hits(ev):
    return apo.DeviceHits.from_events(ev)


def _true_idx(g, level, params):
    idx = []
    for a in range(5):
        n = int(g.bins[a]) << level
        lo, hi = g.cell_edges(level, a, np.arange(n))
        j = np.nonzero((lo <= params[a]) & (params[a] <= hi))[0]
        idx.append(int(j[0]) if j.size else 0)
    return np.array(idx)


@pytest.mark.parametrize("prec", [apo.F64 | OUT, apo.F32 | OUT, apo.F64_FILTERED | OUT,
                                  apo.F64_EXACT | OUT])
def test_direction_coarse_votes_bit_exact(wires, prec):
    g = G.make_grid([10] * 5, 4, 16)
    geom = apo.Geometry(g, wires)
    ev = chamber.single_track_events(3, seed=91, w=wires)
    got = apo.vote(geom, _hits(ev), precision=prec).cpu().numpy()
    tab = O.Tables(g, wires)
    base = prec & ~OUT
    oprec = {apo.F64: 0, apo.F32: 1, apo.F64_FILTERED: 0, apo.F64_EXACT: 4}[base] | O.OUTGOING
    plain = apo.vote(geom, _hits(ev), precision=base).cpu().numpy()
    for e in range(ev.n_events):
        a, b = ev.offsets[e], ev.offsets[e + 1]
        ref = O.vote_coarse(tab, ev.wire_id[a:b], ev.drift[a:b], oprec)
        np.testing.assert_array_equal(got[e], ref)
        assert np.all(got[e] <= plain[e]) and got[e].sum() < plain[e].sum()


@pytest.mark.parametrize("prec", [apo.F64 | OUT, apo.F32 | OUT])
def test_direction_cells_and_pair_ends_bit_exact(wires, prec):
    """Explicit keys at every level of an anisotropic grid with a 13-bit phi0 axis, near the
    helix and its reversed twin, and the program's end points pair by pair."""
    g = G.make_grid([2, 256, 16, 2, 8], 5, 64)
    geom = apo.Geometry(g, wires)
    tab = O.Tables(g, wires)
    ev = chamber.single_track_events(2, seed=92, w=wires)
    rng = np.random.default_rng(92)
    oprec = (0 if prec & ~OUT == apo.F64 else 1) | O.OUTGOING
    cells, hits9, ref = [], [], []
    for level in range(6):
        keys = np.zeros((ev.n_events, 96), np.uint64)
        for e in range(ev.n_events):
            tp = ev.tracks[e][0].params
            rev = np.array([-tp[0], (tp[1] + np.pi) % (2 * np.pi), -tp[2], tp[3], -tp[4]])
            for j in range(96):
                c = _true_idx(g, level, tp if j % 2 == 0 else rev)
                c = np.clip(c + rng.integers(-2, 3, 5), 0, (g.bins.astype(np.int64) << level) - 1)
                keys[e, j] = G.cell_key(c, g)
                if j < 8:
                    for wid in ev.wire_id[ev.offsets[e]:ev.offsets[e + 1]][:4]:
                        cells.append(O.cell12(g, level, c))
                        hits9.append(O.hit9(wires, wid, ev.drift[ev.offsets[e]]))
                        v, o = O.vote_pair(cells[-1], hits9[-1], oprec)
                        ref.append(np.concatenate([[v], o]))
        got = apo.vote(geom, _hits(ev), keys=torch.as_tensor(keys.view(np.int64), device="cuda"),
                       level=level, precision=prec).cpu().numpy()
        for e in range(ev.n_events):
            a, b = ev.offsets[e], ev.offsets[e + 1]
            np.testing.assert_array_equal(
                got[e], O.vote_cells(tab, ev.wire_id[a:b], ev.drift[a:b], level, keys[e], oprec))
    out = apo.vote_pair_ends(geom, torch.as_tensor(np.array(cells), device="cuda"),
                             torch.as_tensor(np.array(hits9), device="cuda"), precision=prec)
    np.testing.assert_array_equal(out.cpu().numpy(), np.array(ref))
    assert np.any(np.array(ref)[:, 5] == 2)          # some pairs refused by the direction


def _maxset_opts(levels, prec, keep, slack, ne, **kw):
    fl = torch.zeros(ne, dtype=torch.int32, device="cuda")
    nf = torch.zeros(ne, dtype=torch.int32, device="cuda")
    tc = torch.zeros(ne * (levels + 1), dtype=torch.int32, device="cuda")
    tk = torch.zeros(ne * (levels + 1) * keep, dtype=torch.int64, device="cuda")
    tv = torch.zeros(ne * (levels + 1) * keep, dtype=torch.int32, device="cuda")
    o = apo.solve_opts(precision=prec, schedule=apo.SCHED_MAXSET, max_keep=keep, slack=slack,
                       final_level=fl, n_final=nf, trace_count=tc, trace_keys=tk, trace_votes=tv,
                       **kw)
    return o, (fl, nf, tc, tk, tv)


def _check_against_oracle(g, tab, ev, events, tracks, outs, prec, keep, slack):
    fl, nf, tc, tk, tv = (x.cpu().numpy() for x in outs)
    lv = g.levels
    tc = tc.reshape(-1, lv + 1)
    tk = tk.view(np.uint64).reshape(-1, lv + 1, keep)
    tv = tv.reshape(-1, lv + 1, keep)
    t = apo.tracks_to_numpy(tracks, ev.n_events)[:, 0]
    oprec = [(1 if (p & ~OUT) == apo.F32 else 0) | (O.OUTGOING if p & OUT else 0) for p in prec]
    for e in events:
        a, b = ev.offsets[e], ev.offsets[e + 1]
        r = O.solve_event_maxset(tab, ev.wire_id[a:b], ev.drift[a:b], keep, slack, oprec, trace=True)
        assert fl[e] == r["final_level"] and nf[e] == r["n_final"] and t[e]["votes"] == r["votes"], e
        assert np.array_equal(t[e]["p"], r["p"]) and np.array_equal(t[e]["w"], r["w"]), \
            (e, t[e]["p"] - r["p"], t[e]["w"] - r["w"])
        for L in range(r["final_level"]):
            rk, rv = r["trace"][L]
            assert tc[e, L] == len(rk), (e, L)
            o = np.argsort(tk[e, L, :tc[e, L]])
            np.testing.assert_array_equal(tk[e, L, :tc[e, L]][o], rk)
            np.testing.assert_array_equal(tv[e, L, :tc[e, L]][o], rv)


@pytest.mark.parametrize("slack,keep", [(0, 3000), (1, 3000), (2, 40)])
def test_maxset_search_bit_exact(wires, slack, keep):
    g = G.make_grid([2, 64, 8, 2, 4], 3, 64)
    tab = O.Tables(g, wires)
    geom = apo.Geometry(g, wires)
    ev = chamber.single_track_events(6, seed=93, w=wires)
    prec = [apo.F32 | OUT, apo.F32 | OUT, apo.F64 | OUT, apo.F64 | OUT]
    o, outs = _maxset_opts(3, prec, keep, slack, ev.n_events)
    tracks, nt = apo.solve_batch(geom, _hits(ev), o)
    torch.cuda.synchronize()
    assert np.all(nt.cpu().numpy() == 1)
    _check_against_oracle(g, tab, ev, range(ev.n_events), tracks, outs, prec, keep, slack)
    if keep == 40:   # some events stop early because their vmax group overflows
        assert np.any(outs[0].cpu().numpy() < 3)


def test_maxset_chunks_graph_and_plain_fp64(wires):
    """Chunking and graph replay change nothing; the all-FP64 schedule matches the oracle
    too, and a malformed event is reported without stopping the batch."""
    g = G.make_grid([2, 64, 8, 2, 4], 3, 64)
    tab = O.Tables(g, wires)
    geom = apo.Geometry(g, wires)
    ev = chamber.single_track_events(5, seed=94, w=wires)
    dr = ev.drift.copy()
    dr[ev.offsets[2]] = -1.0                        # event 2 is malformed
    bad = chamber.Events(offsets=ev.offsets, wire_id=ev.wire_id, drift=dr, tracks=ev.tracks)
    prec = [apo.F64 | OUT] * 4
    o, outs = _maxset_opts(3, prec, 2000, 0, ev.n_events)
    tracks, nt = apo.solve_batch(geom, _hits(bad), o)
    torch.cuda.synchronize()
    t = apo.tracks_to_numpy(tracks, ev.n_events)[:, 0]
    assert t[2]["votes"] == apo.APO_EINVAL and nt.cpu().numpy()[2] == 0
    _check_against_oracle(g, tab, bad, [0, 1, 3, 4], tracks, outs, prec, 2000, 0)
    ref = t.copy()
    tune = apo.ApoTune(0, 1, 128, 2)
    o2 = apo.solve_opts(precision=prec, schedule=apo.SCHED_MAXSET, max_keep=2000, tune=tune,
                        use_graph=True)
    for _ in range(2):
        tr2, _ = apo.solve_batch(geom, _hits(bad), o2)
        torch.cuda.synchronize()
        assert np.array_equal(apo.tracks_to_numpy(tr2, ev.n_events)[:, 0].view(np.uint8),
                              ref.view(np.uint8))


def test_maxset_full_batch_sampled(wires):
    """The benchmark's max-set workload in its launch configuration: 1024 events, the
    2 x 256 x 16 x 2 x 8 grid, 5 levels, FP32 levels 0-3 and FP64 levels 4-5, direction
    condition, max_keep 32768; three events recomputed whole by the oracle."""
    g = G.make_grid([2, 256, 16, 2, 8], 5, 64)
    tab = O.Tables(g, wires)
    geom = apo.Geometry(g, wires)
    ev = chamber.single_track_events(1024, seed=2, w=wires)
    prec = [apo.F32 | OUT] * 4 + [apo.F64 | OUT] * 2
    keep = 32768
    fl = torch.zeros(ev.n_events, dtype=torch.int32, device="cuda")
    nf = torch.zeros(ev.n_events, dtype=torch.int32, device="cuda")
    o = apo.solve_opts(precision=prec, schedule=apo.SCHED_MAXSET, max_keep=keep, final_level=fl,
                       n_final=nf)
    tracks, nt = apo.solve_batch(geom, _hits(ev), o)
    torch.cuda.synchronize()
    t = apo.tracks_to_numpy(tracks, ev.n_events)[:, 0]
    fl, nf = fl.cpu().numpy(), nf.cpu().numpy()
    oprec = [1 | O.OUTGOING] * 4 + [0 | O.OUTGOING] * 2
    for e in (0, 511, 1023):
        a, b = ev.offsets[e], ev.offsets[e + 1]
        r = O.solve_event_maxset(tab, ev.wire_id[a:b], ev.drift[a:b], keep, 0, oprec)
        assert fl[e] == r["final_level"] and nf[e] == r["n_final"] and t[e]["votes"] == r["votes"]
        assert np.array_equal(t[e]["p"], r["p"]) and np.array_equal(t[e]["w"], r["w"]), e
    # the estimate's box holds the generated helix in nearly every event
    truth = np.array([tr[0].params for tr in ev.tracks])
    inside = np.all(np.abs(t["p"] - truth) <= t["w"], axis=1)
    assert inside.mean() >= 0.95, inside.mean()


def _tied_event(w, rng):
    """Two noiseless tracks with equal hit counts on disjoint wires (phi0 >= 1 rad apart)."""
    while True:
        a, b = chamber.draw_track(rng), chamber.draw_track(rng)
        ha, hb = chamber.simulate_track(a, w, None), chamber.simulate_track(b, w, None)
        dphi = abs((a.params[1] - b.params[1] + np.pi) % (2 * np.pi) - np.pi)
        if len(ha) == len(hb) >= 8 and dphi > 1.0 and not ({h.wire for h in ha} & {h.wire for h in hb}):
            items = sorted([(h.wire, h.drift) for h in ha + hb])
            return [i[0] for i in items], [i[1] for i in items]


def _multi_batch(w, n_multi, seed):
    ev = chamber.multi_track_events(n_multi, seed=seed, w=w)
    wid, dr, off = list(ev.wire_id), list(ev.drift), list(ev.offsets)
    rng = np.random.default_rng(seed)
    for _ in range(2):   # two events of two tied tracks
        a, b = _tied_event(w, rng)
        wid += a
        dr += b
        off.append(off[-1] + len(a))
    return chamber.Events(offsets=np.array(off, np.int32), wire_id=np.array(wid, np.int32),
                          drift=np.array(dr))


def _multi_opts(prec, keep, slack, mt, ne, nhits, **kw):
    fl = torch.full((ne * mt,), -7, dtype=torch.int32, device="cuda")
    nf = torch.full((ne * mt,), -7, dtype=torch.int32, device="cuda")
    ht = torch.full((max(nhits, 1),), -5, dtype=torch.int32, device="cuda")
    o = apo.solve_opts(precision=prec, schedule=apo.SCHED_MAXSET, max_keep=keep, slack=slack,
                       max_tracks=mt, min_votes=6, final_level=fl, n_final=nf, hit_track=ht, **kw)
    return o, (fl, nf, ht)


def _check_multi(tab, ev, events, tracks, nt, outs, prec, keep, slack, mt):
    fl, nf, ht = (x.cpu().numpy() for x in outs)
    t = apo.tracks_to_numpy(tracks, ev.n_events, mt)
    nt = nt.cpu().numpy()
    oprec = [(1 if (p & ~OUT) == apo.F32 else 0) | (O.OUTGOING if p & OUT else 0) for p in prec]
    n_found = 0
    for e in events:
        a, b = ev.offsets[e], ev.offsets[e + 1]
        r = O.solve_event_maxset_multi(tab, ev.wire_id[a:b], ev.drift[a:b], keep, mt, 6, slack=slack,
                                       prec_per_level=oprec)
        assert nt[e] == r["n_tracks"], (e, nt[e], r["n_tracks"])
        for k in range(r["n_tracks"]):
            assert t[e, k]["votes"] == r["votes"][k], (e, k)
            assert fl[e * mt + k] == r["final_level"][k] and nf[e * mt + k] == r["n_final"][k], (e, k)
            assert np.array_equal(t[e, k]["p"], r["p"][k]) and np.array_equal(t[e, k]["w"], r["w"][k]), (e, k)
        np.testing.assert_array_equal(ht[a:b], r["hit_track"])
        n_found += r["n_tracks"]
    return n_found


@pytest.mark.parametrize("tune", [apo.ApoTune(0, 1, 256, 0), apo.ApoTune(0, 0, 128, 3)])
def test_maxset_multi_track_bit_exact(wires, tune):
    """Multi-track rounds (one hit-set cluster of the final group per round): tracks, final
    levels, cluster sizes and every hit's track equal to the oracle, on config-4-like
    events and on two events of two tied noiseless tracks, which must come out as two."""
    g = G.make_grid([2, 64, 8, 2, 4], 3, 64)
    tab = O.Tables(g, wires)
    geom = apo.Geometry(g, wires)
    ev = _multi_batch(wires, 6, 96)
    prec = [apo.F32 | OUT, apo.F32 | OUT, apo.F64 | OUT, apo.F64 | OUT]
    mt = 4
    o, outs = _multi_opts(prec, 3000, 2, mt, ev.n_events, int(ev.offsets[-1]), tune=tune)
    tracks, nt = apo.solve_batch(geom, _hits(ev), o)
    torch.cuda.synchronize()
    assert _check_multi(tab, ev, range(ev.n_events), tracks, nt, outs, prec, 3000, 2, mt) >= 8
    assert np.all(nt.cpu().numpy()[-2:] == 2)


def test_maxset_multi_track_config4_sampled(wires):
    """The multi-track workload in the benchmark's form: config-4 events (1-5 tracks, 10-30 %
    noise), the 2 x 256 x 16 x 2 x 8 grid, 5 levels, FP32 levels 0-3 / FP64 4-5 with the
    direction condition, max_keep 32768, slack 2, up to 5 tracks, min 6 votes; 256 events,
    the two with the fewest hits recomputed whole by the oracle; most true tracks found."""
    g = G.make_grid([2, 256, 16, 2, 8], 5, 64)
    tab = O.Tables(g, wires)
    geom = apo.Geometry(g, wires)
    ev = chamber.multi_track_events(256, seed=4, w=wires)
    prec = [apo.F32 | OUT] * 4 + [apo.F64 | OUT] * 2
    o, outs = _multi_opts(prec, 32768, 2, 5, ev.n_events, int(ev.offsets[-1]))
    tracks, nt = apo.solve_batch(geom, _hits(ev), o)
    torch.cuda.synchronize()
    small = np.argsort(np.diff(ev.offsets), kind="stable")[:2]
    _check_multi(tab, ev, small, tracks, nt, outs, prec, 32768, 2, 5)
    t = apo.tracks_to_numpy(tracks, ev.n_events, 5)
    nt = nt.cpu().numpy()
    found = true = 0
    for e in range(ev.n_events):
        truth = np.array([tr.params for tr in ev.tracks[e]])
        true += len(truth)
        hit = np.zeros(len(truth), bool)
        for k in range(nt[e]):
            hit |= np.all(np.abs(t[e, k]["p"] - truth) <= t[e, k]["w"], axis=1)
        found += int(hit.sum())
    assert found >= 0.6 * true, (found, true)


def test_maxset_multi_track_edges_chunks_and_graph(wires):
    """Multi-track rounds with an empty event, a malformed event and an event whose hits
    cannot reach min_votes in one batch, processed in chunks of 3 events and replayed from
    a CUDA graph: every other event equal to the oracle, the malformed one flagged with no
    track, and chunking and replay change nothing."""
    g = G.make_grid([2, 64, 8, 2, 4], 3, 64)
    tab = O.Tables(g, wires)
    geom = apo.Geometry(g, wires)
    base = chamber.multi_track_events(5, seed=97, w=wires)
    wid, dr, off = list(base.wire_id), list(base.drift), list(base.offsets)
    off.append(off[-1])                                   # event 5: no hit
    few = chamber.single_track_events(1, seed=98, w=wires)
    wid += list(few.wire_id[:4]); dr += list(few.drift[:4]); off.append(off[-1] + 4)   # event 6: 4 hits
    bad_at = len(wid)
    wid += list(few.wire_id); dr += list(few.drift); off.append(off[-1] + len(few.wire_id))  # event 7
    dr[bad_at + 1] = -2.0                                 # malformed
    ev = chamber.Events(offsets=np.array(off, np.int32), wire_id=np.array(wid, np.int32), drift=np.array(dr))
    prec = [apo.F32 | OUT, apo.F32 | OUT, apo.F64 | OUT, apo.F64 | OUT]
    mt = 3
    runs = []
    for tune, graph in ((apo.ApoTune(0, 1, 256, 0), False), (apo.ApoTune(0, 1, 256, 3), False),
                        (apo.ApoTune(0, 1, 128, 3), True)):
        o, outs = _multi_opts(prec, 2000, 2, mt, ev.n_events, int(ev.offsets[-1]), tune=tune, use_graph=graph)
        for _ in range(2 if graph else 1):
            tracks, nt = apo.solve_batch(geom, _hits(ev), o)
            torch.cuda.synchronize()
        runs.append((apo.tracks_to_numpy(tracks, ev.n_events, mt), nt.cpu().numpy(),
                     [x.cpu().numpy() for x in outs]))
    for r in runs[1:]:
        assert np.array_equal(r[0].view(np.uint8), runs[0][0].view(np.uint8))
        assert np.array_equal(r[1], runs[0][1])
        for a, b in zip(r[2], runs[0][2]):
            np.testing.assert_array_equal(a, b)
    t, nt, (fl, nf, ht) = runs[0]
    assert t[7, 0]["votes"] == apo.APO_EINVAL and nt[7] == 0
    assert np.all(ht[off[7]:off[8]] == -1)
    assert nt[5] == 0 and nt[6] == 0
    o2, outs2 = _multi_opts(prec, 2000, 2, mt, ev.n_events, int(ev.offsets[-1]), tune=apo.ApoTune(0, 1, 256, 3))
    tr2, nt2 = apo.solve_batch(geom, _hits(ev), o2)
    torch.cuda.synchronize()
    _check_multi(tab, ev, [0, 1, 2, 3, 4, 5, 6], tr2, nt2, outs2, prec, 2000, 2, mt)
