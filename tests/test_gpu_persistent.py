"""The persistent batch launch (apo_tune.persistent): one launch whose blocks pull events
from a device counter and run each event's whole search.  It must give exactly what the
per-level launches give (and so what the oracle gives), track by track and hit by hit,
on single-track batches and on the full 4096-event multi-track batch."""
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


def _solve(geom, ev, prec, persistent, cells_filter=1, **kw):
    ne = ev.n_events
    ht = torch.full((max(int(ev.offsets[-1]), 1),), -5, dtype=torch.int32, device="cuda")
    o = apo.solve_opts(precision=prec, hit_track=ht, tune=apo.ApoTune(0, cells_filter, 256, 0, persistent=persistent), **kw)
    tr, nt = apo.solve_batch(geom, apo.DeviceHits.from_events(ev), o)
    torch.cuda.synchronize()
    mt = int(o.max_tracks)
    return apo.tracks_to_numpy(tr, ne, mt), nt.cpu().numpy(), ht.cpu().numpy()[:int(ev.offsets[-1])]


@pytest.mark.parametrize("prec", [[apo.F64] * 5, [apo.F32] * 3 + [apo.F64] * 2,
                                  [apo.F32 | apo.OUTGOING] * 5])
def test_persistent_single_track_equals_per_level_launches(wires, prec):
    g = G.make_grid([10] * 5, 4, 16)
    geom = apo.Geometry(g, wires)
    ev = chamber.single_track_events(40, seed=101, w=wires)
    for cf in (0, 1):
        a = _solve(geom, ev, prec, 0, cf)
        b = _solve(geom, ev, prec, 1, cf)
        assert np.array_equal(a[0].view(np.uint8), b[0].view(np.uint8))
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    tab = O.Tables(g, wires)
    oprec = [(1 if (p & ~apo.OUTGOING) == apo.F32 else 0) | (O.OUTGOING if p & apo.OUTGOING else 0)
             for p in prec]
    for e in (0, 39):
        x, y = ev.offsets[e], ev.offsets[e + 1]
        r = O.solve_event(tab, ev.wire_id[x:y], ev.drift[x:y], oprec)
        assert b[0][e, 0]["votes"] == r["votes"]
        assert np.array_equal(b[0][e, 0]["p"], r["p"]) and np.array_equal(b[0][e, 0]["w"], r["w"])


def test_persistent_multi_track_full_batch(wires):
    """The 4096-event multi-track batch (10^5 grid, top-64, 6 levels, FP32 levels 0-4 and
    FP64 5-6, up to 5 tracks, min 6 votes): every track, count and hit assignment equal to
    the per-level launches; two events recomputed whole by the oracle."""
    g = G.make_grid([10] * 5, 6, 64)
    geom = apo.Geometry(g, wires)
    ev = chamber.multi_track_events(4096, seed=4, w=wires)
    prec = [apo.F32] * 5 + [apo.F64] * 2
    a = _solve(geom, ev, prec, 0, max_tracks=5, min_votes=6)
    b = _solve(geom, ev, prec, 1, max_tracks=5, min_votes=6)
    assert np.array_equal(a[0].view(np.uint8), b[0].view(np.uint8))
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    tab = O.Tables(g, wires)
    for e in (7, 4000):
        x, y = ev.offsets[e], ev.offsets[e + 1]
        r = O.solve_event_multi(tab, ev.wire_id[x:y], ev.drift[x:y], 5, 6, prec_per_level=[1] * 5 + [0] * 2)
        assert b[1][e] == r["n_tracks"]
        for k in range(r["n_tracks"]):
            assert b[0][e, k]["votes"] == r["votes"][k]
            assert np.array_equal(b[0][e, k]["p"], r["p"][k]) and np.array_equal(b[0][e, k]["w"], r["w"][k])
        assert np.array_equal(b[2][x:y], r["hit_track"])


def test_autotune_considers_the_persistent_launch(wires):
    g = G.make_grid([10] * 5, 6, 64)
    geom = apo.Geometry(g, wires)
    ev = chamber.multi_track_events(256, seed=5, w=wires)
    o = apo.solve_opts(precision=[apo.F32] * 5 + [apo.F64] * 2, max_tracks=5, min_votes=6)
    best, ms = apo.autotune(geom, apo.DeviceHits.from_events(ev), o)
    assert ms > 0 and best.persistent in (0, 1)
    ref = _solve(geom, ev, [apo.F32] * 5 + [apo.F64] * 2, 0, max_tracks=5, min_votes=6)
    o2 = apo.solve_opts(precision=[apo.F32] * 5 + [apo.F64] * 2, max_tracks=5, min_votes=6, tune=best)
    tr, nt = apo.solve_batch(geom, apo.DeviceHits.from_events(ev), o2)
    assert np.array_equal(apo.tracks_to_numpy(tr, ev.n_events, 5).view(np.uint8), ref[0].view(np.uint8))
