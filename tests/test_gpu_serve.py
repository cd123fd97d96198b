"""Serving (continuous batching): each event's result is the same alone and in a mix of
concurrent batches, back-pressure, admission by device memory, and a failure injected on
the host side (no GPU fault)."""
import time

import numpy as np
import pytest

from gen import chamber, grid as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2401_04576_gb300 import apo  # noqa: E402


@pytest.fixture(scope="module")
def setup():
    w = chamber.make_wires()
    g = G.make_grid([8] * 5, 3, 16)
    geom = apo.Geometry(g, w)
    ev = chamber.multi_track_events(48, seed=51, w=w)
    solve = apo.solve_opts(precision=[apo.F32, apo.F32, apo.F64, apo.F64], max_tracks=4,
                           min_votes=6)
    return geom, ev, solve


def _events(ev):
    return [(ev.wire_id[ev.offsets[e]:ev.offsets[e + 1]], ev.drift[ev.offsets[e]:ev.offsets[e + 1]])
            for e in range(ev.n_events)]


def _collect(srv, n, timeout=60.0):
    out = {}
    t0 = time.time()
    while len(out) < n and time.time() - t0 < timeout:
        for rid, tr, nt in srv.poll():
            out[rid] = (tr, nt)
        time.sleep(0.001)
    return out


def test_same_result_alone_and_in_the_mix(setup):
    geom, ev, solve = setup
    evs = _events(ev)
    # reference: the whole set as one apo_solve_batch call
    tr, nt = apo.solve_batch(geom, apo.DeviceHits.from_events(ev), solve)
    ref = apo.tracks_to_numpy(tr, ev.n_events, 4)
    ref_nt = nt.cpu().numpy()
    # alone: one event at a time through the server
    srv = apo.Server(geom, solve, batch_events=8, max_slots=4)
    alone = {}
    for e, (w, d) in enumerate(evs):
        assert srv.submit(w, d, e) == apo.APO_OK
        assert srv.drain(60000) == apo.APO_OK
        alone.update({rid: v for rid, v in [(r, (t, n)) for r, t, n in srv.poll()]})
    # in the mix: everything submitted at once (shuffled), batches overlapping
    order = np.random.default_rng(3).permutation(len(evs))
    for e in order:
        w, d = evs[e]
        assert srv.submit(w, d, 1000 + int(e)) == apo.APO_OK
    assert srv.drain(60000) == apo.APO_OK
    mix = _collect(srv, len(evs))
    batches, max_busy = srv.stats()
    p50, p99, n_lat = srv.latency()      # measured inside the library, every finished event
    srv.close()
    assert n_lat == 2 * len(evs) and 0.0 < p50 <= p99
    assert len(alone) == len(evs) and len(mix) == len(evs)
    for e in range(len(evs)):
        ta, na = alone[e]
        tm, nm = mix[1000 + e]
        assert na == nm == ref_nt[e], e
        assert np.array_equal(ta.view(np.uint8), tm.view(np.uint8)), e
        assert np.array_equal(tm.view(np.uint8), ref[e].view(np.uint8)), e
    assert max_busy > 1 and batches >= len(evs) + len(evs) // 8


def test_backpressure_and_admission(setup):
    geom, ev, solve = setup
    evs = _events(ev)
    srv = apo.Server(geom, solve, batch_events=4, max_slots=1, max_pending=3)
    busy = 0
    sent = 0
    for e, (w, d) in enumerate(evs):
        rc = srv.submit(w, d, e)
        busy += rc == apo.APO_EBUSY
        sent += rc == apo.APO_OK
    assert busy > 0 and sent >= 3
    assert srv.drain(60000) == apo.APO_OK
    assert len(_collect(srv, sent)) == sent
    srv.close()
    ws1 = apo.Server(geom, solve, batch_events=16, max_slots=1)
    one, slot_bytes = ws1.slots, ws1.slot_bytes
    ws1.close()
    assert one == 1 and slot_bytes > geom.workspace_bytes(16, solve)
    # a budget for two and a half slots admits two
    srv = apo.Server(geom, solve, batch_events=16, max_slots=8, device_bytes=int(2.5 * slot_bytes))
    assert srv.slots == 2
    srv.close()
    with pytest.raises(apo.ApoError) as ex:
        apo.Server(geom, solve, batch_events=16, device_bytes=1024)
    assert ex.value.code == apo.APO_ENOMEM


def test_injected_batch_failure_is_reported(setup):
    geom, ev, solve = setup
    evs = _events(ev)
    srv = apo.Server(geom, solve, batch_events=4, max_slots=2, inject_error_after=3)
    for e, (w, d) in enumerate(evs[:20]):
        rc = srv.submit(w, d, e)
        assert rc in (apo.APO_OK, apo.APO_ECUDA)
    assert srv.drain(30000) == apo.APO_ECUDA
    with pytest.raises(apo.ApoError):
        srv.poll()
    srv.close()
    # the device is still usable afterwards
    tr, nt = apo.solve_batch(geom, apo.DeviceHits.from_events(ev.subset([0])), solve)
    torch.cuda.synchronize()
    assert int(nt.cpu()[0]) >= 0


def test_max_set_schedule_through_the_server(setup):
    """The max-set schedule with the direction condition served: each event's track is
    the one apo_solve_batch gives for the whole set."""
    geom, ev, _ = setup
    lv = geom.levels
    solve = apo.solve_opts(precision=[apo.F32 | apo.OUTGOING] * (lv - 1) + [apo.F64 | apo.OUTGOING] * 2,
                           schedule=apo.SCHED_MAXSET, max_keep=4096)
    tr, nt = apo.solve_batch(geom, apo.DeviceHits.from_events(ev), solve)
    ref = apo.tracks_to_numpy(tr, ev.n_events)
    srv = apo.Server(geom, solve, batch_events=4, max_slots=3)
    for e, (w, d) in enumerate(_events(ev)):
        assert srv.submit(w, d, e) == apo.APO_OK
    assert srv.drain(60000) == apo.APO_OK
    got = _collect(srv, ev.n_events)
    srv.close()
    for e in range(ev.n_events):
        assert np.array_equal(got[e][0].view(np.uint8), ref[e].view(np.uint8)), e
