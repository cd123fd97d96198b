"""apo_vote_coarse_noalloc: the allocation-free variant of full-grid voting, for callers
that may not allocate device memory while they vote (their framework allocator owns the
device budget, or allocation's device synchronisation is not allowed in their loop).

Called through the C ABI and compared with apo_vote (workspace from the caller) on two
calls in a row: the fixed scratch array keeps the previous call's contents, so the second
call checks that whatever must start at zero is cleared, and the device's free memory is
unchanged across it.  The status word in the same array is read back through
apo_vote_coarse_noalloc_status: malformed events and a device wait that runs out of its
poll limit (forced on the host's request, no device fault) are reported.  Vote counts are integers and
must match exactly.  Collected last so that a run stopping at the first failure has run
every other test first."""
import numpy as np
import pytest

from gen import chamber, grid as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2401_04576_gb300 import apo  # noqa: E402

MAX_EVENTS = 64


def _noalloc(geom, hits, precision, out):
    return apo.vote_coarse_noalloc(geom, hits, out, precision)


@pytest.mark.parametrize("prec", [apo.F64, apo.F32, apo.F64_MID, apo.F64_EXACT])
def test_noalloc_matches_workspace_entry_twice(prec):
    w = chamber.make_wires()
    g = G.make_grid([10] * 5, 4, 16)
    geom = apo.Geometry(g, w)
    # two different batches, so stale scratch from the first call would show in the second
    for k, (seed, n) in enumerate(((31, 7), (32, 5))):
        ev = chamber.single_track_events(n, seed=seed, w=w)
        hits = apo.DeviceHits.from_events(ev)
        ref = apo.vote(geom, hits, precision=prec)
        got = torch.full_like(ref, -7)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        rc = _noalloc(geom, hits, prec, got)
        assert rc == apo.APO_OK, apo.lib().apo_last_error()
        assert apo.noalloc_status() == (apo.APO_OK, 0)
        torch.cuda.synchronize()
        if k == 1:   # the first call on the device may look up the array's address only
            assert torch.cuda.mem_get_info()[0] == free0
        assert torch.equal(got, ref)
        assert int(ref.sum()) > 0


def test_noalloc_reports_malformed_events_and_timeouts():
    w = chamber.make_wires()
    g = G.make_grid([6] * 5, 2, 8)
    geom = apo.Geometry(g, w)
    ev = chamber.single_track_events(3, seed=33, w=w)
    good = apo.DeviceHits.from_events(ev)
    out = torch.zeros((ev.n_events, geom.n_coarse), dtype=torch.int32, device="cuda")
    assert _noalloc(geom, good, apo.F64, out) == apo.APO_OK
    assert apo.noalloc_status() == (apo.APO_OK, 0)
    ref = out.clone()
    # a negative drift in event 1: that event gets no votes, the others are unaffected
    bad_drift = torch.tensor(ev.drift, dtype=torch.float64, device="cuda")
    bad_drift[int(ev.offsets[1])] = -1e-3
    bad = apo.DeviceHits(good.offsets, good.wire_id, bad_drift)
    assert _noalloc(geom, bad, apo.F64, out) == apo.APO_OK
    rc, flags = apo.noalloc_status()
    assert rc == apo.APO_EINVAL and flags & apo.STATUS_BADHIT
    assert int(out[1].abs().sum()) == 0
    assert torch.equal(out[0], ref[0]) and torch.equal(out[2], ref[2])
    # a device wait on the array's status word that runs out of its poll limit
    assert apo.noalloc_wait_timeout_test(1000) == apo.APO_OK
    rc, flags = apo.noalloc_status()
    assert rc == apo.APO_ETIMEOUT and flags & apo.STATUS_TIMEOUT
    # the next call clears the word again
    assert _noalloc(geom, good, apo.F64, out) == apo.APO_OK
    assert apo.noalloc_status() == (apo.APO_OK, 0)
    assert torch.equal(out, ref)


def test_noalloc_rejects_batches_above_its_limit():
    w = chamber.make_wires()
    g = G.make_grid([6] * 5, 2, 8)
    geom = apo.Geometry(g, w)
    n = MAX_EVENTS + 1
    offs = torch.arange(n + 1, dtype=torch.int32, device="cuda")
    hits = apo.DeviceHits(offs, torch.zeros(n, dtype=torch.int32, device="cuda"),
                          torch.full((n,), 1e-3, dtype=torch.float64, device="cuda"))
    out = torch.zeros((n, geom.n_coarse), dtype=torch.int32, device="cuda")
    rc = _noalloc(geom, hits, apo.F64, out)
    assert rc == apo.APO_EINVAL
    assert b"limit" in apo.lib().apo_last_error()
    assert int(out.abs().sum()) == 0
