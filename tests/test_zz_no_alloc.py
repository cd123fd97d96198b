"""apo_vote_coarse_noalloc: the allocation-free variant of full-grid voting, for callers
that may not allocate device memory while they vote (their framework allocator owns the
device budget, or allocation's device synchronisation is not allowed in their loop).

Called through the C ABI and compared with apo_vote (workspace from the caller) on two
calls in a row: the fixed scratch array keeps the previous call's contents, so the second
call checks that whatever must start at zero is cleared.  Vote counts are integers and
must match exactly.  Collected last so that a run stopping at the first failure has run
every other test first."""
import ctypes as C

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
    L = apo.lib()
    L.apo_vote_coarse_noalloc.argtypes = [C.c_void_p, C.POINTER(apo.ApoHits), C.c_int32,
                                          C.c_void_p, C.c_void_p]
    hc = hits.c()
    return L.apo_vote_coarse_noalloc(geom.handle, C.byref(hc), int(precision), apo._ptr(out),
                                     apo._stream_ptr(None))


@pytest.mark.parametrize("prec", [apo.F64, apo.F32])
def test_noalloc_matches_workspace_entry_twice(prec):
    w = chamber.make_wires()
    g = G.make_grid([10] * 5, 4, 16)
    geom = apo.Geometry(g, w)
    # two different batches, so stale scratch from the first call would show in the second
    for seed, n in ((31, 7), (32, 5)):
        ev = chamber.single_track_events(n, seed=seed, w=w)
        hits = apo.DeviceHits.from_events(ev)
        ref = apo.vote(geom, hits, precision=prec)
        got = torch.full_like(ref, -7)
        rc = _noalloc(geom, hits, prec, got)
        assert rc == apo.APO_OK, apo.lib().apo_last_error()
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
        assert int(ref.sum()) > 0


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
