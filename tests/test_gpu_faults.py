"""Failure detection without any GPU fault: a device wait on a barrier that nothing
completes runs out of its short poll limit, reports APO_ETIMEOUT through the status word,
and the device keeps working; normal work reports no timeout."""
import pytest

from gen import chamber, grid as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2401_04576_gb300 import apo  # noqa: E402


def test_device_wait_limit_reports_timeout_and_context_survives():
    assert apo.wait_timeout_test(1000) == apo.APO_ETIMEOUT
    assert b"poll limit" in apo.lib().apo_last_error()
    w = chamber.make_wires()
    g = G.make_grid([6] * 5, 2, 8)
    geom = apo.Geometry(g, w)
    ev = chamber.single_track_events(4, seed=61, w=w)
    ws = geom.workspace(ev.n_events)
    tr, nt = apo.solve_batch(geom, apo.DeviceHits.from_events(ev), workspace=ws)
    torch.cuda.synchronize()
    assert int(nt.sum()) == ev.n_events
    assert apo.workspace_status(geom, ev.n_events, ws) == apo.APO_OK
