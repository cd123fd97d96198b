"""GPU parity of the paper's own 4-D search (include/apo4.h) against the oracle
(or4_vote_grid / or4_solve_event): every voxel's votes in both accumulators, and every
iteration's estimate, errors, sign, maximum, reference point and hit selection, bit for
bit, in FP64 and FP32, on reduced grids, on the paper's grids (sampled events), and with a
malformed event."""
import numpy as np
import pytest

from gen import comet, grid as G
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2401_04576_gb300 import apo  # noqa: E402

# reduced grids over the same boxes as Table tabGridDef (4-8x fewer voxels)
RW = ((0.045, 0.045, 0.009375, 0.15), (0.025, 0.025, 0.009375, 0.15), (0.0025, 0.0025, 0.0025, 0.08))
RN = ((20, 20, 16, 10), (36, 36, 16, 10), (20, 20, 20, 10))


@pytest.fixture(scope="module")
def wires():
    return comet.make_wires()


@pytest.fixture(scope="module")
def tab(wires):
    return O.Tables(G.make_grid([4] * 5, 1, 4), wires)


@pytest.fixture(scope="module")
def ch(wires):
    return apo.Chamber4(wires)


def _hits(ev):
    return apo.DeviceHits.from_events(ev)


def _compare(got, ref, e, k):
    for f in ("value", "err", "ref"):
        assert np.array_equal(got[f], ref[f]), (e, k, f, got[f], ref[f])
    for f in ("sign", "vmax", "n_max", "n_sel"):
        assert int(got[f]) == ref[f], (e, k, f, int(got[f]), ref[f])


@pytest.mark.parametrize("prec", [apo.F64, apo.F32])
def test_four_vote_grid_bit_exact(wires, tab, ch, prec):
    ev = comet.events(3, seed=61, w=wires)
    rng = np.random.default_rng(7)
    n = (10, 10, 8, 6)
    w = (0.09, 0.09, 0.01875, 0.25)
    opts = apo.four_opts(precision=prec, n=(n, n, n), w=(w, w, w))
    lo = np.array([[-0.45, -0.45, 0.225, -0.75], [-0.40, -0.35, 0.23, -0.70],
                   [-0.45, -0.42, 0.226, -0.74]])
    refs, act = [], np.zeros(int(ev.offsets[-1]), np.uint8)
    for e in range(ev.n_events):
        a, b = ev.offsets[e], ev.offsets[e + 1]
        h = ev.wire_id[a + (b - a) // 2]
        refs.append([wires.x0[h], wires.y0[h]] if e else [0.0, 0.0])
        act[a:b] = rng.random(b - a) < 0.8
    refs = np.array(refs)
    got = apo.vote4(ch, _hits(ev), opts, 0, torch.as_tensor(lo, device="cuda"),
                    torch.as_tensor(refs, device="cuda"),
                    active=torch.as_tensor(act, device="cuda")).cpu().numpy()
    oo = O.four_opts(precision=0 if prec == apo.F64 else 1)
    for e in range(ev.n_events):
        a, b = ev.offsets[e], ev.offsets[e + 1]
        ref = O.four_vote_grid(oo, O.four_grid(lo[e], w, n), refs[e], tab, ev.wire_id[a:b],
                               ev.drift[a:b], act[a:b])
        np.testing.assert_array_equal(got[e], ref, err_msg=f"event {e}")
        assert got[e].max() > 0


@pytest.mark.parametrize("prec", [apo.F64, apo.F32])
def test_four_vote_tiles_without_disk_columns(wires, tab, ch, prec):
    """Event 0's grid lies far from the origin, so no column of any tile passes the disk
    pre-filter (every vote 0); event 1's 1,152 columns fill two tiles of 512 and a
    ragged third, mixing passing and failing columns."""
    ev = comet.events(2, seed=65, w=wires)
    n = (12, 12, 8, 6)
    w = (0.075, 0.075, 0.01875, 0.25)
    opts = apo.four_opts(precision=prec, n=(n, n, n), w=(w, w, w))
    lo = np.array([[2.0, 2.0, 0.225, -0.75], [-0.45, -0.45, 0.225, -0.75]])
    refs = np.zeros((2, 2))
    act = np.ones(int(ev.offsets[-1]), np.uint8)
    got = apo.vote4(ch, _hits(ev), opts, 0, torch.as_tensor(lo, device="cuda"),
                    torch.as_tensor(refs, device="cuda"),
                    active=torch.as_tensor(act, device="cuda")).cpu().numpy()
    oo = O.four_opts(precision=0 if prec == apo.F64 else 1)
    for e in range(2):
        a, b = ev.offsets[e], ev.offsets[e + 1]
        ref = O.four_vote_grid(oo, O.four_grid(lo[e], w, n), refs[e], tab, ev.wire_id[a:b],
                               ev.drift[a:b], act[a:b])
        np.testing.assert_array_equal(got[e], ref, err_msg=f"event {e}")
    assert got[0].max() == 0 and got[1].max() > 0


@pytest.mark.parametrize("prec,per_sign", [(apo.F64, 1), (apo.F32, 1), (apo.F64, 0), (apo.F32, 0)])
def test_four_solve_reduced_grids_bit_exact(wires, tab, ch, prec, per_sign):
    ev = comet.events(5, seed=62, w=wires)
    opts = apo.four_opts(precision=prec, w=RW, n=RN, per_sign=per_sign)
    out, sel = apo.solve4(ch, _hits(ev), opts)
    got = apo.iters4_to_numpy(out, ev.n_events, 3)
    sel = sel.cpu().numpy()
    oo = O.four_opts(w=RW, n=RN, precision=0 if prec == apo.F64 else 1, per_sign=per_sign)
    for e in range(ev.n_events):
        a, b = ev.offsets[e], ev.offsets[e + 1]
        its, rsel = O.four_solve_event(oo, tab, ev.wire_id[a:b], ev.drift[a:b])
        for k in range(3):
            _compare(got[e, k], its[k], e, k)
        assert np.array_equal(sel[a:b].astype(bool), rsel), e


@pytest.mark.parametrize("prec", [apo.F64, apo.F32])
def test_four_paper_grids_sampled(wires, tab, ch, prec):
    """The paper's grids (Table tabGridDef) on 48 events in one batch, as the benchmark runs
    them; two events recomputed whole by the oracle."""
    ev = comet.events(48, seed=63, w=wires)
    opts = apo.four_opts(precision=prec)
    out, sel = apo.solve4(ch, _hits(ev), opts)
    got = apo.iters4_to_numpy(out, ev.n_events, 3)
    sel = sel.cpu().numpy()
    oo = O.four_opts(precision=0 if prec == apo.F64 else 1)
    for e in (3, 40):
        a, b = ev.offsets[e], ev.offsets[e + 1]
        its, rsel = O.four_solve_event(oo, tab, ev.wire_id[a:b], ev.drift[a:b])
        for k in range(3):
            _compare(got[e, k], its[k], e, k)
        assert np.array_equal(sel[a:b].astype(bool), rsel), e
    # the searches find the generated helices
    dx = [abs(got[e, 2]["value"][0] - comet.helix_centre(ev.tracks[e][0])[0]) for e in range(ev.n_events)]
    assert np.median(dx) < 1e-3


def test_four_malformed_event(wires, ch):
    ev = comet.events(3, seed=64, w=wires)
    wid = ev.wire_id.copy()
    wid[ev.offsets[1] + 2] = wires.n + 7                   # event 1: a wire id out of range
    bad = apo.DeviceHits(torch.as_tensor(ev.offsets, device="cuda"),
                         torch.as_tensor(wid, device="cuda"),
                         torch.as_tensor(ev.drift, device="cuda"))
    opts = apo.four_opts(w=RW, n=RN)
    out, sel = apo.solve4(ch, bad, opts)
    got = apo.iters4_to_numpy(out, ev.n_events, 3)
    sel = sel.cpu().numpy()
    assert all(got[1, k]["vmax"] == apo.APO_EINVAL and got[1, k]["n_sel"] == 0 for k in range(3))
    assert not sel[ev.offsets[1]:ev.offsets[2]].any()
    assert got[0, 2]["vmax"] > 0 and got[2, 2]["vmax"] > 0


@pytest.mark.parametrize("prec", [apo.F64, apo.F32])
def test_four_per_sign_iteration_three(wires, tab, ch, prec):
    """Steep tracks whose iteration 2 picks the wrong tan(lambda) sign or a box 20-50 mm off
    (events 2, 41 and 56 of the benchmark's batch): with iteration 3 per sign the search is
    bit-exact against the oracle and ends within 1 mm (x_c, y_c, R) and 10 mm (z0) of the
    generated helix; on iteration 2's box alone it does not."""
    ev = comet.events(57, seed=70, w=wires).subset([2, 41, 56])
    res = {}
    for ps in (1, 0):
        out, sel = apo.solve4(ch, _hits(ev), apo.four_opts(precision=prec, per_sign=ps))
        res[ps] = (apo.iters4_to_numpy(out, ev.n_events, 3), sel.cpu().numpy())
    got, sel = res[1]
    oo = O.four_opts(precision=0 if prec == apo.F64 else 1, per_sign=1)
    n_ok = {0: 0, 1: 0}
    for e in range(ev.n_events):
        a, b = ev.offsets[e], ev.offsets[e + 1]
        its, rsel = O.four_solve_event(oo, tab, ev.wire_id[a:b], ev.drift[a:b])
        for k in range(3):
            _compare(got[e, k], its[k], e, k)
        assert np.array_equal(sel[a:b].astype(bool), rsel), e
        tr = ev.tracks[e][0]
        xc, yc, R = comet.helix_centre(tr)
        for ps in (0, 1):
            r = res[ps][0][e, 2]
            d = np.abs(r["value"] - [xc, yc, R, comet.z_at_point(tr, *r["ref"])])
            n_ok[ps] += bool(np.all(d[:3] < 1e-3) and d[3] < 1e-2)
    assert n_ok[1] == 3 and n_ok[0] < 3, n_ok
