"""GPU parity of the midpoint form (APO_F64_MID): the CUDA path through the C ABI against
the oracle's midpoint form (or_vote_cells / or_solve_event with precision 3), bit-exact
vote counts and estimates, on ragged grids, every refinement level, whole searches, the
full-size batch (sampled), and a mixed midpoint / interval precision schedule."""
import dataclasses

import numpy as np
import pytest

from gen import chamber, grid as G
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2401_04576_gb300 import apo  # noqa: E402

MID = 3   # the oracle's code of the midpoint form


@pytest.fixture(scope="module")
def wires():
    return chamber.make_wires()


@pytest.fixture(scope="module")
def grid1():
    return G.make_grid([10] * 5, 4, 16)


@pytest.fixture(scope="module")
def grid2():
    return G.make_grid([16] * 5, 6, 64)


@pytest.fixture(scope="module")
def ev1(wires):
    return chamber.single_track_events(6, seed=1, w=wires)


@pytest.fixture(scope="module")
def ev2(wires):
    return chamber.single_track_events(1024, seed=2, w=wires)


def _hits(ev):
    return apo.DeviceHits.from_events(ev)


def test_mid_coarse_votes_ragged_grid(wires):
    """Uneven bins on every axis (several (d0, z0) thread shapes, 9 tan(lambda) bins)."""
    grid = G.make_grid([7, 6, 8, 5, 9], 3, 16)
    ev = chamber.single_track_events(5, seed=41, w=wires)
    geom = apo.Geometry(grid, wires)
    got = apo.vote(geom, _hits(ev), precision=apo.F64_MID).cpu().numpy()
    tab = O.Tables(grid, wires)
    for e in range(ev.n_events):
        a, b = ev.offsets[e], ev.offsets[e + 1]
        np.testing.assert_array_equal(got[e], O.vote_coarse(tab, ev.wire_id[a:b], ev.drift[a:b], MID))


def test_mid_cell_votes_every_level(wires, grid2, ev2):
    geom = apo.Geometry(grid2, wires)
    sub = ev2.subset([5, 6, 7])
    tab = O.Tables(grid2, wires)
    rng = np.random.default_rng(42)
    for L in range(grid2.levels + 1):
        keys = np.zeros((sub.n_events, 200), np.uint64)
        for e in range(sub.n_events):
            p = sub.tracks[e][0].params
            near = [int(np.searchsorted(grid2.lo_edge[a][::1 << (grid2.levels - L)], p[a],
                                        side="right") - 1) for a in range(5)]
            n = [int(grid2.bins[a]) << L for a in range(5)]
            idx = np.array([[min(max(near[a] + int(rng.integers(-2, 3)), 0), n[a] - 1)
                             for a in range(5)] for _ in range(100)] +
                           [[int(rng.integers(0, n[a])) for a in range(5)] for _ in range(100)])
            keys[e] = G.cell_key(idx)
        kt = torch.as_tensor(keys.view(np.int64), device="cuda")
        got = apo.vote(geom, _hits(sub), keys=kt, level=L, precision=apo.F64_MID).cpu().numpy()
        for e in range(sub.n_events):
            a, b = sub.offsets[e], sub.offsets[e + 1]
            ref = O.vote_cells(tab, sub.wire_id[a:b], sub.drift[a:b], L, keys[e], MID)
            np.testing.assert_array_equal(got[e], ref, err_msg=f"level {L} event {e}")


def _solve_and_compare(wires, grid, ev, precision, oprec):
    geom = apo.Geometry(grid, wires)
    ne, K, lv = ev.n_events, grid.topk, grid.levels
    tk = torch.zeros((ne, lv + 1, K), dtype=torch.int64, device="cuda")
    tv = torch.zeros((ne, lv + 1, K), dtype=torch.int32, device="cuda")
    tracks, nt = apo.solve_batch(geom, _hits(ev), apo.solve_opts(precision=precision,
                                                                  trace_keys=tk, trace_votes=tv))
    tr = apo.tracks_to_numpy(tracks, ne)[:, 0]
    tk = tk.cpu().numpy().view(np.uint64)
    tv = tv.cpu().numpy()
    tab = O.Tables(grid, wires)
    for e in range(ne):
        a, b = ev.offsets[e], ev.offsets[e + 1]
        r = O.solve_event(tab, ev.wire_id[a:b], ev.drift[a:b], oprec)
        assert sorted(zip(tk[e, 0].tolist(), tv[e, 0].tolist())) == \
            sorted(zip(r["trace_keys"][0].tolist(), r["trace_votes"][0].tolist()))
        for L in range(1, lv):
            assert tk[e, L].tolist() == r["trace_keys"][L].tolist(), (e, L)
            assert tv[e, L].tolist() == r["trace_votes"][L].tolist(), (e, L)
        assert tr[e]["votes"] == r["votes"]
        assert np.array_equal(tr[e]["p"], r["p"]) and np.array_equal(tr[e]["w"], r["w"])
    assert np.all(nt.cpu().numpy() == 1)


def test_mid_solve_bit_exact(wires, grid1, ev1):
    lv = grid1.levels
    _solve_and_compare(wires, grid1, ev1, [apo.F64_MID] * (lv + 1), [MID] * (lv + 1))


def test_mid_then_interval_solve_bit_exact(wires, grid1, ev1):
    """Midpoint form on the coarse levels, FP32 and FP64 intervals on the fine ones."""
    prec = [apo.F64_MID, apo.F64_MID, apo.F32, apo.F64, apo.F64]
    _solve_and_compare(wires, grid1, ev1, prec, [MID, MID, 1, 0, 0])


def test_mid_full_size_sampled(wires, grid2, ev2):
    """All 1024 events on the 16^5 grid in the benchmark's launch shape; sampled cells of
    sampled events against the oracle one by one."""
    geom = apo.Geometry(grid2, wires)
    votes = apo.vote(geom, _hits(ev2), precision=apo.F64_MID)
    tab = O.Tables(grid2, wires)
    rng = np.random.default_rng(43)
    for e in rng.integers(0, ev2.n_events, 24):
        lin = rng.integers(0, geom.n_coarse, 64)
        keys = G.cell_key(G.coarse_index_to_idx5(lin, grid2.bins))
        a, b = ev2.offsets[e], ev2.offsets[e + 1]
        ref = O.vote_cells(tab, ev2.wire_id[a:b], ev2.drift[a:b], 0, keys, MID)
        got = votes[int(e)][torch.as_tensor(lin, device="cuda")].cpu().numpy()
        np.testing.assert_array_equal(got, ref)


def test_mid_needs_the_centre_table(wires, grid1, ev1):
    """A geometry made without the centre table refuses the midpoint form (and only it)."""
    g = dataclasses.replace(grid1, sincos_mid=None)
    geom = apo.Geometry(g, wires)
    h = _hits(ev1.subset([0]))
    with pytest.raises(apo.ApoError) as ei:
        apo.vote(geom, h, precision=apo.F64_MID)
    assert ei.value.code == apo.APO_EINVAL
    apo.vote(geom, h, precision=apo.F64)
