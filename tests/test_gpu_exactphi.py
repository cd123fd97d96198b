"""GPU parity of the exact-phase vote program (APO_F64_EXACT: Eq. CSAXtoPHI_a enclosed by an
interval fixed point) against the oracle's (or_vote_cells / or_solve_event with precision
4): full-grid votes, cells at every level, whole searches, and the full-size batch
(sampled), bit for bit."""
import numpy as np
import pytest

from gen import chamber, grid as G
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2401_04576_gb300 import apo  # noqa: E402

EXACT = 4   # the oracle's code


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
    return chamber.single_track_events(256, seed=2, w=wires)


def _hits(ev):
    return apo.DeviceHits.from_events(ev)


def test_exact_coarse_votes(wires, grid1, ev1):
    geom = apo.Geometry(grid1, wires)
    sub = ev1.subset(range(3))
    got = apo.vote(geom, _hits(sub), precision=apo.F64_EXACT).cpu().numpy()
    tab = O.Tables(grid1, wires)
    for e in range(sub.n_events):
        a, b = sub.offsets[e], sub.offsets[e + 1]
        np.testing.assert_array_equal(got[e], O.vote_coarse(tab, sub.wire_id[a:b], sub.drift[a:b], EXACT))


def test_exact_cells_every_level(wires, grid2, ev2):
    geom = apo.Geometry(grid2, wires)
    sub = ev2.subset([0, 1])
    tab = O.Tables(grid2, wires)
    rng = np.random.default_rng(21)
    for L in range(grid2.levels + 1):
        keys = np.zeros((sub.n_events, 160), np.uint64)
        for e in range(sub.n_events):
            p = sub.tracks[e][0].params
            near = [int(np.searchsorted(grid2.lo_edge[a][::1 << (grid2.levels - L)], p[a],
                                        side="right") - 1) for a in range(5)]
            n = [int(grid2.bins[a]) << L for a in range(5)]
            idx = np.array([[min(max(near[a] + int(rng.integers(-2, 3)), 0), n[a] - 1)
                             for a in range(5)] for _ in range(120)] +
                           [[int(rng.integers(0, n[a])) for a in range(5)] for _ in range(40)])
            keys[e] = G.cell_key(idx)
        kt = torch.as_tensor(keys.view(np.int64), device="cuda")
        got = apo.vote(geom, _hits(sub), keys=kt, level=L, precision=apo.F64_EXACT).cpu().numpy()
        for e in range(sub.n_events):
            a, b = sub.offsets[e], sub.offsets[e + 1]
            ref = O.vote_cells(tab, sub.wire_id[a:b], sub.drift[a:b], L, keys[e], EXACT)
            np.testing.assert_array_equal(got[e], ref, err_msg=f"level {L} event {e}")


def test_exact_solve_bit_exact(wires, grid1, ev1):
    geom = apo.Geometry(grid1, wires)
    lv = grid1.levels
    prec = [apo.F64_EXACT] * (lv + 1)
    ne, K = ev1.n_events, grid1.topk
    tk = torch.zeros((ne, lv + 1, K), dtype=torch.int64, device="cuda")
    tv = torch.zeros((ne, lv + 1, K), dtype=torch.int32, device="cuda")
    tracks, nt = apo.solve_batch(geom, _hits(ev1), apo.solve_opts(precision=prec, trace_keys=tk,
                                                                   trace_votes=tv))
    tr = apo.tracks_to_numpy(tracks, ne)[:, 0]
    tk = tk.cpu().numpy().view(np.uint64)
    tv = tv.cpu().numpy()
    tab = O.Tables(grid1, wires)
    for e in range(ne):
        a, b = ev1.offsets[e], ev1.offsets[e + 1]
        r = O.solve_event(tab, ev1.wire_id[a:b], ev1.drift[a:b], [EXACT] * (lv + 1))
        assert sorted(zip(tk[e, 0].tolist(), tv[e, 0].tolist())) == \
            sorted(zip(r["trace_keys"][0].tolist(), r["trace_votes"][0].tolist()))
        for L in range(1, lv):
            assert tk[e, L].tolist() == r["trace_keys"][L].tolist(), (e, L)
        assert tr[e]["votes"] == r["votes"]
        assert np.array_equal(tr[e]["p"], r["p"]) and np.array_equal(tr[e]["w"], r["w"])


def test_exact_full_size_sampled(wires, grid2, ev2):
    """256 events of the 16^5 grid in one call; sampled cells against the oracle."""
    geom = apo.Geometry(grid2, wires)
    votes = apo.vote(geom, _hits(ev2), precision=apo.F64_EXACT)
    tab = O.Tables(grid2, wires)
    rng = np.random.default_rng(22)
    for e in rng.integers(0, ev2.n_events, 12):
        lin = rng.integers(0, geom.n_coarse, 48)
        keys = G.cell_key(G.coarse_index_to_idx5(lin, grid2.bins))
        a, b = ev2.offsets[e], ev2.offsets[e + 1]
        ref = O.vote_cells(tab, ev2.wire_id[a:b], ev2.drift[a:b], 0, keys, EXACT)
        got = votes[int(e)][torch.as_tensor(lin, device="cuda")].cpu().numpy()
        np.testing.assert_array_equal(got, ref)
