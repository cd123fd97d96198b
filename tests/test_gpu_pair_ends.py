"""End points of the vote program, GPU against oracle, bit for bit: for explicit (cell, hit)
pairs the kernels' program (apo_diag_vote_pair_ends) and the oracle's (or_vote_pair) must
give the same vote and the same intervals G+ and G- (Eq. ApoVote, G = rho F per drift sign),
the same guard flag and the same phase corrections delta+ and delta- (Eq. ApproxPhi_a), in
FP64 and in FP32.  Zeros compare equal whatever their sign.  Pairs: cells of every level of
the 16^5 grid near the generated helices and at random (both signs of omega, so both sides
take the mirror), each against the event's hits, plus cells whose omega interval holds 0
(the guard)."""
import numpy as np
import pytest

from gen import chamber, grid as G
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2401_04576_gb300 import apo  # noqa: E402


def _pairs():
    w = chamber.make_wires()
    g = G.make_grid([16] * 5, 6, 64)
    ev = chamber.single_track_events(6, seed=91, w=w)
    rng = np.random.default_rng(92)
    cells, hits = [], []
    for e in range(ev.n_events):
        p = ev.tracks[e][0].params
        hs = [O.hit9(w, ev.wire_id[i], ev.drift[i]) for i in range(ev.offsets[e], ev.offsets[e + 1])]
        for L in range(g.levels + 1):
            n = [int(g.bins[a]) << L for a in range(5)]
            near = [int(np.searchsorted(g.lo_edge[a][::1 << (g.levels - L)], p[a], side="right") - 1)
                    for a in range(5)]
            for k in range(24):
                if k < 16:
                    idx = [min(max(near[a] + int(rng.integers(-1, 2)), 0), n[a] - 1) for a in range(5)]
                else:
                    idx = [int(rng.integers(0, n[a])) for a in range(5)]
                c = O.cell12(g, L, idx)
                for h in hs:
                    cells.append(c)
                    hits.append(h)
        # omega straddling 0: the guard
        c = O.cell12(g, 0, [0, 0, 0, 0, 0]).copy()
        c[6], c[7] = -0.05, 0.05
        for h in hs:
            cells.append(c)
            hits.append(h)
    return w, g, np.array(cells), np.array(hits)


@pytest.fixture(scope="module")
def data():
    return _pairs()


@pytest.mark.parametrize("prec", [apo.F64, apo.F32])
def test_vote_program_end_points_bit_exact(data, prec):
    w, g, cells, hits = data
    geom = apo.Geometry(g, w)
    got = apo.vote_pair_ends(geom, torch.as_tensor(cells, device="cuda"),
                             torch.as_tensor(hits, device="cuda"), precision=prec).cpu().numpy()
    oprec = 0 if prec == apo.F64 else 1
    n_guard = n_mirror = 0
    for i in range(cells.shape[0]):
        v, out = O.vote_pair(cells[i], hits[i], oprec)
        assert int(got[i, 0]) == v, (i, got[i], v, out)
        # exact equality of values: +0 == -0, every other value bit for bit
        assert np.all(got[i, 1:] == out), (i, cells[i], hits[i], got[i, 1:], out)
        n_guard += out[4] == 1
        n_mirror += cells[i][7] < 0
    assert cells.shape[0] > 5000 and n_guard >= 6 and n_mirror > 100
