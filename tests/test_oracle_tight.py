"""How much looser the oracle's interval program is than a tight reference evaluation of
the same equations (CPU; Section 3.1: a cell votes when the interval extension of
Eq. ApoVote contains 0, so a looser enclosure can only add votes).

The reference variant is the oracle's own source compiled with APO_TIGHT: the atan series
with twelve terms (through x^23, remainder |x|^25 / 25), sin / cos of the phase
correction through delta^13 / delta^12 (remainders |delta|^15 / 15!, |delta|^14 / 14!),
and sin Phi, cos Phi and u_d of Eq. normudi evaluated per drift sign instead of over the
hull of both signs.  It exists only for these tests.

Both programs enclose the same real function, and each of the shipped program's
simplifications only widens an interval, so every (cell, hit) pair that the tight variant
votes for must also vote in the shipped oracle.  The tests check that pair by pair and
report how many pairs and cells the looser program adds."""
import numpy as np
import pytest

from gen import chamber, grid as G
from oracle import build as ob, oracle as O


@pytest.fixture(scope="module")
def tight():
    return O.load(ob.build(variant="tight", defines=["APO_TIGHT"]))


def _pair_votes(tab, wid, dr, level, keys, L=None):
    """votes[i, j]: hit i votes for cell j (one oracle call per hit)."""
    return np.stack([O.vote_cells(tab, wid[i:i + 1], dr[i:i + 1], level, keys, 0, L=L)
                     for i in range(len(wid))])


def _compare(tab, wid, dr, level, keys, tight):
    shipped = _pair_votes(tab, wid, dr, level, keys)
    ref = _pair_votes(tab, wid, dr, level, keys, L=tight)
    bad = np.argwhere(ref > shipped)
    assert bad.size == 0, f"tight variant votes where the oracle does not: {bad[:5]}"
    extra_pairs = int(np.sum(shipped > ref))
    extra_cells = int(np.sum(shipped.sum(0) > ref.sum(0)))
    return extra_pairs, extra_cells, int(shipped.sum()), int(ref.sum())


def test_tight_enclosures_contain_libm():
    """The reference variant's series are themselves enclosures (libm values inside)."""
    L = O.load(ob.build(variant="tight", defines=["APO_TIGHT"]))
    import ctypes as C
    rng = np.random.default_rng(5)
    for _ in range(300):
        a = rng.uniform(-3, 3)
        b = a + rng.uniform(0, 0.2)
        out = np.zeros(2)
        L.or_atan_iv(a, b, 0, out.ctypes.data_as(C.POINTER(C.c_double)))
        assert out[0] <= np.arctan(a) and np.arctan(b) <= out[1]
        L.or_atan_iv(a, a, 0, out.ctypes.data_as(C.POINTER(C.c_double)))   # a point: tight
        assert out[0] <= np.arctan(a) <= out[1] and out[1] - out[0] <= 1e-12
        d = rng.uniform(-0.3, 0.3)
        e = d + rng.uniform(0, 0.05)
        sc = np.zeros(4)
        L.or_sincos_iv(d, e, 0, sc.ctypes.data_as(C.POINTER(C.c_double)))
        for x in (d, e, 0.5 * (d + e)):
            assert sc[0] <= np.sin(x) <= sc[1] and sc[2] <= np.cos(x) <= sc[3]
        L.or_sincos_iv(d, d, 0, sc.ctypes.data_as(C.POINTER(C.c_double)))
        assert sc[0] <= np.sin(d) <= sc[1] and sc[1] - sc[0] <= 1e-15


def test_oracle_contains_tight_variant_on_the_ten_cubed_grid(tight):
    """All 10^5 level-0 cells and the cells kept at levels 1-4 of the search (10^5 grid,
    top-16, 4 levels), three events."""
    w = chamber.make_wires()
    g = G.make_grid([10] * 5, 4, 16)
    tab = O.Tables(g, w)
    ev = chamber.single_track_events(3, seed=1, w=w)
    keys0 = O.coarse_keys(tab)
    tot = np.zeros(4, np.int64)
    for e in range(ev.n_events):
        a, b = ev.offsets[e], ev.offsets[e + 1]
        wid, dr = ev.wire_id[a:b], ev.drift[a:b]
        tot += _compare(tab, wid, dr, 0, keys0, tight)
        r = O.solve_event(tab, wid, dr)
        for lev in range(1, 5):
            kept = r["trace_keys"][lev - 1]
            tot += _compare(tab, wid, dr, lev, O.children(kept), tight)
    print(f"\n10^5 grid, levels 0-4, 3 events: the oracle adds {tot[0]} voting pairs "
          f"({tot[0] / max(tot[3], 1):.2e} of the tight variant's {tot[3]}) in {tot[1]} cells")
    assert tot[0] <= 0.01 * tot[3]


def test_oracle_contains_tight_variant_on_one_sixteen_to_the_fifth_event(tight):
    """One event, every cell of the 16^5 level-0 grid."""
    w = chamber.make_wires()
    g = G.make_grid([16] * 5, 6, 64)
    tab = O.Tables(g, w)
    ev = chamber.single_track_events(1, seed=2, w=w)
    pairs, cells, n_shipped, n_ref = _compare(tab, ev.wire_id, ev.drift, 0, O.coarse_keys(tab), tight)
    print(f"\n16^5 level 0, one event: the oracle adds {pairs} voting pairs "
          f"({pairs / max(n_ref, 1):.2e} of the tight variant's {n_ref}) in {cells} cells")
    assert pairs <= 0.01 * n_ref
