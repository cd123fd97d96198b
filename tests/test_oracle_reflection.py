"""The vote program's symmetry under the reflection z -> -z (CPU).

Reflecting the cell and the wire in the plane z = 0 maps (z0, tan(lambda)) to (-z0,
-tan(lambda)) and the wire's stereo terms (tan tau, sin phi tan tau, cos phi tan tau) to
their negatives.  The helix and the wire are the same curves mirrored, so every distance
is the same; the interval program keeps this exactly, because an interval product with
both operands negated has the same four end-point products and one with a single operand
negated is an exact negation.  The FP32 kernels rely on it to evaluate a tan(lambda) bin
with L <= 0 as its reflection (L >= 0).  Checked on the oracle: the vote, both drift
signs' end points of G, the guard flag and the phase corrections delta+-, equal value for
value, in FP64 and FP32, with and without the direction condition.
"""
import numpy as np
import pytest

from gen import chamber, grid as G
from oracle import oracle as O


def _reflect_cell(c):
    r = c.copy()
    r[8], r[9] = -c[9], -c[8]      # z0
    r[10], r[11] = -c[11], -c[10]  # tan(lambda)
    return r


def _reflect_hit(h):
    r = h.copy()
    r[4], r[5], r[6] = -h[4], -h[5], -h[6]   # tan tau, sin phi tan tau, cos phi tan tau
    return r


@pytest.mark.parametrize("prec", [0, 1, 0 | O.OUTGOING, 1 | O.OUTGOING])
def test_vote_program_is_symmetric_under_z_reflection(prec):
    w = chamber.make_wires()
    g = G.make_grid([16] * 5, 6, 64)
    ev = chamber.single_track_events(3, seed=211, w=w)
    rng = np.random.default_rng(211)
    n_votes = n_pairs = 0
    for e in range(ev.n_events):
        tp = ev.tracks[e][0].params
        for level in (0, 2, 4, 6):
            for _ in range(6):
                idx = []
                for a in range(5):
                    nb = int(g.bins[a]) << level
                    lo, hi = g.cell_edges(level, a, np.arange(nb))
                    j = np.nonzero((lo <= tp[a]) & (tp[a] <= hi))[0]
                    i0 = int(j[0]) if j.size else nb // 2
                    idx.append(int(np.clip(i0 + rng.integers(-2, 3), 0, nb - 1)))
                c = O.cell12(g, level, idx)
                for wid in ev.wire_id[ev.offsets[e]:ev.offsets[e + 1]]:
                    h = O.hit9(w, wid, float(rng.uniform(0, 0.008)))
                    v, out = O.vote_pair(c, h, prec)
                    vr, outr = O.vote_pair(_reflect_cell(c), _reflect_hit(h), prec)
                    assert v == vr, (level, idx, wid)
                    np.testing.assert_array_equal(out, outr)
                    n_votes += v
                    n_pairs += 1
    assert n_pairs > 500 and 0 < n_votes < n_pairs
