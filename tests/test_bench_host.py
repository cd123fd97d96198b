"""Host-side logic of bench.py (no GPU): the op-count constants against the oracle's
instrumented counter, pair counting, and the multi-rank max reduction over gloo."""
import os

import numpy as np
import pytest

import bench
from gen import chamber, grid as G
from oracle import oracle as O


def test_op_constants_match_oracle_counter():
    w = chamber.make_wires()
    g = G.make_grid([16] * 5, 6, 64)
    ev = chamber.single_track_events(2, seed=5, w=w)
    p = ev.tracks[0][0].params
    for L in (0, 3, 6):
        idx = [int(np.searchsorted(g.lo_edge[a][::1 << (g.levels - L)], p[a], side="right") - 1)
               for a in range(5)]
        cell = O.cell12(g, L, idx)
        for i in range(ev.n_hits(0)):
            wid = ev.wire_id[ev.offsets[0] + i]
            for prec in (0, 1):   # FP64 and FP32 run the same sequence of operations
                c = O.op_counts(cell, O.hit9(w, wid, ev.drift[ev.offsets[0] + i]), prec)
                assert c.tolist() == [bench.OPS_CELL, bench.OPS_PREFIX, bench.OPS_LPART, bench.OPS_SIGNS]
    assert bench.OPS_FULL == sum([bench.OPS_CELL, bench.OPS_PREFIX, bench.OPS_LPART, bench.OPS_SIGNS])


def test_pairs_decided():
    nh = np.array([10, 20])
    assert bench.pairs_decided(nh, 100, 2, 4) == 30 * (100 + 2 * 4 * 32)


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    q.put((rank, bench.reduce_max(1.0 + rank, world)))
    dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    import multiprocessing as mp
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
    assert out == {0: 2.0, 1: 2.0}


def test_multi_track_figures():
    """The multi-track figures on a hand-made extraction: two events, three true tracks and
    two noise hits; one found track's box holds a true helix, another holds none."""
    from paper_2401_04576_gb300.apo import TRACK_DTYPE
    w = chamber.make_wires()
    ev = chamber.multi_track_events(2, seed=9, w=w)
    n_true = [len(t) for t in ev.tracks]
    tracks = np.zeros((2, 5), TRACK_DTYPE)
    nt = np.zeros(2, np.int32)
    # event 0: track 0 centred on the first generated helix (box 1e-6 wide), track 1 far away
    tracks[0, 0]["p"] = ev.tracks[0][0].params
    tracks[0, 0]["w"] = 1e-6
    tracks[0, 1]["p"] = np.array(ev.tracks[0][0].params) + 10.0
    tracks[0, 1]["w"] = 1e-6
    nt[0] = 2
    a, b = ev.offsets[0], ev.offsets[2]
    ht = np.full(b - a, -1, np.int32)
    truth0 = ev.hit_truth[0]
    sig0 = [i for i, h in enumerate(truth0) if h is not None]
    noise0 = [i for i, h in enumerate(truth0) if h is None]
    ht[sig0[:3]] = 0                      # three signal hits taken
    if noise0:
        ht[noise0[0]] = 1                 # one noise hit taken
    f = bench.multi_track_figures(ev, tracks, nt, ht)
    n_sig = sum(h is not None for e in range(2) for h in ev.hit_truth[e])
    n_noise = sum(h is None for e in range(2) for h in ev.hit_truth[e])
    assert f["signal_hits_taken"] == pytest.approx(3 / n_sig)
    assert f["noise_hits_rejected"] == pytest.approx(1 - (1 if noise0 else 0) / max(n_noise, 1))
    assert f["tracks_found_per_true_track"] == pytest.approx(2 / sum(n_true))
    assert f["true_tracks_in_a_found_box"] == pytest.approx(1 / sum(n_true))
    assert f["found_tracks_holding_no_true_helix"] == pytest.approx(0.5)


def test_headline_latency_is_at_the_highest_sustained_load():
    loads = [
        {"offered_per_s": 1000, "rejected": 0, "sustained_per_s": 1030, "p50_ms": 15.0, "p99_ms": 30.0},
        {"offered_per_s": 2000, "rejected": 0, "sustained_per_s": 1930, "p50_ms": 31.0, "p99_ms": 58.0},
        {"offered_per_s": 5000, "rejected": 0, "sustained_per_s": 2540, "p50_ms": 590.0, "p99_ms": 999.0},
        {"offered_per_s": 10000, "rejected": 3000, "sustained_per_s": 2550, "p50_ms": 1100.0, "p99_ms": 1800.0},
    ]
    assert bench.headline_latency(loads)["offered_per_s"] == 2000
    assert bench.headline_latency(loads[2:]) is None
