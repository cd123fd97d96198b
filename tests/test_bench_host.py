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
