"""Benchmark of the interval-voting hot path on GB300.

One step = apo_solve_batch over a batch of synthetic single-track events of the toy
stereo chamber: coarse 16^5-cell voting, top-64, six rounds of bisection + voting + top-64,
and the max-vote estimate (arXiv:2401.04576, Sections 3.1 and 3.3), FP64 intervals.
The metric is (cell, hit) interval evaluations decided per second (coarse cells x hits +
bisected cells x hits, summed over events), with events per second beside it.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl apo|reference]
Under torchrun (N > 1) every rank runs its own batch on its own GPU (weak scaling); the
step time is the maximum over ranks.  --impl reference times the CPU oracle instead (rank
0 only) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("cell-hit interval evals/s and events/s at 1 GB300 (FP32-bulk vs plain FP64); "
          "p50/p99 ms")
WORKLOAD = dict(name="1024 single-track events, 16^5 coarse cells, top-64, 6 bisection levels, "
                     "FP64 intervals", n_events=1024, seed=2, bins=16, levels=6, topk=64)

# Directed floating-point operations of one evaluation of the vote program, by phase:
# per (cell, hit) without tan(lambda), tan(lambda)-dependent part, both drift signs.
# Counted by the oracle's instrumented interval operations (2 per rounding interval
# operation); tests/test_bench_host.py checks these against it.
OPS_PREFIX, OPS_LPART, OPS_SIGNS, OPS_CELL = 176, 117, 60, 2
OPS_FULL = OPS_CELL + OPS_PREFIX + OPS_LPART + OPS_SIGNS
OPS_TAIL = OPS_LPART + OPS_SIGNS


# DRAM bytes (read + write) of one k_vote_coarse<FP64> launch per event: an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, --clock-control none) of one 64-event
# launch of that kernel on the 16^5 grid, in the search's form (each block keeps its K
# best cells), read 496,384 B and wrote 0 B; scaled by events to the benchmark's launch.
# Must be re-captured (or set to None) whenever that kernel changes.
COARSE_F64_DRAM_BYTES_PER_EVENT = 496384 / 64


def coarse_kernel_ops(n_parent: int, n_prefix: int, n_tail: int) -> int:
    """Algorithmic directed FP operations of the coarse vote kernel from its work counters:
    parent-cell tests are full evaluations, each (cell, hit) prefix and each tan(lambda)
    tail as counted."""
    return n_parent * OPS_FULL + n_prefix * OPS_PREFIX + n_tail * OPS_TAIL


def coarse_linear_index(g, params) -> int:
    """Level-0 linear index (d0 fastest, tan(lambda) slowest) of the cell holding params."""
    lin, mul = 0, 1
    for a in range(5):
        n = int(g.bins[a])
        edges = g.lo_edge[a][::1 << g.levels]
        i = int(np.clip(np.searchsorted(edges, params[a], side="right") - 1, 0, n - 1))
        lin += i * mul
        mul *= n
    return lin


def pairs_decided(n_hits: np.ndarray, n_coarse: int, levels: int, topk: int) -> float:
    """(cell, hit) pairs whose vote one step decides: all coarse cells and the topk * 32
    children of every bisection level, times the hits of each event."""
    return float(np.sum(n_hits.astype(np.float64)) * (n_coarse + levels * topk * 32))


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(value: float, world: int) -> float:
    """Maximum of a per-rank number over ranks (identity for one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def make_inputs(seed_offset: int = 0):
    from gen import chamber, grid as G
    w = chamber.make_wires()
    g = G.make_grid([WORKLOAD["bins"]] * 5, WORKLOAD["levels"], WORKLOAD["topk"])
    ev = chamber.single_track_events(WORKLOAD["n_events"], seed=WORKLOAD["seed"] + seed_offset,
                                     w=w)
    return w, g, ev


def headline_latency(loads):
    """The load whose p50 / p99 head the JSON line: the highest offered rate the server
    sustains (nothing rejected and at least 90 % of the offered rate completed per second);
    above it the latencies measure the queue's backlog, not the service.  None if no load
    qualifies."""
    ok = [x for x in loads if x["rejected"] == 0 and x["p50_ms"] is not None
          and x["sustained_per_s"] >= 0.9 * x["offered_per_s"]]
    return max(ok, key=lambda x: x["offered_per_s"]) if ok else None


def serve_sweep(geom, ev, rates, seconds: float, solve, batch_events: int = 64, max_slots: int = 8,
                max_pending: int = 4096) -> list:
    """Poisson arrivals at each offered rate (events/s) into the continuous-batching server
    (search options `solve`), cycling through the batch's events; per rate: sustained
    completions/s, p50 / p99 latency (measured in the library from submission to the batch
    seen complete), rejected submissions (queue full)."""
    import threading
    from paper_2401_04576_gb300 import apo
    evs = [(np.ascontiguousarray(ev.wire_id[ev.offsets[e]:ev.offsets[e + 1]], np.int32),
            np.ascontiguousarray(ev.drift[ev.offsets[e]:ev.offsets[e + 1]], np.float64))
           for e in range(ev.n_events)]
    out = []
    rng = np.random.default_rng(5)
    import sys
    import torch
    switch = sys.getswitchinterval()
    sys.setswitchinterval(2e-4)    # the poller thread sees completions within ~0.2 ms
    for rate in rates:
        srv = apo.Server(geom, solve, batch_events=batch_events, max_slots=max_slots,
                         max_pending=max_pending)
        n = max(64, int(rate * seconds))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, n))
        t_arr = {}
        t_done = {}
        stop = threading.Event()

        def poller():
            while not stop.is_set() or len(t_done) < len(t_arr):
                for rid, _, _ in srv.poll(4096):
                    t_done[rid] = time.perf_counter()
                if stop.is_set() and srv.drain(0) == apo.APO_OK and len(t_done) >= len(t_arr):
                    break
                time.sleep(0.0002)

        th = threading.Thread(target=poller)
        th.start()
        rejected = 0
        clk = ClockSampler(torch.cuda.current_device())
        clk.__enter__()
        t0 = time.perf_counter()
        for i in range(n):
            due = t0 + arrivals[i]
            # sleep (releasing the interpreter lock for the poller) until just before the
            # arrival, then spin the last few hundred microseconds
            while True:
                left = due - time.perf_counter()
                if left <= 0:
                    break
                if left > 4e-4:
                    time.sleep(left - 3e-4)
            w, d = evs[i % len(evs)]
            if srv.submit(w, d, i) == apo.APO_OK:
                t_arr[i] = due
            else:
                rejected += 1
        srv.drain(120000)
        clk.__exit__(None, None, None)
        stop.set()
        th.join(timeout=120)
        lat = np.array([1e3 * (t_done[i] - t_arr[i]) for i in t_arr if i in t_done])
        t_end = max(t_done.values()) if t_done else t0
        batches, max_busy = srv.stats()
        c50, c99, cn = srv.latency()
        srv.close()
        out.append({"offered_per_s": rate, "completed": int(lat.size), "rejected": rejected,
                    "sustained_per_s": lat.size / max(t_end - t0, 1e-9),
                    "p50_ms": c50 if cn else None, "p99_ms": c99 if cn else None,
                    "latency_clock": "library: submit accepted -> batch seen complete",
                    "python_p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
                    "python_p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
                    "batches": batches, "max_slots_in_flight": max_busy,
                    "sm_mhz": clk.summary().get("sm_mhz")})
    sys.setswitchinterval(switch)
    return out


MAXSET = dict(name="1024 single-track events, 2 x 256 x 16 x 2 x 8 coarse cells (d0, phi0, "
                   "omega, z0, tanl), max-set schedule (whole maximum-vote groups, up to "
                   "32768 cells per level), 5 bisection levels, direction condition",
              bins=[2, 256, 16, 2, 8], levels=5, max_keep=32768)


def truth_recovery(g, level_of, tracks_p, tracks_w, truth) -> dict:
    """How the final estimates relate to the generated helices: the fraction of events
    whose estimate box (value +- error, per axis) holds the generated helix, the fraction
    within 1 and within 3 final cells of it on every axis, and the median distance in final
    cells per axis (d0, phi0, omega, z0, tanl).  level_of: the level whose cells are the
    "final cells" of each event."""
    cw = np.stack([[g.hi_edge[a][0] - g.lo_edge[a][0] for a in range(5)]])   # finest cell
    cw = cw * (2.0 ** (g.levels - np.asarray(level_of, np.float64)))[:, None]
    dist = np.abs(tracks_p - truth) / cw
    inside = np.all(np.abs(tracks_p - truth) <= tracks_w * (1 + 1e-12), axis=1)
    return {"in_estimate_box": float(inside.mean()),
            "within_1_final_cell": float(np.mean(np.all(dist <= 1.0, axis=1))),
            "within_3_final_cells": float(np.mean(np.all(dist <= 3.0, axis=1))),
            "median_final_cells": [float(x) for x in np.median(dist, axis=0)],
            "events": int(len(inside))}


def maxset_leg(w, ev, steps: int, flush, world: int = 1, per_event: int = 32) -> dict:
    """The max-set schedule on the anisotropic grid: events/s of the FP32-bulk form (FP32
    levels 0-4, FP64 on the last level) and of the plain FP64 form (every level FP64), both with
    the direction condition; (cell, hit) pairs evaluated per second; the truth recovery of
    each; and the plain FP64 form one event per call (the per-event path: latency and
    events/s)."""
    import torch
    from gen import grid as G
    from paper_2401_04576_gb300 import apo
    g = G.make_grid(MAXSET["bins"], MAXSET["levels"], 64)
    geom = apo.Geometry(g, w)
    hits = apo.DeviceHits.from_events(ev)
    lv, K, ne = g.levels, MAXSET["max_keep"], ev.n_events
    nh = np.diff(ev.offsets).astype(np.float64)
    truth = np.array([t[0].params for t in ev.tracks])
    stream = torch.cuda.current_stream()
    out = {"workload": MAXSET["name"], "n_events": ne, "coarse_cells": geom.n_coarse,
           "levels": lv, "max_keep": K}
    forms = {"fp32_bulk": [apo.F32 | apo.OUTGOING] * lv + [apo.F64 | apo.OUTGOING],
             "fp64": [apo.F64 | apo.OUTGOING] * (lv + 1)}
    sample = apo.DeviceHits.from_events(ev.subset(range(min(128, ne))))
    for name, prec in forms.items():
        fl = torch.zeros(ne, dtype=torch.int32, device="cuda")
        tc = torch.zeros(ne * (lv + 1), dtype=torch.int32, device="cuda")
        # execution knobs picked by apo_autotune on a 128-event sample (no knob changes a result)
        tune, _ = apo.autotune(geom, sample, apo.solve_opts(precision=prec, schedule=apo.SCHED_MAXSET,
                                                            max_keep=K))
        o = apo.solve_opts(precision=prec, schedule=apo.SCHED_MAXSET, max_keep=K,
                           final_level=fl, trace_count=tc, tune=tune)
        ws = geom.workspace(ne, opts=o)
        tracks = torch.zeros(ne * apo.TRACK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        ntr = torch.zeros(ne, dtype=torch.int32, device="cuda")
        apo.solve_batch(geom, hits, o, tracks=tracks, n_tracks=ntr, workspace=ws, stream=stream)
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush.fill_(1)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            apo.solve_batch(geom, hits, o, tracks=tracks, n_tracks=ntr, workspace=ws, stream=stream)
            s1.record(stream)
            s1.synchronize()
            ms.append(s0.elapsed_time(s1))
        t = reduce_max(statistics.mean(ms), world)
        tr = apo.tracks_to_numpy(tracks, ne)[:, 0]
        flv = fl.cpu().numpy()
        kept = tc.cpu().numpy().reshape(ne, lv + 1).astype(np.float64)
        # cells voted per event: the level-0 grid, then 32 children of every kept cell
        cells = geom.n_coarse + 32.0 * kept.sum(axis=1)
        pairs = float(np.sum(cells * nh))
        out[name] = {"precision": ("FP32 levels 0-4, FP64 level 5" if name == "fp32_bulk"
                                   else "FP64 at every level") + ", direction condition",
                     "ms_per_step": t, "events_per_s": ne * world / (t * 1e-3),
                     "tune": tune.as_dict(),
                     "pairs_evaluated_per_s": pairs * world / (t * 1e-3),
                     "cells_per_event_mean": float(cells.mean()),
                     "kept_cells_per_level_max": [int(x) for x in kept.max(axis=0)],
                     "events_ending_early": int(np.sum(flv < lv)),
                     "truth_recovery": truth_recovery(g, flv, tr["p"], tr["w"], truth)}
        del ws
    # the plain FP64 form one event per call, synchronised after each (per-event path)
    o1 = apo.solve_opts(precision=forms["fp64"], schedule=apo.SCHED_MAXSET, max_keep=K)
    ws1 = geom.workspace(1, opts=o1)
    lat = []
    for e in range(min(per_event, ne) + 1):
        sub = apo.DeviceHits.from_events(ev.subset([e]))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        apo.solve_batch(geom, sub, o1, workspace=ws1, stream=stream)
        torch.cuda.synchronize()
        if e > 0:
            lat.append(1e3 * (time.perf_counter() - t0))
    out["fp64_per_event"] = {"events": len(lat), "p50_ms": float(np.percentile(lat, 50)),
                             "p99_ms": float(np.percentile(lat, 99)),
                             "events_per_s": len(lat) / (sum(lat) * 1e-3)}
    out["fp32_bulk_vs_fp64_per_event"] = (out["fp32_bulk"]["events_per_s"] /
                                          out["fp64_per_event"]["events_per_s"])
    geom.close()
    return out


def config1_latency(w, n: int = 50) -> dict:
    """The plain method on one event at a time (10^5 coarse cells, top-16, 4 levels, FP64):
    latency of apo_solve_batch_host (host arrays in, track out) per event, p50 / p99."""
    from gen import chamber, grid as G
    from paper_2401_04576_gb300 import apo
    g = G.make_grid([10] * 5, 4, 16)
    geom = apo.Geometry(g, w)
    ev = chamber.single_track_events(n + 1, seed=1, w=w)
    o = apo.solve_opts(precision=[apo.F64] * 5)
    import torch
    ws = torch.empty(apo.host_workspace_bytes(geom, 1, apo.HIT_CAP, o), dtype=torch.uint8,
                     device="cuda")
    lat = []
    for e in range(n + 1):
        sub = ev.subset([e])
        t0 = time.perf_counter()
        apo.solve_batch_host(geom, sub.offsets, sub.wire_id, sub.drift, o, workspace=ws)
        if e > 0:
            lat.append(1e3 * (time.perf_counter() - t0))
    geom.close()
    return {"workload": "one single-track event per call (seed 1), 10^5 coarse cells, top-16, "
                        "4 levels, FP64, through apo_solve_batch_host",
            "events": n, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99))}


def serving_leg(w, seconds: float) -> dict:
    """Serving (the fifth configuration): Poisson arrivals of uneven multi-track events
    (1-5 helices plus noise, 10-200 hits; "the config-3 distribution" read as the fourth
    configuration, index 3 counted from 0) into apo_serve at 1k-50k events/s, each slot's
    batch through the per-level launches (FP32 levels 0-4, FP64 levels 5-6, up to 5 tracks;
    a 64-event batch is too small for the persistent launch),
    next to the plain FP64 per-event path on the same events (one event per call,
    synchronised)."""
    import torch
    from gen import chamber, grid as G
    from paper_2401_04576_gb300 import apo
    g4 = G.make_grid([10] * 5, 6, 64)
    ev = chamber.multi_track_events(2048, seed=5, w=w)
    geom = apo.Geometry(g4, w)
    solve = apo.solve_opts(precision=[apo.F32] * 5 + [apo.F64] * 2, max_tracks=5, min_votes=6)
    serve_sweep(geom, ev, [1000], 0.25, solve)   # warm-up pass (first-use costs), discarded
    sweep = serve_sweep(geom, ev, [1000, 2000, 5000, 10000, 20000, 50000], seconds, solve)
    o64 = apo.solve_opts(precision=[apo.F64] * 7, max_tracks=5, min_votes=6)
    ws = geom.workspace(1, opts=o64)
    lat = []
    for e in range(65):
        sub = apo.DeviceHits.from_events(ev.subset([e]))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        apo.solve_batch(geom, sub, o64, workspace=ws)
        torch.cuda.synchronize()
        if e > 0:
            lat.append(1e3 * (time.perf_counter() - t0))
    geom.close()
    return {"workload": "Poisson arrivals of 2048 multi-track events (seed 5; 1-5 helices plus "
                        "noise, mean %.1f hits) into apo_serve (64-event slots, 8 slots), "
                        "10^5 coarse cells, top-64, 6 levels, FP32 "
                        "levels 0-4 / FP64 5-6, up to 5 tracks" % (ev.offsets[-1] / ev.n_events),
            "reading": "the config-3 distribution = the uneven multi-track configuration "
                       "(fourth in the list, index 3 counted from 0)",
            "loads": sweep,
            "fp64_per_event_path": {"events": len(lat), "p50_ms": float(np.percentile(lat, 50)),
                                    "p99_ms": float(np.percentile(lat, 99)),
                                    "events_per_s": len(lat) / (sum(lat) * 1e-3),
                                    "precision": "FP64 at every level, one event per call"}}


def background_study(w, n_events: int = 1024, seed: int = 4, n_maxset: int = 512) -> dict:
    """Background-hit rejection of the multi-track hit finding (the study the paper leaves
    for later, Conclusion), on multi-track events with 10-30 % noise occupancy: 10^5 coarse
    cells, top-64, 6 levels, FP32 levels 0-4 / FP64 levels 5-6, up to 5 tracks, min 6 votes.
    A hit counts as taken when a found track's final maximum-vote cells take it (d +- 3
    sigma).  Reported per bin of the event's noise fraction: signal hits taken (efficiency)
    and noise hits left (rejection)."""
    import torch
    from gen import chamber, grid as G
    from paper_2401_04576_gb300 import apo
    g = G.make_grid([10] * 5, 6, 64)
    ev = chamber.multi_track_events(n_events, seed=seed, w=w)
    geom = apo.Geometry(g, w)
    hits = apo.DeviceHits.from_events(ev)
    ht = torch.empty(int(ev.offsets[-1]), dtype=torch.int32, device="cuda")
    prec = [apo.F32] * 5 + [apo.F64] * 2
    launch = {}
    results = {}
    # the same search through the per-level launches recorded as one CUDA graph, through the
    # persistent launch, and with the knobs apo_autotune picks on a 1024-event sample (the
    # persistent launch needs many more events than resident blocks to pay)
    sample = apo.DeviceHits.from_events(ev.subset(range(min(1024, ev.n_events))))
    best, _ = apo.autotune(geom, sample, apo.solve_opts(precision=prec, max_tracks=5, min_votes=6))
    for name, tune, graph in (("graph", apo.ApoTune(0, 1, 256, 0, persistent=0), True),
                              ("persistent", apo.ApoTune(0, 1, 256, 0, persistent=1), False),
                              ("autotuned", best, best.persistent == 0)):
        o = apo.solve_opts(precision=prec, max_tracks=5, min_votes=6, hit_track=ht, tune=tune,
                           use_graph=graph)
        ws = geom.workspace(ev.n_events, opts=o)
        apo.solve_batch(geom, hits, o, workspace=ws)      # warm-up (and graph recording)
        torch.cuda.synchronize()
        mss = []
        for _ in range(2):
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record()
            tracks, nt = apo.solve_batch(geom, hits, o, workspace=ws)
            s1.record()
            s1.synchronize()
            mss.append(s0.elapsed_time(s1))
        launch[name] = {"ms": min(mss), "events_per_s": ev.n_events / (min(mss) * 1e-3),
                        "tune": tune.as_dict()}
        results[name] = (apo.tracks_to_numpy(tracks, ev.n_events, 5).copy(), nt.cpu().numpy().copy(),
                         ht.cpu().numpy().copy())
        del ws
    same = all(np.array_equal(results["graph"][i].view(np.uint8), results[k][i].view(np.uint8))
               for i in range(3) for k in ("persistent", "autotuned"))
    fastest = min(launch, key=lambda k: launch[k]["ms"])
    ms = launch[fastest]["ms"]
    tracks, nt, hts = results[fastest]
    geom.close()
    out = {"workload": f"{ev.n_events} multi-track events (1-5 helices, noise fraction "
                       "0.08-0.31, mean %.1f hits), 10^5 coarse cells, top-64, 6 levels, "
                       "FP32 L0-4 / FP64 L5-6, <= 5 tracks, min 6 votes" % (ev.offsets[-1] / ev.n_events),
           "events_per_s": ev.n_events / (ms * 1e-3),
           "launch_schedules": launch, "schedules_give_identical_results": bool(same)}
    out.update(multi_track_figures(ev, tracks, nt, hts))
    # the max-set extraction on the first n_maxset of the events (it runs about 130x
    # longer per event than the top-K one)
    out["maxset"] = multi_maxset_leg(w, ev.subset(range(min(n_maxset, ev.n_events))))
    return out


def multi_track_figures(ev, tracks, nt, hit_track) -> dict:
    """Hit and track figures of a multi-track extraction against the generator's truth: the
    signal hits taken and noise hits left (overall and per bin of the event's noise
    fraction), the true tracks whose helix lies in some found track's estimate box (value
    +- error per axis) per true track, and the found tracks whose box holds no true helix."""
    taken = hit_track >= 0
    bins = [(0.0, 0.15), (0.15, 0.20), (0.20, 0.25), (0.25, 1.0)]
    acc = {b: [0, 0, 0, 0, 0, 0, 0, 0] for b in bins}   # sig, sig taken, noise, noise taken, ev, found, true, matched
    fakes = 0
    for e in range(ev.n_events):
        a, b = int(ev.offsets[e]), int(ev.offsets[e + 1])
        noise = np.array([h is None for h in ev.hit_truth[e]])
        frac = noise.mean()
        key = next(k for k in bins if k[0] <= frac < k[1])
        t = taken[a:b]
        truth = np.array([tr.params for tr in ev.tracks[e]])
        matched = np.zeros(len(truth), bool)
        for k in range(int(nt[e])):
            ins = np.all(np.abs(tracks[e, k]["p"] - truth) <= tracks[e, k]["w"] * (1 + 1e-12), axis=1)
            matched |= ins
            fakes += int(not ins.any())
        x = acc[key]
        x[0] += int((~noise).sum()); x[1] += int((t & ~noise).sum())
        x[2] += int(noise.sum()); x[3] += int((t & noise).sum())
        x[4] += 1; x[5] += int(nt[e]); x[6] += len(truth); x[7] += int(matched.sum())
    rows = []
    tot = np.zeros(8, np.int64)
    for k in bins:
        x = acc[k]
        tot += np.array(x)
        if x[4]:
            rows.append({"noise_fraction": [k[0], min(k[1], 1.0)], "events": x[4],
                         "signal_hits_taken": x[1] / max(x[0], 1),
                         "noise_hits_rejected": 1.0 - x[3] / max(x[2], 1),
                         "tracks_found_per_event": x[5] / x[4],
                         "true_tracks_per_event": x[6] / x[4],
                         "true_tracks_in_a_found_box": x[7] / max(x[6], 1)})
    return {"signal_hits_taken": tot[1] / max(tot[0], 1),
            "noise_hits_rejected": 1.0 - tot[3] / max(tot[2], 1),
            "tracks_found_per_true_track": tot[5] / max(tot[6], 1),
            "true_tracks_in_a_found_box": tot[7] / max(tot[6], 1),
            "found_tracks_holding_no_true_helix": fakes / max(tot[5], 1),
            "by_noise_fraction": rows}


def multi_maxset_leg(w, ev) -> dict:
    """The same multi-track events through the max-set schedule (anisotropic grid, FP32
    levels 0-4 / FP64 level 5, direction condition, max_keep 32768, slack 6, <= 5 tracks,
    min 6 votes): each round keeps one hit-set cluster of the final maximum-vote group."""
    import torch
    from gen import grid as G
    from paper_2401_04576_gb300 import apo
    g = G.make_grid(MAXSET["bins"], MAXSET["levels"], 64)
    geom = apo.Geometry(g, w)
    hits = apo.DeviceHits.from_events(ev)
    ht = torch.empty(int(ev.offsets[-1]), dtype=torch.int32, device="cuda")
    prec = [apo.F32 | apo.OUTGOING] * MAXSET["levels"] + [apo.F64 | apo.OUTGOING]
    tune = apo.ApoTune(0, 1, 256, 0)
    o = apo.solve_opts(precision=prec, schedule=apo.SCHED_MAXSET, max_keep=MAXSET["max_keep"], slack=6,
                       max_tracks=5, min_votes=6, hit_track=ht, tune=tune)
    ws = geom.workspace(ev.n_events, opts=o)
    tracks, nt = apo.solve_batch(geom, hits, o, workspace=ws)      # warm-up
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record()
    tracks, nt = apo.solve_batch(geom, hits, o, tracks=tracks, n_tracks=nt, workspace=ws)
    s1.record()
    s1.synchronize()
    ms = s0.elapsed_time(s1)
    res = {"workload": "the same events; 2 x 256 x 16 x 2 x 8 coarse cells, max-set schedule "
                       "(max_keep 32768, slack 6), 5 bisection levels, direction condition; FP32 "
                       "levels 0-4, FP64 level 5; <= 5 tracks, min 6 votes; one hit-set cluster "
                       "of the final maximum-vote group per round",
           "events_per_s": ev.n_events / (ms * 1e-3), "ms": ms, "tune": tune.as_dict()}
    res.update(multi_track_figures(ev, apo.tracks_to_numpy(tracks, ev.n_events, 5), nt.cpu().numpy(),
                                   ht.cpu().numpy()))
    del ws
    geom.close()
    return res


def paper_search_leg(n_events: int = 512, seed: int = 70, cpu_events: int = 1, n_fp64: int = 64) -> dict:
    """The paper's own search (Sections 3.1-3.3): COMET-like toy, 105 MeV/c electrons, 4-D
    voxels x_c x y_c x R x z0 with two tan(lambda) accumulators, disk pre-filter, midpoint
    form, the three iterations of Table tabGridDef with hit finding and the moving
    reference point; time per track in FP64 and FP32 and the resolution per iteration
    (Table HelixParametes' quantities).  FP64 runs on the first n_fp64 events (its time
    per track is the same on any batch of thousands of blocks), FP32 on all.  cpu_events
    > 0 also times the oracle on that many events (host cores)."""
    import torch
    from gen import comet
    from paper_2401_04576_gb300 import apo
    w = comet.make_wires()
    ev = comet.events(n_events, seed=seed, w=w)
    ch = apo.Chamber4(w)
    hits = apo.DeviceHits.from_events(ev)
    res = {"workload": f"{ev.n_events} electrons of 105 MeV/c from the origin in a 20-layer, "
                       f"4,986-wire chamber (mean {ev.offsets[-1] / ev.n_events:.1f} hits, noiseless), "
                       "3 iterations of Table tabGridDef (2M / 6.5M / 2.5M voxels x 2 signs before "
                       "the disk filter), midpoint form",
           "paper_context": {"s_per_track_4xK80": 1.2, "s_per_track_V100": 0.2,
                             "rms_mm_iter3": {"x_c": 0.23, "y_c": 0.23, "R": 0.19, "z0": 2.68},
                             "wrong_sign_fraction": [0.166, 0.047, 0.0],
                             "within_1mm_10mm": 0.997}}
    ev_all, hits_all = ev, hits
    # iteration 3 per tan(lambda) sign (the default), and FP32 on iteration 2's box alone
    for prec, name, ps in ((apo.F64, "fp64", 1), (apo.F32, "fp32", 1), (apo.F32, "fp32_one_box", 0)):
        ev = ev_all.subset(range(min(n_fp64, ev_all.n_events))) if prec == apo.F64 else ev_all
        hits = apo.DeviceHits.from_events(ev) if prec == apo.F64 else hits_all
        o = apo.four_opts(precision=prec, per_sign=ps)
        ws = ch.workspace(ev.n_events, o)
        out, sel = apo.solve4(ch, hits, o, workspace=ws)
        torch.cuda.synchronize()
        ms = []
        for _ in range(2):
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record()
            apo.solve4(ch, hits, o, out=out, selected=sel, workspace=ws)
            s1.record()
            s1.synchronize()
            ms.append(s0.elapsed_time(s1))
        r = apo.iters4_to_numpy(out, ev.n_events, 3)
        iters = []
        for k in range(3):
            d = []
            for e in range(ev.n_events):
                tr = ev.tracks[e][0]
                xc, yc, R = comet.helix_centre(tr)
                z0 = comet.z_at_point(tr, *r[e, k]["ref"])
                v = r[e, k]["value"]
                d.append([v[0] - xc, v[1] - yc, v[2] - R, v[3] - z0,
                          float(r[e, k]["sign"] != (1 if tr.tanl > 0 else -1))])
            d = np.array(d)
            iters.append({"mean_mm": dict(zip(("x_c", "y_c", "R", "z0"), (d[:, :4].mean(0) * 1e3).round(3).tolist())),
                          "rms_mm": dict(zip(("x_c", "y_c", "R", "z0"), (d[:, :4].std(0) * 1e3).round(3).tolist())),
                          "wrong_sign_fraction": float(d[:, 4].mean()),
                          "within_1mm_10mm": float(np.mean((np.abs(d[:, :3]) < 1e-3).all(1) &
                                                           (np.abs(d[:, 3]) < 1e-2)))})
        t = min(ms)
        res[name] = {"ms_per_track": t / ev.n_events, "tracks_per_s": ev.n_events / (t * 1e-3),
                     "batch_ms": t, "tracks": ev.n_events, "iteration_3": "per sign" if ps else
                     "both signs on iteration 2's box", "iterations": iters}
    ch.close()
    ev = ev_all
    if cpu_events > 0:
        from gen import grid as G
        from oracle import oracle as O
        tab = O.Tables(G.make_grid([4] * 5, 1, 4), w)
        oo = O.four_opts()
        t0 = time.perf_counter()
        for e in range(cpu_events):
            a, b = ev.offsets[e], ev.offsets[e + 1]
            O.four_solve_event(oo, tab, ev.wire_id[a:b], ev.drift[a:b])
        dt = time.perf_counter() - t0
        res["cpu_oracle"] = {"s_per_track": dt / cpu_events, "cores": O.num_threads(),
                             "kind": "oracle", "sample": f"{cpu_events} event(s), FP64, all 3 iterations"}
    return res


def cpu_baseline(w, g, ev, n_sample: int) -> dict:
    """The oracle as it stands, on the host cores, over the first n_sample events (full
    coarse-to-fine search each)."""
    from oracle import oracle as O
    tab = O.Tables(g, w)
    nh = np.diff(ev.offsets)[:n_sample]
    t0 = time.perf_counter()
    for e in range(n_sample):
        a, b = ev.offsets[e], ev.offsets[e + 1]
        O.solve_event(tab, ev.wire_id[a:b], ev.drift[a:b])
    dt = time.perf_counter() - t0
    pairs = pairs_decided(nh, g.n_coarse(), g.levels, g.topk)
    return {"value": pairs / dt, "unit": "evals/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{n_sample} of the {ev.n_events} events, full search each "
                      f"({pairs:.3g} pair evaluations, {dt:.1f} s wall)",
            "events_per_s": n_sample / dt}


def run_reference(args) -> None:
    world, rank, _ = dist_env()
    if rank != 0:
        return
    w, g, ev = make_inputs()
    from oracle import oracle as O
    tab = O.Tables(g, w)
    n_sample = 1
    times = []
    for i in range(args.warmup + args.steps):
        e = i % ev.n_events
        a, b = ev.offsets[e], ev.offsets[e + 1]
        t0 = time.perf_counter()
        O.solve_event(tab, ev.wire_id[a:b], ev.drift[a:b])
        if i >= args.warmup:
            times.append((time.perf_counter() - t0, b - a))
    dt = sum(t for t, _ in times)
    pairs = sum(pairs_decided(np.array([n]), g.n_coarse(), g.levels, g.topk) for _, n in times)
    val = pairs / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "evals/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD["name"],
                   "sample": f"{n_sample} event per step (of {WORKLOAD['n_events']})"},
        "events_per_s": len(times) / dt,
        "cpu_baseline": {"value": val, "unit": "evals/s", "cores": O.num_threads(),
                         "kind": "oracle", "sample": f"{n_sample} event per step"},
        "e2e": {"value": val, "unit": "evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


def run_apo(args) -> None:
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2401_04576_gb300 import apo

    w, g, ev = make_inputs(seed_offset=rank)
    nh = np.diff(ev.offsets)
    geom = apo.Geometry(g, w)
    hits = apo.DeviceHits.from_events(ev)
    lv = g.levels
    opts64 = apo.solve_opts(precision=[apo.F64] * (lv + 1))
    # the precision form: knobs from apo_autotune on a 256-event sample (results unchanged)
    tune32, _ = apo.autotune(geom, apo.DeviceHits.from_events(ev.subset(range(256))),
                             apo.solve_opts(precision=[apo.F32] * 5 + [apo.F64] * (lv + 1 - 5)))
    opts32 = apo.solve_opts(precision=[apo.F32] * 5 + [apo.F64] * (lv + 1 - 5), tune=tune32)
    # one workspace for both forms: the larger of their layouts (the tuned chunk size and
    # vote form decide the FP32-bulk one)
    ws = torch.empty(max(geom.workspace_bytes(ev.n_events), geom.workspace_bytes(ev.n_events, opts32)),
                     dtype=torch.uint8, device="cuda")
    tracks = torch.zeros(ev.n_events * apo.TRACK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    ntr = torch.zeros(ev.n_events, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB L2
    stream = torch.cuda.current_stream()

    def step(o):
        apo.solve_batch(geom, hits, o, tracks=tracks, n_tracks=ntr, workspace=ws, stream=stream)

    def timed(o, steps, warmup):
        for _ in range(warmup):
            step(o)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush.fill_(1)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            step(o)
            s1.record(stream)
            s1.synchronize()
            ms.append(s0.elapsed_time(s1))
        torch.cuda.synchronize()
        barrier(world)
        return ms

    with ClockSampler(local) as clk:
        ms64 = timed(opts64, args.steps, args.warmup)
    clocks = clk.summary()
    t_step = reduce_max(sum(ms64) / len(ms64), world)
    pairs = pairs_decided(nh, geom.n_coarse, lv, g.topk)
    value = pairs * world / (t_step * 1e-3)

    tracks64 = apo.tracks_to_numpy(tracks, ev.n_events).copy()
    # the same FP64 search with the knobs apo_autotune picks (the FP32-first filter on the
    # coarse grid gives the same FP64 votes): reported beside the headline, whose roofline
    # stays the plain FP64 kernel's
    tune64, _ = apo.autotune(geom, apo.DeviceHits.from_events(ev.subset(range(256))), opts64)
    ms64t = timed(apo.solve_opts(precision=[apo.F64] * (lv + 1), tune=tune64), max(2, args.steps), 1)
    t64t = reduce_max(sum(ms64t) / len(ms64t), world)
    same64 = bool(np.array_equal(apo.tracks_to_numpy(tracks, ev.n_events).view(np.uint8),
                                 tracks64.view(np.uint8)))
    # FP32-bulk precision form on the same events (FP32 coarse + levels 1-4, FP64 5-6)
    ms32 = timed(opts32, max(2, args.steps), 1)
    t32 = reduce_max(sum(ms32) / len(ms32), world)
    tracks32 = apo.tracks_to_numpy(tracks, ev.n_events).copy()
    # its two correctness figures: final helix within one final cell width of the FP64
    # result (per axis), and FP32 coarse votes >= FP64 coarse votes cell by cell
    fine_w = np.array([g.hi_edge[a][0] - g.lo_edge[a][0] for a in range(5)])
    dp = np.abs(tracks32["p"][:, 0, :] - tracks64["p"][:, 0, :])
    agree = float(np.mean(np.all(dp <= fine_w[None, :] * (1 + 1e-9), axis=1)))
    truth = np.array([t[0].params for t in ev.tracks])
    rec64 = truth_recovery(g, np.full(ev.n_events, lv), tracks64["p"][:, 0, :],
                           tracks64["w"][:, 0, :], truth)
    rec32 = truth_recovery(g, np.full(ev.n_events, lv), tracks32["p"][:, 0, :],
                           tracks32["w"][:, 0, :], truth)

    # roofline of the dominant kernel (coarse vote, in the form the search runs: each block
    # keeps its K best cells): counted work / live launch time
    votes = apo.vote(geom, hits, precision=apo.F64, workspace=ws, stream=stream)
    votes32 = apo.vote(geom, hits, precision=apo.F32, workspace=ws, stream=stream)
    superset_violations = int((votes32 < votes).sum().item())
    n_cells_cmp = int(votes.numel())
    del votes32
    L = apo.lib()
    hc = hits.c()
    import ctypes as C

    def coarse_counts(prec):
        c = torch.zeros(8, dtype=torch.int64, device="cuda")
        apo._check(L.apo_diag_vote_coarse_counts(geom.handle, C.byref(hc), prec, None, apo._ptr(c),
                                                 apo._ptr(ws), ws.numel(), apo._stream_ptr(stream)))
        return [int(x) for x in c.cpu().tolist()]

    def coarse_launch_ms(prec, n_launch, reps, full=None):
        # full: a vote array for the full-vote form; None: each block keeps its K best cells
        out = []
        for _ in range(reps):
            flush.fill_(1)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            apo._check(L.apo_diag_vote_coarse_counts(geom.handle, C.byref(hc), prec,
                                                     None if full is None else apo._ptr(full), None,
                                                     apo._ptr(ws), ws.numel(), apo._stream_ptr(stream)))
            s1.record(stream)
            s1.synchronize()
            out.append(s0.elapsed_time(s1) / max(n_launch, 1))
        return statistics.mean(out)

    n_par, n_pre, n_tail, n_launch, p32, q32, t32c, _ = coarse_counts(apo.F64)
    c32 = coarse_counts(apo.F32)
    # the FP32 coarse kernel (dominant in the FP32-bulk solve): counted FP32 directed
    # operations / live launch time, against the measured FP32 directed add/mul rate
    ops32_coarse = coarse_kernel_ops(c32[4], c32[5], c32[6]) / max(c32[3], 1)
    # in the form the tuned FP32-bulk step runs (full votes or per-block candidates)
    full32 = bool(tune32.coarse_full)
    k32_ms = coarse_launch_ms(apo.F32, c32[3], max(3, args.steps), full=votes if full32 else None)
    peak32 = apo.pipe_peak(apo.F32)
    roofline32 = {"bound": "issue", "kernel": "k_vote_coarse<float>",
                  "form": "full votes" if full32 else "per-block K best cells",
                  "achieved": ops32_coarse / (k32_ms * 1e-3) / 1e12, "peak": peak32 / 1e12,
                  "unit": "TFLOP/s", "frac": ops32_coarse / (k32_ms * 1e-3) / peak32,
                  "launch_ms": k32_ms, "ops_per_launch": ops32_coarse,
                  "peak_source": "measured: libapo directed-rounding FP32 add/mul microbenchmark "
                                 "(apo_diag_pipe_peak) on this GPU, this run",
                  "work": {"fp32_parent": c32[4], "fp32_prefix": c32[5], "fp32_tail": c32[6],
                           "launches": c32[3]}}
    ops_launch = coarse_kernel_ops(n_par, n_pre, n_tail) / max(n_launch, 1)
    ops32_launch = coarse_kernel_ops(p32, q32, t32c) / max(n_launch, 1)
    k_ms = coarse_launch_ms(apo.F64, n_launch, max(2, args.steps))
    peak = apo.pipe_peak(apo.F64)
    achieved = ops_launch / (k_ms * 1e-3)
    ev_per_launch = ev.n_events / max(n_launch, 1)
    traffic = (None if COARSE_F64_DRAM_BYTES_PER_EVENT is None
               else COARSE_F64_DRAM_BYTES_PER_EVENT * ev_per_launch)
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "traffic_source": "ncu dram__bytes_read+write of a 64-event launch, scaled by "
                                  "events to this launch",
                "kernel": "k_vote_coarse<double>",
                "peak_source": "measured: libapo directed-rounding FP64 add/mul microbenchmark "
                               "(apo_diag_pipe_peak) on this GPU, this run",
                "ops_per_launch": ops_launch, "launch_ms": k_ms,
                "fp32_filter_ops_per_launch": ops32_launch,
                "fp32_filter_tflops": ops32_launch / (k_ms * 1e-3) / 1e12,
                "work": {"fp64_parent": n_par, "fp64_prefix": n_pre, "fp64_tail": n_tail,
                         "fp32_parent": p32, "fp32_prefix": q32, "fp32_tail": t32c,
                         "launches": n_launch}}

    # midpoint form (Section 3.1: the quantities of d^Ax at the voxel centre): coarse launch
    # time against the interval program's, solve throughput, and how its votes differ
    midpoint = None
    if not args.no_mid:
        vmid = torch.empty_like(votes)
        mms = []
        for _ in range(max(2, args.steps)):
            flush.fill_(1)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            apo.vote(geom, hits, precision=apo.F64_MID, out=vmid, workspace=ws, stream=stream)
            s1.record(stream)
            s1.synchronize()
            mms.append(s0.elapsed_time(s1) / n_launch)
        m_ms = statistics.mean(mms)
        diff = vmid - votes
        ncell = diff.numel()
        truth_lin = np.array([coarse_linear_index(g, ev.tracks[e][0].params) for e in range(ev.n_events)])
        rows = torch.arange(ev.n_events, device="cuda")
        tl = torch.as_tensor(truth_lin, device="cuda")
        t64 = votes[rows, tl].to(torch.int64)
        tmid = vmid[rows, tl].to(torch.int64)
        opts_mid = apo.solve_opts(precision=[apo.F64_MID] * (lv + 1))
        msm = timed(opts_mid, max(2, args.steps), 1)
        tm = reduce_max(sum(msm) / len(msm), world)
        tracks_mid = apo.tracks_to_numpy(tracks, ev.n_events).copy()
        dpm = np.abs(tracks_mid["p"][:, 0, :] - tracks64["p"][:, 0, :])
        midpoint = {
            "precision": "midpoint form at every level (FP64 point part, FP64 interval part)",
            "coarse_launch_ms": m_ms, "coarse_launch_ms_fp64_intervals": k_ms,
            "coarse_speedup_vs_fp64_intervals": k_ms / m_ms,
            "ms_per_step": tm, "value": pairs * world / (tm * 1e-3), "unit": "evals/s",
            "events_per_s": ev.n_events * world / (tm * 1e-3),
            "coarse_cells_differing": (diff != 0).sum().item() / ncell,
            "coarse_cells_more_votes": (diff > 0).sum().item() / ncell,
            "coarse_cells_fewer_votes": (diff < 0).sum().item() / ncell,
            "coarse_mean_abs_vote_difference": diff.abs().sum(dtype=torch.int64).item() / ncell,
            "truth_cell_votes_lost_mean": float((t64 - tmid).clamp(min=0).float().mean().item()),
            "truth_cell_events_losing_votes": float(((tmid < t64).float().mean()).item()),
            "final_within_one_cell_of_fp64": float(np.mean(np.all(dpm <= fine_w[None, :] * (1 + 1e-9),
                                                                  axis=1))),
        }
        del vmid, diff

    # exact phase (Eq. CSAXtoPHI_a enclosed instead of expanded) on the first 256 events:
    # coarse launch time against the expansion's, vote differences, whole-search time
    exact = None
    if not args.no_exact:
        sub = ev.subset(range(min(256, ev.n_events)))
        hs = apo.DeviceHits.from_events(sub)
        v64 = apo.vote(geom, hs, precision=apo.F64, workspace=ws, stream=stream)
        vex = torch.empty_like(v64)
        ems, fms = [], []
        for _ in range(2):
            for prec_, acc, out_ in ((apo.F64_EXACT, ems, vex), (apo.F64, fms, v64)):
                flush.fill_(1)
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s0.record(stream)
                apo.vote(geom, hs, precision=prec_, out=out_, workspace=ws, stream=stream)
                s1.record(stream)
                s1.synchronize()
                acc.append(s0.elapsed_time(s1))
        dv = vex - v64
        nc = dv.numel()
        tr_sub = torch.zeros(sub.n_events * apo.TRACK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        nt_sub = torch.zeros(sub.n_events, dtype=torch.int32, device="cuda")
        # the expansion on the two coarsest levels (their wide cells defeat the inclusion
        # proof, and a failed proof votes), the exact phase on levels 2 .. lv
        oex = apo.solve_opts(precision=[apo.F64] * 2 + [apo.F64_EXACT] * (lv - 1))
        apo.solve_batch(geom, hs, oex, tracks=tr_sub, n_tracks=nt_sub, workspace=ws, stream=stream)
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        apo.solve_batch(geom, hs, oex, tracks=tr_sub, n_tracks=nt_sub, workspace=ws, stream=stream)
        s1.record(stream)
        s1.synchronize()
        t_ex = s0.elapsed_time(s1)
        tex = apo.tracks_to_numpy(tr_sub, sub.n_events)
        dpx = np.abs(tex["p"][:, 0, :] - tracks64["p"][:sub.n_events, 0, :])
        exact = {"precision": "FP64 intervals; coarse figures: exact phase on the level-0 grid; "
                              "search: expansion on levels 0-1, exact phase on levels 2-6",
                 "events": sub.n_events,
                 "coarse_ms": min(ems), "coarse_ms_expansion": min(fms),
                 "coarse_cost_vs_expansion": min(ems) / min(fms),
                 "coarse_cells_differing": (dv != 0).sum().item() / nc,
                 "coarse_cells_more_votes": (dv > 0).sum().item() / nc,
                 "coarse_cells_fewer_votes": (dv < 0).sum().item() / nc,
                 "search_events_per_s": sub.n_events / (t_ex * 1e-3),
                 "final_within_one_cell_of_expansion": float(np.mean(np.all(dpx <= fine_w[None, :] * (1 + 1e-9), axis=1)))}
        del v64, vex, dv

    # end to end through the host-buffer entry point (pinned host inputs, tracks back)
    off_h = torch.from_numpy(np.ascontiguousarray(ev.offsets, np.int32)).pin_memory()
    wid_h = torch.from_numpy(np.ascontiguousarray(ev.wire_id, np.int32)).pin_memory()
    dr_h = torch.from_numpy(np.ascontiguousarray(ev.drift, np.float64)).pin_memory()
    wsh = torch.empty(apo.host_workspace_bytes(geom, ev.n_events, int(ev.offsets[-1])),
                      dtype=torch.uint8, device="cuda")
    out_h = np.zeros((ev.n_events, 1), apo.TRACK_DTYPE)
    e2e_ms = []
    for i in range(1 + max(2, args.steps)):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        apo.solve_batch_host(geom, off_h.numpy(), wid_h.numpy(), dr_h.numpy(), opts64,
                             workspace=wsh, out=out_h, stream=stream)
        if i > 0:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    t_e2e = reduce_max(statistics.mean(e2e_ms), world)
    h2d = 4 * (ev.n_events + 1) + 12 * int(ev.offsets[-1])
    d2h = apo.TRACK_DTYPE.itemsize * ev.n_events + 4 * ev.n_events

    launches = apo.solve_launches(geom, ev.n_events)
    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD["name"], "n_events": ev.n_events,
                   "coarse_cells": geom.n_coarse, "topk": g.topk, "levels": lv,
                   "hits_per_event_mean": float(nh.mean()),
                   "hits_per_event_reading": "the configuration's hit rule (closest approach "
                                             "under half a cell) gives about one wire per "
                                             "layer of the 10-layer chamber, so ~10 hits, not "
                                             "the ~20 its text estimates; tracks with fewer "
                                             "than 6 hits are redrawn",
                   "l2": "flushed between timed steps (256 MiB write)"},
        "events_per_s": ev.n_events * world / (t_step * 1e-3),
        "pairs": {"decided_per_step": pairs,
                  "note": "value counts every (cell, hit) pair whose vote a step decides: "
                          "coarse cells x hits + bisected cells x hits.  The coarse kernel "
                          "decides most of them without evaluating the pair: the exact "
                          "parent-cell test and the shared tan(lambda)-free prefix",
                  "coarse_decided_per_step": float(np.sum(nh)) * geom.n_coarse,
                  "coarse_tails_evaluated_per_step": float(n_tail),
                  "coarse_prefixes_evaluated_per_step": float(n_pre),
                  "refine_evaluated_per_step": float(np.sum(nh)) * lv * g.topk * 32},
        "truth_recovery": rec64,
        "fp64_autotuned": {"ms_per_step": t64t, "value": pairs * world / (t64t * 1e-3),
                           "unit": "evals/s", "events_per_s": ev.n_events * world / (t64t * 1e-3),
                           "tune": tune64.as_dict(), "tracks_identical_to_headline": same64},
        "fp32_bulk": {"ms_per_step": t32, "value": pairs * world / (t32 * 1e-3),
                      "unit": "evals/s", "events_per_s": ev.n_events * world / (t32 * 1e-3),
                      "precision": "FP32 levels 0-4, FP64 levels 5-6",
                      "tune": tune32.as_dict(),
                      "final_within_one_cell_of_fp64": agree,
                      "truth_recovery": rec32,
                      "coarse_superset_violations": superset_violations,
                      "coarse_cells_compared": n_cells_cmp,
                      "coarse_roofline": roofline32},
        "step_ms_p50": float(np.percentile(ms64, 50)), "step_ms_p99": float(np.percentile(ms64, 99)),
        "e2e": {"value": pairs * world / (t_e2e * 1e-3), "unit": "evals/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": t_e2e},
        "gpu_launches": launches * args.steps,
        "clocks": clocks,
        "roofline": roofline,
    }
    if midpoint is not None:
        line["midpoint"] = midpoint
    if exact is not None:
        line["exact_phase"] = exact
    if not args.no_serve:
        line["serving"] = serving_leg(w, args.serve_seconds)
        best = headline_latency(line["serving"]["loads"])
        if best is not None:
            line["p50_ms"] = best["p50_ms"]
            line["p99_ms"] = best["p99_ms"]
            line["p50_p99_at_offered_per_s"] = best["offered_per_s"]
    if not args.no_maxset:
        line["recovery_maxset"] = maxset_leg(w, ev, max(2, args.steps), flush, world)
    if rank == 0 and not args.no_bg:
        line["background_rejection"] = background_study(w, n_events=args.bg_events,
                                                        n_maxset=args.bg_maxset_events)
    if rank == 0 and not args.no_config1:
        line["config1_latency"] = config1_latency(w)
    if rank == 0 and not args.no_paper4d:
        line["paper_search_4d"] = paper_search_leg(cpu_events=0 if args.no_cpu_baseline else 1)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, g, ev, args.cpu_sample)
    if rank == 0:
        print(json.dumps(line))
    geom.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_case(args) -> None:
    """Small profiling case: one warm-up and one measured call of a single kernel family on
    the first --events events of the workload (for ncu captures of one launch)."""
    import torch
    from paper_2401_04576_gb300 import apo
    if args.case.startswith("four"):
        from gen import comet
        w4 = comet.make_wires()
        ev4 = comet.events(args.events, seed=70, w=w4)
        ch = apo.Chamber4(w4)
        h4 = apo.DeviceHits.from_events(ev4)
        o4 = apo.four_opts(precision=apo.F32 if args.case == "four-f32" else apo.F64)
        ws4 = ch.workspace(ev4.n_events, o4)
        for _ in range(2):
            apo.solve4(ch, h4, o4, workspace=ws4)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "events": ev4.n_events, "ok": True}))
        return
    if args.case in ("solve-maxset", "solve-maxset-multi"):
        # the max-set leg's FP32-bulk form on the first events (single-track events, or the
        # multi-track events of the background study with up to 5 tracks)
        from gen import chamber, grid as G
        w = chamber.make_wires()
        ga = G.make_grid(MAXSET["bins"], MAXSET["levels"], 64)
        multi = args.case == "solve-maxset-multi"
        ev = (chamber.multi_track_events(args.events, seed=4, w=w) if multi else
              chamber.single_track_events(args.events, seed=WORKLOAD["seed"], w=w))
        geom = apo.Geometry(ga, w)
        o = apo.solve_opts(precision=[apo.F32 | apo.OUTGOING] * ga.levels + [apo.F64 | apo.OUTGOING],
                           schedule=apo.SCHED_MAXSET, max_keep=MAXSET["max_keep"],
                           tune=apo.ApoTune(0, 1, 256, 0, 0) if multi else apo.ApoTune(0, 0, 128, 0, 0),
                           slack=6 if multi else 0,
                           max_tracks=5 if multi else 1, min_votes=6 if multi else 0)
        hits = apo.DeviceHits.from_events(ev)
        for _ in range(2):
            apo.solve_batch(geom, hits, o)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "events": ev.n_events, "ok": True}))
        return
    if args.case == "solve-persist":   # the multi-track batch through the persistent launch
        from gen import chamber, grid as G
        w = chamber.make_wires()
        g4 = G.make_grid([10] * 5, 6, 64)
        ev = chamber.multi_track_events(args.events, seed=4, w=w)
        geom = apo.Geometry(g4, w)
        o = apo.solve_opts(precision=[apo.F32] * 5 + [apo.F64] * 2, max_tracks=5, min_votes=6,
                           tune=apo.ApoTune(0, 1, 256, 0, persistent=1))
        hits = apo.DeviceHits.from_events(ev)
        for _ in range(2):
            apo.solve_batch(geom, hits, o)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "events": ev.n_events, "ok": True}))
        return
    w, g, ev = make_inputs()
    ev = ev.subset(range(args.events))
    geom = apo.Geometry(g, w)
    hits = apo.DeviceHits.from_events(ev)
    ws = geom.workspace(ev.n_events)
    prec = (apo.F64_MID if args.case == "coarse-mid" else
            apo.F64 if args.case.endswith("f64") else apo.F32)
    if args.case == "coarse-mid":
        votes = torch.empty((ev.n_events, geom.n_coarse), dtype=torch.int32, device="cuda")
        for _ in range(2):
            apo.vote(geom, hits, precision=prec, out=votes, workspace=ws)
    elif args.case.startswith("coarse"):   # each block keeps its K best cells, or (-full) every vote
        import ctypes as C
        hc = hits.c()
        full = (torch.empty((ev.n_events, geom.n_coarse), dtype=torch.int32, device="cuda")
                if args.case.endswith("-full") else None)
        for _ in range(2):
            apo._check(apo.lib().apo_diag_vote_coarse_counts(geom.handle, C.byref(hc), prec,
                                                             None if full is None else apo._ptr(full),
                                                             None, apo._ptr(ws), ws.numel(),
                                                             apo._stream_ptr(None)))
    else:
        precision = ([apo.F32] * 5 + [apo.F64] * (g.levels + 1 - 5) if args.case == "solve-bulk"
                     else [prec] * (g.levels + 1))
        o = apo.solve_opts(precision=precision)
        for _ in range(2):
            apo.solve_batch(geom, hits, o, workspace=ws)
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "events": ev.n_events, "ok": True}))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="apo", choices=["apo", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-mid", action="store_true", help="skip the midpoint-form leg")
    ap.add_argument("--no-bg", action="store_true", help="skip the background-rejection study")
    ap.add_argument("--no-paper4d", action="store_true", help="skip the paper's own 4-D search")
    ap.add_argument("--no-exact", action="store_true", help="skip the exact-phase leg")
    ap.add_argument("--no-maxset", action="store_true", help="skip the max-set (recovery) leg")
    ap.add_argument("--no-config1", action="store_true", help="skip the one-event latency leg")
    ap.add_argument("--bg-events", type=int, default=4096,
                    help="events of the multi-track background study")
    ap.add_argument("--bg-maxset-events", type=int, default=512,
                    help="of them, events of its max-set extraction (about 35 events/s)")
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--case", default=None,
                    choices=["coarse-f64", "coarse-f32", "coarse-f32-full", "coarse-mid", "solve-f64",
                             "solve-f32", "solve-bulk", "solve-maxset", "solve-maxset-multi", "solve-persist",
                             "four-f32", "four-f64"],
                    help="run one small profiling case instead of the benchmark")
    ap.add_argument("--events", type=int, default=64)
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.case:
        run_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_apo(args)


if __name__ == "__main__":
    main()
