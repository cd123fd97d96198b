"""Thin ctypes binding of libapo.so (include/apo.h): argument marshalling only.

Device memory and streams come from PyTorch; every step of the hot path runs in the
library's CUDA kernels.  There is no CPU fallback: loading fails loudly when the library
is missing, and calls raise when CUDA is unusable.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

APO_OK, APO_EINVAL, APO_ENOMEM, APO_ECUDA, APO_ETIMEOUT, APO_EBUSY = 0, -1, -2, -3, -4, -5
F64, F32, F64_FILTERED, F64_MID, F64_EXACT = 0, 1, 2, 3, 4
OUTGOING = 16                      # precision flag: the direction condition
SCHED_TOPK, SCHED_MAXSET = 0, 1
HIT_CAP = 256
STATUS_TIMEOUT, STATUS_BADHIT, STATUS_TOOMANY, STATUS_BADOFFS = 1, 2, 4, 8
MAX_LEVELS = 8
MAX_TRACKS = 8

TRACK_DTYPE = np.dtype([("p", "<f8", (5,)), ("w", "<f8", (5,)), ("votes", "<i4"),
                        ("n_hits", "<i4")])
assert TRACK_DTYPE.itemsize == 88

_dp = C.POINTER(C.c_double)


class ApoWires(C.Structure):
    _fields_ = [("n_wires", C.c_int32)] + [(n, _dp) for n in
                ("x0", "y0", "sin_phis", "cos_phis", "tan_tau", "sphi_t", "cphi_t", "t2")]


class ApoGrid(C.Structure):
    _fields_ = [("bins", C.c_int32 * 5), ("levels", C.c_int32), ("topk", C.c_int32),
                ("lo_edge", _dp * 5), ("hi_edge", _dp * 5), ("sincos", _dp),
                ("sincos_mid", _dp)]


class ApoHits(C.Structure):
    _fields_ = [("n_events", C.c_int32), ("offsets", C.c_void_p), ("wire_id", C.c_void_p),
                ("drift", C.c_void_p)]


class ApoTune(C.Structure):
    _fields_ = [("coarse_filter", C.c_int32), ("cells_filter", C.c_int32),
                ("cells_block", C.c_int32), ("chunk_events", C.c_int32),
                ("coarse_full", C.c_int32), ("persistent", C.c_int32)]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class ApoSolveOpts(C.Structure):
    _fields_ = [("precision", C.c_int32 * (MAX_LEVELS + 1)), ("max_tracks", C.c_int32),
                ("min_votes", C.c_int32), ("mask_sigma", C.c_double),
                ("trace_keys", C.c_void_p), ("trace_votes", C.c_void_p),
                ("tune", ApoTune), ("use_graph", C.c_int32), ("hit_track", C.c_void_p),
                ("schedule", C.c_int32), ("max_keep", C.c_int32), ("slack", C.c_int32),
                ("final_level", C.c_void_p), ("n_final", C.c_void_p),
                ("trace_count", C.c_void_p)]


class Apo4Opts(C.Structure):
    _fields_ = [("p_gev", C.c_double), ("b_tesla", C.c_double), ("disk_radius", C.c_double),
                ("hit_factor", C.c_double), ("glo", C.c_double * 4),
                ("w", (C.c_double * 4) * 3), ("n", (C.c_int32 * 4) * 3),
                ("precision", C.c_int32), ("n_iter", C.c_int32), ("per_sign", C.c_int32)]


APO4_ITER_DTYPE = np.dtype([("value", "<f8", (4,)), ("err", "<f8", (4,)), ("ref", "<f8", (2,)),
                            ("sign", "<i4"), ("vmax", "<i4"), ("n_max", "<i4"), ("n_sel", "<i4")])


class ApoServeOpts(C.Structure):
    _fields_ = [("solve", ApoSolveOpts), ("batch_events", C.c_int32), ("max_slots", C.c_int32),
                ("device_bytes", C.c_size_t), ("max_pending", C.c_int32),
                ("inject_error_after", C.c_int32)]


_lib = None


def lib():
    """Loads (building if needed) the in-tree libapo.so."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            path = _build.build()
        L = C.CDLL(path)
        vp, i32, i64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
        L.apo_last_error.restype = C.c_char_p
        L.apo_solve_opts_default.argtypes = [C.POINTER(ApoSolveOpts)]
        L.apo_geometry_create.argtypes = [C.POINTER(ApoWires), C.POINTER(ApoGrid), C.POINTER(vp)]
        L.apo_geometry_destroy.argtypes = [vp]
        L.apo_coarse_cells.argtypes = [vp]
        L.apo_coarse_cells.restype = i64
        L.apo_workspace_bytes.argtypes = [vp, i32, C.POINTER(ApoSolveOpts), C.POINTER(sz)]
        L.apo_vote.argtypes = [vp, C.POINTER(ApoHits), vp, i64, i32, i32, vp, vp, sz, vp]
        L.apo_refine.argtypes = [vp, C.POINTER(ApoHits), vp, vp, i64, i32, vp, vp, vp, vp, sz, vp]
        L.apo_solve_batch.argtypes = [vp, C.POINTER(ApoHits), C.POINTER(ApoSolveOpts), vp, vp, vp,
                                      sz, vp]
        L.apo_host_extra_bytes.argtypes = [i32, i64]
        L.apo_host_extra_bytes.restype = sz
        L.apo_solve_batch_host.argtypes = [vp, i32, vp, vp, vp, C.POINTER(ApoSolveOpts), vp, vp,
                                           vp, sz, vp]
        L.apo_serve_opts_default.argtypes = [C.POINTER(ApoServeOpts)]
        L.apo_serve_create.argtypes = [vp, C.POINTER(ApoServeOpts), C.POINTER(vp)]
        L.apo_serve_slot_bytes.argtypes = [vp, C.POINTER(ApoServeOpts)]
        L.apo_serve_slot_bytes.restype = sz
        L.apo_serve_slots.argtypes = [vp]
        L.apo_serve_slots.restype = i32
        L.apo_serve_submit.argtypes = [vp, vp, vp, i32, C.c_uint64]
        L.apo_serve_poll.argtypes = [vp, vp, vp, vp, i32, C.POINTER(i32)]
        L.apo_serve_drain.argtypes = [vp, i32]
        L.apo_serve_stats.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
        L.apo_serve_destroy.argtypes = [vp]
        L.apo_serve_latency.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                        C.POINTER(C.c_int64)]
        L.apo_autotune.argtypes = [vp, C.POINTER(ApoHits), C.POINTER(ApoSolveOpts), vp, sz, vp,
                                   C.POINTER(ApoTune), C.POINTER(C.c_float)]
        L.apo_diag_vote_coarse_counts.argtypes = [vp, C.POINTER(ApoHits), i32, vp, vp, vp, sz, vp]
        L.apo_diag_coarse_launches.argtypes = [vp, i32]
        L.apo_diag_coarse_launches.restype = i32
        L.apo_diag_pipe_peak.argtypes = [i32, i32, C.POINTER(C.c_double)]
        L.apo_diag_wait_timeout.argtypes = [i32]
        L.apo_diag_dops.argtypes = [i32, vp, vp, C.c_int64, vp]
        L.apo_diag_vote_pair_ends.argtypes = [vp, i32, vp, vp, vp, C.c_int64, vp]
        L.apo_workspace_status.argtypes = [vp, i32, vp, vp]
        L.apo_vote_coarse_noalloc.argtypes = [vp, C.POINTER(ApoHits), i32, vp, vp]
        L.apo_vote_coarse_noalloc_status.argtypes = [C.POINTER(C.c_uint32), vp]
        L.apo_diag_noalloc_wait_timeout.argtypes = [i32, vp]
        L.apo4_opts_default.argtypes = [C.POINTER(Apo4Opts)]
        L.apo4_chamber_create.argtypes = [C.POINTER(ApoWires), C.POINTER(vp)]
        L.apo4_chamber_destroy.argtypes = [vp]
        L.apo4_workspace_bytes.argtypes = [vp, i32, C.POINTER(Apo4Opts), C.POINTER(sz)]
        L.apo4_solve_batch.argtypes = [vp, C.POINTER(ApoHits), C.POINTER(Apo4Opts), vp, vp, vp, sz, vp]
        L.apo4_vote.argtypes = [vp, C.POINTER(ApoHits), C.POINTER(Apo4Opts), i32, vp, vp, vp, vp, vp,
                                sz, vp]
        _lib = L
    return _lib


class ApoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"apo error {code}: {msg}")
        self.code = code


def _check(rc):
    if rc != APO_OK:
        raise ApoError(rc, lib().apo_last_error().decode())


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(0 if t is None else int(t.data_ptr()))


class Geometry:
    """Device copy of a wire table (gen.chamber.Wires-like) and grid (gen.grid.Grid-like)."""

    def __init__(self, grid, wires):
        self.grid, self.wires = grid, wires
        keep = []

        def dp(a):
            a = np.ascontiguousarray(a, np.float64)
            keep.append(a)
            return a.ctypes.data_as(_dp)

        w = ApoWires()
        w.n_wires = int(wires.n)
        for name in ("x0", "y0", "sin_phis", "cos_phis", "tan_tau", "sphi_t", "cphi_t", "t2"):
            setattr(w, name, dp(getattr(wires, name)))
        g = ApoGrid()
        for a in range(5):
            g.bins[a] = int(grid.bins[a])
            g.lo_edge[a] = dp(grid.lo_edge[a])
            g.hi_edge[a] = dp(grid.hi_edge[a])
        g.levels = int(grid.levels)
        g.topk = int(grid.topk)
        g.sincos = dp(grid.sincos)
        mid = getattr(grid, "sincos_mid", None)
        g.sincos_mid = dp(mid) if mid is not None else None
        h = C.c_void_p()
        _check(lib().apo_geometry_create(C.byref(w), C.byref(g), C.byref(h)))
        self.handle = h
        self.n_coarse = int(lib().apo_coarse_cells(h))
        self.levels, self.topk = int(grid.levels), int(grid.topk)

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().apo_geometry_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_bytes(self, n_events: int, opts: ApoSolveOpts | None = None) -> int:
        n = C.c_size_t()
        _check(lib().apo_workspace_bytes(self.handle, int(n_events),
                                         None if opts is None else C.byref(opts), C.byref(n)))
        return int(n.value)

    def workspace(self, n_events: int, extra: int = 0, opts: ApoSolveOpts | None = None):
        torch = _torch()
        return torch.empty(self.workspace_bytes(n_events, opts) + extra, dtype=torch.uint8,
                           device="cuda")


class DeviceHits:
    """CSR hits on the device (torch tensors)."""

    def __init__(self, offsets, wire_id, drift):
        self.offsets, self.wire_id, self.drift = offsets, wire_id, drift
        self.n_events = int(offsets.shape[0] - 1)

    @classmethod
    def from_events(cls, ev, device="cuda"):
        torch = _torch()
        return cls(torch.as_tensor(np.asarray(ev.offsets, np.int32), device=device),
                   torch.as_tensor(np.asarray(ev.wire_id, np.int32), device=device),
                   torch.as_tensor(np.asarray(ev.drift, np.float64), device=device))

    def c(self) -> ApoHits:
        h = ApoHits()
        h.n_events = self.n_events
        h.offsets, h.wire_id, h.drift = _ptr(self.offsets), _ptr(self.wire_id), _ptr(self.drift)
        return h


def solve_opts(precision=None, levels: int = 0, max_tracks: int = 1, min_votes: int = 0,
               mask_sigma: float = 150e-6, trace_keys=None, trace_votes=None, tune=None,
               use_graph: bool = False, hit_track=None, schedule: int = SCHED_TOPK,
               max_keep: int | None = None, slack: int = 0, final_level=None, n_final=None,
               trace_count=None) -> ApoSolveOpts:
    o = ApoSolveOpts()
    lib().apo_solve_opts_default(C.byref(o))
    if tune is not None:
        o.tune = tune
    o.use_graph = 1 if use_graph else 0
    if precision is not None:
        for i, p in enumerate(precision):
            o.precision[i] = int(p)
    o.max_tracks, o.min_votes, o.mask_sigma = int(max_tracks), int(min_votes), float(mask_sigma)
    o.trace_keys = _ptr(trace_keys).value
    o.trace_votes = _ptr(trace_votes).value
    o.hit_track = _ptr(hit_track).value
    o.schedule, o.slack = int(schedule), int(slack)
    if max_keep is not None:
        o.max_keep = int(max_keep)
    o.final_level = _ptr(final_level).value
    o.n_final = _ptr(n_final).value
    o.trace_count = _ptr(trace_count).value
    return o


def vote(geom: Geometry, hits: DeviceHits, keys=None, level: int = 0, precision: int = F64,
         n_per_event: int | None = None, out=None, workspace=None, stream=None):
    """apo_vote: votes (int32, n_events x n_cells) of the given keys or the full coarse grid."""
    torch = _torch()
    n = geom.n_coarse if keys is None else int(n_per_event if n_per_event is not None
                                                 else keys.shape[-1])
    if out is None:
        out = torch.empty((hits.n_events, n), dtype=torch.int32, device="cuda")
    ws = geom.workspace(hits.n_events) if workspace is None else workspace
    hc = hits.c()
    _check(lib().apo_vote(geom.handle, C.byref(hc), _ptr(keys), n, int(level), int(precision),
                          _ptr(out), _ptr(ws), ws.numel(), _stream_ptr(stream)))
    return out


def refine(geom: Geometry, hits: DeviceHits, votes, keys=None, level: int = 0, workspace=None,
           stream=None):
    """apo_refine: (kept_keys, kept_votes, children) per event."""
    torch = _torch()
    ne, K = hits.n_events, geom.topk
    n_in = geom.n_coarse if keys is None else int(keys.shape[-1])
    kk = torch.empty((ne, K), dtype=torch.int64, device="cuda")
    kv = torch.empty((ne, K), dtype=torch.int32, device="cuda")
    ch = torch.empty((ne, K * 32), dtype=torch.int64, device="cuda")
    ws = geom.workspace(ne) if workspace is None else workspace
    hc = hits.c()
    _check(lib().apo_refine(geom.handle, C.byref(hc), _ptr(keys), _ptr(votes), n_in, int(level),
                            _ptr(kk), _ptr(kv), _ptr(ch), _ptr(ws), ws.numel(),
                            _stream_ptr(stream)))
    return kk, kv, ch


def solve_batch(geom: Geometry, hits: DeviceHits, opts: ApoSolveOpts | None = None,
                tracks=None, n_tracks=None, workspace=None, stream=None):
    """apo_solve_batch: device tracks (uint8 tensor of apo_track records) and per-event
    track counts."""
    torch = _torch()
    o = opts if opts is not None else solve_opts()
    mt = int(o.max_tracks)
    if tracks is None:
        tracks = torch.zeros(hits.n_events * mt * TRACK_DTYPE.itemsize, dtype=torch.uint8,
                             device="cuda")
    if n_tracks is None:
        n_tracks = torch.zeros(hits.n_events, dtype=torch.int32, device="cuda")
    ws = geom.workspace(hits.n_events, opts=o) if workspace is None else workspace
    hc = hits.c()
    _check(lib().apo_solve_batch(geom.handle, C.byref(hc), C.byref(o), _ptr(tracks),
                                 _ptr(n_tracks), _ptr(ws), ws.numel(), _stream_ptr(stream)))
    return tracks, n_tracks


def autotune(geom: Geometry, hits: DeviceHits, opts: ApoSolveOpts | None = None, workspace=None,
             stream=None):
    """apo_autotune: the fastest execution knobs for this batch (results never change)."""
    o = opts if opts is not None else solve_opts()
    if workspace is None:   # room for every candidate, the persistent launch's scratch included
        op = ApoSolveOpts.from_buffer_copy(o)
        op.tune.persistent = 1
        of = ApoSolveOpts.from_buffer_copy(o)
        of.tune.coarse_full = 1
        torch = _torch()
        ws = torch.empty(max(geom.workspace_bytes(hits.n_events, x) for x in (o, op, of)),
                         dtype=torch.uint8, device="cuda")
    else:
        ws = workspace
    best = ApoTune()
    ms = C.c_float()
    hc = hits.c()
    _check(lib().apo_autotune(geom.handle, C.byref(hc), C.byref(o), _ptr(ws), ws.numel(),
                              _stream_ptr(stream), C.byref(best), C.byref(ms)))
    return best, float(ms.value)


def tracks_to_numpy(tracks, n_events: int, max_tracks: int = 1) -> np.ndarray:
    a = tracks.cpu().numpy() if hasattr(tracks, "cpu") else np.asarray(tracks)
    return a.view(TRACK_DTYPE).reshape(n_events, max_tracks)


def host_workspace_bytes(geom: Geometry, n_events: int, n_hits: int,
                         opts: ApoSolveOpts | None = None) -> int:
    return geom.workspace_bytes(n_events, opts) + int(lib().apo_host_extra_bytes(int(n_events),
                                                                                 int(n_hits)))


def solve_batch_host(geom: Geometry, offsets: np.ndarray, wire_id: np.ndarray, drift: np.ndarray,
                     opts: ApoSolveOpts | None = None, workspace=None, out=None, stream=None):
    """apo_solve_batch_host: host arrays in, host tracks out (synchronous)."""
    o = opts if opts is not None else solve_opts()
    offsets = np.ascontiguousarray(offsets, np.int32)
    wire_id = np.ascontiguousarray(wire_id, np.int32)
    drift = np.ascontiguousarray(drift, np.float64)
    n_ev = int(offsets.shape[0] - 1)
    ws = workspace
    if ws is None:
        torch = _torch()
        ws = torch.empty(host_workspace_bytes(geom, n_ev, int(offsets[-1]), o), dtype=torch.uint8,
                         device="cuda")
    if out is None:
        out = np.zeros((n_ev, int(o.max_tracks)), TRACK_DTYPE)
    nt = np.zeros(n_ev, np.int32)

    def hp(a):
        return C.c_void_p(a.ctypes.data)

    _check(lib().apo_solve_batch_host(geom.handle, n_ev, hp(offsets), hp(wire_id), hp(drift),
                                      C.byref(o), hp(out), hp(nt), _ptr(ws), ws.numel(),
                                      _stream_ptr(stream)))
    return out, nt


def wait_timeout_test(limit_polls: int = 1000) -> int:
    """apo_diag_wait_timeout: status of a device wait on a barrier nothing completes
    (APO_ETIMEOUT expected)."""
    return int(lib().apo_diag_wait_timeout(int(limit_polls)))


def vote_coarse_noalloc(geom: Geometry, hits: DeviceHits, out, precision: int = F64,
                        stream=None) -> int:
    """apo_vote_coarse_noalloc into `out` (device int32, n_events x n_coarse); returns the
    status code."""
    hc = hits.c()
    return int(lib().apo_vote_coarse_noalloc(geom.handle, C.byref(hc), int(precision), _ptr(out),
                                             _stream_ptr(stream)))


def noalloc_status(stream=None):
    """(status code, raw status bits) of the last apo_vote_coarse_noalloc call."""
    f = C.c_uint32(0)
    rc = lib().apo_vote_coarse_noalloc_status(C.byref(f), _stream_ptr(stream))
    return int(rc), int(f.value)


def noalloc_wait_timeout_test(limit_polls: int = 1000, stream=None) -> int:
    return int(lib().apo_diag_noalloc_wait_timeout(int(limit_polls), _stream_ptr(stream)))


def workspace_status(geom: Geometry, n_events: int, workspace, stream=None) -> int:
    return int(lib().apo_workspace_status(geom.handle, int(n_events), _ptr(workspace),
                                          _stream_ptr(stream)))


def pipe_peak(precision: int = F64) -> float:
    """Measured directed-rounding add / mul throughput of the current GPU (operations per
    second, the best of add, mul and an alternating chain)."""
    best = 0.0
    for op in (0, 1, 2):
        r = C.c_double()
        _check(lib().apo_diag_pipe_peak(int(precision), op, C.byref(r)))
        best = max(best, r.value)
    return best


def pipe_rate(precision: int, op: int) -> float:
    """One op of the directed-rounding pipe microbenchmark (apo_diag_pipe_peak)."""
    r = C.c_double()
    _check(lib().apo_diag_pipe_peak(int(precision), int(op), C.byref(r)))
    return r.value


def dops(op: int, x, stream=None):
    """apo_diag_dops: elementwise FP64 reciprocal / square root (op 0-5 the library's
    integer-pipe forms rd / ru / rn, 6-11 the CUDA library's) of a float64 CUDA tensor."""
    assert x.dtype == _torch().float64 and x.is_cuda and x.is_contiguous()
    out = _torch().empty_like(x)
    _check(lib().apo_diag_dops(int(op), _ptr(x), _ptr(out), x.numel(), _stream_ptr(stream)))
    return out


def vote_pair_ends(geom: Geometry, cells, hits, precision: int = F64, stream=None):
    """apo_diag_vote_pair_ends: (n, 10) float64 CUDA tensor (vote, G+ lo/hi, G- lo/hi,
    guard, delta+ lo/hi, delta- lo/hi) for float64 CUDA tensors cells (n, 12), hits (n, 9)."""
    torch = _torch()
    assert cells.dtype == torch.float64 and hits.dtype == torch.float64
    cells, hits = cells.contiguous(), hits.contiguous()
    n = cells.shape[0]
    assert hits.shape[0] == n
    out = torch.empty((n, 10), dtype=torch.float64, device=cells.device)
    _check(lib().apo_diag_vote_pair_ends(geom.handle, int(precision), _ptr(cells), _ptr(hits),
                                         _ptr(out), n, _stream_ptr(stream)))
    return out


def coarse_launches(geom: Geometry, n_events: int) -> int:
    return int(lib().apo_diag_coarse_launches(geom.handle, int(n_events)))


def solve_launches(geom: Geometry, n_events: int) -> int:
    """Kernel launches of one single-track apo_solve_batch: staging, then per chunk of
    events the coarse vote, the coarse selection, per level the child vote and top-K,
    and the estimate."""
    return 1 + coarse_launches(geom, n_events) * (3 + 2 * geom.levels)


class Server:
    """apo_serve_*: continuous batching of events submitted one by one (host arrays)."""

    def __init__(self, geom: Geometry, solve: ApoSolveOpts | None = None, batch_events: int = 64,
                 max_slots: int = 4, device_bytes: int = 0, max_pending: int = 4096,
                 inject_error_after: int = 0):
        o = ApoServeOpts()
        lib().apo_serve_opts_default(C.byref(o))
        if solve is not None:
            o.solve = solve
        o.batch_events, o.max_slots, o.device_bytes = int(batch_events), int(max_slots), int(device_bytes)
        o.max_pending, o.inject_error_after = int(max_pending), int(inject_error_after)
        self.max_tracks = int(o.solve.max_tracks)
        self.geom = geom
        self.slot_bytes = int(lib().apo_serve_slot_bytes(geom.handle, C.byref(o)))
        h = C.c_void_p()
        _check(lib().apo_serve_create(geom.handle, C.byref(o), C.byref(h)))
        self.handle = h
        self.slots = int(lib().apo_serve_slots(h))

    def submit(self, wire_id, drift, request_id: int) -> int:
        """Returns the status (APO_OK, or APO_EBUSY when the queue is full)."""
        w = np.ascontiguousarray(wire_id, np.int32)
        d = np.ascontiguousarray(drift, np.float64)
        rc = lib().apo_serve_submit(self.handle, C.c_void_p(w.ctypes.data), C.c_void_p(d.ctypes.data),
                                    int(w.shape[0]), int(request_id))
        if rc not in (APO_OK, APO_EBUSY):
            _check(rc)
        return rc

    def poll(self, max_items: int = 1024):
        """[(request_id, tracks[max_tracks] (TRACK_DTYPE), n_tracks)] of finished events."""
        tr = np.zeros(max_items * self.max_tracks, TRACK_DTYPE)
        nt = np.zeros(max_items, np.int32)
        ids = np.zeros(max_items, np.uint64)
        n = C.c_int32()
        _check(lib().apo_serve_poll(self.handle, C.c_void_p(tr.ctypes.data), C.c_void_p(nt.ctypes.data),
                                    C.c_void_p(ids.ctypes.data), int(max_items), C.byref(n)))
        k = int(n.value)
        tr = tr.reshape(max_items, self.max_tracks)
        return [(int(ids[i]), tr[i].copy(), int(nt[i])) for i in range(k)]

    def drain(self, timeout_ms: int = 60000) -> int:
        return int(lib().apo_serve_drain(self.handle, int(timeout_ms)))

    def stats(self):
        b, m = C.c_int32(), C.c_int32()
        _check(lib().apo_serve_stats(self.handle, C.byref(b), C.byref(m)))
        return int(b.value), int(m.value)

    def latency(self):
        """(p50 ms, p99 ms, events) measured inside the library (accepted -> batch done)."""
        p50, p99, n = C.c_double(), C.c_double(), C.c_int64()
        _check(lib().apo_serve_latency(self.handle, C.byref(p50), C.byref(p99), C.byref(n)))
        return float(p50.value), float(p99.value), int(n.value)

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().apo_serve_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------------------- #
# The paper's own 4-D search (include/apo4.h)
# ---------------------------------------------------------------------------------------- #
def four_opts(precision: int = F64, n_iter: int = 3, per_sign: int = 1, **kw) -> Apo4Opts:
    """apo4_opts_default (Table tabGridDef in metres) with overrides: p_gev, b_tesla,
    disk_radius, hit_factor, glo (4), w (3 x 4), n (3 x 4)."""
    o = Apo4Opts()
    lib().apo4_opts_default(C.byref(o))
    o.precision, o.n_iter, o.per_sign = int(precision), int(n_iter), int(per_sign)
    for k in ("p_gev", "b_tesla", "disk_radius", "hit_factor"):
        if k in kw:
            setattr(o, k, float(kw[k]))
    if "glo" in kw:
        for a in range(4):
            o.glo[a] = kw["glo"][a]
    for key in ("w", "n"):
        if key in kw:
            for i in range(3):
                for a in range(4):
                    getattr(o, key)[i][a] = kw[key][i][a]
    return o


class Chamber4:
    """Device wire table for the 4-D search (apo4_chamber)."""

    def __init__(self, wires):
        keep = []

        def dp(a):
            a = np.ascontiguousarray(a, np.float64)
            keep.append(a)
            return a.ctypes.data_as(_dp)

        w = ApoWires()
        w.n_wires = int(wires.n)
        for name in ("x0", "y0", "sin_phis", "cos_phis", "tan_tau", "sphi_t", "cphi_t", "t2"):
            setattr(w, name, dp(getattr(wires, name)))
        h = C.c_void_p()
        _check(lib().apo4_chamber_create(C.byref(w), C.byref(h)))
        self.handle = h

    def workspace(self, n_events: int, opts: Apo4Opts):
        n = C.c_size_t()
        _check(lib().apo4_workspace_bytes(self.handle, int(n_events), C.byref(opts), C.byref(n)))
        return _torch().empty(int(n.value), dtype=_torch().uint8, device="cuda")

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().apo4_chamber_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve4(ch: Chamber4, hits: DeviceHits, opts: Apo4Opts, out=None, selected=None,
           workspace=None, stream=None):
    """apo4_solve_batch: (uint8 tensor of apo4_iter records, n_events x n_iter; uint8
    selection per hit)."""
    torch = _torch()
    ne = hits.n_events
    if out is None:
        out = torch.zeros(ne * opts.n_iter * APO4_ITER_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    if selected is None:
        selected = torch.zeros(max(int(hits.wire_id.shape[0]), 1), dtype=torch.uint8, device="cuda")
    ws = ch.workspace(ne, opts) if workspace is None else workspace
    hc = hits.c()
    _check(lib().apo4_solve_batch(ch.handle, C.byref(hc), C.byref(opts), _ptr(out), _ptr(selected),
                                  _ptr(ws), ws.numel(), _stream_ptr(stream)))
    return out, selected


def iters4_to_numpy(out, n_events: int, n_iter: int) -> np.ndarray:
    a = out.cpu().numpy() if hasattr(out, "cpu") else np.asarray(out)
    return a.view(APO4_ITER_DTYPE).reshape(n_events, n_iter)


def vote4(ch: Chamber4, hits: DeviceHits, opts: Apo4Opts, it: int, lo, ref, active=None,
          out=None, workspace=None, stream=None):
    """apo4_vote: int32 votes (n_events, 2, n_z0, n_R, n_y, n_x) of iteration it's grid."""
    torch = _torch()
    ne = hits.n_events
    n = [opts.n[it][a] for a in range(4)]
    if out is None:
        out = torch.zeros((ne, 2, n[3], n[2], n[1], n[0]), dtype=torch.int32, device="cuda")
    ws = ch.workspace(ne, opts) if workspace is None else workspace
    hc = hits.c()
    _check(lib().apo4_vote(ch.handle, C.byref(hc), C.byref(opts), int(it), _ptr(lo), _ptr(ref),
                           _ptr(active), _ptr(out), _ptr(ws), ws.numel(), _stream_ptr(stream)))
    return out
