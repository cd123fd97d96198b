"""ctypes binding of the C oracle (oracle/apo_oracle.c).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
reference leg use this module.  It never touches the CUDA library.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None


class OrWires(C.Structure):
    _fields_ = [("n_wires", C.c_int32)] + [(n, C.POINTER(C.c_double)) for n in
                ("x0", "y0", "sin_phis", "cos_phis", "tan_tau", "sphi_t", "cphi_t", "t2")]


class OrGrid(C.Structure):
    _fields_ = [("bins", C.c_int32 * 5), ("levels", C.c_int32), ("topk", C.c_int32),
                ("lo_edge", C.POINTER(C.c_double) * 5), ("hi_edge", C.POINTER(C.c_double) * 5),
                ("sincos", C.POINTER(C.c_double)), ("sincos_offset", C.POINTER(C.c_int64)),
                ("sincos_mid", C.POINTER(C.c_double))]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp, ip, up = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_uint64)
        L.or_vote_pair.argtypes = [dp, dp, C.c_int, dp]
        L.or_vote_pair.restype = C.c_int
        L.or_vote_pair_mid.argtypes = [dp, dp, dp, dp]
        L.or_vote_pair_mid.restype = C.c_int
        L.or_vote_cells.argtypes = [C.POINTER(OrGrid), C.POINTER(OrWires), C.c_int32, ip, dp,
                                    C.c_int32, C.c_int32, up, C.c_int64, ip]
        L.or_vote_cells.restype = None
        L.or_coarse_keys.argtypes = [C.POINTER(OrGrid), up]
        L.or_topk.argtypes = [up, ip, C.c_int64, C.c_int32, up, ip]
        L.or_topk.restype = C.c_int64
        L.or_children.argtypes = [up, C.c_int64, up]
        L.or_solve_event.argtypes = [C.POINTER(OrGrid), C.POINTER(OrWires), C.c_int32, ip, dp,
                                     ip, dp, dp, ip, up, ip, up, ip]
        L.or_solve_event.restype = C.c_int
        L.or_solve_event_multi.argtypes = [C.POINTER(OrGrid), C.POINTER(OrWires), C.c_int32, ip, dp,
                                           ip, C.c_int32, C.c_int32, C.c_double, dp, dp, ip, ip, ip]
        L.or_solve_event_multi.restype = C.c_int
        L.or_atan_iv.argtypes = [C.c_double, C.c_double, C.c_int, dp]
        L.or_sincos_iv.argtypes = [C.c_double, C.c_double, C.c_int, dp]
        L.or_op_counts.argtypes = [dp, dp, C.c_int, C.POINTER(C.c_ulonglong)]
        L.or_num_threads.restype = C.c_int
        L.or_set_num_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class Tables:
    """Keeps the numpy arrays alive while the C structs point at them."""

    def __init__(self, grid, wires):
        self.grid, self.wires = grid, wires
        self._keep = []
        w = OrWires()
        w.n_wires = wires.n
        for name in ("x0", "y0", "sin_phis", "cos_phis", "tan_tau", "sphi_t", "cphi_t", "t2"):
            arr = np.ascontiguousarray(getattr(wires, name), np.float64)
            self._keep.append(arr)
            setattr(w, name, _p(arr, C.c_double))
        g = OrGrid()
        for a in range(5):
            g.bins[a] = int(grid.bins[a])
            lo = np.ascontiguousarray(grid.lo_edge[a], np.float64)
            hi = np.ascontiguousarray(grid.hi_edge[a], np.float64)
            self._keep += [lo, hi]
            g.lo_edge[a] = _p(lo, C.c_double)
            g.hi_edge[a] = _p(hi, C.c_double)
        g.levels = grid.levels
        g.topk = grid.topk
        sc = np.ascontiguousarray(grid.sincos, np.float64)
        so = np.ascontiguousarray(grid.sincos_offset, np.int64)
        self._keep += [sc, so]
        g.sincos = _p(sc, C.c_double)
        g.sincos_offset = _p(so, C.c_int64)
        sm = np.ascontiguousarray(grid.sincos_mid, np.float64)
        self._keep.append(sm)
        g.sincos_mid = _p(sm, C.c_double)
        self.cw, self.cg = w, g


def set_threads(n: int) -> None:
    lib().or_set_num_threads(int(n))


def num_threads() -> int:
    return int(lib().or_num_threads())


def vote_pair(cell12, hit9, prec: int = 0):
    """Vote (0/1) of one (cell, hit) pair and the evaluated intervals
    (G+ lo, G+ hi, G- lo, G- hi, guard flag, delta+ lo, delta+ hi, delta- lo, delta- hi),
    delta = Phi - Phi^Ax of each drift sign."""
    c = np.ascontiguousarray(cell12, np.float64)
    h = np.ascontiguousarray(hit9, np.float64)
    out = np.zeros(9)
    v = lib().or_vote_pair(_p(c, C.c_double), _p(h, C.c_double), int(prec), _p(out, C.c_double))
    return int(v), out


def vote_pair_mid(cell12, scm2, hit9):
    """Midpoint-form vote (0/1) of one (cell, hit) pair and (G+ lo, G+ hi, G- lo, G- hi,
    guard flags, d^Ax+, d^Ax-); scm2 = sin, cos of the phi0 centre."""
    c = np.ascontiguousarray(cell12, np.float64)
    m = np.ascontiguousarray(scm2, np.float64)
    h = np.ascontiguousarray(hit9, np.float64)
    out = np.zeros(7)
    v = lib().or_vote_pair_mid(_p(c, C.c_double), _p(m, C.c_double), _p(h, C.c_double),
                               _p(out, C.c_double))
    return int(v), out


def op_counts(cell12, hit9, prec: int = 0) -> np.ndarray:
    """Directed operations of one evaluation of the vote program by phase: per cell, per
    (cell, hit) without tan(lambda), tan(lambda)-dependent part, both drift signs."""
    c = np.ascontiguousarray(cell12, np.float64)
    h = np.ascontiguousarray(hit9, np.float64)
    out = (C.c_ulonglong * 4)()
    lib().or_op_counts(_p(c, C.c_double), _p(h, C.c_double), int(prec), out)
    return np.array(list(out), np.int64)


def atan_iv(lo: float, hi: float, prec: int = 0) -> np.ndarray:
    out = np.zeros(2)
    lib().or_atan_iv(float(lo), float(hi), int(prec), _p(out, C.c_double))
    return out


def sincos_iv(lo: float, hi: float, prec: int = 0) -> np.ndarray:
    """(sin lo, sin hi, cos lo, cos hi) enclosures over [lo, hi]."""
    out = np.zeros(4)
    lib().or_sincos_iv(float(lo), float(hi), int(prec), _p(out, C.c_double))
    return out


def hit9(wires, wid: int, drift: float) -> np.ndarray:
    return np.array([wires.x0[wid], wires.y0[wid], wires.sin_phis[wid], wires.cos_phis[wid],
                     wires.tan_tau[wid], wires.sphi_t[wid], wires.cphi_t[wid], wires.t2[wid],
                     drift])


def cell12(grid, level: int, idx5) -> np.ndarray:
    lo = [grid.cell_edges(level, a, idx5[a])[0] for a in range(5)]
    hi = [grid.cell_edges(level, a, idx5[a])[1] for a in range(5)]
    sc = grid.sincos[grid.sincos_offset[level] + idx5[1]]
    return np.array([lo[0], hi[0], sc[0], sc[1], sc[2], sc[3], lo[2], hi[2], lo[3], hi[3],
                     lo[4], hi[4]], np.float64)


def scm2(grid, level: int, idx5) -> np.ndarray:
    """sin, cos of the phi0 centre of a cell (from the grid's centre table)."""
    return np.array(grid.sincos_mid[grid.sincos_offset[level] + idx5[1]], np.float64)


def vote_cells(tab: Tables, wire_id, drift, level: int, keys, prec: int = 0) -> np.ndarray:
    wid = np.ascontiguousarray(wire_id, np.int32)
    dr = np.ascontiguousarray(drift, np.float64)
    k = np.ascontiguousarray(keys, np.uint64)
    out = np.zeros(k.shape[0], np.int32)
    lib().or_vote_cells(C.byref(tab.cg), C.byref(tab.cw), int(wid.shape[0]), _p(wid, C.c_int32),
                        _p(dr, C.c_double), int(level), int(prec), _p(k, C.c_uint64),
                        int(k.shape[0]), _p(out, C.c_int32))
    return out


def coarse_keys(tab: Tables) -> np.ndarray:
    out = np.zeros(tab.grid.n_coarse(), np.uint64)
    lib().or_coarse_keys(C.byref(tab.cg), _p(out, C.c_uint64))
    return out


def vote_coarse(tab: Tables, wire_id, drift, prec: int = 0) -> np.ndarray:
    return vote_cells(tab, wire_id, drift, 0, coarse_keys(tab), prec)


def topk(keys, votes, K: int):
    k = np.ascontiguousarray(keys, np.uint64)
    v = np.ascontiguousarray(votes, np.int32)
    ok = np.zeros(K, np.uint64)
    ov = np.zeros(K, np.int32)
    m = lib().or_topk(_p(k, C.c_uint64), _p(v, C.c_int32), int(k.shape[0]), int(K),
                      _p(ok, C.c_uint64), _p(ov, C.c_int32))
    return ok[:m], ov[:m]


def children(keys) -> np.ndarray:
    k = np.ascontiguousarray(keys, np.uint64)
    out = np.zeros(k.shape[0] * 32, np.uint64)
    lib().or_children(_p(k, C.c_uint64), int(k.shape[0]), _p(out, C.c_uint64))
    return out


def solve_event(tab: Tables, wire_id, drift, prec_per_level=None):
    """Coarse-to-fine search of one event.  Returns dict with the estimate, its errors, the
    best vote count, the frontier (keys, votes) kept after each level and the last level's
    (keys, votes)."""
    g = tab.grid
    K, lv = g.topk, g.levels
    prec = np.zeros(lv + 1, np.int32) if prec_per_level is None else \
        np.ascontiguousarray(prec_per_level, np.int32)
    wid = np.ascontiguousarray(wire_id, np.int32)
    dr = np.ascontiguousarray(drift, np.float64)
    p = np.zeros(5)
    werr = np.zeros(5)
    best = np.zeros(1, np.int32)
    tk = np.zeros((lv + 1) * K, np.uint64)
    tv = np.zeros((lv + 1) * K, np.int32)
    lk = np.zeros(K * 32, np.uint64)
    lvv = np.zeros(K * 32, np.int32)
    lib().or_solve_event(C.byref(tab.cg), C.byref(tab.cw), int(wid.shape[0]), _p(wid, C.c_int32),
                         _p(dr, C.c_double), _p(prec, C.c_int32), _p(p, C.c_double),
                         _p(werr, C.c_double), _p(best, C.c_int32), _p(tk, C.c_uint64),
                         _p(tv, C.c_int32), _p(lk, C.c_uint64), _p(lvv, C.c_int32))
    return dict(p=p, w=werr, votes=int(best[0]), trace_keys=tk.reshape(lv + 1, K),
                trace_votes=tv.reshape(lv + 1, K), last_keys=lk, last_votes=lvv)


def solve_event_multi(tab: Tables, wire_id, drift, max_tracks: int, min_votes: int,
                      mask_sigma: float = 150e-6, prec_per_level=None):
    """Multi-track extraction of one event (see or_solve_event_multi).  Returns dict with
    per-track estimates / errors / votes, the number of tracks and, per hit, the index of
    the track that masked it (-1: none)."""
    g = tab.grid
    prec = np.zeros(g.levels + 1, np.int32) if prec_per_level is None else \
        np.ascontiguousarray(prec_per_level, np.int32)
    wid = np.ascontiguousarray(wire_id, np.int32)
    dr = np.ascontiguousarray(drift, np.float64)
    n = wid.shape[0]
    p = np.zeros(5 * max_tracks)
    werr = np.zeros(5 * max_tracks)
    votes = np.zeros(max_tracks, np.int32)
    nf = np.zeros(1, np.int32)
    ht = np.zeros(max(n, 1), np.int32)
    lib().or_solve_event_multi(C.byref(tab.cg), C.byref(tab.cw), int(n), _p(wid, C.c_int32),
                               _p(dr, C.c_double), _p(prec, C.c_int32), int(max_tracks),
                               int(min_votes), float(mask_sigma), _p(p, C.c_double),
                               _p(werr, C.c_double), _p(votes, C.c_int32), _p(nf, C.c_int32),
                               _p(ht, C.c_int32))
    k = int(nf[0])
    return dict(n_tracks=k, p=p.reshape(max_tracks, 5)[:k], w=werr.reshape(max_tracks, 5)[:k],
                votes=votes[:k], hit_track=ht[:n])
