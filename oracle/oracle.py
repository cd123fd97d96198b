"""ctypes binding of the C oracle (oracle/apo_oracle.c).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
reference leg use this module.  It never touches the CUDA library.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None
OUTGOING = 16   # precision flag bit: the direction condition of the vote program


class OrWires(C.Structure):
    _fields_ = [("n_wires", C.c_int32)] + [(n, C.POINTER(C.c_double)) for n in
                ("x0", "y0", "sin_phis", "cos_phis", "tan_tau", "sphi_t", "cphi_t", "t2")]


class OrGrid(C.Structure):
    _fields_ = [("bins", C.c_int32 * 5), ("levels", C.c_int32), ("topk", C.c_int32),
                ("lo_edge", C.POINTER(C.c_double) * 5), ("hi_edge", C.POINTER(C.c_double) * 5),
                ("sincos", C.POINTER(C.c_double)), ("sincos_offset", C.POINTER(C.c_int64)),
                ("sincos_mid", C.POINTER(C.c_double))]


class Or4Grid(C.Structure):
    _fields_ = [("lo", C.c_double * 4), ("w", C.c_double * 4), ("n", C.c_int32 * 4)]


class Or4Opts(C.Structure):
    _fields_ = [("p_gev", C.c_double), ("b_tesla", C.c_double), ("disk_radius", C.c_double),
                ("hit_factor", C.c_double), ("glo", C.c_double * 4),
                ("w", (C.c_double * 4) * 3), ("n", (C.c_int32 * 4) * 3),
                ("precision", C.c_int32), ("n_iter", C.c_int32), ("per_sign", C.c_int32)]


class Or4Iter(C.Structure):
    _fields_ = [("value", C.c_double * 4), ("err", C.c_double * 4), ("ref", C.c_double * 2),
                ("sign", C.c_int32), ("vmax", C.c_int32), ("n_max", C.c_int32),
                ("n_sel", C.c_int32)]


def lib():
    global _lib
    if _lib is None:
        _lib = load(_build.build())
    return _lib


def load(path):
    """Loads a build of the oracle (liboracle.so or a reference variant) with its
    signatures."""
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
    L.or_children.argtypes = [C.c_void_p, up, C.c_int64, up]
    L.or_solve_event_maxset.argtypes = [C.POINTER(OrGrid), C.POINTER(OrWires), C.c_int32, ip, dp,
                                        ip, C.c_int32, C.c_int32, dp, dp, ip, ip,
                                        C.POINTER(C.c_int64), ip, up, ip]
    L.or_solve_event_maxset.restype = C.c_int
    L.or_solve_event.argtypes = [C.POINTER(OrGrid), C.POINTER(OrWires), C.c_int32, ip, dp,
                                 ip, dp, dp, ip, up, ip, up, ip]
    L.or_solve_event.restype = C.c_int
    L.or_solve_event_multi.argtypes = [C.POINTER(OrGrid), C.POINTER(OrWires), C.c_int32, ip, dp,
                                       ip, C.c_int32, C.c_int32, C.c_double, dp, dp, ip, ip, ip]
    L.or_solve_event_multi.restype = C.c_int
    L.or_solve_event_maxset_multi.argtypes = [C.POINTER(OrGrid), C.POINTER(OrWires), C.c_int32, ip, dp,
                                              ip, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                              C.c_double, dp, dp, ip, ip, C.POINTER(C.c_int64), ip, ip]
    L.or_solve_event_maxset_multi.restype = C.c_int
    L.or_mask_hits.argtypes = [C.POINTER(OrGrid), C.POINTER(OrWires), C.c_int32, ip, dp,
                               C.POINTER(C.c_uint8), C.c_int32, up, C.c_int64, C.c_double,
                               C.c_int, C.POINTER(C.c_uint8)]
    L.or_atan_iv.argtypes = [C.c_double, C.c_double, C.c_int, dp]
    L.or_sincos_iv.argtypes = [C.c_double, C.c_double, C.c_int, dp]
    L.or_op_counts.argtypes = [dp, dp, C.c_int, C.POINTER(C.c_ulonglong)]
    L.or_num_threads.restype = C.c_int
    L.or4_vote_pair.argtypes = [dp, C.c_int32, dp, dp, C.c_double, C.c_double, C.c_int32, dp]
    L.or4_vote_pair.restype = C.c_int
    L.or4_vote_grid.argtypes = [C.POINTER(Or4Opts), C.POINTER(Or4Grid), dp, C.POINTER(OrWires),
                                C.c_int32, ip, dp, C.POINTER(C.c_uint8), ip]
    L.or4_estimate.argtypes = [C.POINTER(Or4Grid), ip, C.POINTER(Or4Iter)]
    L.or4_disk.argtypes = [dp, C.c_double, C.c_int32]
    L.or4_disk.restype = C.c_int
    L.or4_solve_event.argtypes = [C.POINTER(Or4Opts), C.POINTER(OrWires), C.c_int32, ip, dp,
                                  C.POINTER(Or4Iter), C.POINTER(C.c_uint8)]
    L.or_set_num_threads.argtypes = [C.c_int]
    return L


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


def vote_cells(tab: Tables, wire_id, drift, level: int, keys, prec: int = 0,
               L=None) -> np.ndarray:
    """Votes of cells (keys at `level`) for one event's hits; L: another build of the
    oracle (default: liboracle.so)."""
    wid = np.ascontiguousarray(wire_id, np.int32)
    dr = np.ascontiguousarray(drift, np.float64)
    k = np.ascontiguousarray(keys, np.uint64)
    out = np.zeros(k.shape[0], np.int32)
    (L or lib()).or_vote_cells(C.byref(tab.cg), C.byref(tab.cw), int(wid.shape[0]), _p(wid, C.c_int32),
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


def children(keys, tab: Tables | None = None) -> np.ndarray:
    """The 32 children of each key (key layout of tab's grid; 10 bits per axis without)."""
    k = np.ascontiguousarray(keys, np.uint64)
    out = np.zeros(k.shape[0] * 32, np.uint64)
    lib().or_children(None if tab is None else C.byref(tab.cg), _p(k, C.c_uint64),
                      int(k.shape[0]), _p(out, C.c_uint64))
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


def solve_event_maxset(tab: Tables, wire_id, drift, max_keep: int, slack: int = 0,
                       prec_per_level=None, trace: bool = False):
    """Max-set search of one event (see or_solve_event_maxset).  prec_per_level: codes as
    vote_cells (e.g. F32 | OUTGOING).  Returns dict p, w, votes, final_level, n_final and,
    with trace, per level the kept (keys, votes) in key order."""
    g = tab.grid
    lv = g.levels
    prec = np.zeros(lv + 1, np.int32) if prec_per_level is None else \
        np.ascontiguousarray(prec_per_level, np.int32)
    wid = np.ascontiguousarray(wire_id, np.int32)
    dr = np.ascontiguousarray(drift, np.float64)
    p, werr = np.zeros(5), np.zeros(5)
    best, fl = np.zeros(1, np.int32), np.zeros(1, np.int32)
    nf = np.zeros(1, np.int64)
    tc = np.zeros(lv + 1, np.int32)
    tk = np.zeros((lv + 1) * max_keep if trace else 1, np.uint64)
    tv = np.zeros((lv + 1) * max_keep if trace else 1, np.int32)
    lib().or_solve_event_maxset(C.byref(tab.cg), C.byref(tab.cw), int(wid.shape[0]),
                                _p(wid, C.c_int32), _p(dr, C.c_double), _p(prec, C.c_int32),
                                int(max_keep), int(slack), _p(p, C.c_double),
                                _p(werr, C.c_double), _p(best, C.c_int32), _p(fl, C.c_int32),
                                _p(nf, C.c_int64), _p(tc, C.c_int32) if trace else None,
                                _p(tk, C.c_uint64) if trace else None,
                                _p(tv, C.c_int32) if trace else None)
    r = dict(p=p, w=werr, votes=int(best[0]), final_level=int(fl[0]), n_final=int(nf[0]))
    if trace:
        tk, tv = tk.reshape(lv + 1, max_keep), tv.reshape(lv + 1, max_keep)
        r["trace"] = [(tk[L, :tc[L]].copy(), tv[L, :tc[L]].copy()) for L in range(lv + 1)]
    return r


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


def solve_event_maxset_multi(tab: Tables, wire_id, drift, max_keep: int, max_tracks: int,
                             min_votes: int, slack: int = 0, mask_sigma: float = 150e-6,
                             prec_per_level=None):
    """Multi-track extraction with the max-set search (see or_solve_event_maxset_multi).
    Returns dict with per-track p, w, votes, final_level, n_final, the number of tracks and,
    per hit, the index of the track that took it (-1: none)."""
    g = tab.grid
    prec = np.zeros(g.levels + 1, np.int32) if prec_per_level is None else \
        np.ascontiguousarray(prec_per_level, np.int32)
    wid = np.ascontiguousarray(wire_id, np.int32)
    dr = np.ascontiguousarray(drift, np.float64)
    n = wid.shape[0]
    p = np.zeros(5 * max_tracks)
    werr = np.zeros(5 * max_tracks)
    votes = np.zeros(max_tracks, np.int32)
    fl = np.zeros(max_tracks, np.int32)
    nfin = np.zeros(max_tracks, np.int64)
    nf = np.zeros(1, np.int32)
    ht = np.zeros(max(n, 1), np.int32)
    lib().or_solve_event_maxset_multi(C.byref(tab.cg), C.byref(tab.cw), int(n), _p(wid, C.c_int32),
                                      _p(dr, C.c_double), _p(prec, C.c_int32), int(max_keep),
                                      int(slack), int(max_tracks), int(min_votes), float(mask_sigma),
                                      _p(p, C.c_double), _p(werr, C.c_double), _p(votes, C.c_int32),
                                      _p(fl, C.c_int32), _p(nfin, C.c_int64), _p(nf, C.c_int32),
                                      _p(ht, C.c_int32))
    k = int(nf[0])
    return dict(n_tracks=k, p=p.reshape(max_tracks, 5)[:k], w=werr.reshape(max_tracks, 5)[:k],
                votes=votes[:k], final_level=fl[:k], n_final=nfin[:k], hit_track=ht[:n])


def mask_hits(tab: Tables, wire_id, drift, level: int, keys, width: float, active=None,
              outgoing: bool = False) -> np.ndarray:
    """Hit finding on a set of cells (see or_mask_hits): bool per hit, taken by a cell."""
    wid = np.ascontiguousarray(wire_id, np.int32)
    dr = np.ascontiguousarray(drift, np.float64)
    k = np.ascontiguousarray(keys, np.uint64)
    n = wid.shape[0]
    act = None if active is None else np.ascontiguousarray(active, np.uint8)
    out = np.zeros(max(n, 1), np.uint8)
    lib().or_mask_hits(C.byref(tab.cg), C.byref(tab.cw), int(n), _p(wid, C.c_int32),
                       _p(dr, C.c_double), None if act is None else _p(act, C.c_uint8), int(level),
                       _p(k, C.c_uint64), int(k.shape[0]), float(width), int(bool(outgoing)),
                       _p(out, C.c_uint8))
    return out[:n].astype(bool)


# ---------------------------------------------------------------------------------------- #
# The paper's own 4-D search (x_c, y_c, R, z0; Sections 3.1-3.3, Table tabGridDef)
# ---------------------------------------------------------------------------------------- #
def four_opts(p_gev=0.105, b_tesla=1.0, disk_radius=0.10, hit_factor=5.0, glo=None, w=None,
              n=None, precision=0, n_iter=3, per_sign=1) -> Or4Opts:
    """Defaults: Table tabGridDef read in metres with z0 centred on the chamber middle:
    iterations 1 and 2 on x_c, y_c in [-0.45, 0.45], R in [0.225, 0.375], z0 in [-0.75, 0.75]
    with voxels 18 x 18 x 3.75 x 75 mm and 10 x 10 x 3.75 x 75 mm; iteration 3 on the
    estimate +- (25, 25, 25, 400) mm with 1 x 1 x 1 x 40 mm voxels."""
    o = Or4Opts()
    o.p_gev, o.b_tesla, o.disk_radius, o.hit_factor = p_gev, b_tesla, disk_radius, hit_factor
    glo = (-0.45, -0.45, 0.225, -0.75) if glo is None else glo
    w = ((0.018, 0.018, 0.00375, 0.075), (0.010, 0.010, 0.00375, 0.075),
         (0.001, 0.001, 0.001, 0.040)) if w is None else w
    n = ((50, 50, 40, 20), (90, 90, 40, 20), (50, 50, 50, 20)) if n is None else n
    for a in range(4):
        o.glo[a] = glo[a]
    for k in range(3):
        for a in range(4):
            o.w[k][a] = w[k][a]
            o.n[k][a] = n[k][a]
    o.precision, o.n_iter, o.per_sign = precision, n_iter, per_sign
    return o


def four_vote_pair(box8, sign, ref, hit9, p_gev=0.105, b_tesla=1.0, prec=0):
    """4-D midpoint-form vote of one (voxel, hit) pair and (d^Ax+, d^Ax-, guard flags,
    |tan(lambda)| at the centre, psi)."""
    b = np.ascontiguousarray(box8, np.float64)
    r = np.ascontiguousarray(ref, np.float64)
    h = np.ascontiguousarray(hit9, np.float64)
    out = np.zeros(5)
    v = lib().or4_vote_pair(_p(b, C.c_double), int(sign), _p(r, C.c_double), _p(h, C.c_double),
                            float(p_gev), float(b_tesla), int(prec), _p(out, C.c_double))
    return int(v), out


def four_grid(lo, w, n) -> Or4Grid:
    g = Or4Grid()
    for a in range(4):
        g.lo[a], g.w[a], g.n[a] = lo[a], w[a], n[a]
    return g


def four_vote_grid(opts: Or4Opts, grid: Or4Grid, ref, tab: Tables, wire_id, drift, active=None):
    """Votes (2, n_z0, n_R, n_y, n_x) of every voxel of one grid for one event; index 0 of
    the first axis is tan(lambda) > 0."""
    wid = np.ascontiguousarray(wire_id, np.int32)
    dr = np.ascontiguousarray(drift, np.float64)
    r = np.ascontiguousarray(ref, np.float64)
    nvox = int(np.prod([grid.n[a] for a in range(4)]))
    out = np.zeros(2 * nvox, np.int32)
    act = None if active is None else np.ascontiguousarray(active, np.uint8)
    lib().or4_vote_grid(C.byref(opts), C.byref(grid), _p(r, C.c_double), C.byref(tab.cw),
                        int(wid.shape[0]), _p(wid, C.c_int32), _p(dr, C.c_double),
                        None if act is None else _p(act, C.c_uint8), _p(out, C.c_int32))
    return out.reshape(2, grid.n[3], grid.n[2], grid.n[1], grid.n[0])


def four_disk(box6, radius=0.10, prec=0) -> bool:
    """Disk pre-filter (Eq. ApoVoteDisk) of one voxel (x_c, y_c, R as lo, hi)."""
    b = np.ascontiguousarray(box6, np.float64)
    return bool(lib().or4_disk(_p(b, C.c_double), float(radius), int(prec)))


def four_estimate(grid: Or4Grid, votes) -> dict:
    v = np.ascontiguousarray(votes, np.int32).reshape(-1)
    it = Or4Iter()
    lib().or4_estimate(C.byref(grid), _p(v, C.c_int32), C.byref(it))
    return _iter_dict(it)


def _iter_dict(it) -> dict:
    return dict(value=np.array(it.value[:]), err=np.array(it.err[:]), ref=np.array(it.ref[:]),
                sign=int(it.sign), vmax=int(it.vmax), n_max=int(it.n_max), n_sel=int(it.n_sel))


def four_solve_event(opts: Or4Opts, tab: Tables, wire_id, drift):
    """The three iterations for one event: list of per-iteration dicts and the last hit
    selection."""
    wid = np.ascontiguousarray(wire_id, np.int32)
    dr = np.ascontiguousarray(drift, np.float64)
    its = (Or4Iter * 3)()
    sel = np.zeros(max(wid.shape[0], 1), np.uint8)
    lib().or4_solve_event(C.byref(opts), C.byref(tab.cw), int(wid.shape[0]), _p(wid, C.c_int32),
                          _p(dr, C.c_double), its, _p(sel, C.c_uint8))
    return [_iter_dict(its[k]) for k in range(opts.n_iter)], sel[:wid.shape[0]].astype(bool)
