"""Parameter grid of the 5-D helix voxel space and its shared input tables.

The paper discretises the helix parameter space into voxels (multidimensional intervals,
Section 3.1).  Here a voxel ("cell") is a box over the five axes

    a = 0: d0      signed transverse distance of the POCA to the origin  [m]
    a = 1: phi0    azimuth of the helix tangent at the POCA              [rad]
    a = 2: omega   signed curvature rho = 1/R                            [1/m]
    a = 3: z0      z of the helix at the POCA                            [m]
    a = 4: tanl    lambda = tan(dip angle)

Level 0 has bins[a] cells along axis a; every level halves each cell along every axis, so a
level-L cell index is idx_a in [0, bins[a] * 2**L) and its 32 children are 2 idx_a + bit_a.
The omega axis is split into two equal halves [-1, -0.15] and [0.15, 1] so that no cell
straddles omega = 0.

This module only defines the grid: the finest-level cell edges (rounded to nearest once
here), a table of outward-rounded enclosures of sin/cos over every phi0 cell of every
level, and a table of sin/cos at every phi0 cell's centre (lo + hi) / 2 (libm values, for
the midpoint form of the vote).  All are inputs shared by every consumer; none of the
voting arithmetic is here.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

AXES = ("d0", "phi0", "omega", "z0", "tanl")
N_AXES = 5
KEY_BITS = 10            # minimum bits per axis in a cell key


def key_bits_for(bins, levels: int) -> list:
    """Bits of each axis in a cell key: max(10, ceil(log2(bins[a] << levels))); axis a
    starts at bit sum(bits[:a]), d0 lowest (so a grid whose finest level has at most 1024
    cells per axis uses 10 bits per axis)."""
    out = []
    for b in bins:
        n, bits = int(b) << int(levels), KEY_BITS
        while (1 << bits) < n:
            bits += 1
        out.append(bits)
    return out


@dataclass
class Grid:
    bins: np.ndarray        # int32[5], level-0 bins per axis
    levels: int             # number of bisection levels after level 0
    topk: int
    lo_edge: list           # per axis: float64[bins[a] << levels], finest-cell lower edges
    hi_edge: list           # per axis: float64[bins[a] << levels], finest-cell upper edges
    sincos: np.ndarray      # float64[sum_L bins[1] << L, 4]: (sin_lo, sin_hi, cos_lo, cos_hi)
    sincos_offset: np.ndarray   # int64[levels + 1]: first row of level L in `sincos`
    ranges: tuple = ()
    sincos_mid: np.ndarray = None   # float64[rows, 2]: (sin c, cos c), c = phi0 cell centre

    def n_fine(self, a: int) -> int:
        return int(self.bins[a]) << self.levels

    def cell_edges(self, level: int, a: int, idx):
        """Lower and upper edge of cell idx (any array) on axis a at `level`."""
        sh = self.levels - level
        idx = np.asarray(idx, np.int64)
        return self.lo_edge[a][idx << sh], self.hi_edge[a][((idx + 1) << sh) - 1]

    def n_coarse(self) -> int:
        return int(np.prod(self.bins.astype(np.int64)))

    def key_bits(self) -> list:
        return key_bits_for(self.bins, self.levels)


def _uniform_edges(lo: float, hi: float, n: int):
    w = (hi - lo) / n
    e = lo + np.arange(n + 1, dtype=np.float64) * w
    return e[:-1].copy(), e[1:].copy()


def _widen(x: np.ndarray, k: int, direction: float) -> np.ndarray:
    for _ in range(k):
        x = np.nextafter(x, direction)
    return x


def sincos_enclosures(a: np.ndarray, b: np.ndarray, ulps: int = 2):
    """Outward enclosures of sin and cos over [a_i, b_i]: hull of the end-point values
    widened by `ulps` ulp each way, joined with +-1 wherever a multiple of pi/2 where sin or
    cos reaches an extremum may lie inside the cell (tested with a margin), clamped to
    [-1, 1]."""
    sa, sb, ca, cb = np.sin(a), np.sin(b), np.cos(a), np.cos(b)
    s_lo = _widen(np.minimum(sa, sb), ulps, -np.inf)
    s_hi = _widen(np.maximum(sa, sb), ulps, np.inf)
    c_lo = _widen(np.minimum(ca, cb), ulps, -np.inf)
    c_hi = _widen(np.maximum(ca, cb), ulps, np.inf)
    eps = 1e-12
    half_pi = np.pi / 2.0
    k_lo = np.floor((a - eps) / half_pi).astype(np.int64)
    k_hi = np.ceil((b + eps) / half_pi).astype(np.int64)
    for i in range(a.shape[0]):
        for k in range(k_lo[i], k_hi[i] + 1):
            x = k * half_pi
            if a[i] - eps <= x <= b[i] + eps:
                m = k % 4          # 0: cos=1, 1: sin=1, 2: cos=-1, 3: sin=-1
                if m == 0:
                    c_hi[i] = 1.0
                elif m == 1:
                    s_hi[i] = 1.0
                elif m == 2:
                    c_lo[i] = -1.0
                else:
                    s_lo[i] = -1.0
    clip = lambda x: np.clip(x, -1.0, 1.0)
    return clip(s_lo), clip(s_hi), clip(c_lo), clip(c_hi)


def make_grid(bins, levels: int, topk: int,
              d0=(-0.01, 0.01), phi0=(0.0, 2.0 * np.pi), omega_abs=(0.15, 1.0),
              z0=(-0.10, 0.10), tanl=(-0.8, 0.8)) -> Grid:
    bins = np.asarray(bins, np.int32)
    assert bins.shape == (5,) and bins[2] % 2 == 0, "omega bins are split evenly per sign"
    assert sum(key_bits_for(bins, levels)) <= 64 and all(int(b) << levels <= 1 << 16 for b in bins)
    lo_e, hi_e = [], []
    for a, rng in enumerate((d0, phi0, None, z0, tanl)):
        n = int(bins[a]) << levels
        if a == 2:
            h = n // 2
            nlo, nhi = _uniform_edges(-omega_abs[1], -omega_abs[0], h)
            plo, phi_ = _uniform_edges(omega_abs[0], omega_abs[1], h)
            lo_e.append(np.concatenate([nlo, plo]))
            hi_e.append(np.concatenate([nhi, phi_]))
        else:
            l_, h_ = _uniform_edges(rng[0], rng[1], n)
            lo_e.append(l_)
            hi_e.append(h_)
    g = Grid(bins=bins, levels=levels, topk=topk, lo_edge=lo_e, hi_edge=hi_e,
             sincos=np.zeros((0, 4)), sincos_offset=np.zeros(levels + 1, np.int64),
             ranges=(d0, phi0, omega_abs, z0, tanl))
    rows, mids, offs, parent = [], [], [], None
    off = 0
    for L in range(levels + 1):
        n = int(bins[1]) << L
        a, b = g.cell_edges(L, 1, np.arange(n))
        s_lo, s_hi, c_lo, c_hi = sincos_enclosures(a, b)
        if parent is not None:   # a child's enclosure never exceeds its parent's
            p = parent[np.arange(n) >> 1]
            s_lo = np.maximum(s_lo, p[:, 0])
            s_hi = np.minimum(s_hi, p[:, 1])
            c_lo = np.maximum(c_lo, p[:, 2])
            c_hi = np.minimum(c_hi, p[:, 3])
        tab = np.stack([s_lo, s_hi, c_lo, c_hi], axis=1)
        rows.append(tab)
        c = (a + b) * 0.5
        mids.append(np.stack([np.sin(c), np.cos(c)], axis=1))
        offs.append(off)
        off += n
        parent = tab
    g.sincos = np.ascontiguousarray(np.concatenate(rows, axis=0))
    g.sincos_offset = np.asarray(offs, np.int64)
    g.sincos_mid = np.ascontiguousarray(np.concatenate(mids, axis=0))
    return g


def _layout(grid):
    bits = [KEY_BITS] * N_AXES if grid is None else grid.key_bits()
    return bits, [int(sum(bits[:a])) for a in range(N_AXES)]


def cell_key(idx5, grid: Grid | None = None) -> np.ndarray:
    """Packed uint64 key sum_a idx_a << s_a (s_a from key_bits_for; 10 a without a grid);
    idx5 has shape (..., 5)."""
    bits, sh = _layout(grid)
    idx5 = np.asarray(idx5, np.uint64)
    k = np.zeros(idx5.shape[:-1], np.uint64)
    for a in range(N_AXES):
        k |= idx5[..., a] << np.uint64(sh[a])
    return k


def key_indices(keys, grid: Grid | None = None) -> np.ndarray:
    bits, sh = _layout(grid)
    keys = np.asarray(keys, np.uint64)
    return np.stack([(keys >> np.uint64(sh[a])) & np.uint64((1 << bits[a]) - 1)
                     for a in range(N_AXES)], axis=-1).astype(np.int64)


def coarse_index_to_idx5(lin, bins) -> np.ndarray:
    """Level-0 linear index (d0 fastest, tanl slowest) -> per-axis indices.  This order
    is the key order, so sorting by linear index sorts by key."""
    lin = np.asarray(lin, np.int64)
    out = []
    for a in range(N_AXES):
        out.append(lin % int(bins[a]))
        lin = lin // int(bins[a])
    return np.stack(out, axis=-1)
