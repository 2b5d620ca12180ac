"""Cluster geometries for the single-band Hubbard model (Eq. 1).

A cluster is a number of sites L and a list of unordered bonds (i, j, t_ij),
each bond listed once.  Site i corresponds to bit i of the occupation string
(Sec. II A: site index increasing right-to-left).  The hopping amplitude enters
Eq. 1 as -t_ij (c^dag_i c_j + h.c.), so a bond with t_ij = t' = -0.3 gives a
matrix element of +0.3 times the fermion sign.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Tuple


@dataclass(frozen=True)
class Cluster:
    name: str
    L: int
    bonds: Tuple[Tuple[int, int], ...]
    t: Tuple[float, ...]
    coords: Tuple[Tuple[int, int], ...] = field(default=(), compare=False)

    @property
    def n_bonds(self) -> int:
        return len(self.bonds)

    def bond_array(self):
        import numpy as np
        return np.asarray(self.bonds, dtype=np.int32).reshape(-1, 2)

    def t_array(self):
        import numpy as np
        return np.asarray(self.t, dtype=np.float64)


def _dedup(pairs: List[Tuple[int, int, float]]) -> List[Tuple[int, int, float]]:
    seen = set()
    out = []
    for i, j, t in pairs:
        if i == j:
            raise ValueError(f"self bond at site {i}")
        key = (min(i, j), max(i, j))
        if key in seen:
            raise ValueError(f"bond {key} listed twice; cluster too small for this bond pattern")
        seen.add(key)
        out.append((i, j, t))
    return out


def _make(name, L, pairs, coords=()):
    pairs = _dedup(pairs)
    return Cluster(name=name, L=L, bonds=tuple((i, j) for i, j, _ in pairs),
                   t=tuple(float(t) for _, _, t in pairs), coords=tuple(coords))


def dimer(t: float = 1.0) -> Cluster:
    """Two sites joined by one bond."""
    return _make("dimer", 2, [(0, 1, t)], [(0, 0), (1, 0)])


def ring(L: int, t: float = 1.0) -> Cluster:
    """1D periodic chain 0-1-...-(L-1)-0 (the loop of the Sec. II B example)."""
    if L < 3:
        raise ValueError("ring needs L >= 3 (use dimer() for two sites)")
    return _make(f"ring{L}", L, [(i, (i + 1) % L, t) for i in range(L)], [(i, 0) for i in range(L)])


def rect_periodic(Lx: int, Ly: int, t: float = 1.0, tprime: float = 0.0) -> Cluster:
    """Lx x Ly periodic square lattice, site = x + Lx*y.

    Nearest-neighbour bonds (x+1, y) and (x, y+1) with amplitude t; if tprime is
    nonzero, next-nearest (diagonal) bonds (x+1, y+1) and (x+1, y-1) with t'.
    """
    pairs = []
    coords = []
    for y in range(Ly):
        for x in range(Lx):
            coords.append((x, y))
    for y in range(Ly):
        for x in range(Lx):
            s = x + Lx * y
            pairs.append((s, (x + 1) % Lx + Lx * y, t))
            pairs.append((s, x + Lx * ((y + 1) % Ly), t))
    if tprime != 0.0:
        for y in range(Ly):
            for x in range(Lx):
                s = x + Lx * y
                pairs.append((s, (x + 1) % Lx + Lx * ((y + 1) % Ly), tprime))
                pairs.append((s, (x + 1) % Lx + Lx * ((y - 1) % Ly), tprime))
    name = f"rect{Lx}x{Ly}" + (f"_tp{tprime:g}" if tprime else "")
    return _make(name, Lx * Ly, pairs, coords)


def square_periodic(n: int, t: float = 1.0, tprime: float = 0.0) -> Cluster:
    return rect_periodic(n, n, t, tprime)


def tilted_18(t: float = 1.0) -> Cluster:
    """18-site tilted square cluster with periodic vectors a1=(3,3), a2=(3,-3).

    Sites are the classes of Z^2 modulo the lattice spanned by a1, a2.  The
    representative of a class is (x, y) with 0 <= x < 3 and 0 <= y < 6, obtained
    by reducing x and y mod 6 (since (6,0)=a1+a2 and (0,6)=a1-a2) and then, if
    x >= 3, subtracting a1 = (3,3).  Site index = x + 3*y.  Bonds: (x+1, y) and
    (x, y+1) from every site, 36 in total, every site of degree 4.
    """
    def canon(x, y):
        x %= 6
        y %= 6
        if x >= 3:
            x -= 3
            y = (y - 3) % 6
        return x + 3 * y

    pairs = []
    coords = [(x, y) for y in range(6) for x in range(3)]
    for y in range(6):
        for x in range(3):
            s = canon(x, y)
            pairs.append((s, canon(x + 1, y), t))
            pairs.append((s, canon(x, y + 1), t))
    return _make("tilted18", 18, pairs, coords)
