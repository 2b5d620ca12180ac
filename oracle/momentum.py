"""Momentum-space Paradeisos by definition (oracle; test infrastructure only).

Sec. IV A of the paper: on a periodic cluster the single-particle momenta
k_0 .. k_{N-1} label the bits of a spin string (bit i = occupation of k_i), the
total momentum K of a string is the sum of its occupied momenta modulo the
Brillouin zone, and a fixed-K sector of the spin-full basis is indexed by the
extended combinatorial tables C_i^m(k) (recursion of Sec. IV A) and their
spin-full version C~_i^m(k; n_dn) (Eq. 6).

Readings used here (each listed with the paper's words it resolves):

* momentum grid of an Lx x Ly cluster (Ly = 1: ring): k_i = 2 pi (mx / Lx,
  my / Ly) with i = mx + Lx * my; adding momenta adds (mx, my) modulo (Lx, Ly);
* C_i^m(k) counts the placements of m particles on bits 0 .. i-1 with total
  momentum k.  With that reading the forward map of Sec. IV A (k updated to
  include k_i before C_i^m(k) is added) gives the position of a string among the
  strings of the same sector in ascending order, and the recursion reads
  C_i^m(k) = C_{i-1}^m(k) + C_{i-1}^{m-1}(k - k_{i-1}), C_0^0(k) = [k = 0];
  the paper's own index on k in the recursion and its C_i^1 initial condition
  are one bit off from this (taken as a typesetting slip; pinned below by
  counting);
* the spin-full order is ascending in the combined integer (up << N) | dn, the
  same order as Sec. III (spin-down string in the low bits);
* the backward maps stop taking particles once m = 0;
* H of Eq. 4 with eps_k = -2t (cos kx + cos ky) - 4t' cos kx cos ky (the
  paper's dispersion; -2t cos k on a ring) and the interaction written as
  (U/N) sum_q rho_up(q) rho_dn(-q) with rho(q) = sum_k c^dag_{k+q} c_k (moving
  c_{k up} to the right through the two spin-down operators costs no sign);
  the sign of c^dag_a c_b on a string is (-1)^(occupied momenta strictly between
  positions a and b), as for a real-space hop.

Pins (tests/test_oracle_momentum.py): the tables against brute-force counting;
the maps against positions in the sorted sector list, for every state; the
sector dimensions sum to the full dimension; the union of the spectra of all
sectors equals the spectrum of the real-space Hamiltonian of Eq. 1 on the same
cluster (dense, small clusters); the U = 0 sector ground energies equal the
lowest free-fermion occupations.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


# ---------------------------------------------------------------- momentum grid
@dataclass(frozen=True)
class Grid:
    Lx: int
    Ly: int

    @property
    def N(self) -> int:
        return self.Lx * self.Ly

    def m(self, i: int):
        return i % self.Lx, i // self.Lx

    def add(self, a: int, b: int) -> int:
        ax, ay = self.m(a)
        bx, by = self.m(b)
        return (ax + bx) % self.Lx + self.Lx * ((ay + by) % self.Ly)

    def neg(self, a: int) -> int:
        ax, ay = self.m(a)
        return (-ax) % self.Lx + self.Lx * ((-ay) % self.Ly)

    def sub(self, a: int, b: int) -> int:
        return self.add(a, self.neg(b))

    def total(self, s: int) -> int:
        """Total momentum (grid index) of the occupied bits of s."""
        k = 0
        for i in range(self.N):
            if (s >> i) & 1:
                k = self.add(k, i)
        return k

    def eps(self, t: float, tp: float) -> np.ndarray:
        """Bare band energies eps_k (Sec. IV A) on the grid."""
        e = np.zeros(self.N)
        for i in range(self.N):
            mx, my = self.m(i)
            kx, ky = 2 * math.pi * mx / self.Lx, 2 * math.pi * my / self.Ly
            if self.Ly == 1:
                e[i] = -2.0 * t * math.cos(kx)
            else:
                e[i] = -2.0 * t * (math.cos(kx) + math.cos(ky)) - 4.0 * tp * math.cos(kx) * math.cos(ky)
        return e


# ---------------------------------------------------------------- sector basis by definition
def strings(N: int, n: int) -> list:
    return [s for s in range(1 << N) if bin(s).count("1") == n]


def sector_list(g: Grid, n_up: int, n_dn: int, K: int) -> np.ndarray:
    """Ascending combined integers (up << N) | dn of the sector with total momentum K."""
    N = g.N
    ups, dns = strings(N, n_up), strings(N, n_dn)
    kd = {d: g.total(d) for d in dns}
    out = []
    for u in ups:
        ku = g.total(u)
        for d in dns:
            if g.add(ku, kd[d]) == K:
                out.append((u << N) | d)
    return np.array(sorted(out), dtype=np.uint64)


# ---------------------------------------------------------------- tables (Sec. IV A recursion, Eq. 6)
def c_table(g: Grid, n: int) -> np.ndarray:
    """C[i, m, k] for 0 <= i <= N, 0 <= m <= n by the recursion."""
    N = g.N
    C = np.zeros((N + 1, n + 1, N), dtype=np.int64)
    C[0, 0, 0] = 1
    for i in range(1, N + 1):
        for m in range(n + 1):
            for k in range(N):
                C[i, m, k] = C[i - 1, m, k]
                if m >= 1:
                    C[i, m, k] += C[i - 1, m - 1, g.sub(k, i - 1)]
    return C


def c_table_by_counting(g: Grid, n: int) -> np.ndarray:
    """The same table by listing: placements of m particles on bits below i with momentum k."""
    N = g.N
    C = np.zeros((N + 1, n + 1, N), dtype=np.int64)
    for i in range(N + 1):
        for s in range(1 << i):
            m = bin(s).count("1")
            if m <= n:
                C[i, m, g.total(s)] += 1
    return C


def ct_table(g: Grid, n_up: int, n_dn: int) -> np.ndarray:
    """C~[i, m, k] = sum_kd C[i, m, k - kd] C[N, n_dn, kd] (Eq. 6)."""
    N = g.N
    Cu, Cd = c_table(g, n_up), c_table(g, n_dn)
    T = np.zeros((N + 1, n_up + 1, N), dtype=np.int64)
    for i in range(N + 1):
        for m in range(n_up + 1):
            for k in range(N):
                T[i, m, k] = sum(Cu[i, m, g.sub(k, kd)] * Cd[N, n_dn, kd] for kd in range(N))
    return T


# ---------------------------------------------------------------- maps (Sec. IV A)
def forward_map_k(g: Grid, C: np.ndarray, s: int):
    """(index within its momentum sector, total momentum) of one spin string."""
    idx, m, k = 0, 0, 0
    for i in range(g.N):
        if (s >> i) & 1:
            m += 1
            k = g.add(k, i)
            idx += int(C[i, m, k])
    return idx, k


def backward_map_k(g: Grid, C: np.ndarray, idx: int, n: int, K: int) -> int:
    s, k, m, p = 0, K, n, idx
    for i in range(g.N - 1, -1, -1):
        if m > 0 and p >= C[i, m, k]:
            s |= 1 << i
            p -= int(C[i, m, k])
            m -= 1
            k = g.sub(k, i)
    return s


def forward_map_spin(g: Grid, Cd: np.ndarray, Ct: np.ndarray, u: int, d: int) -> int:
    """Index of (up, dn) in its spin-full sector: spin-down map first, then the up bits with C~."""
    idx_d, k = forward_map_k(g, Cd, d)
    idx, m = 0, 0
    for i in range(g.N):
        if (u >> i) & 1:
            m += 1
            k = g.add(k, i)
            idx += int(Ct[i, m, k])
    return idx + idx_d


def backward_map_spin(g: Grid, Cd: np.ndarray, Ct: np.ndarray, idx: int, n_up: int, n_dn: int, K: int):
    u, k, m, p = 0, K, n_up, idx
    for i in range(g.N - 1, -1, -1):
        if m > 0 and p >= Ct[i, m, k]:
            u |= 1 << i
            p -= int(Ct[i, m, k])
            m -= 1
            k = g.sub(k, i)
    return u, backward_map_k(g, Cd, p, n_dn, k)


# ---------------------------------------------------------------- Hamiltonian of Eq. 4
@dataclass
class KModel:
    grid: Grid
    t: float
    tp: float
    U: float
    N_up: int
    N_dn: int
    K: int


def _mask_between(a: int, b: int) -> int:
    lo, hi = min(a, b), max(a, b)
    return ((1 << hi) - 1) & ~((1 << (lo + 1)) - 1)


def _move(s: int, a: int, b: int):
    """c^dag_b c_a on string s: (new string, sign) or None."""
    if not (s >> a) & 1:
        return None
    if a == b:
        return s, 1
    if (s >> b) & 1:
        return None
    sign = -1 if bin(s & _mask_between(a, b)).count("1") % 2 else 1
    return s ^ (1 << a) ^ (1 << b), sign


def row(model: KModel, lst: np.ndarray, r: int):
    """Canonical row r of H (Eq. 4) in the sector: (columns ascending, values)."""
    g, N = model.grid, model.grid.N
    s = int(lst[r])
    u, d = s >> N, s & ((1 << N) - 1)
    e = g.eps(model.t, model.tp)
    terms = {}
    diag = sum(e[i] for i in range(N) if (u >> i) & 1) + sum(e[i] for i in range(N) if (d >> i) & 1)
    terms[s] = diag
    for q in range(N):
        for k in range(N):
            mu = _move(u, k, g.add(k, q))
            if mu is None:
                continue
            for kp in range(N):
                md = _move(d, kp, g.sub(kp, q))
                if md is None:
                    continue
                t2 = (mu[0] << N) | md[0]
                terms[t2] = terms.get(t2, 0.0) + model.U / N * mu[1] * md[1]
    cols = np.searchsorted(lst, np.array(list(terms.keys()), dtype=np.uint64))
    vals = np.array(list(terms.values()))
    o = np.argsort(cols)
    return cols[o], vals[o]


def dense(model: KModel) -> np.ndarray:
    lst = sector_list(model.grid, model.N_up, model.N_dn, model.K)
    H = np.zeros((len(lst), len(lst)))
    for r in range(len(lst)):
        c, v = row(model, lst, r)
        H[r, c] = v
    return H


def apply(model: KModel, x: np.ndarray) -> np.ndarray:
    lst = sector_list(model.grid, model.N_up, model.N_dn, model.K)
    y = np.zeros(len(lst))
    for r in range(len(lst)):
        c, v = row(model, lst, r)
        y[r] = np.dot(v, x[c])
    return y
