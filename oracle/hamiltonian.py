"""Hubbard Hamiltonian of Eq. 1 by definition (oracle; test infrastructure only).

H = -sum_{<ij>,sigma} t_ij (c^dag_{i sigma} c_{j sigma} + h.c.) + U sum_i n_{i up} n_{i dn}

Readings of the paper used here (Sec. II A-B):

* every bond (i, j) is listed once and contributes both hop directions, so the
  matrix element between two strings connected by it is -t_ij times a sign;
* the sign is (-1)^(number of particles of the same spin on sites strictly
  between i and j): moving c_j and then c^dag_i through the higher-index
  creators of the normal-ordered product (Sec. II A) leaves exactly the
  particles between the two sites as the net exchange count, and the other
  spin species contributes no sign because its creators are crossed twice;
* the interaction is U times the number of doubly occupied sites, the popcount
  of (up AND dn) (Sec. II B);
* the row of a basis state r holds H[r, c] for all states c; rows are returned
  in canonical form, sorted by column.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .basis import Basis, position, spin_list


def popcount64(a: np.ndarray) -> np.ndarray:
    a = np.asarray(a, dtype=np.uint64)
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(a).astype(np.int64)
    c = np.zeros(a.shape, dtype=np.int64)
    v = a.copy()
    while np.any(v):
        c += (v & np.uint64(1)).astype(np.int64)
        v >>= np.uint64(1)
    return c


def between_mask(i: int, j: int) -> int:
    """Bits strictly between sites i and j."""
    lo, hi = min(i, j), max(i, j)
    return ((1 << hi) - 1) & ~((1 << (lo + 1)) - 1)


@dataclass
class Model:
    L: int
    bonds: np.ndarray  # (n_bonds, 2) int
    t: np.ndarray      # (n_bonds,) float64
    U: float
    N_up: int
    N_dn: int

    @classmethod
    def from_cluster(cls, cluster, U, N_up, N_dn):
        return cls(cluster.L, cluster.bond_array(), cluster.t_array(), float(U), int(N_up), int(N_dn))


def hop_targets(s: np.ndarray, i: int, j: int):
    """For strings s: whether bond (i, j) can move a particle, the new string, and the sign."""
    s = np.asarray(s, dtype=np.uint64)
    bi = (s >> np.uint64(i)) & np.uint64(1)
    bj = (s >> np.uint64(j)) & np.uint64(1)
    valid = bi != bj
    new = s ^ np.uint64((1 << i) | (1 << j))
    nb = popcount64(s & np.uint64(between_mask(i, j)))
    sign = np.where(nb % 2 == 0, 1.0, -1.0)
    return valid, new, sign


def row(model: Model, basis: Basis, r: int):
    """Canonical row r of H: (columns sorted ascending, values)."""
    L = model.L
    state = int(basis.state_at(r))
    up, dn = state >> L, state & ((1 << L) - 1)
    cols = [r]
    vals = [model.U * bin(up & dn).count("1")]
    for b in range(len(model.t)):
        i, j = int(model.bonds[b, 0]), int(model.bonds[b, 1])
        for spin in (0, 1):
            s = up if spin == 0 else dn
            if ((s >> i) & 1) == ((s >> j) & 1):
                continue
            s2 = s ^ ((1 << i) | (1 << j))
            nbetween = bin(s & between_mask(i, j)).count("1")
            sign = -1.0 if nbetween % 2 else 1.0
            target = (s2 << L) | dn if spin == 0 else (up << L) | s2
            c = int(basis.index_of(np.uint64(target)))
            assert c >= 0
            cols.append(c)
            vals.append(-model.t[b] * sign)
    order = np.argsort(np.asarray(cols, dtype=np.int64), kind="stable")
    return np.asarray(cols, dtype=np.int64)[order], np.asarray(vals, dtype=np.float64)[order]


def row_by_counting(model: Model, r: int):
    """Canonical row r for clusters too large to list (e.g. 18 sites at half filling).

    Same terms as `row`; positions come from the counting definition of the
    sorted order (`count_below` / `string_at`) instead of a stored list:
    combined position = C(L, N_dn) * position_up + position_dn (the order of
    the sorted combined integers, up string in the high bits).
    """
    import math

    from .basis import count_below, string_at
    L = model.L
    D_dn = math.comb(L, model.N_dn)
    pu, pd_ = divmod(int(r), D_dn)
    up, dn = string_at(pu, L, model.N_up), string_at(pd_, L, model.N_dn)
    cols = [int(r)]
    vals = [model.U * bin(up & dn).count("1")]
    for b in range(len(model.t)):
        i, j = int(model.bonds[b, 0]), int(model.bonds[b, 1])
        for spin in (0, 1):
            s = up if spin == 0 else dn
            if ((s >> i) & 1) == ((s >> j) & 1):
                continue
            s2 = s ^ ((1 << i) | (1 << j))
            sign = -1.0 if bin(s & between_mask(i, j)).count("1") % 2 else 1.0
            if spin == 0:
                c = count_below(s2, L, model.N_up) * D_dn + pd_
            else:
                c = pu * D_dn + count_below(s2, L, model.N_dn)
            cols.append(c)
            vals.append(-model.t[b] * sign)
    order = np.argsort(np.asarray(cols, dtype=np.int64), kind="stable")
    return np.asarray(cols, dtype=np.int64)[order], np.asarray(vals, dtype=np.float64)[order]


def apply(model: Model, basis: Basis, x: np.ndarray) -> np.ndarray:
    """y = H x for the whole basis, evaluated term by term of Eq. 1.

    Every state is its own row; for each bond and spin the hop target is located
    in the sorted list by binary search.  Terms are added in the order diagonal,
    then bonds in list order with spin up before spin down.
    """
    L = model.L
    states = basis.combined
    up, dn = basis.split(states)
    x = np.asarray(x, dtype=np.float64)
    y = model.U * popcount64(up & dn).astype(np.float64) * x
    for b in range(len(model.t)):
        i, j = int(model.bonds[b, 0]), int(model.bonds[b, 1])
        for spin in (0, 1):
            s = up if spin == 0 else dn
            valid, s2, sign = hop_targets(s, i, j)
            if spin == 0:
                target = (s2 << np.uint64(L)) | dn
            else:
                target = (up << np.uint64(L)) | s2
            rows = np.nonzero(valid)[0]
            cols = basis.index_of(target[rows])
            assert np.all(cols >= 0)
            y[rows] += -model.t[b] * sign[rows] * x[cols]
    return y


def apply_rows(model: Model, basis: Basis, x: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """(H x)[rows]: the same term-by-term evaluation as `apply`, restricted to some rows."""
    L = model.L
    rows = np.asarray(rows, dtype=np.int64)
    states = basis.combined[rows]
    up, dn = basis.split(states)
    y = model.U * popcount64(up & dn).astype(np.float64) * x[rows]
    for b in range(len(model.t)):
        i, j = int(model.bonds[b, 0]), int(model.bonds[b, 1])
        for spin in (0, 1):
            s = up if spin == 0 else dn
            valid, s2, sign = hop_targets(s, i, j)
            target = (s2 << np.uint64(L)) | dn if spin == 0 else (up << np.uint64(L)) | s2
            k = np.nonzero(valid)[0]
            cols = basis.index_of(target[k])
            assert np.all(cols >= 0)
            y[k] += -model.t[b] * sign[k] * x[cols]
    return y


def dense(model: Model, basis: Basis) -> np.ndarray:
    """Dense H (small clusters only), assembled row by row from `row`."""
    if basis.D > 6000:
        raise ValueError("dense H only for D <= 6000")
    H = np.zeros((basis.D, basis.D))
    for r in range(basis.D):
        c, v = row(model, basis, r)
        H[r, c] = v
    return H


def spin_hop_matrix(L: int, n: int, bonds: np.ndarray, t: np.ndarray):
    """Single-spin hopping matrix on the sorted n-particle list, by definition (scipy CSR).

    Entry [r, c] = -t_b * sign for the string c reached from string r through bond b.
    """
    import scipy.sparse as sp
    lst = spin_list(L, n)
    rows, cols, vals = [], [], []
    for b in range(len(t)):
        i, j = int(bonds[b, 0]), int(bonds[b, 1])
        valid, s2, sign = hop_targets(lst, i, j)
        rr = np.nonzero(valid)[0]
        cc = position(lst, s2[rr])
        assert np.all(cc >= 0)
        rows.append(rr)
        cols.append(cc)
        vals.append(-t[b] * sign[rr])
    D = len(lst)
    if rows:
        m = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(D, D))
    else:
        m = sp.csr_matrix((D, D))
    return m, lst


def _load_c_helper():
    """The OpenMP helper compiled from oracle/kron_hv.c (built here with gcc when absent or stale)."""
    import ctypes

    from oracle.build import build
    lib = ctypes.CDLL(build())
    lib.oracle_kron_apply.restype = None
    return lib


class KronOperator:
    """y = H x using the tensor-product structure of the basis (Sec. II A).

    With x viewed as a D_up x D_dn matrix X (row = up position, column = down
    position, the combined-index order of Sec. III), the spin-up hops act on the
    row index only and the spin-down hops on the column index only, with no sign
    from the other species, so  Y = A X + X B^T + U * docc o X,  where A, B are
    the single-spin hopping matrices from `spin_hop_matrix`.  This is the same
    operator as `apply`, evaluated in an order that finishes on a laptop for
    D ~ 1e8; the tests pin it to `apply` and `row` on small clusters.

    backend "c" evaluates the products in oracle/kron_hv.c (compiled on first
    use; a failed build raises), "numpy" with scipy sparse products.  The
    choice is explicit: nothing switches from one to the other on its own.
    """

    def __init__(self, model: Model, backend: str = "c"):
        if backend not in ("c", "numpy"):
            raise ValueError("backend must be 'c' or 'numpy'")
        self.model = model
        self.A, self.up = spin_hop_matrix(model.L, model.N_up, model.bonds, model.t)
        self.B, self.dn = spin_hop_matrix(model.L, model.N_dn, model.bonds, model.t)
        self.D_up, self.D_dn = len(self.up), len(self.dn)
        self.D = self.D_up * self.D_dn
        self.backend = backend
        self._lib = _load_c_helper() if backend == "c" else None
        self._docc = None

    @property
    def docc(self):
        if self._docc is None:
            self._docc = popcount64(self.up[:, None] & self.dn[None, :]).astype(np.float64)
        return self._docc

    def __call__(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        if self._lib is not None:
            return self._call_c(x)
        X = x.reshape(self.D_up, self.D_dn)
        Y = self.model.U * self.docc * X
        Y += self.A @ X
        Y += (self.B @ X.T).T
        return Y.reshape(-1)

    def _call_c(self, x, absolute: bool = False):
        import ctypes
        y = np.empty_like(x)
        A, B = self.A, self.B
        av, bv, U = (np.abs(A.data), np.abs(B.data), abs(self.model.U)) if absolute else (A.data, B.data, self.model.U)
        keep = [np.ascontiguousarray(a) for a in (A.indptr.astype(np.int64), A.indices.astype(np.int64), av,
                                                  B.indptr.astype(np.int64), B.indices.astype(np.int64), bv,
                                                  self.up, self.dn)]
        P = ctypes.c_void_p
        self._lib.oracle_kron_apply(ctypes.c_int64(self.D_up), ctypes.c_int64(self.D_dn),
                                    *[P(k.ctypes.data) for k in keep], ctypes.c_double(U),
                                    P(x.ctypes.data), P(y.ctypes.data))
        return y

    def abs_apply(self, x: np.ndarray) -> np.ndarray:
        """|H| |x| (entrywise absolute values): the scale of the rounding error of every row sum."""
        if self._lib is not None:
            return self._call_c(np.abs(np.ascontiguousarray(x, dtype=np.float64)), absolute=True)
        X = np.abs(np.asarray(x, dtype=np.float64)).reshape(self.D_up, self.D_dn)
        Y = abs(self.model.U) * self.docc * X
        Y += abs(self.A) @ X
        Y += (abs(self.B) @ X.T).T
        return Y.reshape(-1)

    def diag_row_sums(self):
        """Row sums of |H| (used for error bounds in tests)."""
        ra = np.abs(self.A).sum(axis=1).A.ravel()
        rb = np.abs(self.B).sum(axis=1).A.ravel()
        return (abs(self.model.U) * self.docc + ra[:, None] + rb[None, :]).reshape(-1)
