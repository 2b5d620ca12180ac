"""Pins of the oracle Hamiltonian (CPU only)."""
import json
import os

import numpy as np
import pytest

import workloads as wl
from oracle.basis import Basis
from oracle.hamiltonian import KronOperator, Model, apply, dense, row
from oracle.lanczos import start_vector
from tests.conftest import GOLDEN

EX = json.load(open(os.path.join(GOLDEN, "paper_examples.json")))


def test_hop_example_from_paper():
    """Spin-up hops of 0101 x 1011 on the 4-site loop (Sec. II B), including the minus sign."""
    g = EX["hop_example"]
    L = g["L"]
    bonds = np.array(g["bonds"], dtype=np.int32)
    t = 0.7
    m = Model(L, bonds, np.full(len(bonds), t), U=0.0, N_up=2, N_dn=3)
    b = Basis(L, 2, 3)
    up, dn = int(g["up"], 2), int(g["dn"], 2)
    r = int(b.index_of(np.uint64((up << L) | dn)))
    cols, vals = row(m, b, r)
    got = {}
    for c, v in zip(cols, vals):
        st = int(b.state_at(c))
        u2, d2 = st >> L, st & ((1 << L) - 1)
        if d2 == dn and u2 != up:
            got[format(u2, "04b")] = v
    want = {k: -t * s for k, s in g["terms"].items()}
    assert got == want


def test_hop_example_full_index_form():
    """The same row in combined indices: C(4,3) * idx_up + idx_dn with the paper's tables."""
    g = EX["hop_example"]
    tab_up = EX["spin_tables"]["n2"]
    tab_dn = EX["spin_tables"]["n3"]
    b = Basis(4, 2, 3)
    m = Model(4, np.array(g["bonds"]), np.ones(4), U=0.0, N_up=2, N_dn=3)
    r = 4 * tab_up.index(0b0101) + tab_dn.index(0b1011)
    assert r == 5
    cols, vals = row(m, b, r)
    up_cols = {4 * tab_up.index(int(k, 2)) + tab_dn.index(0b1011): -s for k, s in g["terms"].items()}
    got = {int(c): float(v) for c, v in zip(cols, vals) if c in up_cols}
    assert got == {9: -1.0, 1: -1.0, 13: -1.0, 21: 1.0}
    assert got == up_cols


@pytest.mark.parametrize("cl,nu,nd,U", [(wl.ring(8), 4, 4, 4.0), (wl.ring(6), 2, 3, 1.5),
                                        (wl.rect_periodic(3, 3, 1.0, -0.3), 2, 2, 3.0)])
def test_hermitian_bit_exact(cl, nu, nd, U):
    m = Model.from_cluster(cl, U, nu, nd)
    b = Basis(cl.L, nu, nd)
    H = dense(m, b)
    assert np.array_equal(H, H.T)


def test_row_count_is_one_plus_hops():
    cl = wl.square_periodic(4, 1.0, -0.3)
    m = Model.from_cluster(cl, 8.0, 2, 2)
    b = Basis(16, 2, 2)
    rng = np.random.default_rng(5)
    for r in rng.integers(0, b.D, 20):
        st = int(b.state_at(r))
        up, dn = st >> 16, st & 0xFFFF
        nh = 0
        for (i, j) in cl.bonds:
            for s in (up, dn):
                nh += ((s >> i) & 1) != ((s >> j) & 1)
        cols, _ = row(m, b, int(r))
        assert len(cols) == 1 + nh
        assert len(set(cols.tolist())) == len(cols)


@pytest.mark.parametrize("cl,nu,nd,U", [(wl.ring(8), 4, 4, 4.0), (wl.ring(7), 3, 2, 2.0),
                                        (wl.rect_periodic(4, 3), 3, 4, 5.0),
                                        (wl.rect_periodic(3, 3, 1.0, -0.3), 4, 4, 8.0)])
@pytest.mark.parametrize("backend", ["c", "numpy"])
def test_apply_matches_dense_and_kron(cl, nu, nd, U, backend):
    """Both evaluations of the tensor-product form (the C helper of
    oracle/kron_hv.c, which the full-size GPU checks and the CPU baseline use,
    and the scipy one) against the term-by-term definition and the dense matrix."""
    m = Model.from_cluster(cl, U, nu, nd)
    b = Basis(cl.L, nu, nd)
    x = start_vector(3, b.D)
    y = apply(m, b, x)
    k = KronOperator(m, backend=backend)
    assert (k._lib is not None) == (backend == "c")
    yk = k(x)
    assert np.max(np.abs(y - yk)) <= 1e-13 * np.max(np.abs(y))
    if b.D <= 6000:
        H = dense(m, b)
        yd = H @ x
        assert np.max(np.abs(y - yd)) <= 1e-13 * np.max(np.abs(y))
    # symmetry of the operator: <x, H z> = <H x, z>
    z = start_vector(4, b.D)
    assert abs(np.dot(x, k(z)) - np.dot(yk, z)) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(z) * 50


def test_basis_vector_gives_row():
    cl = wl.ring(8)
    m = Model.from_cluster(cl, 4.0, 4, 4)
    b = Basis(8, 4, 4)
    k = KronOperator(m)
    for r in (0, 17, 2450, 4899):
        e = np.zeros(b.D)
        e[r] = 1.0
        col = k(e)  # column r of H == row r by symmetry
        cols, vals = row(m, b, r)
        nz = np.nonzero(col)[0]
        assert nz.tolist() == cols.tolist()
        assert np.array_equal(col[nz], vals)


@pytest.mark.parametrize("backend", ["c", "numpy"])
def test_abs_apply_is_entrywise_absolute_product(backend):
    cl = wl.rect_periodic(3, 3, 1.0, -0.3)
    m = Model.from_cluster(cl, -3.0, 4, 3)  # negative U: the absolute value must reach the diagonal too
    b = Basis(9, 4, 3)
    x = start_vector(2, b.D)
    want = np.abs(dense(m, b)) @ np.abs(x) if b.D <= 6000 else None
    got = KronOperator(m, backend=backend).abs_apply(x)
    if want is None:
        # row by row from the canonical rows
        for r in range(0, b.D, 997):
            c, v = row(m, b, r)
            assert abs(got[r] - np.dot(np.abs(v), np.abs(x[c]))) <= 1e-13 * got[r]
    else:
        assert np.allclose(got, want, rtol=1e-13, atol=0)


def test_apply_rows_matches_apply():
    from oracle.hamiltonian import apply_rows
    cl = wl.rect_periodic(4, 3)
    m = Model.from_cluster(cl, 5.0, 5, 4)
    b = Basis(12, 5, 4)
    x = start_vector(6, b.D)
    rows = np.array([0, 5, 777, b.D - 1])
    assert np.array_equal(apply_rows(m, b, x, rows), apply(m, b, x)[rows])


@pytest.mark.parametrize("cl,nu,nd,U", [(wl.ring(8), 4, 4, 4.0), (wl.rect_periodic(3, 3, 1.0, -0.3), 4, 3, 2.0),
                                        (wl.tilted_18(), 2, 3, 6.0)])
def test_row_by_counting_matches_list_rows(cl, nu, nd, U):
    from oracle.hamiltonian import row_by_counting
    m = Model.from_cluster(cl, U, nu, nd)
    b = Basis(cl.L, nu, nd)
    for r in np.unique(np.linspace(0, b.D - 1, 37).astype(np.int64)):
        c1, v1 = row(m, b, int(r))
        c2, v2 = row_by_counting(m, int(r))
        assert np.array_equal(c1, c2) and np.array_equal(v1, v2)
