"""Momentum-space oracle (Sec. IV A) pinned to counting, to sorted positions and to the
real-space Hamiltonian of Eq. 1."""
import numpy as np
import pytest

import workloads as wl
from oracle import momentum as M
from oracle.basis import Basis
from oracle.hamiltonian import Model, dense as real_dense
from oracle.lanczos import one_body_ground


@pytest.mark.parametrize("Lx,Ly,n", [(6, 1, 3), (3, 3, 4), (4, 4, 3)])
def test_tables_match_counting(Lx, Ly, n):
    g = M.Grid(Lx, Ly)
    assert np.array_equal(M.c_table(g, n), M.c_table_by_counting(g, n))


@pytest.mark.parametrize("Lx,Ly,nu,nd", [(6, 1, 2, 3), (3, 3, 2, 2), (4, 4, 2, 1)])
def test_maps_are_sorted_positions(Lx, Ly, nu, nd):
    """Forward map = position in the ascending sector list, backward map its inverse, every state."""
    g = M.Grid(Lx, Ly)
    Cd, Ct = M.c_table(g, nd), M.ct_table(g, nu, nd)
    total = 0
    for K in range(g.N):
        lst = M.sector_list(g, nu, nd, K)
        total += len(lst)
        for r, s in enumerate(lst):
            u, d = int(s) >> g.N, int(s) & ((1 << g.N) - 1)
            assert M.forward_map_spin(g, Cd, Ct, u, d) == r
            assert M.backward_map_spin(g, Cd, Ct, r, nu, nd, K) == (u, d)
        # the sector size is the last table entry: C~_N^{n_up}(K)
        assert len(lst) == Ct[g.N, nu, K]
    assert total == len(M.strings(g.N, nu)) * len(M.strings(g.N, nd))


def _real_cluster(Lx, Ly, tp):
    return wl.ring(Lx) if Ly == 1 else wl.rect_periodic(Lx, Ly, 1.0, tp)


@pytest.mark.parametrize("Lx,Ly,tp,U,nu,nd", [(6, 1, 0.0, 3.0, 2, 2), (5, 1, 0.0, 7.0, 3, 2),
                                             (3, 3, -0.3, 4.0, 2, 2), (4, 4, -0.3, 8.0, 1, 2)])
def test_sector_spectra_union_is_real_space_spectrum(Lx, Ly, tp, U, nu, nd):
    """H of Eq. 4 block-diagonalises H of Eq. 1: the eigenvalues of all momentum sectors together are
    exactly those of the real-space Hamiltonian on the same cluster (same t, t', U, filling)."""
    g = M.Grid(Lx, Ly)
    ev = []
    for K in range(g.N):
        H = M.dense(M.KModel(g, 1.0, tp, U, nu, nd, K))
        assert np.array_equal(H, H.T)
        ev.extend(np.linalg.eigvalsh(H))
    m = Model.from_cluster(_real_cluster(Lx, Ly, tp), U, nu, nd)
    er = np.linalg.eigvalsh(real_dense(m, Basis(m.L, nu, nd)))
    assert len(ev) == len(er)
    assert np.max(np.abs(np.sort(ev) - er)) < 1e-11


def test_u0_sector_energies_are_free_fermion_sums():
    """At U = 0 the sector ground energy is the lowest sum of eps over n_up + n_dn occupied momenta
    with total momentum K; the overall minimum equals the filled one-body levels."""
    g = M.Grid(4, 4)
    e = g.eps(1.0, -0.3)
    nu, nd = 2, 1
    best = {}
    for u in M.strings(g.N, nu):
        for d in M.strings(g.N, nd):
            K = g.add(g.total(u), g.total(d))
            E = sum(e[i] for i in range(g.N) if (u >> i) & 1) + sum(e[i] for i in range(g.N) if (d >> i) & 1)
            best[K] = min(best.get(K, np.inf), E)
    for K in range(g.N):
        H = M.dense(M.KModel(g, 1.0, -0.3, 0.0, nu, nd, K))
        assert abs(np.linalg.eigvalsh(H)[0] - best[K]) < 1e-12
    cl = wl.rect_periodic(4, 4, 1.0, -0.3)
    assert abs(min(best.values()) - one_body_ground(cl.L, cl.bond_array(), cl.t_array(), nu, nd)) < 1e-12


def test_row_apply_matches_dense_and_is_hermitian():
    g = M.Grid(3, 3)
    mod = M.KModel(g, 1.0, -0.3, 5.0, 2, 2, 4)
    H = M.dense(mod)
    x = np.random.default_rng(1).standard_normal(len(H))
    assert np.allclose(M.apply(mod, x), H @ x, rtol=0, atol=1e-12)
    y = np.random.default_rng(2).standard_normal(len(H))
    assert abs(x @ (H @ y) - (H @ x) @ y) < 1e-10
