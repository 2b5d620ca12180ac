"""Continued-fraction Green's function oracle pinned to spectral sums, the sum rule, the free
limit and the real-space operators of Eq. 1."""
import cmath

import numpy as np
import pytest

import workloads as wl
from oracle import momentum as M
from oracle import response as R
from oracle.basis import Basis
from oracle.hamiltonian import Model, dense as real_dense

Z = np.linspace(-6, 6, 25) + 0.3j


def _sector_data(g, t, tp, U, nu, nd):
    best = None
    for K in range(g.N):
        lst = M.sector_list(g, nu, nd, K)
        if len(lst) == 0:
            continue
        w, V = R.sector_ground(g, t, tp, U, nu, nd, K)
        if best is None or w[0] < best[0]:
            best = (w[0], K, V[:, 0], lst, w[1] - w[0] if len(w) > 1 else np.inf)
    return best


def test_full_continued_fraction_equals_spectral_sum():
    g = M.Grid(6, 1)
    E0, K0, psi, lst, _ = _sector_data(g, 1.0, 0.0, 4.0, 3, 3)
    for k in range(g.N):
        dst = M.sector_list(g, 2, 3, g.sub(K0, k))
        phi = R.apply_op(g, lst, dst, "c", 0, k, psi, 3)
        if np.linalg.norm(phi) < 1e-12:
            continue
        H = M.dense(M.KModel(g, 1.0, 0.0, 4.0, 2, 3, g.sub(K0, k)))
        a, b = R.lanczos_coefficients(H, phi, len(dst))
        cf = R.continued_fraction(a, b, float(phi @ phi), E0, Z)
        assert np.max(np.abs(cf - R.spectral_sum(H, phi, E0, Z))) < 1e-10


def test_removal_plus_addition_weight_is_one():
    g = M.Grid(3, 3)
    E0, K0, psi, lst, _ = _sector_data(g, 1.0, -0.3, 5.0, 2, 2)
    for spin in (0, 1):
        for k in range(g.N):
            nu_r, nd_r = (1, 2) if spin == 0 else (2, 1)
            nu_a, nd_a = (3, 2) if spin == 0 else (2, 3)
            rem = R.apply_op(g, lst, M.sector_list(g, nu_r, nd_r, g.sub(K0, k)), "c", spin, k, psi, 2)
            add = R.apply_op(g, lst, M.sector_list(g, nu_a, nd_a, g.add(K0, k)), "cdag", spin, k, psi, 2)
            assert abs(rem @ rem + add @ add - 1.0) < 1e-12


def test_free_fermions_have_one_removal_pole():
    g = M.Grid(6, 1)
    E0, K0, psi, lst, _ = _sector_data(g, 1.0, 0.0, 0.0, 3, 3)
    eps = g.eps(1.0, 0.0)
    for k in range(g.N):
        dst = M.sector_list(g, 2, 3, g.sub(K0, k))
        phi = R.apply_op(g, lst, dst, "c", 0, k, psi, 3)
        wgt = phi @ phi
        if wgt < 1e-12:
            continue
        assert abs(wgt - 1.0) < 1e-12
        H = M.dense(M.KModel(g, 1.0, 0.0, 0.0, 2, 3, g.sub(K0, k)))
        w, V = np.linalg.eigh(H)
        amp = (V.T @ phi) ** 2
        n = int(np.argmax(amp))
        assert abs(amp[n] - 1.0) < 1e-10 and abs((w[n] - E0) + eps[k]) < 1e-10


def _real_c(L, nu, nd, src, dst, j, spin):
    """Matrix of the site operator c_{j spin} from the (nu, nd) real-space basis to its (nu-1, nd) or
    (nu, nd-1) neighbour, with the descending-creator order (up left of down)."""
    pos = {int(s): i for i, s in enumerate(dst.combined)}
    C = np.zeros((dst.D, src.D))
    for i, s in enumerate(src.combined):
        s = int(s)
        u, d = s >> L, s & ((1 << L) - 1)
        part = u if spin == 0 else d
        if not (part >> j) & 1:
            continue
        sgn = R.sign_above(part, j) * ((-1) ** nu if spin == 1 else 1)
        part2 = part ^ (1 << j)
        t = (part2 << L) | d if spin == 0 else (u << L) | part2
        C[pos[t], i] = sgn
    return C


@pytest.mark.parametrize("U,spin", [(4.0, 0), (4.0, 1), (0.0, 0)])
def test_momentum_green_function_equals_real_space(U, spin):
    """c_k = N^-1/2 sum_j e^(-i k r_j) c_j on the real-space ring reproduces the momentum-space G_k(z)."""
    L, nu, nd = 6, 3, 3
    g = M.Grid(L, 1)
    E0, K0, psi_k, lst, gap = _sector_data(g, 1.0, 0.0, U, nu, nd)
    m = Model.from_cluster(wl.ring(L), U, nu, nd)
    src = Basis(L, nu, nd)
    Hr = real_dense(m, src)
    w, V = np.linalg.eigh(Hr)
    assert abs(w[0] - E0) < 1e-10 and w[1] - w[0] > 1e-6  # non-degenerate ground state
    psi_r = V[:, 0]
    nu2, nd2 = (nu - 1, nd) if spin == 0 else (nu, nd - 1)
    dst = Basis(L, nu2, nd2)
    Hd = real_dense(Model.from_cluster(wl.ring(L), U, nu2, nd2), dst)
    wd, Vd = np.linalg.eigh(Hd)
    for k in range(L):
        ck = sum(cmath.exp(-2j * np.pi * k * j / L) * _real_c(L, nu, nd, src, dst, j, spin) for j in range(L)) / np.sqrt(L)
        phi_r = ck @ psi_r
        g_real = np.array([np.sum(np.abs(Vd.T @ phi_r) ** 2 / (zz - (wd - E0))) for zz in Z])
        dstk = M.sector_list(g, nu2, nd2, g.sub(K0, k))
        phi_k = R.apply_op(g, lst, dstk, "c", spin, k, psi_k, nu)
        Hk = M.dense(M.KModel(g, 1.0, 0.0, U, nu2, nd2, g.sub(K0, k)))
        g_mom = R.spectral_sum(Hk, phi_k, E0, Z)
        assert np.max(np.abs(g_real - g_mom)) < 1e-10
