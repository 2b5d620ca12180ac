"""Ground-energy pins of the oracle against closed forms and invariants (CPU only)."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle.basis import Basis
from oracle.hamiltonian import KronOperator, Model, dense
from oracle.lanczos import lanczos, one_body_ground, splitmix64_stream, start_vector


def ground_dense(cl, U, nu, nd):
    m = Model.from_cluster(cl, U, nu, nd)
    return float(np.linalg.eigvalsh(dense(m, Basis(cl.L, nu, nd)))[0])


def ground_lanczos(cl, U, nu, nd, seed=0, maxit=400, reorth=False, tol=1e-11):
    m = Model.from_cluster(cl, U, nu, nd)
    k = KronOperator(m)
    return lanczos(k, start_vector(seed, k.D), maxit, reorth=reorth, tol=tol)


@pytest.mark.parametrize("U,t", [(4.0, 1.0), (0.0, 1.0), (8.0, 0.5), (1.3, 2.0)])
def test_dimer_closed_form(U, t):
    """Two sites, one particle per spin, half filling: E0 = (U - sqrt(U^2 + 16 t^2)) / 2."""
    e = ground_dense(wl.dimer(t), U, 1, 1)
    assert abs(e - (U - math.sqrt(U * U + 16 * t * t)) / 2) < 1e-13


@pytest.mark.parametrize("cl,nu,nd", [(wl.ring(8), 4, 4), (wl.ring(8), 3, 5), (wl.ring(6), 3, 3),
                                      (wl.rect_periodic(3, 3, 1.0, -0.3), 4, 3)])
def test_U0_is_filled_one_body_levels(cl, nu, nd):
    if math.comb(cl.L, nu) * math.comb(cl.L, nd) <= 6000:
        e, tol = ground_dense(cl, 0.0, nu, nd), 1e-12
    else:
        e, tol = ground_lanczos(cl, 0.0, nu, nd, reorth=True).E0, 1e-10
    e1 = one_body_ground(cl.L, cl.bonds, cl.t, nu, nd)
    assert abs(e - e1) < tol * max(1, abs(e1))


def test_U0_ring8_closed_form():
    """Ring of 8, 4+4 particles: 2 * (-2 - 2 sqrt 2) from eps_k = -2t cos k."""
    e = ground_dense(wl.ring(8), 0.0, 4, 4)
    assert abs(e - 2 * (-2 - 2 * math.sqrt(2))) < 1e-12


def test_U0_square4x4_tprime_matches_paper_dispersion():
    """4x4 periodic with t, t': U=0 energy equals the lowest eps_k of Sec. III A's dispersion.

    eps_k = -2t (cos kx + cos ky) - 4 t' cos kx cos ky, k = 2 pi (mx, my) / 4.
    """
    t, tp = 1.0, -0.3
    cl = wl.square_periodic(4, t, tp)
    ks = [(2 * math.pi * mx / 4, 2 * math.pi * my / 4) for mx in range(4) for my in range(4)]
    eps = sorted(-2 * t * (math.cos(kx) + math.cos(ky)) - 4 * tp * math.cos(kx) * math.cos(ky) for kx, ky in ks)
    for nu, nd in [(1, 1), (2, 1), (3, 2)]:
        want = sum(eps[:nu]) + sum(eps[:nd])
        assert abs(one_body_ground(16, cl.bonds, cl.t, nu, nd) - want) < 1e-12
        r = ground_lanczos(cl, 0.0, nu, nd, maxit=300, reorth=True)
        assert abs(r.E0 - want) < 1e-9


@pytest.mark.parametrize("cl,nu,nd,U", [(wl.ring(8), 5, 4, 4.0), (wl.ring(6), 4, 5, 2.0),
                                        (wl.rect_periodic(3, 3), 5, 6, 7.0)])
def test_t0_is_U_times_min_double_occupancy(cl, nu, nd, U):
    cl0 = wl.Cluster(cl.name + "_t0", cl.L, cl.bonds, tuple(0.0 for _ in cl.t))
    if math.comb(cl.L, nu) * math.comb(cl.L, nd) <= 6000:
        e = ground_dense(cl0, U, nu, nd)
    else:
        e = ground_lanczos(cl0, U, nu, nd).E0
    assert abs(e - U * max(0, nu + nd - cl.L)) < 1e-12


def test_spin_flip_symmetry():
    cl = wl.ring(8)
    assert abs(ground_dense(cl, 3.0, 5, 3) - ground_dense(cl, 3.0, 3, 5)) < 1e-12


def test_monotone_in_U():
    """dE0/dU = <double occupancy> >= 0 (Hellmann-Feynman), so E0 is non-decreasing in U."""
    cl = wl.ring(8)
    es = [ground_dense(cl, U, 4, 4) for U in (0.0, 1.0, 2.0, 4.0, 8.0)]
    assert all(b >= a for a, b in zip(es, es[1:]))


def test_lanczos_full_reorth_matches_dense_ring8():
    """Ring of 8, (4,4), U=4: 100 steps with full reorthogonalisation vs dense eigh."""
    cl = wl.ring(8)
    ed = ground_dense(cl, 4.0, 4, 4)
    r = ground_lanczos(cl, 4.0, 4, 4, maxit=100, reorth=True, tol=None)
    assert r.iterations == 100
    assert abs(r.E0 - ed) < 1e-10 * max(1, abs(ed))
    # Ritz values of the lowest pair never increase
    th = np.array(r.thetas)
    assert np.all(np.diff(th) <= 1e-12)
    # every Ritz value lies in the spectrum's range (Cauchy interlacing)
    assert th[-1] >= ed - 1e-12


def test_lanczos_stops_at_tolerance():
    cl = wl.ring(8)
    ed = ground_dense(cl, 4.0, 4, 4)
    r = ground_lanczos(cl, 4.0, 4, 4, maxit=400, reorth=False, tol=1e-10)
    assert r.converged and r.iterations < 400
    assert abs(r.E0 - ed) <= 1e-10 * max(1, abs(ed))


def test_splitmix64_published_outputs():
    """First outputs of SplitMix64 seeded with 0 (reference implementation's known sequence)."""
    assert splitmix64_stream(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_start_vector_range_and_determinism():
    v = start_vector(11, 10000)
    assert v.min() >= -1.0 and v.max() < 1.0
    assert np.array_equal(v, start_vector(11, 10000))
    assert abs(v.mean()) < 0.05
    # element i is output i+1 of the stream
    z = splitmix64_stream(11, 5)
    assert np.array_equal(v[:5], np.array([(q >> 11) * 2.0 ** -52 - 1.0 for q in z]))
