"""C-ABI checks that need no GPU: the library loads, exports every declared symbol,
rejects bad arguments before touching the device, and its host tridiagonal solver
agrees with LAPACK."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1707_03974_gb300 as pd
from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "paradeisos.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1707_03974_gb300.build import build
    build()
    return pd.load()


def declared_functions(header=HEADER):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:hb_status|const char \*)\s*(\w+)\s*\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(pd.EXPORTED_SYMBOLS)


def test_every_mlp_symbol_is_exported(lib):
    names = declared_functions(os.path.join(ROOT, "include", "paradeisos_mlp.h"))
    assert set(names) == set(pd.MLP_SYMBOLS)
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    assert lib.hb_status_string(0) == b"HB_OK"
    assert lib.hb_status_string(8) == b"HB_ERR_TIMEOUT"


@pytest.mark.parametrize("L,bonds,nu,nd", [(0, [], 0, 0), (33, [], 1, 1), (4, [(0, 0)], 1, 1),
                                            (4, [(0, 1), (1, 0)], 1, 1), (4, [(0, 4)], 1, 1), (4, [(0, 1)], 5, 1),
                                            (4, [(0, 1)], -1, 1)])
def test_create_rejects_bad_arguments(lib, L, bonds, nu, nd):
    with pytest.raises(pd.HubbardError) as e:
        pd.Handle(L, bonds, [1.0] * len(bonds), 1.0, nu, nd)
    assert e.value.name == "HB_ERR_INVALID_ARG"


@pytest.mark.parametrize("Lx,Ly,nu,nd,Kx,Ky", [(0, 1, 1, 1, 0, 0), (1, 1, 1, 1, 0, 0), (8, 5, 1, 1, 0, 0),
                                                (4, 4, 17, 1, 0, 0), (4, 4, 1, -1, 0, 0), (4, 4, 1, 1, 4, 0),
                                                (4, 4, 1, 1, 0, -1), (6, 1, 1, 1, 0, 1)])
def test_create_k_rejects_bad_arguments(lib, Lx, Ly, nu, nd, Kx, Ky):
    """Momentum-sector handles: grid of 2 .. 32 momenta, fillings and K inside the zone."""
    with pytest.raises(pd.HubbardError) as e:
        pd.Handle.momentum(Lx, Ly, 1.0, 0.0, 1.0, nu, nd, Kx, Ky)
    assert e.value.name == "HB_ERR_INVALID_ARG"


def test_null_pointer_arguments(lib):
    assert lib.hubbard_basis_create(4, 0, None, None, 1.0, 1, 1, None) == 1
    assert lib.hubbard_basis_create_k(4, 4, 1.0, 0.0, 1.0, 1, 1, 0, 0, None) == 1
    assert lib.hubbard_basis_dim(None, None, None, None) == 1
    assert lib.hubbard_apply(None, 0, None, None, None) == 1
    assert lib.paradeisos_rank(None, None, None, 0, None) == 1


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (7, 2), (60, 3), (400, 4)])
def test_tridiag_lowest_matches_lapack(lib, n, seed):
    from scipy.linalg import eigh_tridiagonal
    rng = np.random.default_rng(seed)
    a = rng.normal(size=n) * 3
    b = np.abs(rng.normal(size=max(n - 1, 0))) + 0.1
    th, sl = pd.hb_tridiag_lowest(a, b)
    if n == 1:
        assert th == a[0] and sl == 1.0
        return
    w, v = eigh_tridiagonal(a, b, select="i", select_range=(0, 0))
    assert abs(th - w[0]) <= 1e-13 * max(1, abs(w[0]))
    assert abs(abs(sl) - abs(v[-1, 0])) <= 1e-9


def test_tridiag_lowest_lanczos_like_spectrum(lib):
    """Nearly converged Lanczos tridiagonals have tiny trailing betas and clustered Ritz values."""
    from scipy.linalg import eigh_tridiagonal
    a = np.array([-3.0, -1.0, 0.5, 2.0, -2.9999999, 1.0])
    b = np.array([0.5, 0.3, 0.2, 1e-6, 1e-9])
    th, sl = pd.hb_tridiag_lowest(a, b)
    w, v = eigh_tridiagonal(a, b, select="i", select_range=(0, 0))
    assert abs(th - w[0]) <= 1e-13 * abs(w[0])
    assert abs(abs(sl) - abs(v[-1, 0])) <= 1e-8


def test_continued_fraction_matches_oracle(lib):
    """hb_continued_fraction (host utility) against the oracle's evaluation of the same fraction."""
    from oracle import response as R
    rng = np.random.default_rng(3)
    for n in (1, 2, 7, 40):
        a = rng.normal(size=n) * 2
        b = np.abs(rng.normal(size=n - 1)) + 0.1
        z = np.linspace(-5, 5, 11) + 0.2j
        got = pd.hb_continued_fraction(a, b, 0.7, -1.3, z)
        want = R.continued_fraction(a, b, 0.7, -1.3, z)
        assert np.max(np.abs(got - want)) <= 1e-12 * max(1.0, np.max(np.abs(want)))


def test_host_alloc_argument_errors(lib):
    """The pinned-buffer entry points refuse bad arguments before touching the driver."""
    import ctypes
    p = ctypes.c_void_p()
    assert lib.hb_host_alloc(0, ctypes.byref(p)) == 1  # HB_ERR_INVALID_ARG
    assert p.value is None
    assert lib.hb_host_alloc(4096, None) == 1
    assert lib.hb_host_free(None) == 0
    x = ctypes.create_string_buffer(64)
    assert lib.hb_host_free(ctypes.cast(x, ctypes.c_void_p)) == 1  # not one of its buffers
