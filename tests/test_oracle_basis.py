"""Pins of the oracle's basis and position definitions (CPU only)."""
import json
import math
import os

import numpy as np
import pytest

from oracle.basis import Basis, count_below, next_string, position, spin_list, string_at
from tests.conftest import GOLDEN

EX = json.load(open(os.path.join(GOLDEN, "paper_examples.json")))


def test_spin_tables_match_paper():
    g = EX["spin_tables"]
    assert spin_list(g["L"], 2).tolist() == g["n2"]
    assert spin_list(g["L"], 3).tolist() == g["n3"]


def test_dimension_example():
    g = EX["dimension"]
    b = Basis(g["L"], g["N_up"], g["N_dn"])
    assert b.D == g["D"] == len(b.combined)


def test_basis_element_encoding():
    g = EX["basis_element"]
    up = sum(1 << i for i in g["up_sites"])
    dn = sum(1 << i for i in g["dn_sites"])
    assert up == int(g["up"], 2) and dn == int(g["dn"], 2)


def test_forward_map_example():
    g = EX["forward_map_example"]
    s = int(g["string"], 2)
    lst = spin_list(g["L"], g["n"])
    assert int(position(lst, s)) == g["index"]
    assert count_below(s, g["L"], g["n"]) == g["index"]


@pytest.mark.parametrize("L", range(1, 15))
def test_count_below_equals_sorted_position(L):
    for n in range(L + 1):
        lst = spin_list(L, n)
        assert len(lst) == math.comb(L, n)
        # brute force: position = number of smaller strings with the same popcount
        for p in range(0, len(lst), max(1, len(lst) // 97)):
            s = int(lst[p])
            assert count_below(s, L, n) == p
            assert string_at(p, L, n) == s


@pytest.mark.parametrize("L", range(1, 15))
def test_next_string_walks_the_sorted_list(L):
    """The bit-operation successor (Sec. II A) visits the sorted list in order."""
    for n in range(1, L + 1):
        lst = spin_list(L, n)
        for a, b in zip(lst[:-1], lst[1:]):
            assert next_string(int(a)) == int(b)
        assert next_string(int(lst[-1])) >> L  # past the last string the successor leaves L bits


@pytest.mark.parametrize("L,n", [(32, 16), (32, 1), (32, 31), (31, 9), (24, 12), (28, 5)])
def test_count_below_steps_by_one_at_large_L(L, n):
    """Above the enumerable sizes: walking with the successor, which counts
    nothing, count_below must grow by exactly one per step and string_at must
    return the walked string -- from the first string, around a random interior
    position and up to the last string."""
    D = math.comb(L, n)
    rng = np.random.default_rng(L * 100 + n)
    starts = [0, max(0, D - 1500)] + ([int(rng.integers(1500, D - 3000))] if D > 6000 else [])
    for p0 in starts:
        s = string_at(p0, L, n)
        assert count_below(s, L, n) == p0
        p = p0
        for _ in range(min(1499, D - 1 - p0)):
            s = next_string(s)
            p += 1
            assert count_below(s, L, n) == p
            assert string_at(p, L, n) == s
    assert string_at(0, L, n) == (1 << n) - 1
    assert string_at(D - 1, L, n) == ((1 << n) - 1) << (L - n)


def test_count_below_edge_sectors():
    for L in (1, 5, 20, 32):
        assert count_below(0, L, 0) == 0
        assert count_below((1 << L) - 1, L, L) == 0
        assert string_at(0, L, 0) == 0
    # last string of L=32, n=16 sits at C(32,16) - 1
    s = ((1 << 16) - 1) << 16
    assert count_below(s, 32, 16) == math.comb(32, 16) - 1
    assert string_at(math.comb(32, 16) - 1, 32, 16) == s


def test_combined_position_is_tensor_product_index():
    """Position in the sorted combined list equals C(L, n_dn) * idx_up + idx_dn (Sec. III)."""
    for (L, nu, nd) in [(4, 2, 3), (6, 3, 2), (7, 0, 4), (5, 5, 1)]:
        b = Basis(L, nu, nd)
        for iu, u in enumerate(b.up):
            for idn, d in enumerate(b.dn):
                st = (int(u) << L) | int(d)
                assert int(b.index_of(np.uint64(st))) == math.comb(L, nd) * iu + idn


def test_position_rejects_absent_values():
    lst = spin_list(6, 3)
    assert int(position(lst, np.uint64(0b1))) == -1
    assert int(position(lst, np.uint64(0b111000))) == len(lst) - 1
