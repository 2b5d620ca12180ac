"""Inversion-symmetric maps (Sec. IV B) pinned to orbit counting and brute force."""
from math import comb

import pytest

from oracle import inversion as V


def palindromes(N, n):
    if N % 2 == 0:
        return comb(N // 2, n // 2) if n % 2 == 0 else 0
    return comb((N - 1) // 2, n // 2)


@pytest.mark.parametrize("N", range(1, 15))
def test_counts_are_orbit_numbers(N):
    """S_N^n = (C(N,n) + number of palindromes) / 2, the number of orbits of the inversion."""
    for n in range(N + 1):
        assert V.S(N, n) == (comb(N, n) + palindromes(N, n)) // 2
        assert V.S(N, n) == len(V.representatives(N, n))


@pytest.mark.parametrize("N", range(2, 13))
def test_maps_biject_representatives(N):
    for n in range(N + 1):
        reps = V.representatives(N, n)
        idx = [V.forward_map(s, N, n) for s in reps]
        assert sorted(idx) == list(range(len(reps)))
        for s, i in zip(reps, idx):
            assert V.backward_map(i, N, n) == s
            assert V.forward_map(V.reverse(s, N), N, n) == i  # both members of an orbit share the index


def test_tree_order_a_before_b_before_c():
    """At depth 0 the class-A leaf comes first, then the B subtree, then the C subtree."""
    N, n = 8, 4
    for s in V.representatives(N, n):
        i = V.forward_map(s, N, n)
        hi, lo = (s >> (N - 1)) & 1, s & 1
        a, b = V.C(N - 2, n - 1), V.S(N - 2, n)
        if (hi, lo) == (0, 1):
            assert i < a
        elif (hi, lo) == (0, 0):
            assert a <= i < a + b
        else:
            assert a + b <= i
