"""Basis enumeration and positions by definition (oracle; test infrastructure only).

Sec. II A: a spin string of an L-site cluster is the integer whose bit i is the
occupation of site i; the per-spin basis with n particles is the list of such
integers sorted ascending (the paper's table for L=4, n=2 and n=3).  The full
basis is the tensor product, with the spin-down string in the L low bits of the
combined integer (up << L) | dn (Sec. III, combined index), so sorting combined
integers orders first by the up string, then by the down string.

Positions are found the conventional way (Sec. II C): binary search in the
stored sorted list.  For clusters too large to enumerate, ``count_below`` counts
the fixed-popcount strings below a given one directly from its definition.
"""
from __future__ import annotations

import math

import numpy as np

MAX_ENUM_L = 26


def spin_list(L: int, n: int) -> np.ndarray:
    """Sorted array (uint64) of all L-bit integers with exactly n bits set."""
    if not (0 <= n <= L):
        raise ValueError("need 0 <= n <= L")
    if L > MAX_ENUM_L:
        raise ValueError(f"L={L} too large to enumerate in the oracle")
    allv = np.arange(1 << L, dtype=np.uint64)
    pc = np.zeros(allv.shape, dtype=np.uint8)
    v = allv.copy()
    for _ in range(L):
        pc += (v & np.uint64(1)).astype(np.uint8)
        v >>= np.uint64(1)
    return allv[pc == n]


def position(sorted_list: np.ndarray, value) -> np.ndarray:
    """Index of value(s) in a sorted list by binary search; -1 where absent."""
    value = np.asarray(value, dtype=np.uint64)
    idx = np.searchsorted(sorted_list, value)
    idx_c = np.minimum(idx, len(sorted_list) - 1)
    found = (idx < len(sorted_list)) & (sorted_list[idx_c] == value)
    return np.where(found, idx, -1).astype(np.int64)


def count_below(s: int, L: int, n: int) -> int:
    """Number of L-bit strings with n bits set that are smaller than s (s must have n bits).

    Definition of the position, evaluated by counting instead of listing: a
    string t < s with the same popcount first differs from s at some bit i where
    s has 1 and t has 0, agrees above i, and places the remaining particles
    anywhere below i.  Summing those counts over the set bits of s gives the
    number of smaller strings.
    """
    if bin(s).count("1") != n or s >> L:
        raise ValueError("string has wrong popcount or bits beyond L")
    total = 0
    above = 0
    for i in range(L - 1, -1, -1):
        if (s >> i) & 1:
            remaining = n - above
            # t has 0 at i, agrees above i: it must place `remaining` particles in i positions
            total += math.comb(i, remaining)
            above += 1
    return total


def string_at(p: int, L: int, n: int) -> int:
    """Inverse of count_below: the string with exactly p smaller strings (by search).

    Walks from the top bit, deciding each bit by comparing p with the number of
    strings that have a 0 there -- the plain counting definition, no tables.
    """
    total = math.comb(L, n)
    if not (0 <= p < total):
        raise ValueError("position out of range")
    s = 0
    m = n
    for i in range(L - 1, -1, -1):
        zeros_here = math.comb(i, m)  # strings with 0 at bit i and m particles below
        if p >= zeros_here:
            s |= 1 << i
            p -= zeros_here
            m -= 1
    return s


def next_string(s: int) -> int:
    """The next larger integer with the same popcount (Sec. II A: advancing the
    position p -> p + 1 of a spin string takes a few bit operations).

    Gosper's successor (HAKMEM item 175, 1972): the lowest block of ones moves
    its top bit one place up and the rest of the block to the bottom.  Unlike
    count_below and string_at it counts nothing, so stepping with it checks
    those two independently.
    """
    if s <= 0:
        raise ValueError("need a positive string")
    low = s & -s                # lowest set bit
    ripple = s + low            # clears the lowest block of ones, sets the bit above it
    ones = ((ripple ^ s) >> 2) // low  # the block's remaining ones, shifted to bit 0
    return ripple | ones


class Basis:
    """Full tensor-product basis of an (L, N_up, N_dn) sector, stored as a sorted list."""

    def __init__(self, L: int, N_up: int, N_dn: int, store_combined: bool = True):
        self.L, self.N_up, self.N_dn = L, N_up, N_dn
        self.up = spin_list(L, N_up)
        self.dn = spin_list(L, N_dn)
        self.D_up = len(self.up)
        self.D_dn = len(self.dn)
        self.D = self.D_up * self.D_dn
        self.combined = None
        if store_combined:
            # all (up << L) | dn; sorting is by definition of the ordered list
            comb = (self.up[:, None] << np.uint64(L)) | self.dn[None, :]
            comb = comb.ravel()
            self.combined = np.sort(comb, kind="stable")

    def index_of(self, states) -> np.ndarray:
        """Position of combined integers in the sorted combined list (binary search)."""
        if self.combined is None:
            raise RuntimeError("combined list not stored")
        return position(self.combined, states)

    def state_at(self, idx) -> np.ndarray:
        if self.combined is None:
            raise RuntimeError("combined list not stored")
        return self.combined[np.asarray(idx, dtype=np.int64)]

    def split(self, states):
        states = np.asarray(states, dtype=np.uint64)
        mask = np.uint64((1 << self.L) - 1)
        return states >> np.uint64(self.L), states & mask
