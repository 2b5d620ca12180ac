"""Inversion-symmetric Paradeisos maps by definition (oracle; test infrastructure only).

Sec. IV B of the paper: on a chain of N sites the inversion F maps site i to
N-1-i, so a string phi and its bit reversal F(phi) belong to one orbit, and the
symmetric subspace has one basis element per orbit.  Representatives and their
order come from a recursive classification of the outermost pair of still
unclassified bits (N-1-d, d) at depth d:

* class A, bits (0, 1): a leaf; the representative of its orbit (the partner
  with bits (1, 0) is not listed); the inner N-2-2d bits carry m-1 particles in
  any arrangement, ordered by the standard forward map (Eq. 3);
* class B, bits (0, 0): recurse one level deeper with the same m;
* class C, bits (1, 1): recurse one level deeper with m-2.

At every depth the A states come first, then the B subtree, then the C subtree.
The counts are C_{i-2}^{m-1} for the A leaf and S_i^m for a subtree, with
S_i^m = C_{i-2}^{m-1} + S_{i-2}^m + S_{i-2}^{m-2}.

Readings: S_0^0 = 1 (the empty middle of an even chain), S_1^0 = S_1^1 = 1 (the
middle bit of an odd chain is its own mirror image), S_i^m = 0 outside
0 <= m <= i; the forward map starts from idx = 0 (the paper's listing does not
initialise it); a string whose first unequal pair is (1, 0) is represented by
its reversal.

Pins (tests/test_oracle_inversion.py): S_N^n equals the number of orbits
(C(N,n) + palindromes) / 2; the forward map is a bijection from the
representatives onto [0, S_N^n) and the backward map its inverse; every orbit
has exactly one representative, found by brute force over all strings.
"""
from __future__ import annotations

from math import comb


def reverse(s: int, N: int) -> int:
    r = 0
    for i in range(N):
        if (s >> i) & 1:
            r |= 1 << (N - 1 - i)
    return r


def C(i: int, m: int) -> int:
    return comb(i, m) if 0 <= m <= i else 0


def S(i: int, m: int) -> int:
    """Number of representatives with i unclassified bits and m particles (the recursion above)."""
    if m < 0 or m > i:
        return 0
    if i == 0:
        return 1 if m == 0 else 0
    if i == 1:
        return 1
    return C(i - 2, m - 1) + S(i - 2, m) + S(i - 2, m - 2)


def representative(s: int, N: int) -> int:
    """The member of the orbit {s, F(s)} that the classification lists."""
    for d in range(N // 2):
        hi, lo = (s >> (N - 1 - d)) & 1, (s >> d) & 1
        if hi != lo:
            return s if (hi, lo) == (0, 1) else reverse(s, N)
    return s  # a palindrome


def forward_rank(s: int, n_bits: int) -> int:
    """Standard forward map (Eq. 3) of an n_bits-bit string."""
    idx, m = 0, 0
    for j in range(n_bits):
        if (s >> j) & 1:
            m += 1
            idx += C(j, m)
    return idx


def backward_rank(p: int, m: int, n_bits: int) -> int:
    s = 0
    for i in range(n_bits - 1, -1, -1):
        if m > 0 and p >= C(i, m):
            s |= 1 << i
            p -= C(i, m)
            m -= 1
    return s


def forward_map(s: int, N: int, n: int) -> int:
    """Index of the orbit of s in the symmetric subspace (tree order)."""
    s = representative(s, N)
    idx, m = 0, n
    for d in range(N // 2):
        i = N - 2 * d
        hi, lo = (s >> (N - 1 - d)) & 1, (s >> d) & 1
        if (hi, lo) == (0, 1):
            inner = (s >> (d + 1)) & ((1 << (i - 2)) - 1)
            return idx + forward_rank(inner, i - 2)
        if (hi, lo) == (0, 0):
            idx += C(i - 2, m - 1)
        else:  # (1, 1)
            idx += C(i - 2, m - 1) + S(i - 2, m)
            m -= 2
    return idx


def backward_map(p: int, N: int, n: int) -> int:
    s, m = 0, n
    for d in range(N // 2):
        i = N - 2 * d
        a, b = C(i - 2, m - 1), S(i - 2, m)
        if p >= a + b:
            p -= a + b
            s |= (1 << (N - 1 - d)) | (1 << d)
            m -= 2
        elif p >= a:
            p -= a
        else:
            s |= 1 << d
            return s | (backward_rank(p, m - 1, i - 2) << (d + 1))
    if N % 2 == 1 and m == 1:
        s |= 1 << (N // 2)
    return s


def representatives(N: int, n: int) -> list:
    """All representatives, by brute force over the strings with n bits."""
    return sorted({representative(s, N) for s in range(1 << N) if bin(s).count("1") == n})
