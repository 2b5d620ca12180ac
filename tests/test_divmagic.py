"""Quotients by an invariant divisor (pd_divmagic.h, Granlund & Montgomery 1994) on the CPU.

The basis maps split a combined index with this quotient.  Checked against
Python's exact integer division: every divisor 1..300 with numerators at the
ends of the 64-bit range and around multiples of the divisor, powers of two
and their neighbours, the per-spin dimensions C(L, n) of every L <= 32, and
random 64-bit pairs."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1707_03974_gb300", "csrc")
MAX64 = (1 << 64) - 1


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("dm") / "divmagic_driver")
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, os.path.join(HERE, "divmagic_driver.cpp"), "-o", exe],
                   check=True)
    return exe


def quotients(driver, pairs):
    text = f"{len(pairs)}\n" + "\n".join(f"{n} {d}" for n, d in pairs) + "\n"
    out = subprocess.run([driver], input=text, capture_output=True, text=True, check=True).stdout.split()
    return [int(v) for v in out]


def check(driver, pairs):
    got = quotients(driver, pairs)
    bad = [(n, d, g) for (n, d), g in zip(pairs, got) if g != n // d]
    assert not bad, bad[:5]


def test_small_divisors_edge_numerators(driver):
    pairs = []
    for d in range(1, 301):
        for n in (0, 1, d - 1, d, d + 1, 2 * d - 1, 2 * d, MAX64, MAX64 - 1, MAX64 - d, (MAX64 // d) * d,
                  (MAX64 // d) * d - 1):
            if 0 <= n <= MAX64:
                pairs.append((n, d))
    check(driver, pairs)


def test_powers_of_two_and_neighbours(driver):
    pairs = []
    for k in range(64):
        for d in {(1 << k) - 1, 1 << k, (1 << k) + 1}:
            if 1 <= d <= MAX64:
                for n in (0, d, MAX64, MAX64 - 1, (1 << 63), (1 << 63) - 1, 12345678901234567):
                    pairs.append((n, d))
    check(driver, pairs)


def test_spin_dimensions(driver):
    rng = np.random.default_rng(7)
    pairs = []
    for L in range(1, 33):
        for n in range(L + 1):
            d = math.comb(L, n)
            top = d * d
            for x in [0, d - 1, d, top - 1, top, *rng.integers(0, 1 << 62, 6, dtype=np.uint64).tolist()]:
                pairs.append((int(x) % (MAX64 + 1), d))
    check(driver, pairs)


def test_random_pairs(driver):
    rng = np.random.default_rng(11)
    n = rng.integers(0, 1 << 63, 4000, dtype=np.uint64).astype(object) * 2 + rng.integers(0, 2, 4000).astype(object)
    bits = rng.integers(1, 64, 4000)
    d = [max(1, int(rng.integers(0, 1 << 62, dtype=np.uint64)) >> (62 - int(b)) if b < 62 else
             int(rng.integers(1, 1 << 62, dtype=np.uint64))) for b in bits]
    check(driver, [(int(a), int(b)) for a, b in zip(n, d)])
