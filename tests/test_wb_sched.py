"""Slot schedule of the warp-blocked spin-down table (host C++, pd_wb_sched.h), on the CPU.

The row pass of the split H·v reads, per slot, one shared-memory element per
lane; a slot costs as many wavefronts as the most used bank group among the
lanes served together (8 lanes over t % 8 for 16-byte elements, 32 lanes over
t % 32 for 4-byte elements).  The schedule may only permute each lane's hops
among that lane's slots (the sums are exact integers, or float32 sums in the
table's fixed order).  Checked here: every lane keeps exactly its hops; the
cost never drops below the lower bound max(slots, most hops on one group) of
each lane set; and the cost falls well below the natural order's.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1707_03974_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("wb") / "wb_sched_driver")
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, os.path.join(HERE, "wb_sched_driver.cpp"), "-o", exe],
                   check=True)
    return exe


def run(driver, layout, grids):
    NL, G = layout
    lines = [f"{NL} {G} {len(grids)}"]
    for g in grids:
        lines.append(f"{g.shape[1]} " + " ".join(str(int(v)) for v in g.reshape(-1)))
    out = subprocess.run([driver], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True).stdout
    res = []
    for line, g in zip(out.strip().splitlines(), grids):
        vals = np.array(line.split(), dtype=np.int64)
        assert vals[0] == g.shape[1]
        res.append(vals[1:].reshape(32, g.shape[1]))
    assert len(res) == len(grids)
    return res


def cost(g, layout):
    NL, G = layout
    total = 0
    for l0 in range(0, 32, NL):
        for s in range(g.shape[1]):
            t = g[l0:l0 + NL, s]
            t = t[t >= 0]
            total += max(1, np.bincount(t % G, minlength=G).max()) if len(t) else 1
    return total


def lower_bound(g, layout):
    NL, G = layout
    total = 0
    for l0 in range(0, 32, NL):
        t = g[l0:l0 + NL].reshape(-1)
        t = t[t >= 0]
        most = np.bincount(t % G, minlength=G).max() if len(t) else 0
        total += max(g.shape[1], most)
    return total


def random_grids(seed, n, D=20000):
    rng = np.random.default_rng(seed)
    grids = []
    for k in range(n):
        S = int(rng.choice([2, 4, 6, 8, 12]))
        g = -np.ones((32, S), dtype=np.int64)
        live = 32 if k % 5 else int(rng.integers(1, 32))  # a ragged last warp block
        for lane in range(live):
            kk = int(rng.integers(S // 2, S + 1))
            g[lane, :kk] = rng.integers(0, D, kk)
        grids.append(g)
    return grids


@pytest.mark.parametrize("layout", [(8, 8), (32, 32)])
def test_schedule_keeps_every_lanes_hops(driver, layout):
    grids = random_grids(1, 60)
    out = run(driver, layout, grids)
    for g, h in zip(grids, out):
        for lane in range(32):
            assert sorted(g[lane].tolist()) == sorted(h[lane].tolist()), lane


@pytest.mark.parametrize("layout,gain", [((8, 8), 0.80), ((32, 32), 0.75)])
def test_schedule_cost_between_bound_and_natural(driver, layout, gain):
    grids = random_grids(2, 200)
    out = run(driver, layout, grids)
    natural = sum(cost(g, layout) for g in grids)
    after = sum(cost(h, layout) for h in out)
    bound = sum(lower_bound(g, layout) for g in grids)
    assert all(cost(h, layout) >= lower_bound(g, layout) for g, h in zip(grids, out))
    assert after <= gain * natural, (after, natural, bound)
    assert after <= 1.05 * bound, (after, natural, bound)


def test_conflict_free_instance_reaches_the_bound(driver):
    """Eight lanes whose hops can be arranged with one lane per bank group in every slot
    (a Latin square, shuffled within each lane): the schedule finds a conflict-free order."""
    rng = np.random.default_rng(3)
    S = 8
    g = -np.ones((32, S), dtype=np.int64)
    for lane in range(32):
        q = lane // 8
        groups = [(lane % 8 + s) % 8 for s in range(S)]
        vals = [8 * int(rng.integers(0, 500)) + gr + 4096 * q for gr in groups]
        rng.shuffle(vals)
        g[lane] = vals
    h = run(driver, (8, 8), [g])[0]
    assert cost(h, (8, 8)) == lower_bound(g, (8, 8)) == 4 * S
