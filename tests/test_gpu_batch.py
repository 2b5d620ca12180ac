"""Batched problems: 64 twelve-site instances (ring or 3x4, N_sigma in 3..6, U in [0,12))."""
import json
import os

import numpy as np
import pytest

import workloads as wl
from oracle.lanczos import start_vector
from tests.conftest import GOLDEN
from tests.gpu_util import handle_for, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    torch = need_gpu()
    import paper_1707_03974_gb300 as pd
    insts = wl.draw_batch_instances(64)
    hs = [handle_for(i.cluster, i.U, i.N_up, i.N_dn) for i in insts]
    b = pd.Batch(hs)
    yield torch, pd, insts, hs, b
    b.close()
    for h in hs:
        h.close()


def gold():
    return json.load(open(os.path.join(GOLDEN, "oracle_energies.json")))["batch64"]


@pytest.mark.parametrize("dtype_name", ["float64", "float32", "int64"])
def test_batch_apply_equals_single_applies(batch, dtype_name):
    torch, pd, insts, hs, b = batch
    dt = getattr(torch, dtype_name)
    x = torch.zeros(b.total, dtype=dt, device="cuda")
    for k, h in enumerate(hs):
        v = torch.from_numpy(start_vector(100 + k, h.D)).cuda()
        b.view(x, k).copy_(pd.hubbard_convert(h, v, torch.int64) if dtype_name == "int64" else v.to(dt))
    y = pd.hubbard_batch_apply(b, x)
    for k, h in enumerate(hs):
        ref = pd.hubbard_apply(h, b.view(x, k).contiguous())
        assert torch.equal(b.view(y, k), ref), k


@pytest.mark.parametrize("shape", [(64, 4, 2), (128, 2, 2), (32, 8, 1), (256, 1, 4)])
def test_batch_split_form_equals_single_applies(batch, shape):
    """The split batched H·v (row pass on each instance's warp-blocked table, then the
    column-blocked spin-up pass) gives the same integers as each instance's own H·v."""
    torch, pd, insts, hs, b = batch
    x = torch.zeros(b.total, dtype=torch.int64, device="cuda")
    for k, h in enumerate(hs):
        v = torch.from_numpy(start_vector(300 + k, h.D)).cuda()
        b.view(x, k).copy_(pd.hubbard_convert(h, v, torch.int64))
    pd.hubbard_batch_set_config(b, split=1, rows_per_cta=2, threads_per_cta=256, up_block=shape[0],
                                up_threads=shape[0] * shape[1], up_rows=shape[2])
    y = pd.hubbard_batch_apply(b, x)
    for k, h in enumerate(hs):
        assert torch.equal(b.view(y, k), pd.hubbard_apply(h, b.view(x, k).contiguous())), k


def test_batch_autotune_keeps_results(batch):
    torch, pd, insts, hs, b = batch
    x = torch.zeros(b.total, dtype=torch.float64, device="cuda")
    for k, h in enumerate(hs):
        b.view(x, k).copy_(torch.from_numpy(start_vector(200 + k, h.D)).cuda())
    ref = pd.hubbard_batch_apply(b, x)
    y = torch.empty_like(x)
    best = pd.hubbard_batch_autotune(b, x, y, reps=2)
    assert best["ms"] > 0 and best["rows_per_cta"] in (1, 2, 4)
    assert torch.equal(pd.hubbard_batch_apply(b, x), ref)


@pytest.mark.parametrize("dtype_name", ["int64", "float64"])
def test_batch_lanczos_matches_oracle(batch, dtype_name):
    torch, pd, insts, hs, b = batch
    E0, infos, status = pd.lanczos_batch_ground_state(b, maxit=1500, tol=1e-10, dtype=getattr(torch, dtype_name),
                                                      seed=0, check_every=10)
    assert status == "HB_OK"
    g = gold()
    for k in range(64):
        assert infos[k]["converged"]
        assert abs(E0[k] - g[k]["E0"]) <= 1e-10 * max(1.0, abs(g[k]["E0"])), (k, E0[k], g[k]["E0"])


def test_batch_lanczos_split_form_matches_oracle(batch):
    """The persistent batched solve with the split H·v (row-pass phase, grid barrier, spin-up phase
    whose hook forms w = H v - beta vprev and <w, v>): all 64 E0 within 1e-10 of the oracle."""
    torch, pd, insts, hs, b = batch
    pd.hubbard_batch_set_config(b, split=1, rows_per_cta=2, threads_per_cta=256, up_block=128, up_threads=256,
                                up_rows=2)
    try:
        E0, infos, status = pd.lanczos_batch_ground_state(b, maxit=1500, tol=1e-10, dtype=torch.int64, seed=0,
                                                          check_every=10)
    finally:
        pd.hubbard_batch_set_config(b, split=0, rows_per_cta=2, threads_per_cta=256)
    assert status == "HB_OK"
    g = gold()
    for k in range(64):
        assert infos[k]["converged"]
        assert abs(E0[k] - g[k]["E0"]) <= 1e-10 * max(1.0, abs(g[k]["E0"])), (k, E0[k], g[k]["E0"])


def test_batch_lanczos_uneven_subset_and_iteration_counts(batch):
    """A batch of four very uneven instances (the smallest and largest of the draw, rings and 3x4):
    every E0 within 1e-10 of the oracle, each instance stopping at its own iteration count."""
    torch, pd, insts, hs, b = batch
    g = gold()
    D = [h.D for h in hs]
    pick = sorted({int(np.argmin(D)), int(np.argmax(D)), 0, 63})
    sub = pd.Batch([hs[k] for k in pick])
    E0, infos, status = pd.lanczos_batch_ground_state(sub, maxit=1500, tol=1e-10, dtype=torch.int64, seed=0,
                                                      check_every=7)
    assert status == "HB_OK"
    for i, k in enumerate(pick):
        assert infos[i]["converged"]
        assert infos[i]["iterations"] % 7 == 0 or infos[i]["iterations"] >= hs[k].D
        assert abs(E0[i] - g[k]["E0"]) <= 1e-10 * max(1.0, abs(g[k]["E0"])), (k, E0[i], g[k]["E0"])
    sub.close()


def test_batch_lanczos_maxit_reports_not_converged(batch):
    torch, pd, insts, hs, b = batch
    E0, infos, status = pd.lanczos_batch_ground_state(b, maxit=5, tol=1e-10, dtype=torch.int64, seed=0,
                                                      check_every=10)
    assert status == "HB_ERR_NOT_CONVERGED"
    assert all(i["iterations"] == 5 and not i["converged"] for i in infos)
    g = gold()
    assert all(e >= gk["E0"] - 1e-9 for e, gk in zip(E0, g))  # Ritz values bound E0 from above


@pytest.mark.parametrize("withhold", [0, 5])
def test_batch_grid_wait_gives_up(batch, withhold):
    """A CTA that never arrives at the grid barrier: the other CTAs' waits give up after 50 ms and the
    solve reports HB_ERR_TIMEOUT instead of hanging; the batch solves correctly right after."""
    torch, pd, insts, hs, b = batch
    assert pd.lanczos_batch_wait_selftest(b, withhold_cta=withhold, limit_ms=50) == "HB_ERR_TIMEOUT"
    E0, infos, status = pd.lanczos_batch_ground_state(b, maxit=1500, tol=1e-10, dtype=torch.int64, seed=0,
                                                      check_every=10)
    assert status == "HB_OK"
    g = gold()
    assert max(abs(e - gk["E0"]) / max(1.0, abs(gk["E0"])) for e, gk in zip(E0, g)) <= 1e-10
