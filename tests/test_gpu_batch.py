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
