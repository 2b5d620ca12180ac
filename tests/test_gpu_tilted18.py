"""18-site tilted cluster at half filling (D = 2,363,904,400): sampled-row parity at full size.

The oracle cannot list this basis; it evaluates single rows with the counting
definition of the sorted order (`row_by_counting`).  Inputs are random vectors
drawn on the GPU; only the entries a sampled row needs are copied back.
"""
import numpy as np
import pytest

import workloads as wl
from oracle.hamiltonian import Model, row_by_counting
from tests.gpu_util import handle_for, need_gpu

pytestmark = pytest.mark.gpu
EPS64 = np.finfo(np.float64).eps
EPS32 = np.finfo(np.float32).eps
U = 6.0


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    import paper_1707_03974_gb300 as pd
    cl = wl.tilted_18()
    h = handle_for(cl, U, 9, 9)
    assert h.D == 2363904400
    yield torch, pd, cl, h
    h.close()
    torch.cuda.empty_cache()


def sampled_rows(D, n, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, 1, 48619, 48620, D - 1], rng.integers(0, D, n)]))


@pytest.mark.parametrize("dtype_name", ["float32", "int64"])
def test_hv_tilted18_sampled_rows(env, dtype_name):
    torch, pd, cl, h = env
    m = Model.from_cluster(cl, U, 9, 9)
    g = torch.Generator(device="cuda")
    g.manual_seed(18)
    x = torch.empty(h.D, dtype=torch.float32, device="cuda")
    x.uniform_(-1.0, 1.0, generator=g)
    if dtype_name == "int64":
        F = pd.hubbard_fixed_point_bits(h)
        xin = pd.hubbard_convert(h, x.double(), torch.int64)
        del x
        y = pd.hubbard_apply(h, xin)
        scale = 2.0 ** -F
    else:
        xin = x
        y = pd.hubbard_apply(h, xin)
        scale = 1.0
    rows = sampled_rows(h.D, 120, 3)
    ys = y[torch.from_numpy(rows).cuda()].double().cpu().numpy() * scale
    for r, yv in zip(rows, ys):
        c, v = row_by_counting(m, int(r))
        xc = xin[torch.from_numpy(c).cuda()].double().cpu().numpy() * scale
        ref = float(np.dot(v, xc))
        bound = float(np.dot(np.abs(v), np.abs(xc)))
        tol = 64 * EPS32 * bound if dtype_name == "float32" else 4 * scale + 64 * EPS64 * bound
        assert abs(yv - ref) <= tol, (r, yv, ref)
    del xin, y
    torch.cuda.empty_cache()


def test_hv_tilted18_fx64_split_long_rows(env):
    """Fixed point in the split form, whose row pass gathers rows of 48,620 columns (389 KB,
    longer than shared memory) from global memory: sampled rows against the counting oracle,
    and the whole vector bit for bit against the one-kernel form."""
    torch, pd, cl, h = env
    m = Model.from_cluster(cl, U, 9, 9)
    g = torch.Generator(device="cuda")
    g.manual_seed(81)
    x = torch.empty(h.D, dtype=torch.float64, device="cuda")
    x.uniform_(-1.0, 1.0, generator=g)
    F = pd.hubbard_fixed_point_bits(h)
    xin = pd.hubbard_convert(h, x, torch.int64)
    del x
    pd.hubbard_set_hv_config(h, torch.int64, 0, 0, 1)
    ref = pd.hubbard_apply(h, xin)
    pd.hubbard_set_hv_config(h, torch.int64, 0, 0, 1, split=1, up_block=256, up_threads=1024, up_rows=2)
    y = pd.hubbard_apply(h, xin)
    assert torch.equal(y, ref)
    del ref
    scale = 2.0 ** -F
    rows = sampled_rows(h.D, 60, 5)
    ys = y[torch.from_numpy(rows).cuda()].double().cpu().numpy() * scale
    for r, yv in zip(rows, ys):
        c, v = row_by_counting(m, int(r))
        xc = xin[torch.from_numpy(c).cuda()].double().cpu().numpy() * scale
        ref_r = float(np.dot(v, xc))
        assert abs(yv - ref_r) <= 4 * scale + 64 * EPS64 * float(np.dot(np.abs(v), np.abs(xc))), (r, yv, ref_r)
    pd.hubbard_set_hv_config(h, torch.int64, 0, 0, 1)
    assert pd.hubbard_last_error(h) == "HB_OK"
    del xin, y
    torch.cuda.empty_cache()


def test_tilted18_mixed_precision_matches_fixed_point_run(env):
    """float32 Krylov vectors + fixed-point finish vs an all-fixed-point run of the same cluster:
    E0 within 1e-10 (there is no CPU oracle at this size)."""
    torch, pd, cl, h = env
    r_fx = pd.lanczos_ground_state(h, maxit=1500, tol=1e-10, seed=0, dtype=torch.int64)
    torch.cuda.empty_cache()
    r_mx = pd.lanczos_ground_state(h, maxit=1500, tol=1e-10, seed=0, dtype=torch.float32, fp64_finish="fx64")
    torch.cuda.empty_cache()
    assert r_fx.converged and r_mx.converged
    assert abs(r_mx.E0 - r_fx.E0) <= 1e-10 * abs(r_fx.E0)
    # float32-only solve: error reported scale (~1e-6 relative), not the 1e-10 target
    r_32 = pd.lanczos_ground_state(h, maxit=1500, tol=1e-6, seed=0, dtype=torch.float32)
    torch.cuda.empty_cache()
    assert abs(r_32.E0 - r_fx.E0) <= 1e-5 * abs(r_fx.E0)
