"""GPU parity of the matrix-free H·v against the oracle.

Tolerances: float64 vectors, normwise |y - y_ref|_inf <= 1e-12 |y_ref|_inf (the
1e-12 relative bar) and, per element, <= 64 eps64 * sum_c |H_rc x_c| (the
rounding bound of a sum of at most 1 + 2 n_bonds products).  float32 vectors:
per element <= 64 eps32 * sum_c |H_rc x_c| against the float64 oracle applied to
the same (float32-rounded) input.
"""
import json
import os

import numpy as np
import pytest

import workloads as wl
from oracle.basis import Basis
from oracle.hamiltonian import KronOperator, Model, apply, row
from oracle.lanczos import start_vector
from tests.conftest import GOLDEN
from tests.gpu_util import handle_for, need_gpu

pytestmark = pytest.mark.gpu
EPS64 = np.finfo(np.float64).eps
EPS32 = np.finfo(np.float32).eps


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    import paper_1707_03974_gb300 as pd
    return torch, pd


def abs_bound(m, b, x):
    """sum_c |H_rc x_c| for every row (the |H| |x| product), from the oracle."""
    return KronOperator(m, backend="numpy").abs_apply(x)


CASES = [(wl.ring(8), 4, 4, 4.0), (wl.ring(8), 3, 5, 1.0), (wl.ring(6), 2, 3, 2.5), (wl.dimer(), 1, 1, 4.0),
         (wl.rect_periodic(4, 3), 5, 3, 7.5), (wl.rect_periodic(3, 3, 1.0, -0.3), 4, 5, 8.0),
         (wl.ring(12), 6, 6, 3.0), (wl.ring(10), 0, 5, 2.0), (wl.ring(10), 10, 3, 2.0), (wl.ring(7), 7, 7, 5.0)]


@pytest.mark.parametrize("cl,nu,nd,U", CASES)
def test_hv_f64_matches_oracle(env, cl, nu, nd, U):
    torch, pd = env
    m = Model.from_cluster(cl, U, nu, nd)
    b = Basis(cl.L, nu, nd)
    x = start_vector(7, b.D)
    yr = apply(m, b, x)
    h = handle_for(cl, U, nu, nd)
    y = pd.hubbard_apply(h, torch.from_numpy(x).cuda()).cpu().numpy()
    err = np.abs(y - yr)
    assert err.max() <= 1e-12 * max(np.abs(yr).max(), 1e-300)
    assert np.all(err <= 64 * EPS64 * abs_bound(m, b, x) + 1e-300)
    h.close()


@pytest.mark.parametrize("cl,nu,nd,U", CASES)
def test_hv_f32_matches_oracle(env, cl, nu, nd, U):
    torch, pd = env
    m = Model.from_cluster(cl, U, nu, nd)
    b = Basis(cl.L, nu, nd)
    x32 = start_vector(8, b.D).astype(np.float32)
    x = x32.astype(np.float64)
    yr = apply(m, b, x)
    h = handle_for(cl, U, nu, nd)
    bound = 64 * EPS32 * abs_bound(m, b, x) + 1e-30
    y = pd.hubbard_apply(h, torch.from_numpy(x32).cuda()).cpu().numpy().astype(np.float64)
    assert np.all(np.abs(y - yr) <= bound)
    # split form (float32 row pass on the warp-blocked table, where the handle has one)
    for rows in (1, 2, 4):
        pd.hubbard_set_hv_config(h, torch.float32, rows, 256, 1, split=1)
        y = pd.hubbard_apply(h, torch.from_numpy(x32).cuda()).cpu().numpy().astype(np.float64)
        assert np.all(np.abs(y - yr) <= bound), rows
    h.close()


def test_hv_no_bonds_is_diagonal(env):
    torch, pd = env
    cl = wl.Cluster("isolated6", 6, (), ())
    b = Basis(6, 3, 2)
    x = start_vector(9, b.D)
    h = pd.Handle(6, [], [], 3.0, 3, 2)
    y = pd.hubbard_apply(h, torch.from_numpy(x).cuda()).cpu().numpy()
    up, dn = b.split(b.combined)
    docc = np.array([bin(int(u) & int(d)).count("1") for u, d in zip(up, dn)])
    assert np.array_equal(y, 3.0 * docc * x)
    h.close()


def test_hv_rejects_aliasing_and_bad_sizes(env):
    torch, pd = env
    cl = wl.ring(6)
    h = handle_for(cl, 1.0, 3, 3)
    x = torch.zeros(h.D, dtype=torch.float64, device="cuda")
    with pytest.raises(pd.HubbardError):
        pd.hubbard_apply(h, x, x)
    with pytest.raises(ValueError):
        pd.hubbard_apply(h, torch.zeros(h.D + 1, dtype=torch.float64, device="cuda"))
    h.close()


def test_hv_hermitian_property(env):
    """<x, H z> == <H x, z> on a mid-size cluster, on the GPU alone."""
    torch, pd = env
    cl = wl.rect_periodic(4, 3)
    h = handle_for(cl, 5.0, 6, 5)
    x = torch.from_numpy(start_vector(1, h.D)).cuda()
    z = torch.from_numpy(start_vector(2, h.D)).cuda()
    lhs = torch.dot(x, pd.hubbard_apply(h, z)).item()
    rhs = torch.dot(pd.hubbard_apply(h, x), z).item()
    assert abs(lhs - rhs) <= 1e-12 * x.norm().item() * z.norm().item() * 60
    h.close()


@pytest.fixture(scope="module")
def square4x4():
    cl = wl.square_periodic(4, 1.0, -0.3)
    return cl, Model.from_cluster(cl, 8.0, 8, 8), Basis(16, 8, 8)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_hv_square4x4_full_size_sampled(env, square4x4, dtype):
    """D = 165,636,900 in the benchmark's launch configuration: sampled outputs vs oracle rows."""
    torch, pd = env
    cl, m, b = square4x4
    x = start_vector(0, b.D)
    if dtype == "f32":
        x = x.astype(np.float32).astype(np.float64)
    h = handle_for(cl, 8.0, 8, 8)
    xt = torch.from_numpy(x).cuda()
    if dtype == "f32":
        xt = xt.float()
    y = pd.hubbard_apply(h, xt)
    rng = np.random.default_rng(3)
    rows = np.unique(np.concatenate([[0, 1, b.D - 1, b.D - 2, 12869, 12870], rng.integers(0, b.D, 400)]))
    ys = y[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    for r, yv in zip(rows, ys):
        c, v = row(m, b, int(r))
        ref = float(np.dot(v, x[c]))
        bound = float(np.dot(np.abs(v), np.abs(x[c])))
        eps = EPS64 if dtype == "f64" else EPS32
        assert abs(yv - ref) <= 64 * eps * bound, (r, yv, ref)
    h.close()


def test_hv_square4x4_full_vector_vs_tensor_product_oracle(env, square4x4):
    """Whole-vector comparison at full size against the oracle's tensor-product operator."""
    torch, pd = env
    cl, m, b = square4x4
    k = KronOperator(m)
    x = start_vector(5, k.D)
    yr = k(x)
    h = handle_for(cl, 8.0, 8, 8)
    y = pd.hubbard_apply(h, torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.max(np.abs(y - yr)) <= 1e-12 * np.max(np.abs(yr))
    h.close()


# The split launch configuration the autotuner picks for fixed-point vectors on
# the 4x4 benchmark workload (and which bench.py then times).
BENCH_SPLIT_FX = {"rows_per_cta": 2, "threads_per_cta": 1024, "visit_order": 0, "split": 1, "up_block": 128,
                  "up_threads": 512, "up_rows": 4}
BENCH_SPLIT_F32 = {"rows_per_cta": 4, "threads_per_cta": 1024, "visit_order": 0, "split": 1, "up_block": 128,
                   "up_threads": 512, "up_rows": 4}


@pytest.mark.parametrize("dtype", ["fx64", "f32"])
def test_hv_square4x4_bench_split_config_full_vector(env, square4x4, dtype):
    """D = 165,636,900, the split H·v in the configuration the benchmark runs
    (and in whatever the autotuner picks on this GPU): every element of y
    against the oracle's tensor-product operator (C helper) applied to the same
    input, within the rounding bound of each vector type."""
    torch, pd = env
    cl, m, b = square4x4
    k = KronOperator(m)
    assert k._lib is not None
    h = handle_for(cl, 8.0, 8, 8)
    x = start_vector(9, b.D)
    xt = torch.from_numpy(x).cuda()
    if dtype == "fx64":
        F = pd.hubbard_fixed_point_bits(h)
        xin = pd.hubbard_convert(h, xt, torch.int64)
        xref = np.ldexp(xin.cpu().numpy().astype(np.float64), -F)
        tdt, cfg = torch.int64, BENCH_SPLIT_FX
    else:
        xin = xt.float()
        xref = xin.cpu().numpy().astype(np.float64)
        tdt, cfg = torch.float32, BENCH_SPLIT_F32
    del xt
    yr = k(xref)
    habs = k.abs_apply(xref)
    n_classes = len(set(cl.t))
    bound = (n_classes + 2) * 2.0 ** -F + 64 * EPS64 * habs if dtype == "fx64" else 64 * EPS32 * habs + 1e-30
    del habs
    y = torch.empty_like(xin)
    tuned = pd.hubbard_autotune(h, xin, y, reps=1)
    configs = [cfg] + ([tuned] if tuned.get("split") else [])
    for c in configs:
        pd.hubbard_set_hv_config(h, tdt, **{key: c[key] for key in BENCH_SPLIT_FX})
        pd.hubbard_apply(h, xin, y)
        if dtype == "fx64":
            yd = np.ldexp(y.cpu().numpy().astype(np.float64), -F)
        else:
            yd = y.cpu().numpy().astype(np.float64)
        bad = np.count_nonzero(np.abs(yd - yr) > bound)
        assert bad == 0, (c, bad)
        del yd
    assert pd.hubbard_last_error(h) == "HB_OK"
    h.close()


# ---------------------------------------------------------------- fixed point (HB_FX64)

FX_CASES = [(wl.ring(8), 4, 4, 4.0), (wl.rect_periodic(4, 3), 5, 3, 7.5), (wl.rect_periodic(3, 3, 1.0, -0.3), 4, 5, 8.0),
            (wl.ring(12), 6, 6, 3.0), (wl.ring(10), 0, 5, 2.0), (wl.dimer(), 1, 1, 4.0), (wl.tilted_18(), 2, 2, 6.0)]


@pytest.mark.parametrize("cl,nu,nd,U", FX_CASES)
def test_hv_fx64_matches_oracle(env, cl, nu, nd, U):
    """Fixed-point H·v: exact integer hop sums, one rounding per amplitude class and for U docc."""
    torch, pd = env
    m = Model.from_cluster(cl, U, nu, nd)
    b = Basis(cl.L, nu, nd)
    h = handle_for(cl, U, nu, nd)
    F = pd.hubbard_fixed_point_bits(h)
    assert 20 <= F <= 60
    x = start_vector(11, b.D)                      # |x| < 1
    xt = torch.from_numpy(x).cuda()
    q = pd.hubbard_convert(h, xt, torch.int64)
    assert torch.equal(q.cpu(), torch.from_numpy(np.rint(np.ldexp(x, F)).astype(np.int64)))
    xq = np.ldexp(q.cpu().numpy().astype(np.float64), -F)   # the input the fixed-point kernel sees
    yq = pd.hubbard_apply(h, q)
    y = pd.hubbard_convert(h, yq, torch.float64).cpu().numpy()
    yr = apply(m, b, xq)
    n_classes = len(set(cl.t))
    err = np.abs(y - yr)
    assert err.max() <= 1e-12 * max(np.abs(yr).max(), 1e-300)
    assert np.all(err <= (n_classes + 2) * 2.0 ** -F + 64 * EPS64 * abs_bound(m, b, xq))
    h.close()


def test_hv_fx64_square4x4_full_size_sampled(env, square4x4):
    torch, pd = env
    cl, m, b = square4x4
    h = handle_for(cl, 8.0, 8, 8)
    F = pd.hubbard_fixed_point_bits(h)
    x = start_vector(0, b.D)
    q = pd.hubbard_convert(h, torch.from_numpy(x).cuda(), torch.int64)
    yq = pd.hubbard_apply(h, q)
    rng = np.random.default_rng(4)
    rows = np.unique(np.concatenate([[0, 1, b.D - 1, 12869, 12870], rng.integers(0, b.D, 300)]))
    idx = torch.from_numpy(rows).cuda()
    ys = np.ldexp(yq[idx].cpu().numpy().astype(np.float64), -F)
    xq_all = q.cpu().numpy()
    for r, yv in zip(rows, ys):
        c, v = row(m, b, int(r))
        xc = np.ldexp(xq_all[c].astype(np.float64), -F)
        ref = float(np.dot(v, xc))
        assert abs(yv - ref) <= 4 * 2.0 ** -F + 64 * EPS64 * float(np.dot(np.abs(v), np.abs(xc))), (r, yv, ref)
    h.close()


def test_fx64_rejected_for_too_many_amplitudes(env):
    torch, pd = env
    cl = wl.ring(6)
    h = pd.Handle(6, cl.bonds, [1.0, 1.1, 1.2, 1.3, 1.4, 1.5], 1.0, 3, 3)
    q = torch.zeros(h.D, dtype=torch.int64, device="cuda")
    with pytest.raises(pd.HubbardError):
        pd.hubbard_apply(h, q)
    # the float paths still work
    pd.hubbard_apply(h, torch.zeros(h.D, dtype=torch.float64, device="cuda"))
    h.close()


def _many_amplitudes(L, classes):
    """Ring of L sites plus next-nearest bonds, amplitudes cycling through `classes` values."""
    pairs = [(i, (i + 1) % L) for i in range(L)] + [(i, (i + 2) % L) for i in range(0, L, 2)]
    t = tuple(classes[k % len(classes)] for k in range(len(pairs)))
    return wl.Cluster(f"ring{L}_{len(classes)}amp", L, tuple(pairs), t)


@pytest.mark.parametrize("L,classes,nu,nd,U", [(9, (1.0, 0.6, -0.25), 4, 3, 3.0),
                                               (10, (1.0, 0.7, -0.3, 0.45), 5, 4, 6.0)])
def test_hv_split_many_amplitudes(env, L, classes, nu, nd, U):
    """Split H·v with 3 and 4 amplitude classes (6 and 8 segments per warp block of the
    warp-blocked table), fixed point and float32, every row-group size, against the oracle."""
    torch, pd = env
    cl = _many_amplitudes(L, classes)
    m = Model.from_cluster(cl, U, nu, nd)
    b = Basis(cl.L, nu, nd)
    h = handle_for(cl, U, nu, nd)
    F = pd.hubbard_fixed_point_bits(h)
    x = start_vector(21, b.D)
    q = pd.hubbard_convert(h, torch.from_numpy(x).cuda(), torch.int64)
    xq = np.ldexp(q.cpu().numpy().astype(np.float64), -F)
    yr = apply(m, b, xq)
    bound = (len(classes) + 2) * 2.0 ** -F + 64 * EPS64 * abs_bound(m, b, xq)
    for rows in (1, 2):
        for order in (0, 1):
            pd.hubbard_set_hv_config(h, torch.int64, rows, 256, order, split=1, up_block=64, up_threads=256, up_rows=2)
            y = pd.hubbard_convert(h, pd.hubbard_apply(h, q), torch.float64).cpu().numpy()
            assert np.all(np.abs(y - yr) <= bound), (rows, order)
    x32 = x.astype(np.float32)
    yr32 = apply(m, b, x32.astype(np.float64))
    bound32 = 64 * EPS32 * abs_bound(m, b, x32.astype(np.float64)) + 1e-30
    for rows in (1, 2, 4):
        pd.hubbard_set_hv_config(h, torch.float32, rows, 512, 1, split=1)
        y = pd.hubbard_apply(h, torch.from_numpy(x32).cuda()).cpu().numpy().astype(np.float64)
        assert np.all(np.abs(y - yr32) <= bound32), rows
    assert pd.hubbard_last_error(h) == "HB_OK"
    h.close()
