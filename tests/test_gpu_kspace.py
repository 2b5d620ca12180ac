"""Momentum-space Paradeisos on the GPU (Sec. IV A, Eq. 4) against the momentum oracle."""
import json
import os

import numpy as np
import pytest

from oracle import momentum as M
from tests.conftest import GOLDEN
from tests.gpu_util import from_dev_u64, need_gpu, to_dev_u64

pytestmark = pytest.mark.gpu

SMALL = [(6, 1, 2, 3), (3, 3, 2, 2), (4, 4, 2, 1), (4, 2, 2, 2)]


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    import paper_1707_03974_gb300 as pd
    return torch, pd


def _sector(pd, Lx, Ly, nu, nd, K, U=4.0, tp=-0.3):
    g = M.Grid(Lx, Ly)
    tpp = 0.0 if Ly == 1 else tp
    return g, pd.Handle.momentum(Lx, Ly, 1.0, tpp, U, nu, nd, K % Lx, K // Lx), M.KModel(g, 1.0, tpp, U, nu, nd, K)


@pytest.mark.parametrize("Lx,Ly,nu,nd", SMALL)
def test_maps_bit_exact_every_sector(env, Lx, Ly, nu, nd):
    """Rank of every sector state = its position in the ascending oracle list; unrank inverts it;
    states of another sector or popcount are rejected with the sentinel."""
    torch, pd = env
    g = M.Grid(Lx, Ly)
    for K in range(g.N):
        lst = M.sector_list(g, nu, nd, K)
        if len(lst) == 0:
            with pytest.raises(pd.HubbardError):
                pd.Handle.momentum(Lx, Ly, 1.0, 0.0, 1.0, nu, nd, K % Lx, K // Lx)
            continue
        h = pd.Handle.momentum(Lx, Ly, 1.0, 0.0, 1.0, nu, nd, K % Lx, K // Lx)
        assert h.D == len(lst)
        idx = from_dev_u64(pd.paradeisos_rank(h, to_dev_u64(lst)))
        assert np.array_equal(idx, np.arange(len(lst), dtype=np.uint64))
        st = from_dev_u64(pd.paradeisos_unrank(h, to_dev_u64(np.arange(len(lst)))))
        assert np.array_equal(st, lst)
        assert pd.hubbard_last_error(h) == "HB_OK"
        other = M.sector_list(g, nu, nd, (K + 1) % g.N)
        if len(other):
            bad = from_dev_u64(pd.paradeisos_rank(h, to_dev_u64(other[:3])))
            assert np.all(bad == np.uint64(2**64 - 1))
            assert pd.hubbard_last_error(h) == "HB_ERR_INVALID_STATE"
        h.close()


@pytest.mark.parametrize("Lx,Ly,nu,nd", SMALL)
def test_rows_match_oracle(env, Lx, Ly, nu, nd):
    """Canonical rows: columns and off-diagonal values (+-U/N) bit-exact, the diagonal to rounding."""
    torch, pd = env
    g = M.Grid(Lx, Ly)
    for K in range(g.N):
        if len(M.sector_list(g, nu, nd, K)) == 0:
            continue
        _, h, mod = _sector(pd, Lx, Ly, nu, nd, K)
        lst = M.sector_list(g, nu, nd, K)
        me = 1 + nu * nd * (g.N - 1)
        cols, vals, counts = pd.hubbard_row_entries(h, 0, h.D, me)
        cols, vals, counts = cols.cpu().numpy(), vals.cpu().numpy(), counts.cpu().numpy()
        for r in range(h.D):
            c, v = M.row(mod, lst, r)
            n = counts[r]
            assert n == len(c)
            assert np.array_equal(cols[r, :n], c)
            off = c != r
            assert np.array_equal(vals[r, :n][off], v[off])
            assert abs(vals[r, :n][~off][0] - v[~off][0]) <= 1e-13 * max(1.0, abs(v[~off][0]))
        h.close()


@pytest.mark.parametrize("Lx,Ly,nu,nd", SMALL)
def test_hv_matches_oracle(env, Lx, Ly, nu, nd):
    torch, pd = env
    g = M.Grid(Lx, Ly)
    rng = np.random.default_rng(Lx * 7 + nu)
    for K in range(0, g.N, 3):
        if len(M.sector_list(g, nu, nd, K)) == 0:
            continue
        _, h, mod = _sector(pd, Lx, Ly, nu, nd, K, U=6.0)
        x = rng.uniform(-1, 1, h.D)
        ref = M.apply(mod, x)
        xd = torch.from_numpy(x).cuda()
        y = pd.hubbard_apply(h, xd).cpu().numpy()
        assert np.max(np.abs(y - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
        xf = (xd / xd.abs().max()).contiguous()
        q = pd.hubbard_convert(h, xf, torch.int64)
        yq = pd.hubbard_convert(h, pd.hubbard_apply(h, q), torch.float64).cpu().numpy()
        ref2 = M.apply(mod, xf.cpu().numpy())
        F = pd.hubbard_fixed_point_bits(h)
        # two rounded products per element (diagonal, U/N) plus the float64 rounding of the reference
        scale = max(1.0, np.max(np.abs(ref2)))
        assert np.max(np.abs(yq - ref2)) <= 2 * 2.0 ** -F * scale + 32 * np.finfo(float).eps * scale
        y32 = pd.hubbard_apply(h, xd.float()).double().cpu().numpy()
        assert np.max(np.abs(y32 - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))
        h.close()


def test_ring8_sector_minimum_is_real_space_ground_energy(env):
    """Ring L = 8, (4,4), U = 4: the lowest sector energy equals the real-space E0 (golden, oracle)."""
    torch, pd = env
    gold = json.load(open(os.path.join(GOLDEN, "oracle_energies.json")))["ring8_U4_4_4"]["E0"]
    E = []
    for K in range(8):
        h = pd.Handle.momentum(8, 1, 1.0, 0.0, 4.0, 4, 4, K, 0)
        r = pd.lanczos_ground_state(h, maxit=600, tol=1e-10, reorth=True)
        E.append(r.E0)
        h.close()
    assert abs(min(E) - gold) <= 1e-10 * max(1.0, abs(gold))


def test_square4x4_half_filling_sectors(env):
    """4x4 t-t' cluster, U = 8, (8,8): the lowest of the 16 sector energies (fixed-point Lanczos,
    D_K ~ 1.0e7 each) equals the real-space E0 of the float64 oracle to 1e-10."""
    torch, pd = env
    gold = json.load(open(os.path.join(GOLDEN, "oracle_energies.json")))["square4x4_tp-0.3_U8_8_8"]["E0"]
    E, D = [], 0
    for K in range(16):
        h = pd.Handle.momentum(4, 4, 1.0, -0.3, 8.0, 8, 8, K % 4, K // 4)
        D += h.D
        r = pd.lanczos_ground_state(h, maxit=3000, tol=1e-10, dtype=torch.int64)
        E.append(r.E0)
        h.close()
    assert D == 12870 ** 2
    assert abs(min(E) - gold) <= 1e-10 * max(1.0, abs(gold))


def test_autotune_and_step_on_a_sector(env):
    """The configuration and stepping entry points accept a momentum handle (its H·v has one
    launch shape: autotune only times it) and give the same vector as hubbard_apply."""
    import ctypes
    torch, pd = env
    h = pd.Handle.momentum(3, 3, 1.0, -0.3, 5.0, 2, 2, 1, 2)
    x = torch.rand(h.D, dtype=torch.float64, device="cuda") - 0.5
    x /= x.norm()
    ref = pd.hubbard_apply(h, x).clone()
    y = torch.empty_like(x)
    best = pd.hubbard_autotune(h, x, y, reps=2)
    assert best["ms"] > 0
    assert torch.equal(pd.hubbard_apply(h, x), ref)
    scratch = torch.empty(pd.lanczos_step_scratch_bytes(h), dtype=torch.uint8, device="cuda")
    a = torch.zeros(1, dtype=torch.float64, device="cuda")
    b = torch.zeros(1, dtype=torch.float64, device="cuda")
    w = torch.empty_like(x)
    n = ctypes.c_uint32(0)
    pd.lanczos_step(h, x, None, w, None, a, b, scratch, launches=n)
    torch.cuda.synchronize()
    assert n.value == 1 + 5
    alpha = float(torch.dot(ref, x))
    assert abs(a.item() - alpha) < 1e-12
    assert torch.allclose(w * b.item(), ref - alpha * x, atol=1e-12)
    assert pd.hubbard_last_error(h) == "HB_OK"
    h.close()
