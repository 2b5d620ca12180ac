"""Green's function of momentum sectors on the GPU (c / c+ operators, float64 Ritz vector,
Lanczos continued fraction) against the response oracle, plus sum rules at full size."""
import numpy as np
import pytest

from oracle import momentum as M
from oracle import response as R
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

Z = np.linspace(-6, 8, 29) + 0.25j


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    import paper_1707_03974_gb300 as pd
    return torch, pd


def _ground_sector(g, t, tp, U, nu, nd):
    best = None
    for K in range(g.N):
        if len(M.sector_list(g, nu, nd, K)) == 0:
            continue
        w, V = R.sector_ground(g, t, tp, U, nu, nd, K)
        if best is None or w[0] < best[0]:
            best = (w[0], K, V[:, 0], w[1] - w[0])
    return best


@pytest.mark.parametrize("op,spin", [("c", 0), ("c", 1), ("cdag", 0), ("cdag", 1)])
def test_operator_matches_oracle(env, op, spin):
    torch, pd = env
    g = M.Grid(3, 3)
    nu, nd, K = 2, 2, 4
    src = pd.Handle.momentum(3, 3, 1.0, -0.3, 5.0, nu, nd, K % 3, K // 3)
    x = np.random.default_rng(spin + 2 * (op == "c")).uniform(-1, 1, src.D)
    lst = M.sector_list(g, nu, nd, K)
    d = -1 if op == "c" else 1
    nu2, nd2 = (nu + d, nd) if spin == 0 else (nu, nd + d)
    for k in range(g.N):
        K2 = g.sub(K, k) if op == "c" else g.add(K, k)
        dlst = M.sector_list(g, nu2, nd2, K2)
        dst = pd.Handle.momentum(3, 3, 1.0, -0.3, 5.0, nu2, nd2, K2 % 3, K2 // 3)
        y, n2 = pd.hubbard_apply_c(src, dst, op, spin, k, torch.from_numpy(x).cuda())
        want = R.apply_op(g, lst, dlst, op, spin, k, x, nu)
        assert np.array_equal(y.cpu().numpy(), want)
        assert abs(n2.item() - want @ want) <= 1e-12 * max(1.0, want @ want)
        dst.close()
    with pytest.raises(pd.HubbardError):  # wrong target sector
        pd.hubbard_apply_c(src, src, op, spin, 0, torch.from_numpy(x).cuda())
    src.close()


def test_ritz_vector_f64_is_the_ground_state(env):
    torch, pd = env
    g = M.Grid(6, 1)
    E0, K0, psi, gap = _ground_sector(g, 1.0, 0.0, 4.0, 3, 3)
    h = pd.Handle.momentum(6, 1, 1.0, 0.0, 4.0, 3, 3, K0, 0)
    e, v, info = pd.lanczos_ritz_vector_f64(h, tol=1e-12)
    assert info.converged and abs(e - E0) < 1e-10
    assert abs(abs(float(np.dot(v.cpu().numpy(), psi))) - 1.0) < 1e-9
    h.close()


@pytest.mark.parametrize("Lx,Ly,tp,U,nu,nd", [(6, 1, 0.0, 4.0, 3, 3), (3, 3, -0.3, 5.0, 2, 2)])
def test_green_function_matches_spectral_sum(env, Lx, Ly, tp, U, nu, nd):
    """Full-length Lanczos (with reorthogonalisation) from c|psi0> and c+|psi0>: the continued
    fraction equals the oracle's spectral sum over the dense target sector."""
    torch, pd = env
    from paper_1707_03974_gb300 import response
    g = M.Grid(Lx, Ly)
    E0, K0, psi, gap = _ground_sector(g, 1.0, tp, U, nu, nd)
    if gap < 1e-8:
        pytest.skip("degenerate ground state")
    h = pd.Handle.momentum(Lx, Ly, 1.0, tp, U, nu, nd, K0 % Lx, K0 // Lx)
    gs = response.ground(h, tol=1e-12)
    assert abs(gs.E0 - E0) < 1e-10
    lst = M.sector_list(g, nu, nd, K0)
    sgn = np.sign(float(np.dot(gs.psi.cpu().numpy(), psi)))
    for part, op in (("removal", "c"), ("addition", "cdag")):
        for spin in (0, 1):
            for k in range(g.N):
                G, info = response.green(gs, k, spin, part, Z, steps=10_000, reorth=True)
                d = -1 if op == "c" else 1
                nu2, nd2 = (nu + d, nd) if spin == 0 else (nu, nd + d)
                K2 = g.sub(K0, k) if op == "c" else g.add(K0, k)
                dlst = M.sector_list(g, nu2, nd2, K2)
                phi = R.apply_op(g, lst, dlst, op, spin, k, sgn * psi, nu)
                if G is None:
                    assert phi @ phi < 1e-20
                    continue
                H2 = M.dense(M.KModel(g, 1.0, tp, U, nu2, nd2, K2))
                want = R.spectral_sum(H2, phi, E0, Z)
                assert np.max(np.abs(G - want)) <= 1e-8 * max(1.0, np.max(np.abs(want))), (part, spin, k)
    h.close()


def test_sum_rules_at_full_size(env):
    """4x4 t-t' cluster, U = 8, half filling, K = (0,0) ground state (D = 10,353,252): for every k
    the removal and addition weights sum to 1, and the removal weights sum to N_up = 8."""
    torch, pd = env
    from paper_1707_03974_gb300 import response
    h = pd.Handle.momentum(4, 4, 1.0, -0.3, 8.0, 8, 8, 0, 0)
    gs = response.ground(h)
    total = 0.0
    for k in range(16):
        kx, ky = k % 4, k // 4
        dr = pd.Handle.momentum(4, 4, 1.0, -0.3, 8.0, 7, 8, (-kx) % 4, (-ky) % 4)
        da = pd.Handle.momentum(4, 4, 1.0, -0.3, 8.0, 9, 8, kx, ky)
        _, r2 = pd.hubbard_apply_c(h, dr, "c", 0, k, gs.psi)
        _, a2 = pd.hubbard_apply_c(h, da, "cdag", 0, k, gs.psi)
        assert abs(r2.item() + a2.item() - 1.0) < 1e-10
        total += r2.item()
        dr.close()
        da.close()
    assert abs(total - 8.0) < 1e-9
    G, info = response.green(gs, 5, 0, "removal", Z, steps=150)
    assert info["steps"] == 150 and np.all(G.imag <= 1e-12)  # a removal spectral weight is positive
    h.close()
