"""Start-vector network on the GPU vs the CPU oracle (bf16 operands, f32 accumulation)."""
import numpy as np
import pytest

import workloads as wl
from oracle.basis import Basis
from oracle.mlp import bits_of, forward, loss_and_grad
from tests.gpu_util import need_gpu, to_dev_u64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    import paper_1707_03974_gb300 as pd
    return torch, pd


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 128, 32), (384, 32, 128), (128, 128, 1024), (1000, 128, 128)])
def test_tc_gemm_matches_float_reference(env, M, N, K):
    torch, pd = env
    g = torch.Generator().manual_seed(M + N + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    C = pd.mlp_tc_gemm(A.cuda(), B.cuda()).cpu()
    ref = A.double() @ B.double().T   # exact products of bf16 values, float64 sums
    err = (C.double() - ref).abs().max().item()
    assert err <= 2e-6 * K * max(1.0, ref.abs().max().item() / K) + 1e-5 * ref.abs().max().item()


def test_activation_matches_tanh_gelu(env):
    """The network's GELU (tanh form, tanh from the hardware's tanh.approx.f32, relative error about
    2^-11) against the oracle's float64 tanh form over the activation range.  Bounds from that
    error e = 2^-10: |gelu error| <= |x|/2 e + float32 rounding; |gelu' error| <= (1/2 + |x| u'(x)) e
    with u'(x) = sqrt(2/pi) (1 + 3 * 0.044715 x^2).  Both stay inside the bfloat16 rounding
    (2^-9 relative) that every activation then goes through.  The activation also stays within
    5e-4 + that bound of the exact erf form, as the tanh form itself does."""
    torch, pd = env
    import math
    from oracle.mlp import gelu, gelu_grad
    x = torch.linspace(-12.0, 12.0, 200001, dtype=torch.float32)
    xd = x.double().numpy()
    e = 2.0 ** -10
    y = pd.mlp_activation(x.cuda()).cpu().double().numpy()
    dy = pd.mlp_activation(x.cuda(), deriv=True).cpu().double().numpy()
    ax = abs(xd)
    assert (abs(y - gelu(xd)) <= 0.5 * ax * e + 1e-6 * (1 + ax)).all()
    up = math.sqrt(2 / math.pi) * (1 + 3 * 0.044715 * xd * xd)
    assert (abs(dy - gelu_grad(xd)) <= (0.5 + ax * up) * e + 1e-6).all()
    exact = 0.5 * xd * (1.0 + torch.special.erf(torch.from_numpy(xd) / math.sqrt(2.0)).numpy())
    assert (abs(y - exact) <= 5e-4 + 0.5 * ax * e + 1e-6 * (1 + ax)).all()


def test_sampler_matches_inverse_cdf_on_cpu(env):
    """mlp_sample_training against the plain definition on the CPU: the same SplitMix64 draws u_i in
    [0, 1), the first index whose float64 cumulative sum of psi^2 exceeds u_i * total; states by the
    sorted basis, targets log|psi| centred over the draws and the sign after the global sign fix.
    Draws that land within rounding of a cumulative boundary may differ by one index."""
    torch, pd = env
    import workloads as wl
    from oracle.lanczos import splitmix64_outputs
    from tests.gpu_util import handle_for
    cl = wl.rect_periodic(4, 3)
    h = handle_for(cl, 4.0, 5, 4)
    b = Basis(12, 5, 4)
    rng = np.random.default_rng(7)
    psi = rng.standard_normal(b.D).astype(np.float32)
    psi[rng.integers(0, b.D, 300)] = 0.0          # zero entries must never be drawn
    psi[12345] = -40.0                            # the largest magnitude is negative: the sign flips
    n, seed = 20000, 99
    st, t_log, t_sign = pd.mlp_sample_training(h, torch.from_numpy(psi).cuda(), n, seed)
    st = st.cpu().numpy().view(np.uint64)
    t_log, t_sign = t_log.cpu().numpy(), t_sign.cpu().numpy()
    p64 = psi.astype(np.float64)
    cdf = np.cumsum(p64 * p64)
    u = (splitmix64_outputs(seed, 0, n) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53 * cdf[-1]
    idx = np.searchsorted(cdf, u, side="right")
    got_idx = b.index_of(st)
    assert np.all(got_idx >= 0)
    assert np.all(psi[got_idx] != 0.0)
    same = got_idx == idx
    assert same.mean() >= 0.999
    assert np.all(np.abs(got_idx[~same] - idx[~same]) <= 1)
    gsign = -1.0 if psi[np.argmax(np.abs(psi))] < 0 else 1.0
    amp = gsign * p64[got_idx]
    ref_log = np.log(np.abs(amp))
    assert np.allclose(t_log, ref_log - ref_log.mean(), atol=2e-6)
    assert np.array_equal(t_sign, np.where(amp >= 0, 1.0, -1.0).astype(np.float32))
    # the draws follow psi^2: the heaviest entry is drawn about n psi^2 / total times
    heavy = np.count_nonzero(got_idx == 12345)
    expect = n * 1600.0 / cdf[-1]
    assert abs(heavy - expect) <= 5 * np.sqrt(expect) + 1
    h.close()


def test_forward_matches_oracle(env):
    torch, pd = env
    L = 8
    m = pd.Mlp(2 * L, seed=3)
    theta = m.get_params().astype(np.float64)
    b = Basis(L, 4, 3)
    states = b.combined[:777]
    out = pd.mlp_forward(m, to_dev_u64(states)).cpu().numpy()
    ref, _ = forward(theta, bits_of(states, L), 2 * L, 128, emulate_bf16=True)
    assert np.max(np.abs(out - ref)) <= 2e-3 * max(1.0, np.max(np.abs(ref)))
    assert pd.mlp_last_error(m) == "HB_OK"
    m.close()


def test_gradient_matches_oracle(env):
    torch, pd = env
    L = 8
    m = pd.Mlp(2 * L, seed=4)
    theta = m.get_params().astype(np.float64)
    b = Basis(L, 4, 4)
    rng = np.random.default_rng(0)
    idx = rng.choice(b.D, 1500, replace=False)
    states = b.combined[idx]
    t_log = rng.normal(size=idx.size) - 4.0
    t_sign = np.where(rng.random(idx.size) < 0.5, -1.0, 1.0)
    w = rng.random(idx.size)
    w /= w.sum()
    dev = lambda a: torch.from_numpy(np.asarray(a, dtype=np.float32)).cuda()
    g, loss = pd.mlp_gradient(m, to_dev_u64(states), dev(t_log), dev(t_sign), dev(w), lam=1.0)
    g = g.cpu().numpy().astype(np.float64)
    lref, gref = loss_and_grad(theta, bits_of(states, L), t_log, t_sign, w, 2 * L, 128, lam=1.0, emulate_bf16=True)
    assert abs(loss.item() - lref) <= 1e-3 * abs(lref)
    # bf16 rounding of the back-propagated activations: a few parts in a thousand
    assert np.linalg.norm(g - gref) <= 2e-2 * np.linalg.norm(gref)
    assert pd.mlp_last_error(m) == "HB_OK"
    m.close()


def test_training_reduces_loss(env):
    torch, pd = env
    L = 8
    m = pd.Mlp(2 * L, seed=5)
    b = Basis(L, 4, 4)
    rng = np.random.default_rng(1)
    states = to_dev_u64(b.combined)
    bits = bits_of(b.combined, L)
    t_log = torch.from_numpy((bits[:, :L].sum(1) - bits[:, L:].sum(1) * 0.5 - 3.0).astype(np.float32)).cuda()
    t_sign = torch.from_numpy(np.where(bits[:, 0] > 0, 1.0, -1.0).astype(np.float32)).cuda()
    w = torch.full((b.D,), 1.0 / b.D, dtype=torch.float32, device="cuda")
    losses = []
    for _ in range(60):
        _, loss = pd.mlp_gradient(m, states, t_log, t_sign, w)
        losses.append(loss.item())
        pd.mlp_adam_step(m, 3e-3)
    assert losses[-1] < 0.2 * losses[0]
    m.close()


def _expected_start(out):
    """sign(out1) exp(min(out0, 10) - 10), the start-value map, in float64."""
    return np.where(out[:, 1] >= 0, 1.0, -1.0) * np.exp(np.minimum(out[:, 0].astype(np.float64), 10.0) - 10.0)


@pytest.mark.parametrize("dtype_name", ["float32", "float64", "int64"])
def test_fused_start_vector_matches_forward(env, dtype_name):
    """The fused tensor-core inference kernel (unranking on the fly) against mlp_forward on
    every basis state of a small sector (D = 3920: 30 full tiles and a ragged one) and
    against the float64 oracle of the network."""
    torch, pd = env
    from tests.gpu_util import handle_for
    L = 8
    h = handle_for(wl.ring(L), 2.0, 4, 3)
    m = pd.Mlp(2 * L, seed=11)
    b = Basis(L, 4, 3)
    assert len(b.combined) == h.D == 3920
    out = pd.mlp_forward(m, to_dev_u64(b.combined)).cpu().numpy()
    want = _expected_start(out)
    v = pd.mlp_start_vector(m, h, getattr(torch, dtype_name))
    if dtype_name == "int64":
        got = pd.hubbard_convert(h, v, torch.float64).cpu().numpy() * 2.0  # stored as s / 2
    else:
        got = v.double().cpu().numpy()
    assert np.all(np.sign(got) == np.sign(want))
    assert np.max(np.abs(got - want) / np.abs(want)) <= 1e-5
    theta = m.get_params().astype(np.float64)
    ref, _ = forward(theta, bits_of(b.combined, L), 2 * L, 128, emulate_bf16=True)
    assert np.max(np.abs(np.log(np.abs(got)) - np.log(np.abs(_expected_start(ref))))) <= 2e-3 * max(
        1.0, np.max(np.abs(ref)))
    assert pd.mlp_last_error(m) == "HB_OK"
    m.close()
    h.close()


def test_fused_start_vector_sampled_at_853776(env):
    """3x4 cluster, N_up = N_dn = 6 (D = 853,776): 4096 sampled entries against mlp_forward
    on the unranked states."""
    torch, pd = env
    from tests.gpu_util import handle_for
    h = handle_for(wl.rect_periodic(4, 3), 5.0, 6, 6)
    m = pd.Mlp(24, seed=5)
    v = pd.mlp_start_vector(m, h, torch.float32)
    g = torch.Generator().manual_seed(9)
    idx = torch.randint(0, h.D, (4096,), generator=g)
    idx[:2] = torch.tensor([0, h.D - 1])
    states = pd.paradeisos_unrank(h, idx.cuda())
    want = _expected_start(pd.mlp_forward(m, states).cpu().numpy())
    got = v[idx.cuda()].double().cpu().numpy()
    assert np.max(np.abs(got - want) / np.abs(want)) <= 1e-5
    m.close()
    h.close()
