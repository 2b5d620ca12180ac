"""Pins of the start-vector network oracle (CPU only)."""
import numpy as np
import pytest

from oracle.mlp import bf16, bits_of, forward, gelu, gelu_grad, loss_and_grad, unpack


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.normal(size=2000).astype(np.float32) * 10.0 ** rng.integers(-8, 8, 2000),
                        np.array([1.0, -0.0, 1.00390625, 1.01171875, 3.3895e38], dtype=np.float32)])
    want = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(bf16(a), want)


def test_gelu_values_and_derivative():
    """The tanh form of GELU: pinned to the exact erf form x Phi(x) (math.erf, an independent
    definition), which it approximates to within 5e-4 everywhere (a dropped cubic term or a wrong
    scale misses by 1e-2 or more); odd part x/2 exactly, so gelu(x) - gelu(-x) = x; gelu -> x
    and -> 0 far from the origin; the derivative by central differences."""
    import math
    assert gelu(0.0) == 0.0
    xs = np.linspace(-12, 12, 24001)
    exact = np.array([0.5 * v * (1.0 + math.erf(v / math.sqrt(2.0))) for v in xs])
    dev = np.abs(gelu(xs) - exact)
    assert dev.max() < 5e-4 and dev.max() > 1e-4  # the approximation's known size, not the erf form itself
    assert np.max(np.abs(gelu(xs) - gelu(-xs) - xs)) < 1e-12
    assert abs(gelu(10.0) - 10.0) < 1e-12 and abs(gelu(-10.0)) < 1e-12
    xs = np.linspace(-5, 5, 41)
    h = 1e-6
    fd = (gelu(xs + h) - gelu(xs - h)) / (2 * h)
    assert np.max(np.abs(fd - gelu_grad(xs))) < 1e-8


def test_bits_layout():
    b = bits_of(np.array([(0b0101 << 4) | 0b1011], dtype=np.uint64), 4)
    assert b.tolist() == [[1, 1, 0, 1, 1, 0, 1, 0]]


@pytest.mark.parametrize("emulate", [False, True])
def test_gradient_matches_finite_differences(emulate):
    rng = np.random.default_rng(1)
    n_in, hidden, n = 8, 16, 40
    P = hidden * n_in + hidden + hidden * hidden + hidden + 2 * hidden + 2
    theta = rng.normal(size=P) * 0.3
    x = rng.integers(0, 2, size=(n, n_in)).astype(np.float64)
    t_log = rng.normal(size=n)
    t_sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    w = rng.random(n) + 0.1
    loss, g = loss_and_grad(theta, x, t_log, t_sign, w, n_in, hidden, emulate_bf16=False)
    h = 1e-6
    for i in rng.integers(0, P, 60):
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += h
        tm[i] -= h
        lp, _ = loss_and_grad(tp, x, t_log, t_sign, w, n_in, hidden, emulate_bf16=False)
        lm, _ = loss_and_grad(tm, x, t_log, t_sign, w, n_in, hidden, emulate_bf16=False)
        assert abs((lp - lm) / (2 * h) - g[i]) <= 1e-6 * max(1.0, abs(g[i]))
    if emulate:
        loss2, g2 = loss_and_grad(theta, x, t_log, t_sign, w, n_in, hidden, emulate_bf16=True)
        # bf16 rounding of weights and activations changes values by ~2^-8 relative
        assert abs(loss2 - loss) <= 0.05 * abs(loss)
        assert np.linalg.norm(g2 - g) <= 0.05 * np.linalg.norm(g)


def test_unpack_shapes():
    P = 128 * 32 + 128 + 128 * 128 + 128 + 256 + 2
    parts = unpack(np.arange(P, dtype=float), 32, 128)
    assert [p.shape for p in parts] == [(128, 32), (128,), (128, 128), (128,), (2, 128), (2,)]
    assert parts[0][0, 1] == 1 and parts[5][1] == P - 1
