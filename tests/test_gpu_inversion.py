"""Inversion-symmetric maps on the GPU (Sec. IV B) against the oracle: every representative
for N <= 14, sampled strings up to N = 32."""
import numpy as np
import pytest

from oracle import inversion as V
from tests.gpu_util import from_dev_u64, need_gpu, to_dev_u64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    import paper_1707_03974_gb300 as pd
    return torch, pd


@pytest.mark.parametrize("N", [1, 2, 3, 6, 9, 12, 14])
def test_every_representative(env, N):
    torch, pd = env
    for n in range(N + 1):
        inv = pd.Inversion(N, n)
        reps = np.array(V.representatives(N, n), dtype=np.uint64)
        assert inv.D == len(reps)
        want = np.array([V.forward_map(int(s), N, n) for s in reps], dtype=np.uint64)
        got = from_dev_u64(inv.rank(to_dev_u64(reps)))
        assert np.array_equal(got, want)
        rev = np.array([V.reverse(int(s), N) for s in reps], dtype=np.uint64)
        assert np.array_equal(from_dev_u64(inv.rank(to_dev_u64(rev))), want)
        back = from_dev_u64(inv.unrank(to_dev_u64(want)))
        assert np.array_equal(back, reps)
        assert inv.last_error() == "HB_OK"
        inv.close()


@pytest.mark.parametrize("N,n", [(24, 12), (27, 13), (31, 15), (32, 16), (32, 1), (32, 31)])
def test_sampled_large_chains(env, N, n):
    torch, pd = env
    rng = np.random.default_rng(N * 100 + n)
    inv = pd.Inversion(N, n)
    assert inv.D == V.S(N, n)
    idx = np.unique(rng.integers(0, inv.D, 500, dtype=np.uint64))
    idx = np.concatenate([idx, np.array([0, inv.D - 1], dtype=np.uint64)])
    states = from_dev_u64(inv.unrank(to_dev_u64(idx)))
    for i, s in zip(idx, states):
        assert int(s) == V.backward_map(int(i), N, n)
    assert np.array_equal(from_dev_u64(inv.rank(to_dev_u64(states))), idx)
    inv.close()


def test_invalid_inputs_are_flagged(env):
    torch, pd = env
    inv = pd.Inversion(8, 3)
    bad = from_dev_u64(inv.rank(to_dev_u64(np.array([0b111, 0b1111, 1 << 9], dtype=np.uint64))))
    assert bad[0] != np.uint64(2**64 - 1) and bad[1] == np.uint64(2**64 - 1) and bad[2] == np.uint64(2**64 - 1)
    assert inv.last_error() == "HB_ERR_INVALID_STATE"
    out = from_dev_u64(inv.unrank(to_dev_u64(np.array([inv.D], dtype=np.uint64))))
    assert out[0] == np.uint64(2**64 - 1)
    assert inv.last_error() == "HB_ERR_OUT_OF_RANGE"
    inv.close()
