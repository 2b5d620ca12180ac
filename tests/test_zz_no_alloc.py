"""The allocation-free Lanczos step against the regular one (GPU).

Some callers may not allocate device memory at the point where they step the
solver (a host that hands out every device byte from its own pool, a plug-in
inside another framework's memory budget).  They use lanczos_step_noalloc,
whose reduction scratch is a fixed array inside the library instead of a
caller buffer.  Both entry points launch the same kernels, so their outputs
must agree bit for bit.  This file is collected last so that a failure here
comes after every other test has run; it must pass alone in a fresh process as
well.
"""
import numpy as np
import pytest

import workloads as wl
from oracle.lanczos import start_vector
from tests.gpu_util import handle_for, need_gpu

pytestmark = pytest.mark.gpu


def _real_space():
    return handle_for(wl.rect_periodic(4, 3), 5.0, 5, 4)


def _momentum_sector():
    import paper_1707_03974_gb300 as pd
    return pd.Handle.momentum(3, 3, 1.0, -0.3, 4.0, 4, 4, 0, 0)


@pytest.mark.parametrize("make", [_real_space, _momentum_sector], ids=["real_space", "momentum_K00"])
@pytest.mark.parametrize("dtype_name", ["float64", "float32"])
def test_noalloc_step_matches_regular_step_twice(dtype_name, make):
    torch = need_gpu()
    import paper_1707_03974_gb300 as pd
    dtype = getattr(torch, dtype_name)
    h = make()
    dev = torch.device("cuda")
    v0 = torch.from_numpy(start_vector(21, h.D)).to(dev, dtype)
    v0 /= v0.norm()
    pd.hubbard_apply(h, v0)  # builds the handle's tables (the no-alloc call does not)
    scratch = torch.empty(pd.lanczos_step_scratch_bytes(h), dtype=torch.uint8, device=dev)

    def run(no_alloc):
        V = [v0.clone(), torch.empty_like(v0), torch.empty_like(v0)]
        a = torch.zeros(2, dtype=torch.float64, device=dev)
        b = torch.zeros(2, dtype=torch.float64, device=dev)
        for j in range(2):  # two calls in a row: the second reuses the first call's scratch contents
            vprev = V[(j - 1) % 3] if j > 0 else None
            bprev = b[j - 1:j] if j > 0 else None
            if no_alloc:
                pd.lanczos_step_noalloc(h, V[j % 3], vprev, V[(j + 1) % 3], bprev, a[j:j + 1], b[j:j + 1])
            else:
                pd.lanczos_step(h, V[j % 3], vprev, V[(j + 1) % 3], bprev, a[j:j + 1], b[j:j + 1], scratch)
        torch.cuda.synchronize()
        return V[1], V[2], a, b

    ref = run(False)
    got = run(True)
    for r, g in zip(ref, got):
        assert torch.equal(r, g)  # the same kernels on the same inputs
    assert np.all(np.isfinite(got[3].cpu().numpy())) and float(got[3][1]) > 0
    assert pd.hubbard_last_error(h) == "HB_OK"
    h.close()


def test_noalloc_step_refuses_to_build_tables():
    torch = need_gpu()
    import paper_1707_03974_gb300 as pd
    h = handle_for(wl.ring(6), 2.0, 3, 3)
    v = torch.zeros(h.D, dtype=torch.float64, device="cuda")
    v[0] = 1.0
    w = torch.empty_like(v)
    a = torch.zeros(1, dtype=torch.float64, device="cuda")
    b = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(pd.HubbardError) as e:
        pd.lanczos_step_noalloc(h, v, None, w, None, a, b)
    assert e.value.name == "HB_ERR_INVALID_STATE"
    h.close()


def test_noalloc_step_refuses_fixed_point():
    """The fixed-point step needs six doubles of scratch per reduction block,
    more than the library's fixed array holds: refused up front."""
    torch = need_gpu()
    import paper_1707_03974_gb300 as pd
    h = handle_for(wl.ring(6), 2.0, 3, 3)
    x = torch.zeros(h.D, dtype=torch.float64, device="cuda")
    x[0] = 1.0
    pd.hubbard_apply(h, x)  # tables built, so the refusal comes from the vector type
    v = pd.hubbard_convert(h, x, torch.int64)
    w = torch.empty_like(v)
    a = torch.zeros(1, dtype=torch.float64, device="cuda")
    b = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(pd.HubbardError) as e:
        pd.lanczos_step_noalloc(h, v, None, w, None, a, b)
    assert e.value.name == "HB_ERR_INVALID_ARG"
    h.close()


def test_noalloc_step_refuses_another_device():
    torch = need_gpu()
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs to make another device current")
    import paper_1707_03974_gb300 as pd
    with torch.cuda.device(0):
        h = _real_space()
        v = torch.zeros(h.D, dtype=torch.float64, device="cuda:0")
        v[0] = 1.0
        pd.hubbard_apply(h, v)
        w = torch.empty_like(v)
        a = torch.zeros(1, dtype=torch.float64, device="cuda:0")
        b = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    with torch.cuda.device(1):
        with pytest.raises(pd.HubbardError) as e:
            pd.lanczos_step_noalloc(h, v, None, w, None, a, b)
    assert e.value.name == "HB_ERR_INVALID_ARG"
    h.close()
