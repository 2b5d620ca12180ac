"""Pinned huge-page host buffers (hb_host_alloc): page-locked, copy both ways, released with the tensor."""
import gc

import pytest

from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def test_host_empty_is_pinned_and_copies():
    torch = need_gpu()
    import paper_1707_03974_gb300 as pd
    n = 3_000_001  # not a multiple of the 2 MiB rounding
    torch.zeros(1, device="cuda")
    h = pd.host_empty(n, torch.int64)
    assert h.numel() == n and h.dtype == torch.int64 and h.is_pinned()
    assert h.data_ptr() % (2 << 20) == 0
    assert int(h.abs().sum()) == 0  # zero-filled
    src = torch.arange(n, dtype=torch.int64, device="cuda") * 7 - 5
    h.copy_(src, non_blocking=True)
    torch.cuda.synchronize()
    d = torch.empty_like(src)
    d.copy_(h, non_blocking=True)
    torch.cuda.synchronize()
    assert torch.equal(d, src)
    v = h[10:20]  # a view keeps the buffer alive
    del h
    gc.collect()
    assert torch.equal(v, (torch.arange(10, 20, dtype=torch.int64) * 7 - 5))
    del v
    gc.collect()


def test_host_empty_other_dtypes():
    torch = need_gpu()
    import paper_1707_03974_gb300 as pd
    for dt in (torch.float64, torch.float32):
        h = pd.host_empty(1000, dt)
        h.fill_(1.5)
        assert h.is_pinned() and float(h.sum()) == 1500.0
