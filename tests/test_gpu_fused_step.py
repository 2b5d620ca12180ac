"""Fixed-point Lanczos step with its first vector pass inside the split H·v.

Under the split H·v (row pass on the warp-blocked table + spin-up pass) the step
runs the spin-up pass first, storing its term alone, and the row pass then forms
w = H v - beta_prev vprev and the exact sums <w,v>, <w,w>, <v,v> per CTA.  The
one-kernel configuration keeps the separate pass.  Both compute the same integer
operations on every element and exact 128-bit sums, so w, alpha and beta must
agree bit for bit, on the first step (no vprev) and on the general one."""
import numpy as np
import pytest

import workloads as wl
from oracle.lanczos import start_vector
from tests.gpu_util import handle_for, need_gpu

pytestmark = pytest.mark.gpu

BENCH_SPLIT = {"rows_per_cta": 2, "threads_per_cta": 1024, "visit_order": 0, "split": 1,
               "up_block": 128, "up_threads": 512, "up_rows": 4}


def run_steps(torch, pd, h, v0, steps):
    dev = v0.device
    scratch = torch.empty(pd.lanczos_step_scratch_bytes(h), dtype=torch.uint8, device=dev)
    V = [v0.clone(), torch.empty_like(v0), torch.empty_like(v0)]
    a = torch.zeros(steps, dtype=torch.float64, device=dev)
    b = torch.zeros(steps, dtype=torch.float64, device=dev)
    ws = []
    for j in range(steps):
        vp = V[(j - 1) % 3] if j > 0 else None
        bp = b[j - 1:j] if j > 0 else None
        pd.lanczos_step(h, V[j % 3], vp, V[(j + 1) % 3], bp, a[j:j + 1], b[j:j + 1], scratch)
        ws.append(V[(j + 1) % 3].cpu())
    torch.cuda.synchronize()
    return ws, a.cpu(), b.cpu()


def start(torch, pd, h, seed):
    x = torch.from_numpy(start_vector(seed, h.D)).cuda()
    x /= x.norm()
    return pd.hubbard_convert(h, x, torch.int64)


CLUSTERS = {
    # D_up = 495 (odd: the last row group of two holds one row), D_dn = 495
    "4x3_tp_4_4": (lambda: wl.rect_periodic(4, 3, 1.0, -0.3), 4.0, 4, 4),
    "ring7_3_3": (lambda: wl.ring(7), 2.0, 3, 3),               # D_dn = 35, odd column count
    "3x3_tp_4_5": (lambda: wl.rect_periodic(3, 3, 1.0, -0.3), 6.0, 4, 5),  # D_up != D_dn
}


@pytest.mark.parametrize("cluster", sorted(CLUSTERS))
@pytest.mark.parametrize("rows,threads", [(2, 1024), (2, 512), (1, 1024)])
def test_fused_step_bit_identical_to_separate_pass(cluster, rows, threads):
    torch = need_gpu()
    import paper_1707_03974_gb300 as pd
    make, U, nu, nd = CLUSTERS[cluster]
    h = handle_for(make(), U, nu, nd)
    v0 = start(torch, pd, h, 11)
    pd.hubbard_set_hv_config(h, torch.int64, rows, threads, 1)  # one kernel: separate first pass
    ref = run_steps(torch, pd, h, v0, 4)
    pd.hubbard_set_hv_config(h, torch.int64, rows, threads, 1, split=1, up_block=64, up_threads=256, up_rows=2)
    got = run_steps(torch, pd, h, v0, 4)
    for j, (w0, w1) in enumerate(zip(ref[0], got[0])):
        assert torch.equal(w0, w1), j
    assert torch.equal(ref[1], got[1]) and torch.equal(ref[2], got[2])
    h.close()


def test_fused_step_full_size_4x4_bench_configuration():
    """The bench workload (4x4 t-t', U = 8, half filling, D = 165,636,900) under the bench's
    split configuration, against the one-kernel form with its separate first pass."""
    torch = need_gpu()
    import paper_1707_03974_gb300 as pd
    if torch.cuda.get_device_properties(0).total_memory < 40e9:
        pytest.skip("needs ~12 GB of device memory")
    h = handle_for(wl.rect_periodic(4, 4, 1.0, -0.3), 8.0, 8, 8)
    g = torch.Generator(device="cuda")
    g.manual_seed(1234)
    x = torch.empty(h.D, dtype=torch.float64, device="cuda").uniform_(-1.0, 1.0, generator=g)
    x /= x.norm()
    v0 = pd.hubbard_convert(h, x, torch.int64)
    del x
    pd.hubbard_set_hv_config(h, torch.int64, 2, 1024, 0)
    ref = run_steps(torch, pd, h, v0, 2)
    pd.hubbard_set_hv_config(h, torch.int64, **BENCH_SPLIT)
    got = run_steps(torch, pd, h, v0, 2)
    for w0, w1 in zip(ref[0], got[0]):
        assert torch.equal(w0, w1)
    assert torch.equal(ref[1], got[1]) and torch.equal(ref[2], got[2])
    assert pd.lanczos_step_fused(h, torch.int64)
    h.close()


def test_fused_flag_follows_configuration():
    torch = need_gpu()
    import paper_1707_03974_gb300 as pd
    h = handle_for(wl.rect_periodic(4, 3, 1.0, -0.3), 4.0, 4, 4)
    pd.hubbard_set_hv_config(h, torch.int64, 2, 256, 1)
    assert not pd.lanczos_step_fused(h, torch.int64)
    pd.hubbard_set_hv_config(h, torch.int64, 2, 256, 1, split=1)
    assert pd.lanczos_step_fused(h, torch.int64)
    assert not pd.lanczos_step_fused(h, torch.float64)
    assert not pd.lanczos_step_fused(h, torch.float32)
    h.close()
