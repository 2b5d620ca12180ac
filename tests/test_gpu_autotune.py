"""H·v launch configurations: every configuration computes bit-identical results (float32:
every one-kernel configuration, and every split configuration among themselves; the split
float32 row pass sums the spin-down hops per (class, sign) segment of the warp-blocked table,
so it agrees with the one-kernel form to float32 rounding), and the autotuner keeps the
fastest one."""
import numpy as np
import pytest

import workloads as wl
from oracle.lanczos import start_vector
from tests.gpu_util import handle_for, need_gpu

pytestmark = pytest.mark.gpu


CLUSTERS = {
    "3x3_tp_4_4": (lambda: wl.rect_periodic(3, 3, 1.0, -0.3), 5.0, 4, 4),  # D_dn = 126 (even: column pairs)
    "ring7_3_3": (lambda: wl.ring(7), 2.0, 3, 3),                           # D_dn = 35 (odd: single columns)
}


@pytest.mark.parametrize("cluster", sorted(CLUSTERS))
@pytest.mark.parametrize("dtype_name", ["float64", "float32", "int64"])
def test_all_configs_bit_identical(dtype_name, cluster):
    torch = need_gpu()
    import paper_1707_03974_gb300 as pd
    dtype = getattr(torch, dtype_name)
    make, U, nu, nd = CLUSTERS[cluster]
    h = handle_for(make(), U, nu, nd)
    x = torch.from_numpy(start_vector(3, h.D)).cuda()
    x = pd.hubbard_convert(h, x / x.abs().max(), torch.int64) if dtype_name == "int64" else x.to(dtype)
    ref = pd.hubbard_apply(h, x).cpu()
    for rows in (1, 2, 4):
        for threads in (64, 256, 512, 1024):
            for order in (0, 1):
                pd.hubbard_set_hv_config(h, dtype, rows, threads, order)
                y = pd.hubbard_apply(h, x).cpu()
                assert torch.equal(y, ref), (rows, threads, order)
    # split form: row pass then the column-blocked spin-up pass; both row lengths
    # leave ragged column blocks for every block width
    split_ref = None
    for rows, threads in ((1, 256), (2, 1024), (4, 512)):
        for ub, ut in ((32, 64), (64, 512), (128, 1024), (256, 256)):
            for rr in (1, 2, 4):
                pd.hubbard_set_hv_config(h, dtype, rows, threads, 1, split=1, up_block=ub, up_threads=ut, up_rows=rr)
                y = pd.hubbard_apply(h, x).cpu()
                if split_ref is None:
                    split_ref = y
                assert torch.equal(y, split_ref), (rows, threads, ub, ut, rr)
    if dtype_name == "float32":
        assert torch.allclose(split_ref.double(), ref.double(), rtol=0, atol=1e-5 * float(ref.abs().max()))
    else:
        assert torch.equal(split_ref, ref)
    h.close()


@pytest.mark.parametrize("dtype_name", ["float64", "float32", "int64"])
def test_split_matches_fused_on_long_rows(dtype_name):
    """18 sites, N_up = 1, N_dn = 9: rows of 48,620 elements (too long for shared memory
    in 8-byte formats, so the row pass gathers from global memory; one float32 row fits)."""
    torch = need_gpu()
    import paper_1707_03974_gb300 as pd
    dtype = getattr(torch, dtype_name)
    h = handle_for(wl.ring(18), 4.0, 1, 9)
    x = torch.from_numpy(start_vector(5, h.D)).cuda()
    x = pd.hubbard_convert(h, x / x.abs().max(), torch.int64) if dtype_name == "int64" else x.to(dtype)
    pd.hubbard_set_hv_config(h, dtype, 0, 0, 1)
    ref = pd.hubbard_apply(h, x).cpu()
    for ub, ut, rr in ((128, 1024, 1), (256, 512, 2), (512, 1024, 4)):
        pd.hubbard_set_hv_config(h, dtype, 0, 0, 1, split=1, up_block=ub, up_threads=ut, up_rows=rr)
        y = pd.hubbard_apply(h, x).cpu()
        if dtype_name == "float32":  # one 194 KB row fits: the warp-blocked float32 row pass
            assert torch.allclose(y.double(), ref.double(), rtol=0, atol=1e-5 * float(ref.abs().max())), (ub, ut, rr)
        else:
            assert torch.equal(y, ref), (ub, ut, rr)
    h.close()


def test_autotune_keeps_fastest_and_results_unchanged():
    torch = need_gpu()
    import paper_1707_03974_gb300 as pd
    h = handle_for(wl.ring(12), 3.0, 6, 6)
    x = torch.from_numpy(start_vector(4, h.D)).cuda()
    ref = pd.hubbard_apply(h, x).clone()
    y = torch.empty_like(x)
    best = pd.hubbard_autotune(h, x, y, reps=2)
    assert best["ms"] > 0 and best["rows_per_cta"] in (1, 2, 4) and best["threads_per_cta"] in (256, 512, 1024)
    assert best["split"] in (0, 1)
    cur = pd.hubbard_get_hv_config(h, torch.float64)
    keys = ("rows_per_cta", "threads_per_cta", "visit_order", "split", "up_block", "up_threads", "up_rows")
    assert all(cur[k] == best[k] for k in keys)
    assert torch.equal(pd.hubbard_apply(h, x), ref)
    with pytest.raises(pd.HubbardError):
        pd.hubbard_set_hv_config(h, torch.float64, 3, 100, 0)
    with pytest.raises(pd.HubbardError):  # block wider than the CTA
        pd.hubbard_set_hv_config(h, torch.float64, 0, 0, 1, split=1, up_block=512, up_threads=256)
    with pytest.raises(pd.HubbardError):
        pd.hubbard_set_hv_config(h, torch.float64, 0, 0, 1, split=1, up_rows=3)
    h.close()
