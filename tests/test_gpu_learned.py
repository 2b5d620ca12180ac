"""The learned start vector: trained on the method's own ground states at two U, it must
cut the Lanczos iterations at an unseen U (and keep E0 at 1e-10)."""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_util import handle_for, need_gpu

pytestmark = pytest.mark.gpu


def test_learned_start_gains_over_random_start():
    torch = need_gpu()
    import paper_1707_03974_gb300 as pd
    from paper_1707_03974_gb300 import learned
    cl = wl.rect_periodic(4, 3)
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    sets = []
    for U in (3.0, 8.0):
        h = handle_for(cl, U, 6, 6)
        _, psi = learned.ground_state(h, tol=1e-6)
        sets.append(learned.sample(h, psi, 200000, g))
        h.close()
    m = pd.Mlp(24, seed=1)
    rep = learned.train(m, sets, steps=3000, batch=16384, lr=2e-3)
    assert rep.losses[-1] < 0.75 * rep.losses[0]
    assert pd.mlp_last_error(m) == "HB_OK"
    h = handle_for(cl, 5.0, 6, 6)
    E_ref, psi = learned.ground_state(h, tol=1e-8)
    res = learned.compare(m, h, psi, seeds=(0, 1))
    rnd = min(r["iterations"] for r in res["random_f64"])
    assert res["learned_f64"]["converged"] and res["learned_fx64"]["converged"]
    for k in ("learned_f64", "learned_fx64", "learned_mixed_f32_fx64"):
        assert abs(res[k]["E0"] - res["random_f64"][0]["E0"]) <= 1e-10 * abs(res["random_f64"][0]["E0"])
    assert res["overlap"] > 0.0
    # the learned start must save Lanczos steps over the best of two random starts
    assert res["learned_f64"]["iterations"] < rnd
    assert res["learned_fx64"]["iterations"] < rnd + 5
    h.close()
    m.close()
