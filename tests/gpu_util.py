"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_03974_gb300.build import build
    build()
    return torch


def to_dev_u64(arr):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(arr, dtype=np.uint64)).view(np.int64)).cuda()


def from_dev_u64(t):
    return t.cpu().numpy().view(np.uint64)


def handle_for(cluster, U, nu, nd):
    import paper_1707_03974_gb300 as pd
    return pd.Handle(cluster.L, cluster.bonds, cluster.t, U, nu, nd)
