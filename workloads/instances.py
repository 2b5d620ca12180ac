"""Seeded draw of the batched workload: 64 independent 12-site Hubbard problems.

Instance k uses numpy's PCG64 generator seeded with k.  First draw u0 ~ U[0,1):
ring of 12 sites if u0 < 0.5, else the 3x4 periodic lattice (site = x + 4y).
Then N_up and N_dn are drawn independently and uniformly from {3, 4, 5, 6} and
U uniformly from [0, 12); t = 1.  The Lanczos start vector seed of instance k is k.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List

from .lattices import Cluster, ring, rect_periodic


@dataclass(frozen=True)
class BatchInstance:
    index: int
    cluster: Cluster
    N_up: int
    N_dn: int
    U: float
    seed: int


def draw_batch_instances(n: int = 64) -> List[BatchInstance]:
    import numpy as np
    out = []
    ring12 = ring(12)
    rect34 = rect_periodic(4, 3)
    for k in range(n):
        g = np.random.Generator(np.random.PCG64(k))
        shape = g.random()
        nu = int(g.integers(3, 7))
        nd = int(g.integers(3, 7))
        U = float(g.uniform(0.0, 12.0))
        out.append(BatchInstance(k, ring12 if shape < 0.5 else rect34, nu, nd, U, k))
    return out
