"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package only describes *inputs*: cluster geometries (site count and bond
list with hopping amplitudes) and seeded draws of problem instances.  It holds
none of the method's arithmetic (no ranking, no Hamiltonian action, no
eigensolver), so both the CPU oracle side and the CUDA side may consume it.
"""
from .lattices import Cluster, ring, square_periodic, tilted_18, dimer, rect_periodic  # noqa: F401
from .instances import draw_batch_instances, BatchInstance  # noqa: F401
