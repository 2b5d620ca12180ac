"""CPU oracle for the Paradeisos Hubbard hot path -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, obviously correct restatement of what the GPU
path computes, written from the paper (arXiv 1707.03974) in float64.  Only the
test suite, the package's ``__graft_entry__.smoke()`` check and the benchmark's
CPU-baseline leg may import it.  It shares no code with the CUDA library and
never imports it.

Definitions used (each function cites the passage it follows):

* basis positions are positions in the *sorted list* of occupation integers,
  found by binary search (the "conventional" scheme of Sec. II C); Paradeisos
  must reproduce exactly these positions;
* the Hamiltonian is Eq. 1 with the fermion sign fixed by the normal ordering of
  Sec. II A (spin-up creators left of spin-down, higher site index to the left);
* ground energies come from dense ``numpy.linalg.eigh`` on small clusters and a
  textbook Lanczos iteration (which the paper cites but does not specify);
* the momentum-space sectors (Sec. IV A, ``momentum.py``) are ascending lists of
  (up, dn) strings over the single-particle momenta with fixed total momentum,
  and their Hamiltonian is Eq. 4 term by term;
* the inversion-symmetric maps (Sec. IV B, ``inversion.py``) follow the
  classification tree; the single-particle Green's function (``response.py``)
  is the spectral sum over a dense target sector and the continued fraction of
  a textbook Lanczos run.

Parity status: every function here is pinned by tests against values printed in
the paper or fixed by mathematics (closed forms, invariants, brute force).
``count_below`` and ``string_at`` are checked against the sorted list for
L <= 14 and, up to L = 32, along runs of the bit-operation successor of
Sec. II A (which counts nothing): the count must grow by exactly one per step.
"""
