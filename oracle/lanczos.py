"""Start vectors and Lanczos ground-state iteration (oracle; test infrastructure only).

The paper cites Lanczos (Sec. I) without specifying it; this is the textbook
three-term recurrence (Golub & Van Loan, Sec. 10.1):

  w = H v_j - beta_{j-1} v_{j-1};  alpha_j = <w, v_j>;  w -= alpha_j v_j;
  [full reorthogonalisation: w -= V (V^T w), done twice];
  beta_j = ||w||;  v_{j+1} = w / beta_j,

with the lowest eigenpair of the tridiagonal T_j from LAPACK (scipy).  The
Ritz residual of the lowest Ritz pair is beta_j |s_{j,last}|; the iteration
stops when it is <= tol * max(1, |theta|), which bounds |theta - E0| by tol *
max(1, |E0|) for a converged lowest pair.

Random start vectors use SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) as a
counter-based generator: element i of the vector for `seed` is the (i+1)-th
output of the SplitMix64 stream whose state starts at `seed`, mapped to
[-1, 1) as (z >> 11) * 2^-52 - 1 (exact in float64).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

GOLDEN_GAMMA = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


def splitmix64_scalar(state: int) -> int:
    """One SplitMix64 output for an already-advanced state (the published mixing function)."""
    z = state & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def splitmix64_stream(seed: int, n: int) -> List[int]:
    """First n outputs of SplitMix64 seeded with `seed` (state += gamma before each output)."""
    out = []
    s = seed & M64
    for _ in range(n):
        s = (s + GOLDEN_GAMMA) & M64
        out.append(splitmix64_scalar(s))
    return out


def splitmix64_outputs(seed: int, start: int, n: int) -> np.ndarray:
    """Outputs start+1 .. start+n of the stream, vectorised (uint64 arithmetic wraps mod 2^64)."""
    i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & M64) + i * np.uint64(GOLDEN_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def start_vector(seed: int, n: int) -> np.ndarray:
    """Un-normalised uniform[-1, 1) start vector of length n for `seed`."""
    z = splitmix64_outputs(seed, 0, n)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -52) - 1.0


def tridiag_lowest(alpha, beta):
    """Lowest eigenvalue of T (diag alpha, off-diagonal beta) and the last entry of its eigenvector."""
    from scipy.linalg import eigh_tridiagonal
    a = np.asarray(alpha, dtype=np.float64)
    b = np.asarray(beta, dtype=np.float64)
    if len(a) == 1:
        return float(a[0]), 1.0
    w, v = eigh_tridiagonal(a, b, select="i", select_range=(0, 0))
    return float(w[0]), float(v[-1, 0])


@dataclass
class LanczosResult:
    E0: float
    iterations: int
    residual: float
    converged: bool
    alphas: List[float] = field(default_factory=list)
    betas: List[float] = field(default_factory=list)
    thetas: List[float] = field(default_factory=list)


def lanczos(apply: Callable[[np.ndarray], np.ndarray], v0: np.ndarray, maxit: int,
            reorth: bool = False, tol: Optional[float] = 1e-10) -> LanczosResult:
    v = np.asarray(v0, dtype=np.float64).copy()
    v /= np.linalg.norm(v)
    n = v.size
    V = [v.copy()] if reorth else None
    v_prev = np.zeros(n)
    beta_prev = 0.0
    alphas: List[float] = []
    betas: List[float] = []
    thetas: List[float] = []
    theta, res, converged = float("nan"), float("inf"), False
    for j in range(maxit):
        w = apply(v)
        w = w - beta_prev * v_prev
        a = float(np.dot(w, v))
        w = w - a * v
        if reorth:
            Vm = np.asarray(V)
            for _ in range(2):
                w = w - Vm.T @ (Vm @ w)
        b = float(np.linalg.norm(w))
        alphas.append(a)
        theta, s_last = tridiag_lowest(alphas, betas)
        thetas.append(theta)
        res = b * abs(s_last)
        if tol is not None and res <= tol * max(1.0, abs(theta)):
            converged = True
            betas.append(b)
            break
        if b == 0.0 or j == n - 1:
            converged = True  # invariant subspace: T_j eigenvalues are exact
            betas.append(b)
            break
        betas.append(b)
        v_prev, v = v, w / b
        beta_prev = b
        if reorth:
            V.append(v.copy())
    return LanczosResult(theta, len(alphas), res, converged, alphas, betas, thetas)


def one_body_ground(L: int, bonds, t, N_up: int, N_dn: int) -> float:
    """U = 0 ground energy: fill the lowest single-particle levels of h_ij = -t_ij (both spins)."""
    h = np.zeros((L, L))
    for (i, j), tt in zip(np.asarray(bonds).reshape(-1, 2), t):
        h[i, j] += -tt
        h[j, i] += -tt
    eps = np.linalg.eigvalsh(h)
    return float(eps[:N_up].sum() + eps[:N_dn].sum())
