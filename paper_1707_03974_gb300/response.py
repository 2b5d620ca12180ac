"""Single-particle Green's function of a momentum sector by the Lanczos continued fraction.

The paper names the continued-fraction Green's function as the other use of the
Krylov machinery (Sec. I).  For momentum k and spin s, starting from the float64
ground state psi0 of a momentum sector (lanczos_ritz_vector_f64):

* removal part   G(z) = <psi0| c+ [z - (H - E0)]^-1 c |psi0>,  phi = c_{k s} psi0
* addition part  G(z) = <psi0| c [z - (H - E0)]^-1 c+ |psi0>, phi = c+_{k s} psi0

phi lands in the sector with one particle fewer (more) and total momentum K -/+ k
(hubbard_apply_c); a float64 Lanczos run started at phi / ||phi|| gives alpha,
beta, and G(z) = ||phi||^2 / (z + E0 - alpha_0 - beta_0^2 / (...)) (hb_continued_fraction).
Every vector operation runs in the library's kernels; this module only composes
the calls.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

from . import _binding as B


@dataclass
class Ground:
    handle: "B.Handle"
    E0: float
    psi: object  # float64 CUDA tensor, normalised


def ground(h: "B.Handle", tol: float = 1e-10) -> Ground:
    E0, psi, _ = B.lanczos_ritz_vector_f64(h, tol=tol)
    return Ground(h, E0, psi)


def green(g: Ground, k: int, spin: int, part: str, z, steps: int = 200, reorth: bool = False):
    """G(z) of one momentum index k (bit index of the grid), spin (0 up, 1 down), part 'removal' or
    'addition'; returns (G array, dict with the Lanczos steps and seconds)."""
    import torch
    h = g.handle
    op = {"removal": "c", "addition": "cdag"}[part]
    sign = -1 if part == "removal" else 1
    nu = h.N_up + (sign if spin == 0 else 0)
    nd = h.N_dn + (sign if spin == 1 else 0)
    Lx, Ly = h.Lx, h.Ly
    N = Lx * Ly
    Kx, Ky = h.K
    kx, ky = k % Lx, k // Lx
    K2x, K2y = (Kx + sign * kx) % Lx, (Ky + sign * ky) % Ly
    if not (0 <= nu <= N and 0 <= nd <= N):
        return None, {"empty": True}
    t0 = time.perf_counter()
    dst = B.Handle.momentum(Lx, Ly, h.t, h.tp, h.U, nu, nd, K2x, K2y)
    phi, n2 = B.hubbard_apply_c(h, dst, op, spin, k, g.psi)
    norm2 = float(n2.item())
    if norm2 == 0.0:
        dst.close()
        return None, {"empty": True}
    m = int(min(steps, dst.D))
    r = B.lanczos_ground_state(dst, maxit=m, tol=0.0, reorth=reorth, v0=phi, raise_on_error=False,
                               check_every=m)
    G = B.hb_continued_fraction(r.alphas, r.betas[: len(r.alphas) - 1], norm2, g.E0, z)
    torch.cuda.synchronize()
    info = {"steps": len(r.alphas), "norm2": norm2, "seconds": time.perf_counter() - t0, "D_target": dst.D}
    dst.close()
    return G, info
