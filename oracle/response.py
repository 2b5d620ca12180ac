"""Single-particle Green's function by the Lanczos continued fraction (oracle; test
infrastructure only).

The paper names the continued-fraction Green's function as the other use of the
Krylov machinery it serves (Sec. I).  For the removal (annihilation) part of
momentum k and spin sigma,

    G(z) = <psi0| c+_{k s} [z - (H - E0)]^-1 c_{k s} |psi0>,

and the addition part with c and c+ exchanged.  Starting Lanczos from
phi = c|psi0> / ||c psi0|| gives alpha_0 .. alpha_{m-1}, beta_0 .. beta_{m-2} and

    G(z) = ||c psi0||^2 / (z + E0 - alpha_0 - beta_0^2 / (z + E0 - alpha_1 - ...)),

exact when the recursion runs to the dimension of the Krylov space.

Operators on the momentum basis of ``momentum.py`` (bit i = occupation of k_i):
with the many-body state written as the up creators (descending momentum index)
to the left of the down creators (descending), c_{k up} and c+_{k up} carry
(-1)^(number of up particles above k), and the spin-down ones additionally
(-1)^(N_up).

Pins (tests/test_oracle_response.py): the continued fraction of a full-length
Lanczos run equals the spectral sum sum_n |<n|phi>|^2 / (z - (E_n - E0)) of the
dense target sector; removal plus addition weights of one k sum to 1
({c, c+} = 1); at U = 0 an occupied k has a single removal pole, at
E_n - E0 = -eps_k, of weight 1; and the momentum-space G_k(z)
equals the real-space <psi0| c+_k [z - (H - E0)]^-1 c_k |psi0> with
c_k = N^-1/2 sum_j e^(-i k r_j) c_j built from the site operators of Eq. 1.
"""
from __future__ import annotations

import numpy as np

from . import momentum as M


def sign_above(s: int, k: int) -> int:
    return -1 if bin(s >> (k + 1)).count("1") % 2 else 1


def apply_op(g: M.Grid, src_list: np.ndarray, dst_list: np.ndarray, op: str, spin: int, k: int,
             x: np.ndarray, n_up_src: int) -> np.ndarray:
    """y = c_{k spin} x (op 'c') or c+_{k spin} x (op 'cdag'), from a source sector list to a target one."""
    N = g.N
    pos = {int(s): i for i, s in enumerate(dst_list)}
    y = np.zeros(len(dst_list), dtype=np.result_type(x, np.float64))
    for i, s in enumerate(src_list):
        s = int(s)
        u, d = s >> N, s & ((1 << N) - 1)
        part = u if spin == 0 else d
        occupied = (part >> k) & 1
        if (op == "c") != bool(occupied):
            continue
        sgn = sign_above(part, k) * ((-1) ** n_up_src if spin == 1 else 1)
        part2 = part ^ (1 << k)
        t = (part2 << N) | d if spin == 0 else (u << N) | part2
        y[pos[t]] += sgn * x[i]
    return y


def sector_ground(g: M.Grid, t: float, tp: float, U: float, nu: int, nd: int, K: int):
    H = M.dense(M.KModel(g, t, tp, U, nu, nd, K))
    w, V = np.linalg.eigh(H)
    return w, V


def spectral_sum(Hdst: np.ndarray, phi: np.ndarray, E0: float, z: np.ndarray) -> np.ndarray:
    """sum_n |<n|phi>|^2 / (z - (E_n - E0)) for the (unnormalised) vector phi."""
    w, V = np.linalg.eigh(Hdst)
    amp = np.abs(V.T @ phi) ** 2
    return np.array([np.sum(amp / (zz - (w - E0))) for zz in z])


def lanczos_coefficients(H: np.ndarray, phi: np.ndarray, m: int):
    """Textbook Lanczos with full reorthogonalisation from phi / ||phi||: alpha[m], beta[m-1]."""
    v = phi / np.linalg.norm(phi)
    Vs = [v]
    al, be = [], []
    for j in range(m):
        w = H @ Vs[-1]
        a = float(np.vdot(Vs[-1], w).real)
        al.append(a)
        for q in Vs:
            w = w - np.vdot(q, w) * q
        for q in Vs:
            w = w - np.vdot(q, w) * q
        b = float(np.linalg.norm(w))
        if j + 1 == m or b < 1e-14:
            break
        be.append(b)
        Vs.append(w / b)
    return np.array(al), np.array(be)


def continued_fraction(alpha, beta, norm2: float, E0: float, z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=complex) + E0
    m = len(alpha)
    out = []
    for zz in z:
        g = zz - alpha[m - 1]
        for j in range(m - 2, -1, -1):
            g = zz - alpha[j] - beta[j] ** 2 / g
        out.append(norm2 / g)
    return np.array(out)
