"""Learned Lanczos start vectors: training and evaluation driver over the C ABI.

Not part of the paper.  The network (include/paradeisos_mlp.h) is trained on
ground states that the library computes itself (float32 Lanczos + Ritz vector)
at a few values of U, then used to build the start vector of the float64-grade
Lanczos solve at other U or another sector.  Training samples are basis states
drawn with probability |psi|^2 by the library's inverse-CDF sampler, targets
are log|psi| (shifted to zero mean per training problem) and the sign of psi
with the global sign fixed by the largest entry.  Everything numerical runs in
the library's kernels; torch provides memory and the random mini-batch choice.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Dict, List, Sequence

from . import _binding as B


@dataclass
class TrainingSet:
    states: "object"   # int64 CUDA tensor of combined strings
    t_log: "object"    # float32
    t_sign: "object"   # float32, +-1


@dataclass
class TrainReport:
    losses: List[float] = field(default_factory=list)
    seconds: float = 0.0


def ground_state(h: B.Handle, tol: float = 1e-6, maxit: int = 2000, seed: int = 0):
    """(E0, normalised float32 ground-state vector) by float32 Lanczos and the replayed Ritz vector."""
    E0, psi, _ = B.lanczos_ritz_vector_f32(h, maxit=maxit, tol=tol, seed=seed)
    return E0, psi


def sample(h: B.Handle, psi, n: int, seed: int = 0) -> TrainingSet:
    """n basis states drawn with probability psi^2, with their log-amplitude and sign targets
    (the library's inverse-CDF sampler, mlp_sample_training)."""
    states, t_log, t_sign = B.mlp_sample_training(h, psi.float().contiguous(), n, seed)
    return TrainingSet(states, t_log, t_sign)


def train(m: B.Mlp, sets: Sequence[TrainingSet], steps: int, batch: int = 32768, lr: float = 2e-3,
          lam: float = 1.0, seed: int = 0) -> TrainReport:
    import torch
    states = torch.cat([s.states for s in sets])
    t_log = torch.cat([s.t_log for s in sets])
    t_sign = torch.cat([s.t_sign for s in sets])
    g = torch.Generator(device=states.device)
    g.manual_seed(seed)
    w = torch.full((batch,), 1.0 / batch, dtype=torch.float32, device=states.device)
    rep = TrainReport()
    t0 = time.perf_counter()
    for it in range(steps):
        sel = torch.randint(0, states.numel(), (batch,), generator=g, device=states.device)
        _, loss = B.mlp_gradient(m, states[sel].contiguous(), t_log[sel].contiguous(), t_sign[sel].contiguous(), w, lam)
        step_lr = lr * (0.5 * (1 + __import__("math").cos(__import__("math").pi * it / steps)))
        B.mlp_adam_step(m, max(step_lr, lr * 0.02))
        if it % 25 == 0 or it == steps - 1:
            rep.losses.append(float(loss.item()))
    torch.cuda.synchronize()
    rep.seconds = time.perf_counter() - t0
    return rep


def overlap(m: B.Mlp, h: B.Handle, psi) -> float:
    """|<v0 / |v0|, psi>| of the network's start vector with a normalised reference vector."""
    import torch
    v = B.mlp_start_vector(m, h, torch.float32).double()
    return float((torch.dot(v, psi.double()) / v.norm()).abs().item())


def solve_from(h: B.Handle, dtype, v0=None, seed: int = 0, tol: float = 1e-10, fp64_finish=False) -> Dict:
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = B.lanczos_ground_state(h, maxit=3000, tol=tol, dtype=dtype, v0=v0, seed=seed, fp64_finish=fp64_finish,
                               raise_on_error=False)
    torch.cuda.synchronize()
    return {"E0": r.E0, "iterations": r.iterations, "iterations_f32": r.iterations_f32, "converged": r.converged,
            "seconds": time.perf_counter() - t0}


def _timed_start(m: B.Mlp, h: B.Handle, dtype):
    """The network's start vector in `dtype` and the seconds its build took."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    v = B.mlp_start_vector(m, h, dtype)
    torch.cuda.synchronize()
    return v, time.perf_counter() - t0


def tune(h: B.Handle):
    """Autotune the H·v launch configuration of every vector type on this handle (setup, not timed)."""
    import torch
    for dt in (torch.float64, torch.int64, torch.float32):
        x = torch.zeros(h.D, dtype=dt, device="cuda")
        y = torch.empty_like(x)
        B.hubbard_autotune(h, x, y, reps=2)
        del x, y
    torch.cuda.empty_cache()


def compare(m: B.Mlp, h: B.Handle, psi=None, seeds=(0,)) -> Dict:
    """Iterations and wall time to E0 at 1e-10: learned start vs random starts (float64 and fixed point),
    plus the mixed float32 + fixed-point solve from the learned start.  A learned run's seconds include
    building its start vector on the GPU; every run uses the handle's autotuned H·v."""
    import torch
    tune(h)
    out = {"random_f64": [solve_from(h, torch.float64, seed=s) for s in seeds]}
    out["random_fx64"] = [solve_from(h, torch.int64, seed=s) for s in seeds]
    for name, dt, finish in (("learned_f64", torch.float64, False), ("learned_fx64", torch.int64, False),
                             ("learned_mixed_f32_fx64", torch.float32, "fx64")):
        v0, t_build = _timed_start(m, h, dt)
        r = solve_from(h, dt, v0=v0, fp64_finish=finish)
        r["seconds"] += t_build
        r["start_vector_seconds"] = t_build
        out[name] = r
        del v0
    out["start_vector_seconds"] = out["learned_f64"]["start_vector_seconds"]
    if psi is not None:
        out["overlap"] = overlap(m, h, psi)
    return out
