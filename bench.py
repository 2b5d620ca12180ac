"""Benchmark: matrix-free Hubbard H·v + Lanczos step on the 4x4 t-t' cluster (GB300).

Workload (float64): 4x4 periodic square lattice, nearest-neighbour t = 1 and
next-nearest t' = -0.3, U = 8, half filling N_up = N_dn = 8, D = 12870^2 =
165,636,900 basis states.  One step = one three-term Lanczos iteration through
the C ABI (`lanczos_step`): H·v with Paradeisos-ranked hop tables, the
alpha/beta reductions and the vector updates.  The float64 vectors (1.33 GB
each) are larger than L2, so no flush is needed between steps.

Printed (one JSON line on rank 0): Gstates/s of the whole step, the roofline of
the dominant kernel (H·v: 16 algorithmic bytes per state, read x + write y),
end-to-end throughput with host buffers, time to E0 at 1e-10 for plain float64
and for mixed precision, and the CPU oracle timed on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # the benchmark workload
    "hubbard4x4_half": {"workload": "hubbard_4x4_tp-0.3_U8_half_filling", "L": 16,
                        "lattice": "4x4 periodic, t=1, t'=-0.3", "U": 8.0, "N_up": 8, "N_dn": 8, "D": 165636900},
    # smaller sector of the same cluster, for profiler captures (0.5 GB per vector, still > L2)
    "hubbard4x4_n6": {"workload": "hubbard_4x4_tp-0.3_U8_6up_6dn", "L": 16,
                      "lattice": "4x4 periodic, t=1, t'=-0.3", "U": 8.0, "N_up": 6, "N_dn": 6, "D": 64128064},
    # one momentum sector of the benchmark cluster (Sec. IV A, Eq. 4): total momentum K = (0, 0)
    "kspace4x4_K00": {"workload": "hubbard_4x4_tp-0.3_U8_half_filling_momentum_K00", "L": 16,
                      "lattice": "4x4 periodic, t=1, t'=-0.3, momentum basis", "U": 8.0, "N_up": 8, "N_dn": 8,
                      "K": [0, 0], "D": None,
                      "l2": "83 MB per vector; a Lanczos step touches three (249 MB > L2), no flush"},
    # the precision workload: 18-site tilted cluster, run with --dtype f32 (float32 vectors)
    "tilted18_half": {"workload": "hubbard_18site_tilted_U6_half_filling", "L": 18,
                      "lattice": "18-site tilted square, lattice vectors (3,3), (3,-3), t=1", "U": 6.0,
                      "N_up": 9, "N_dn": 9, "D": 2363904400},
}
COMMON = {"vector_dtype": "f64",
          "step": "one three-term Lanczos iteration (H·v + alpha/beta reductions + vector updates)",
          "l2": "inputs larger than L2 (>= 0.5 GB per vector), no flush", "parallelism": "replicas"}
METRIC = "H·v Gstates/s (Lanczos step)"
UNIT = "Gstates/s"
HV_BYTES_PER_STATE = 16  # float64: read x once, write y once
MIXED_F32_TOL_EXP = -6  # residual (10^x max(1,|theta|)) at which a kept-basis float32 phase hands over


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="hubbard4x4_half",
                   choices=sorted(WORKLOADS) + ["batch64", "learned4x4", "start4x4", "green4x4", "ceilings", "tcgemm"])
    p.add_argument("--dtype", default="fx64", choices=["f64", "fx64", "f32"],
                   help="Krylov vector type: fixed-point int64 (default, float64-grade accuracy without the "
                        "float64 pipe), float64 (float64 FMAs), float32")
    p.add_argument("--no-solve", action="store_true", help="skip the time-to-E0 runs")
    p.add_argument("--no-autotune", dest="autotune", action="store_false",
                   help="keep the library's default H·v launch configuration")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--no-extra", action="store_true",
                   help="skip the other configurations (batch, momentum sector, 18-site, learned start)")
    p.add_argument("--basis", default="hubbard4x4_half", choices=sorted(WORKLOADS),
                   help="basis of the start4x4 workload (the start vector is built over all of it)")
    p.add_argument("--hv-config", default=None,
                   help="JSON H·v launch configuration (keys of hubbard_set_hv_config) instead of the autotuner")
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def source_hash():
    """Hash of the file that holds the H·v kernel bodies (the row pass and the spin-up pass):
    the committed DRAM capture is only used while these are the kernels it measured."""
    h = hashlib.sha256()
    h.update(open(os.path.join(ROOT, "paper_1707_03974_gb300", "csrc", "pd_hv_body.cuh"), "rb").read())
    return h.hexdigest()[:16]


def hv_kernel_key(dtype: str, cfg: dict) -> str:
    """Name of the H·v launch(es) under a configuration: one fused kernel, or the row pass
    followed by the column-blocked spin-up pass (their DRAM bytes are summed)."""
    rows = cfg.get("rows_per_cta") or {"f64": 2, "fx64": 2, "f32": 4}[dtype]
    base = {"f64": f"k_hv<{rows},double", "fx64": f"k_hv_fx<{rows},2", "f32": f"k_hv<{rows},float"}[dtype]
    if not cfg.get("split"):
        return base + ",true>"
    up = {"f64": "k_hv_up<{r},double>", "fx64": "k_hv_fx_up<{r},2>", "f32": "k_hv_up<{r},float>"}[dtype]
    # the fixed-point row pass runs on the warp-blocked spin-down table
    row = {"fx64": f"k_hv_fx_wb<{rows},2> (row pass)", "f32": f"k_hv_f_wb<{rows}> (row pass)",
           "f64": f"{base},false> (row pass)"}[dtype]
    return (f"{row} + " + up.format(r=cfg.get("up_rows") or 1)
            + f" (block {cfg.get('up_block') or 256}, {cfg.get('up_threads') or 1024} threads)")


def ncu_traffic(kernel_key: str):
    """DRAM bytes per launch of the H·v kernel from the committed ncu summary, if it matches this source."""
    p = os.path.join(ROOT, "profiles", "hv_dram_traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    if d.get("source_hash") != source_hash() or d.get("kernel") != kernel_key:
        return None
    return d.get("dram_bytes_per_launch")


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Largest value over all ranks (the job's time is its slowest replica's)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(states_per_replica: int, world: int, ms_per_step: float) -> float:
    """Whole-job Gstates/s of `world` independent replicas (weak scaling: each does a full step)."""
    return world * states_per_replica / (ms_per_step * 1e-3) / 1e9


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.remove(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ our arm

def run_ours(args, world, rank, local):
    import torch
    import torch.distributed as dist

    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_1707_03974_gb300.build import build
    if rank == 0:
        build()
    if world > 1:
        dist.barrier()
    import paper_1707_03974_gb300 as pd
    import workloads as wl

    dev = torch.device("cuda", local)
    wk = dict(WORKLOADS[args.workload])
    cl = wl.tilted_18() if wk["L"] == 18 else wl.square_periodic(4, 1.0, -0.3)
    if "K" in wk:
        h = pd.Handle.momentum(4, 4, 1.0, -0.3, wk["U"], wk["N_up"], wk["N_dn"], *wk["K"])
    else:
        h = pd.Handle(cl.L, cl.bonds, cl.t, wk["U"], wk["N_up"], wk["N_dn"])
    D = h.D
    wk["D"] = D
    stream = torch.cuda.current_stream()
    # inputs: a normalised random start vector (plumbing, outside the timed region)
    g = torch.Generator(device=dev)
    g.manual_seed(1234 + rank)
    vdt = {"f64": torch.float64, "fx64": torch.int64, "f32": torch.float32}[args.dtype]
    x0 = torch.empty(D, dtype=torch.float64, device=dev)
    x0.uniform_(-1.0, 1.0, generator=g)
    x0 /= x0.norm()
    if args.dtype == "fx64":
        x0 = pd.hubbard_convert(h, x0, torch.int64)
    V = [x0.to(vdt), torch.empty(D, dtype=vdt, device=dev), torch.empty(D, dtype=vdt, device=dev)]
    del x0
    nsteps = args.warmup + args.steps
    alpha = torch.zeros(nsteps + 1, dtype=torch.float64, device=dev)
    beta = torch.zeros(nsteps + 1, dtype=torch.float64, device=dev)
    scratch = torch.empty(pd.lanczos_step_scratch_bytes(h), dtype=torch.uint8, device=dev)
    pd.hubbard_apply(h, V[0], V[1])  # builds the per-spin tables (setup, untimed)
    if args.hv_config:
        pd.hubbard_set_hv_config(h, vdt, **json.loads(args.hv_config))
        tuned = pd.hubbard_get_hv_config(h, vdt)
    else:
        tuned = pd.hubbard_autotune(h, V[0], V[1], reps=2) if args.autotune else pd.hubbard_get_hv_config(h, vdt)
    torch.cuda.synchronize()

    launches = ctypes.c_uint32(0)
    ev_hv = []

    def step(j, timed):
        iv, ip, iw = j % 3, (j - 1) % 3, (j + 1) % 3
        vprev = V[ip] if j > 0 else None
        bprev = beta[j - 1:j] if j > 0 else None
        e0 = e1 = None
        if timed:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)  # materialise the CUDA events; the library re-records them around H·v
            e1.record(stream)
            ev_hv.append((e0, e1))
        pd.lanczos_step(h, V[iv], vprev, V[iw], bprev, alpha[j:j + 1], beta[j:j + 1], scratch, e0, e1,
                        launches if timed else None)

    for j in range(args.warmup):
        step(j, False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.4)
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t_start.record(stream)
    for j in range(args.warmup, nsteps):
        step(j, True)
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    ms = t_start.elapsed_time(t_end) / args.steps
    hv_ms = statistics.mean(a.elapsed_time(b) for a, b in ev_hv)
    ms = max_over_ranks(ms, world, dev)
    ab = beta[:nsteps].cpu().numpy()
    sane = bool((ab > 0).all())

    # the two passes of the H·v timed separately (events between them), for the on-chip rooflines
    pass_ms = hv_pass_times(pd, h, V[nsteps % 3], V[(nsteps + 1) % 3], torch)
    ceil = measure_ceilings(pd, torch, dev)

    # end to end through the public API with host buffers: every step copies its input vector
    # from pinned host memory and reads alpha, beta back to the host; w stays on the device.
    # Each step is the general three-term step (with vprev and beta_prev, like the timed
    # region).  The copies run on a second stream into a ring of three device buffers, so the
    # copy for step j + 1 overlaps the compute of step j; step j waits for its own copy, and
    # a buffer is refilled only after the last step that read it (as v, then as vprev)
    host_v = pd.host_empty(D, vdt)  # page-locked, on huge pages (hb_host_alloc)
    host_v.copy_(V[nsteps % 3])
    host_ab = torch.empty(2, dtype=torch.float64, pin_memory=True)
    e2e_steps = max(3, args.steps)
    copy_stream = torch.cuda.Stream(device=dev)
    ring = (V[0], V[2], torch.empty(D, dtype=vdt, device=dev))
    w_out = V[1]
    ring[2].copy_(V[0])
    bprev_e2e = beta[nsteps - 1:nsteps]
    copied = [torch.cuda.Event() for _ in range(3)]
    used = [torch.cuda.Event() for _ in range(3)]

    def issue_copy(j):
        b = j % 3
        if j >= 2:  # ring[b] was last read (as vprev) by step j - 2
            copy_stream.wait_event(used[b])
        with torch.cuda.stream(copy_stream):
            ring[b].copy_(host_v, non_blocking=True)
        copied[b].record(copy_stream)

    torch.cuda.synchronize()
    # the link's copy rate for this buffer on its own (best of three), to read the end-to-end figure by
    h2d_ms = []
    for _ in range(3):
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        ring[2].copy_(host_v, non_blocking=True)
        c1.record(stream)
        torch.cuda.synchronize()
        h2d_ms.append(c0.elapsed_time(c1))
    h2d_gbs = D * host_v.element_size() / (min(h2d_ms) * 1e-3) / 1e9
    ring[2].copy_(V[0])
    torch.cuda.synchronize()
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0e.record(stream)
    copy_stream.wait_stream(stream)
    issue_copy(0)
    for j in range(e2e_steps):
        if j + 1 < e2e_steps:
            issue_copy(j + 1)
        b, bp = j % 3, (j - 1) % 3
        stream.wait_event(copied[b])
        pd.lanczos_step(h, ring[b], ring[bp], w_out, bprev_e2e, alpha[0:1], beta[0:1], scratch)
        used[bp].record(stream)  # ring[bp] has been read for the last time (as vprev)
        host_ab[0:1].copy_(alpha[0:1], non_blocking=True)
        host_ab[1:2].copy_(beta[0:1], non_blocking=True)
    t1e.record(stream)
    torch.cuda.synchronize()
    e2e_ms = t0e.elapsed_time(t1e) / e2e_steps
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    host_bytes = host_v.element_size()
    del ring, w_out

    # the same step with plain float64 vectors and float64 FMAs, for comparison
    plain = None
    if args.dtype != "f64" and not args.no_solve:
        del host_v
        for t in V:
            t.data = torch.empty(0, device=dev)
        torch.cuda.empty_cache()
        P = [torch.empty(D, dtype=torch.float64, device=dev) for _ in range(3)]
        P[0].uniform_(-1.0, 1.0, generator=g)
        P[0] /= P[0].norm()
        if args.autotune:  # the float64 comparison gets its own tuned launch configuration
            pd.hubbard_autotune(h, P[0], P[1], reps=2)
        for j in range(args.warmup):
            pd.lanczos_step(h, P[j % 3], P[(j - 1) % 3] if j else None, P[(j + 1) % 3],
                            beta[j - 1:j] if j else None, alpha[j:j + 1], beta[j:j + 1], scratch)
        ev = []
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for j in range(args.warmup, nsteps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            e1.record(stream)
            ev.append((e0, e1))
            pd.lanczos_step(h, P[j % 3], P[(j - 1) % 3], P[(j + 1) % 3], beta[j - 1:j], alpha[j:j + 1], beta[j:j + 1],
                            scratch, e0, e1)
        a1.record(stream)
        torch.cuda.synchronize()
        pms = a0.elapsed_time(a1) / args.steps
        phv = statistics.mean(x.elapsed_time(y) for x, y in ev)
        plain = {"ms_per_step": round(pms, 4), "hv_ms": round(phv, 4), "value": round(job_throughput(D, 1, pms), 4),
                 "hv_roofline_frac": round(16 * D / (phv * 1e-3) / 1e9 / (measured_peaks() or {}).get("hbm_gbs", 6800.0), 4)}
        del P
        torch.cuda.empty_cache()
    else:
        del host_v

    solve = None
    if not args.no_solve and rank == 0 and args.workload in ("hubbard4x4_half", "kspace4x4_K00"):
        solve = time_to_e0(pd, h, torch, tune=args.autotune)
    if not args.no_solve and rank == 0 and args.workload == "tilted18_half":
        solve = precision_e0(pd, h, torch)
    del V
    h.close()
    torch.cuda.empty_cache()
    # the other configurations of the method, measured on rank 0 after the timed steps
    extra = {}
    if args.workload == "hubbard4x4_half" and rank == 0 and not args.no_solve and not args.no_extra:
        extra["batch64"] = measure_batch64(pd, torch, wl, 10, 3, torch.int64)
        extra["kspace4x4_K00"] = measure_kspace(pd, torch)
        extra["tilted18_f32"] = measure_tilted18_f32(pd, torch, wl)
        extra["learned4x4"] = measure_learned_quick(pd, torch, wl)
        extra["maps"] = measure_maps(pd, torch, wl)
    if world > 1:
        dist.barrier()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return None

    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs") if peaks else 6800.0
    bps = HV_BYTES_PER_STATE if args.dtype != "f32" else 8
    achieved = bps * D / (hv_ms * 1e-3) / 1e9
    kname = hv_kernel_key(args.dtype, tuned)
    if "K" in wk:  # momentum sector: one row-factorised kernel
        kname = {"fx64": "k_k_hv_rows2<int64>", "f64": "k_k_hv_rows2<double>", "f32": "k_k_hv_rows2<float>"}[args.dtype]
    traffic = ncu_traffic(kname)
    out = {
        "metric": METRIC, "value": round(job_throughput(D, world, ms), 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"f64": "f64", "fx64": "int64", "f32": "f32"}[args.dtype],
        "precision_note": {"fx64": "64-bit fixed point, 2^-F resolution (F from hubbard_fixed_point_bits, 53 here); "
                                   "H·v within 1e-12 of the float64 oracle, E0 within 1e-10 (tests)",
                           "f64": "IEEE float64 vectors and FMAs", "f32": "float32 vectors, float64 scalars"}[args.dtype],
        "data": "synthetic (seeded random start vector)",
        "config": {**COMMON, **wk, "vector_dtype": args.dtype},
        "hv_ms": round(hv_ms, 4), "hv_gstates_per_s": round(D / (hv_ms * 1e-3) / 1e9, 4),
        "hv_config": tuned,
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     # DRAM bytes the kernels actually move (committed ncu capture) over the same time
                     "dram_gbs": round(traffic / (hv_ms * 1e-3) / 1e9, 1) if traffic else None,
                     "kernel": kname, "bytes_per_state": bps,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks else "fallback 6800 GB/s"},
        "e2e": {"value": round(job_throughput(D, world, e2e_ms), 4), "unit": UNIT,
                "h2d_bytes_per_step": D * host_bytes, "d2h_bytes_per_step": 16,
                "step": "the general three-term step (v from the host, vprev and beta_prev resident), as timed above",
                "output": "alpha and beta are read back each step; w stays on the device",
                "overlap": "each step's input copy runs on a second stream while the previous step computes",
                "host_buffer": "hb_host_alloc: page-locked, 2 MiB-aligned, advised for huge pages, on the host NUMA "
                               "node nearest the GPU",
                "steps": e2e_steps, "h2d_gbs_alone": round(h2d_gbs, 1)},
        "gpu_launches": int(launches.value),
        "clocks": clk,
        "recurrence_sane": sane,
    }
    if "K" not in wk:
        out["roofline"]["onchip"] = onchip_roofline(cl, wk, args.dtype, tuned, pass_ms, ceil, D, peak)
    out["ceilings"] = ceil
    if plain:
        out["plain_f64_step"] = plain
    if solve:
        out["time_to_E0"] = solve
    if extra:
        out["other_workloads"] = extra
    if not args.no_cpu and args.workload == "hubbard4x4_half":
        out["cpu_baseline"] = cpu_baseline(sample_rows=20000)
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    return out


def hv_pass_times(pd, h, x, y, torch, reps=10):
    """Mean ms of the H·v's row pass and spin-up pass over reps applications (events between them)."""
    evs = []
    for _ in range(reps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        pd.hubbard_apply_timed(h, x, y, *e)
        evs.append(e)
    torch.cuda.synchronize()
    row = statistics.mean(a.elapsed_time(b) for a, b, _ in evs)
    up = statistics.mean(b.elapsed_time(c) for _, b, c in evs)
    return {"row_pass_ms": round(row, 4), "up_pass_ms": round(up, 4)}


def measure_ceilings(pd, torch, dev):
    """On-chip rates of this GPU, measured by the library's probe kernels (hb_measure_ceilings)."""
    buf = torch.empty(1 << 31, dtype=torch.uint8, device=dev)
    c = pd.hb_measure_ceilings(buf)
    del buf
    torch.cuda.empty_cache()
    keep = ("sm_clock_mhz", "fp64_fma_tflops", "fp32_fma_tflops", "int32_add_tops", "int64_add_tops",
            "smem_seq16_gbs", "smem_gather8_gbs", "smem_gather16_gbs", "smem_gather8_clk", "smem_gather16_clk",
            "l1_gbs", "l2_gbs", "hbm_read_gbs")
    return {k: round(c[k], 2) for k in keep}


def hops_per_string(cl, n: int) -> float:
    """Average hops of one spin string with n particles: a bond (i, j) moves a particle exactly when one
    of its two sites is occupied, which 2 C(L-2, n-1) of the C(L, n) strings have."""
    import math
    if n <= 0 or n >= cl.L:
        return 0.0
    return len(cl.bonds) * 2 * math.comb(cl.L - 2, n - 1) / math.comb(cl.L, n)


def onchip_roofline(cl, wk, dtype, cfg, pass_ms, ceil, D, hbm_peak):
    """Rooflines of the two H·v passes against the measured on-chip ceilings.

    Row pass: every spin-down hop of every state reads one vector element from the staged rows in
    shared memory (z_dn elements per state); the ceiling is the conflict-free shared-memory load
    rate (the random-gather rate is given beside it).  Spin-up pass: every spin-up hop reads one
    element of a neighbouring row from L2 (z_up per state), plus y read and written once; the
    ceiling is the L2 load rate."""
    es = 4 if dtype == "f32" else 8
    z_dn, z_up = hops_per_string(cl, wk["N_dn"]), hops_per_string(cl, wk["N_up"])
    out = {"z_dn": round(z_dn, 3), "z_up": round(z_up, 3), "element_bytes": es}
    if not cfg.get("split"):
        out["note"] = "one-kernel form: no per-pass split"
        return out
    row_b = D * z_dn * es
    up_b = D * (z_up * es + 2 * es)
    r_gbs = row_b / (pass_ms["row_pass_ms"] * 1e-3) / 1e9
    u_gbs = up_b / (pass_ms["up_pass_ms"] * 1e-3) / 1e9
    out["row_pass"] = {"ms": pass_ms["row_pass_ms"], "bound": "shared memory", "bytes": int(row_b),
                       "achieved_gbs": round(r_gbs, 1), "ceiling_gbs": ceil["smem_seq16_gbs"],
                       "frac": round(r_gbs / ceil["smem_seq16_gbs"], 4),
                       "random_gather16_gbs": ceil["smem_gather16_gbs"],
                       "frac_vs_random_gather16": round(r_gbs / ceil["smem_gather16_gbs"], 4)}
    out["up_pass"] = {"ms": pass_ms["up_pass_ms"], "bound": "L2", "bytes": int(up_b),
                      "achieved_gbs": round(u_gbs, 1), "ceiling_gbs": ceil["l2_gbs"],
                      "frac": round(u_gbs / ceil["l2_gbs"], 4)}
    # the H·v can be no faster than both passes at their ceilings; the HBM fraction it would then reach
    floor = row_b / (ceil["smem_seq16_gbs"] * 1e9) + up_b / (ceil["l2_gbs"] * 1e9)
    out["hv_floor_ms"] = round(floor * 1e3, 4)
    out["hbm_frac_at_floor"] = round(2 * es * D / floor / 1e9 / hbm_peak, 4)
    return out


def time_to_e0(pd, h, torch, tune=True):
    """Wall time to E0 at 1e-10: plain float64 Lanczos vs float32 vectors + float64 finish (same seed)."""
    gold = None
    try:
        gold = json.load(open(os.path.join(ROOT, "tests", "golden", "oracle_energies.json")))["square4x4_tp-0.3_U8_8_8"]["E0"]
    except Exception:
        pass
    if tune:  # the mixed runs' float32 phase on its own autotuned H·v (float64 and fixed point are tuned above)
        xa = torch.zeros(h.D, dtype=torch.float32, device="cuda")
        ya = torch.empty_like(xa)
        pd.hubbard_autotune(h, xa, ya, reps=1)
        del xa, ya
        torch.cuda.empty_cache()
    res = {}
    # the float32 phase with its Krylov vectors kept in HBM (4 D bytes each; 160 of them for the 4x4
    # workload is 106 GB): its Ritz vector is one combination pass instead of a replay of every step
    keep = 160 if 161 * 4 * h.D < 0.6 * torch.cuda.get_device_properties(0).total_memory else 0
    for name, kw in (("plain_f64", dict(dtype=torch.float64)),
                     ("fx64", dict(dtype=torch.int64)),
                     ("mixed_f32_f64finish", dict(dtype=torch.float32, fp64_finish="f64")),
                     ("mixed_f32_fx64finish", dict(dtype=torch.float32, fp64_finish="fx64")),
                     ("mixed_f32_fx64finish_kept_basis", dict(dtype=torch.float32, fp64_finish="fx64",
                                                              store_basis=keep, f32_tol_exp=MIXED_F32_TOL_EXP))):
        if kw.get("store_basis", 1) == 0:
            continue
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = pd.lanczos_ground_state(h, maxit=3000, tol=1e-10, seed=0, raise_on_error=False, **kw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        res[name] = {"seconds": round(dt, 4), "iterations": r.iterations, "iterations_f32": r.iterations_f32,
                     "E0": r.E0, "residual": r.residual, "converged": r.converged,
                     "abs_err_vs_oracle": (abs(r.E0 - gold) if gold is not None else None)}
    return res


def precision_e0(pd, h, torch, runs=("fx64", "plain_f64", "f32_only", "mixed_f32_fx64finish")):
    """18-site tilted cluster: E0 with float32 vectors (float64 scalars) and with the float32 phase plus a
    fixed-point finish, against the float64-grade fixed-point run of the same cluster and seed, and the
    plain float64 solve for time.  Each vector type's H·v launch configuration is autotuned first.
    `runs` picks a subset; errors are stated against the first run's E0."""
    for dt in (torch.int64, torch.float64):
        xa = torch.zeros(h.D, dtype=dt, device="cuda")
        ya = torch.empty_like(xa)
        pd.hubbard_autotune(h, xa, ya, reps=1)
        del xa, ya
        torch.cuda.empty_cache()
    res = {}
    kinds = {"fx64": dict(dtype=torch.int64, tol=1e-10),
             "plain_f64": dict(dtype=torch.float64, tol=1e-10),
             "f32_only": dict(dtype=torch.float32, tol=1e-6),
             "mixed_f32_fx64finish": dict(dtype=torch.float32, fp64_finish="fx64", tol=1e-10)}
    for name in runs:
        kw = kinds[name]
        torch.cuda.empty_cache()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = pd.lanczos_ground_state(h, maxit=3000, seed=0, raise_on_error=False, **kw)
        torch.cuda.synchronize()
        res[name] = {"seconds": round(time.perf_counter() - t0, 3), "iterations": r.iterations,
                     "iterations_f32": r.iterations_f32, "E0": r.E0, "residual": r.residual, "converged": r.converged}
    ref = res[runs[0]]["E0"]
    for v in res.values():
        v["abs_err_vs_" + runs[0]] = abs(v["E0"] - ref)
    return res


def cpu_baseline(sample_rows: int):
    """The CPU oracle as it stands, on the GPU machine's host cores: one full H·v of the workload by the
    tensor-product oracle in C (OpenMP over all host cores), plus the definition itself (sorted list +
    binary search, float64, 1 core) on a bounded sample of rows."""
    import numpy as np

    import workloads as wl
    from oracle import build as oracle_build
    from oracle.basis import Basis
    from oracle.hamiltonian import KronOperator, Model, apply_rows
    from oracle.lanczos import start_vector

    cl = wl.square_periodic(4, 1.0, -0.3)
    m = Model.from_cluster(cl, 8.0, 8, 8)
    x = start_vector(0, 165636900)
    oracle_build.build()
    op = KronOperator(m)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    t0 = time.perf_counter()
    op(x)
    dt_all = time.perf_counter() - t0
    kron = {"value": round(op.D / dt_all / 1e9, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one full H·v (D = {op.D:,}) by the tensor-product oracle in C, OpenMP over "
                      f"{cores} host threads; {dt_all:.2f} s"}
    del op
    b = Basis(16, 8, 8)
    rng = np.random.default_rng(0)
    rows = np.sort(rng.integers(0, b.D, sample_rows))
    t0 = time.perf_counter()
    apply_rows(m, b, x, rows)
    dt = time.perf_counter() - t0
    kron["definition_1core"] = {
        "value": round(sample_rows / dt / 1e9, 9), "unit": UNIT, "cores": 1, "kind": "oracle",
        "sample": f"H·v rows by definition (binary search in the sorted 165,636,900-entry list) for "
                  f"{sample_rows} random rows of the same workload; {dt:.2f} s"}
    return kron


# ------------------------------------------------------------------ reference arm: the CPU oracle

def run_reference(args, world, rank):
    if rank != 0:
        return None
    import numpy as np

    import workloads as wl
    from oracle.basis import Basis
    from oracle.hamiltonian import Model, apply_rows
    from oracle.lanczos import start_vector

    cl = wl.square_periodic(4, 1.0, -0.3)
    m = Model.from_cluster(cl, 8.0, 8, 8)
    b = Basis(16, 8, 8)
    x = start_vector(0, b.D)
    v_prev = start_vector(1, b.D)
    rng = np.random.default_rng(0)
    sample = 10000
    times = []
    for j in range(args.warmup + args.steps):
        rows = np.sort(rng.integers(0, b.D, sample))
        t0 = time.perf_counter()
        w = apply_rows(m, b, x, rows)  # H·v on the sampled rows
        w -= 0.5 * v_prev[rows]           # recurrence on the same rows
        a = float(np.dot(w, x[rows]))
        w -= a * x[rows]
        float(np.linalg.norm(w))
        dt = time.perf_counter() - t0
        if j >= args.warmup:
            times.append(dt)
    ms = 1e3 * statistics.mean(times)
    value = sample / (ms * 1e-3) / 1e9
    out = {"metric": METRIC, "value": round(value, 9), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
           "config": {**WORKLOADS["hubbard4x4_half"], **COMMON},
           "impl": "reference",
           "cpu_baseline": {"value": round(value, 9), "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"{sample} random rows per step of the same workload, oracle H·v by "
                                      f"binary search plus the recurrence on those rows"},
           "e2e": {"value": round(value, 9), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return out


def measure_kspace(pd, torch, steps: int = 10):
    """The K = (0,0) momentum sector of the 4x4 t-t' cluster (Sec. IV A, Eq. 4) in fixed point: H·v and
    Lanczos step times, the H·v against HBM (16 B per sector state), and the time to E0 at 1e-10."""
    h = pd.Handle.momentum(4, 4, 1.0, -0.3, 8.0, 8, 8, 0, 0)
    D = h.D
    V = [torch.zeros(D, dtype=torch.int64, device="cuda") for _ in range(3)]
    x0 = torch.empty(D, dtype=torch.float64, device="cuda").uniform_(-1, 1)
    V[0].copy_(pd.hubbard_convert(h, x0 / x0.norm(), torch.int64))
    del x0
    a = torch.zeros(steps + 4, dtype=torch.float64, device="cuda")
    bt = torch.zeros(steps + 4, dtype=torch.float64, device="cuda")
    scratch = torch.empty(pd.lanczos_step_scratch_bytes(h), dtype=torch.uint8, device="cuda")
    ev = []
    for j in range(steps + 3):
        e = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) if j >= 3 else (None, None)
        if j >= 3:
            e[0].record()
            e[1].record()
            ev.append(e)
        pd.lanczos_step(h, V[j % 3], V[(j - 1) % 3] if j else None, V[(j + 1) % 3], bt[j - 1:j] if j else None,
                        a[j:j + 1], bt[j:j + 1], scratch, e[0], e[1])
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for j in range(3, steps + 3):
        pd.lanczos_step(h, V[j % 3], V[(j - 1) % 3], V[(j + 1) % 3], bt[j - 1:j], a[j:j + 1], bt[j:j + 1], scratch)
    t1.record()
    torch.cuda.synchronize()
    hv_ms = statistics.mean(x.elapsed_time(y) for x, y in ev)
    step_ms = t0.elapsed_time(t1) / steps
    del V
    torch.cuda.synchronize()
    t = time.perf_counter()
    r = pd.lanczos_ground_state(h, maxit=3000, tol=1e-10, seed=0, dtype=torch.int64, raise_on_error=False)
    torch.cuda.synchronize()
    e0_s = time.perf_counter() - t
    peak = (measured_peaks() or {}).get("hbm_gbs", 6800.0)
    gbs = 16 * D / (hv_ms * 1e-3) / 1e9
    h.close()
    return {"workload": "hubbard_4x4_tp-0.3_U8_half_filling_momentum_K00", "D": D, "hv_ms": round(hv_ms, 4),
            "step_ms": round(step_ms, 4), "hv_gstates_per_s": round(D / (hv_ms * 1e-3) / 1e9, 3),
            "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(gbs / peak, 4), "kernel": "k_k_hv_rows2<int64>", "bytes_per_state": 16},
            "time_to_E0_fx64": {"seconds": round(e0_s, 4), "iterations": r.iterations, "E0": r.E0,
                                "converged": r.converged}}


def measure_tilted18_f32(pd, torch, wl, steps: int = 5, with_solve: bool = True):
    """The 18-site tilted cluster (U = 6, (9,9), D = 2,363,904,400) with float32 vectors and float64
    scalars: one Lanczos step and its H·v on the autotuned launch configuration."""
    cl = wl.tilted_18()
    h = pd.Handle(cl.L, cl.bonds, cl.t, 6.0, 9, 9)
    D = h.D
    V = [torch.zeros(D, dtype=torch.float32, device="cuda") for _ in range(3)]
    V[0].uniform_(-1.0, 1.0)
    V[0] /= V[0].norm()
    pd.hubbard_autotune(h, V[0], V[1], reps=1)
    a = torch.zeros(steps + 4, dtype=torch.float64, device="cuda")
    bt = torch.zeros(steps + 4, dtype=torch.float64, device="cuda")
    scratch = torch.empty(pd.lanczos_step_scratch_bytes(h), dtype=torch.uint8, device="cuda")
    ev = []
    for j in range(steps + 2):
        e = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) if j >= 2 else (None, None)
        if j >= 2:
            e[0].record()
            e[1].record()
            ev.append(e)
        pd.lanczos_step(h, V[j % 3], V[(j - 1) % 3] if j else None, V[(j + 1) % 3], bt[j - 1:j] if j else None,
                        a[j:j + 1], bt[j:j + 1], scratch, e[0], e[1])
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for j in range(2, steps + 2):
        pd.lanczos_step(h, V[j % 3], V[(j - 1) % 3], V[(j + 1) % 3], bt[j - 1:j], a[j:j + 1], bt[j:j + 1], scratch)
    t1.record()
    torch.cuda.synchronize()
    hv_ms = statistics.mean(x.elapsed_time(y) for x, y in ev)
    step_ms = t0.elapsed_time(t1) / steps
    peak = (measured_peaks() or {}).get("hbm_gbs", 6800.0)
    gbs = 8 * D / (hv_ms * 1e-3) / 1e9
    del V, scratch
    torch.cuda.empty_cache()
    # time to E0 at 1e-10 from the same seed: plain float64 against the float32 phase with a
    # fixed-point finish (the precision claim of this configuration)
    tte = precision_e0(pd, h, torch, runs=("plain_f64", "mixed_f32_fx64finish")) if with_solve else None
    h.close()
    torch.cuda.empty_cache()
    out = {"workload": "hubbard_18site_tilted_U6_half_filling", "D": D, "vector_dtype": "f32",
           "step_ms": round(step_ms, 3), "hv_ms": round(hv_ms, 3), "value_gstates_per_s": round(D / (step_ms * 1e-3) / 1e9, 3),
           "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(gbs / peak, 4), "bytes_per_state": 8}}
    if tte:
        out["time_to_E0"] = tte
    return out


def measure_maps(pd, torch, wl, reps: int = 5):
    """Rank and unrank over whole bases (Eq. 3 and the backward map; Sec. IV B for the inversion-symmetric
    maps): every index of the 4x4 half-filled basis (D = 165,636,900) unranked to its combined string and
    ranked back, and every representative of the inversion-symmetric basis of 15 particles on 30 sites,
    each timed with CUDA events (best of reps) after one warm-up; the round trips must give back every
    index exactly.  Algorithmic traffic: 8 B read + 8 B written per element."""
    peak = (measured_peaks() or {}).get("hbm_gbs", 6800.0)

    def timed(fn):
        fn()
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = fn()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        return out, best

    def record(n, ms):
        return {"ms": round(ms, 4), "gelements_per_s": round(n / (ms * 1e-3) / 1e9, 3),
                "hbm_frac": round(16 * n / (ms * 1e-3) / 1e9 / peak, 4)}

    out = {}
    cl = wl.square_periodic(4, 1.0, -0.3)
    h = pd.Handle(cl.L, cl.bonds, cl.t, 8.0, 8, 8)
    idx = torch.arange(h.D, dtype=torch.int64, device="cuda")
    states, t_un = timed(lambda: pd.paradeisos_unrank(h, idx))
    back, t_rk = timed(lambda: pd.paradeisos_rank(h, states))
    out["combined_4x4_half"] = {"D": h.D, "unrank": record(h.D, t_un), "rank": record(h.D, t_rk),
                                "round_trip_exact": bool(torch.equal(back, idx)),
                                "status": pd.hubbard_last_error(h)}
    del idx, states, back
    h.close()
    inv = pd.Inversion(30, 15)
    idx = torch.arange(inv.D, dtype=torch.int64, device="cuda")
    states, t_un = timed(lambda: inv.unrank(idx))
    back, t_rk = timed(lambda: inv.rank(states))
    out["inversion_30_15"] = {"D": inv.D, "unrank": record(inv.D, t_un), "rank": record(inv.D, t_rk),
                              "round_trip_exact": bool(torch.equal(back, idx)), "status": inv.last_error()}
    del idx, states, back
    inv.close()
    torch.cuda.empty_cache()
    return out


def measure_learned_quick(pd, torch, wl):
    """The learned start on the 4x4 t-t' cluster, shortened for the default line: trained on the library's
    own ground states at U = 2, 4, 6, 10 (half filling), used at the unseen U = 5; fixed-point Lanczos to
    E0 at 1e-10 from the learned start (its build included) against the same from a random start."""
    from paper_1707_03974_gb300 import learned
    cl = wl.square_periodic(4, 1.0, -0.3)
    t0 = time.perf_counter()
    sets = []
    for U in (2.0, 4.0, 6.0, 10.0):
        h = pd.Handle(cl.L, cl.bonds, cl.t, U, 8, 8)
        _, psi = learned.ground_state(h, tol=1e-6)
        sets.append(learned.sample(h, psi, 500000, seed=int(U)))
        del psi
        h.close()
        torch.cuda.empty_cache()
    t_data = time.perf_counter() - t0
    m = pd.Mlp(32, seed=1)
    rep = learned.train(m, sets, steps=600, batch=32768, lr=2e-3)
    h = pd.Handle(cl.L, cl.bonds, cl.t, 5.0, 8, 8)
    learned.tune(h)
    rnd = learned.solve_from(h, torch.int64, seed=0)
    v0, t_build = learned._timed_start(m, h, torch.int64)
    got = learned.solve_from(h, torch.int64, v0=v0)
    got["seconds"] += t_build
    del v0
    h.close()
    m.close()
    torch.cuda.empty_cache()
    return {"workload": "learned start, 4x4 t-t' U = 5 (8,8), trained at U = 2, 4, 6, 10",
            "data_seconds": round(t_data, 3), "train_seconds": round(rep.seconds, 3),
            "iterations_learned_fx64": got["iterations"], "iterations_random_fx64": rnd["iterations"],
            "seconds_learned_fx64_incl_start": round(got["seconds"], 4), "seconds_random_fx64": round(rnd["seconds"], 4),
            "start_vector_seconds": round(t_build, 4), "abs_E0_diff": abs(got["E0"] - rnd["E0"]),
            "converged": bool(got["converged"] and rnd["converged"])}


def measure_batch64(pd, torch, wl, steps: int, warmup: int, vdt):
    """64 independent 12-site problems solved together: instances/s to E0 at 1e-10 (the persistent
    batched solver), the per-step time with every instance active, and the batched H·v against HBM."""
    insts = wl.draw_batch_instances(64)
    hs = [pd.Handle(i.cluster.L, i.cluster.bonds, i.cluster.t, i.U, i.N_up, i.N_dn) for i in insts]
    b = pd.Batch(hs)
    x = torch.zeros(b.total, dtype=torch.float64, device="cuda")
    x.uniform_(-0.5, 0.5)
    if vdt == torch.int64:
        xs = torch.zeros(b.total, dtype=torch.int64, device="cuda")
        for k, h in enumerate(hs):
            b.view(xs, k).copy_(pd.hubbard_convert(h, b.view(x, k).contiguous(), torch.int64))
        x = xs
    y = torch.empty_like(x)
    tuned = pd.hubbard_batch_autotune(b, x, y, reps=3)
    for _ in range(warmup):
        pd.hubbard_batch_apply(b, x, y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        pd.hubbard_batch_apply(b, x, y)
    e1.record()
    torch.cuda.synchronize()
    hv_ms = e0.elapsed_time(e1) / steps
    gold = None
    try:
        gold = [r["E0"] for r in json.load(open(os.path.join(ROOT, "tests", "golden", "oracle_energies.json")))["batch64"]]
    except Exception:
        pass
    times = []
    for _ in range(max(1, min(steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        E0, infos, status = pd.lanczos_batch_ground_state(b, maxit=2000, tol=1e-10, dtype=vdt, seed=0, check_every=10)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    solve_s = min(times)
    D_total = sum(h.D for h in hs)
    # one persistent-kernel step with every instance active: the difference of two runs without a tolerance
    per = {}
    for n_steps in (2, 34):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pd.lanczos_batch_ground_state(b, maxit=n_steps, tol=0.0, dtype=vdt, seed=0, check_every=10)
        torch.cuda.synchronize()
        per[n_steps] = time.perf_counter() - t0
    step_ms = (per[34] - per[2]) / 32 * 1e3
    err = max(abs(e - g) / max(1, abs(g)) for e, g in zip(E0, gold)) if gold else None
    peak = (measured_peaks() or {}).get("hbm_gbs", 6800.0)
    hv_gbs = 16 * D_total / (hv_ms * 1e-3) / 1e9
    b.close()
    for h in hs:
        h.close()
    return {"instances_per_s": round(64 / solve_s, 3), "solve_seconds": round(solve_s, 4), "status": status,
            "iterations_max": max(i["iterations"] for i in infos), "max_rel_err_vs_oracle": err, "D_total": D_total,
            "step_ms_all_active": round(step_ms, 4),
            "step_gstates_per_s_all_active": round(D_total / (step_ms * 1e-3) / 1e9, 3),
            "batched_hv_ms": round(hv_ms, 4), "batched_hv_gstates_per_s": round(D_total / (hv_ms * 1e-3) / 1e9, 3),
            "batched_hv_roofline": {"bound": "hbm", "achieved": round(hv_gbs, 1), "peak": peak, "unit": "GB/s",
                                    "frac": round(hv_gbs / peak, 4), "bytes_per_state": 16},
            "batched_hv_config": tuned}


def run_batch(args, world, rank, local):
    """64 independent 12-site problems solved together (the persistent batched solver)."""
    import torch
    torch.cuda.set_device(local)
    from paper_1707_03974_gb300.build import build
    build()
    import paper_1707_03974_gb300 as pd
    import workloads as wl
    vdt = {"f64": torch.float64, "fx64": torch.int64}.get(args.dtype, torch.int64)
    r = measure_batch64(pd, torch, wl, args.steps, args.warmup, vdt)
    out = {"metric": "batched Lanczos instances/s to E0 at 1e-10", "value": r["instances_per_s"],
           "unit": "instances/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "int64" if vdt == torch.int64 else "f64",
           "data": "synthetic (seeded draws)",
           "config": {"workload": "64 x 12-site Hubbard (ring-12 / 3x4), N_sigma in 3..6, U in [0,12)",
                      "D_total": r["D_total"], "vector_dtype": args.dtype}, **r}
    print(json.dumps(out))


def run_learned(args, world, rank, local):
    """Learned start vector on the 4x4 t-t' cluster: train at U in {2,4,6,10} (half filling), then
    iterations and wall time to E0 at 1e-10 at U in {3,5,8,12} and in the doped (7,7) sector at U=8."""
    import torch
    torch.cuda.set_device(local)
    from paper_1707_03974_gb300.build import build
    build()
    import paper_1707_03974_gb300 as pd
    from paper_1707_03974_gb300 import learned
    import workloads as wl
    cl = wl.square_periodic(4, 1.0, -0.3)
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    t0 = time.perf_counter()
    sets = []
    for U in (2.0, 4.0, 6.0, 10.0):
        h = pd.Handle(cl.L, cl.bonds, cl.t, U, 8, 8)
        _, psi = learned.ground_state(h, tol=1e-6)
        sets.append(learned.sample(h, psi, 500000, seed=int(U)))
        del psi
        h.close()
    t_data = time.perf_counter() - t0
    m = pd.Mlp(32, seed=1)
    rep = learned.train(m, sets, steps=max(200, args.steps * 50), batch=32768, lr=2e-3)
    cases = {}
    for U, nu, nd in ((3.0, 8, 8), (5.0, 8, 8), (8.0, 8, 8), (12.0, 8, 8), (8.0, 7, 7)):
        h = pd.Handle(cl.L, cl.bonds, cl.t, U, nu, nd)
        _, psi = learned.ground_state(h, tol=1e-7)
        res = learned.compare(m, h, psi, seeds=(0, 1))
        cases[f"U{U:g}_{nu}_{nd}"] = res
        del psi
        h.close()
        torch.cuda.empty_cache()
    rnd = [min(r["iterations"] for r in c["random_f64"]) for c in cases.values()]
    lrn = [c["learned_f64"]["iterations"] for c in cases.values()]
    out = {"metric": "Lanczos iterations to E0 at 1e-10, learned start / random start (4x4 t-t', unseen U and doped)",
           "value": round(sum(lrn) / sum(rnd), 4), "unit": "ratio", "n_gpus": 1, "higher_is_better": False,
           "dtype": "bf16 network (tcgen05), f64/int64 Lanczos", "data": "synthetic (method's own ground states)",
           "config": {"workload": "learned start vector", "train_U": [2, 4, 6, 10], "train_samples_per_U": 500000,
                      "hidden": 128, "steps": len(rep.losses) and max(200, args.steps * 50), "batch": 32768},
           "time_to_E0_speedup_learned_fx64_vs_random_f64": {
               k: round(sum(r["seconds"] for r in c["random_f64"]) / len(c["random_f64"]) / c["learned_fx64"]["seconds"], 3)
               for k, c in cases.items()},
           "train_loss_first_last": [rep.losses[0], rep.losses[-1]], "train_seconds": round(rep.seconds, 3),
           "data_seconds": round(t_data, 3), "cases": cases}
    print(json.dumps(out))
    m.close()


MLP_FLOPS_PER_STATE = 2 * 128 * (32 + 128)  # the two tensor-core layers of the start-vector network


def run_start(args, world, rank, local):
    """Fused tensor-core inference of the start-vector network over the whole 4x4 half-filled
    basis (random-init weights of the same architecture): every basis index is unranked on
    the fly, both layers run on tcgen05, only the start vector is written."""
    import torch
    torch.cuda.set_device(local)
    from paper_1707_03974_gb300.build import build
    build()
    import paper_1707_03974_gb300 as pd
    import workloads as wl
    cfg = WORKLOADS[args.basis]
    cl = wl.square_periodic(4, 1.0, -0.3)
    h = pd.Handle(cl.L, cl.bonds, cl.t, cfg["U"], cfg["N_up"], cfg["N_dn"])
    D = h.D
    m = pd.Mlp(2 * cl.L, seed=1)
    stream = torch.cuda.current_stream()
    v = torch.empty(D, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        pd.mlp_start_vector(m, h, torch.float64)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.4)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        v = pd.mlp_start_vector(m, h, torch.float64)
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1) / args.steps
    assert pd.mlp_last_error(m) == "HB_OK" and bool(torch.isfinite(v).all())
    peaks = measured_peaks() or {}
    peak = peaks.get("bf16_tflops", 1900.0)
    tflops = MLP_FLOPS_PER_STATE * D / (ms * 1e-3) / 1e12
    out = {"metric": "start-vector inference Gstates/s (fused tcgen05 MLP over the whole basis)",
           "value": round(D / (ms * 1e-3) / 1e9, 4), "unit": "Gstates/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "bf16 operands, f32 accumulate, f64 output",
           "data": "synthetic (random-init weights)", "config": {**cfg, "workload": "start_vector_" + cfg["workload"]},
           "roofline": {"bound": "tensor", "achieved": round(tflops, 2), "peak": peak, "unit": "TFLOP/s",
                        "frac": round(tflops / peak, 4), "traffic": None, "kernel": "k_mlp_start<double>",
                        "flops_per_state": MLP_FLOPS_PER_STATE,
                        "peak_source": "MEASURED_PEAKS.json bf16_tflops (measured)" if peaks else "fallback 1900 TFLOP/s"},
           "gpu_launches": args.steps, "clocks": clk}
    print(json.dumps(out))
    m.close()
    h.close()


def run_green(args, world, rank, local):
    """Single-particle spectral function of the 4x4 t-t' ground state (U = 8, half filling, K = (0,0))
    by the Lanczos continued fraction: float64 ground state, then for k = (0,0), (pi/2,pi/2), (pi,0)
    the removal and addition parts (spin up), 200 Lanczos steps each."""
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    from paper_1707_03974_gb300.build import build
    build()
    import paper_1707_03974_gb300 as pd
    from paper_1707_03974_gb300 import response
    h = pd.Handle.momentum(4, 4, 1.0, -0.3, 8.0, 8, 8, 0, 0)
    z = np.linspace(-12.0, 12.0, 481) + 0.1j
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gs = response.ground(h)
    torch.cuda.synchronize()
    t_ground = time.perf_counter() - t0
    parts = {}
    t1 = time.perf_counter()
    for name, k in (("k00", 0), ("kpi2pi2", 5), ("kpi0", 2)):
        for part in ("removal", "addition"):
            G, info = response.green(gs, k, 0, part, z, steps=200)
            parts[f"{name}_{part}"] = {"seconds": round(info["seconds"], 4), "weight": round(info["norm2"], 6),
                                       "D_target": info["D_target"], "steps": info["steps"],
                                       "peak_omega": float(z.real[int(np.argmax(-G.imag))])}
    torch.cuda.synchronize()
    t_all = time.perf_counter() - t1
    out = {"metric": "spectral function A(k, omega): seconds for 3 momenta x (removal + addition), 200 Lanczos steps each",
           "value": round(t_all, 4), "unit": "s", "n_gpus": 1, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (the method's own ground state)",
           "config": {"workload": "green_function_4x4_tp-0.3_U8_half_filling_K00", "D_ground_sector": h.D,
                      "eta": 0.1, "omega_points": len(z)},
           "ground_state_seconds": round(t_ground, 4), "E0": gs.E0, "parts": parts}
    print(json.dumps(out))
    h.close()


def run_tcgemm(args, local):
    """The training product of the start-vector network on the tensor cores: C[4096 x 128] =
    A[4096 x 4096] B[128 x 4096]^T (bf16 operands, float32 accumulation in tensor memory), the shape
    of a layer-2 weight product over a 4096-state slab, through mlp_tc_gemm."""
    import torch
    torch.cuda.set_device(local)
    from paper_1707_03974_gb300.build import build
    build()
    import paper_1707_03974_gb300 as pd
    g = torch.Generator().manual_seed(0)
    M, N, K = 4096, 128, 4096
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    for _ in range(args.warmup):
        C = pd.mlp_tc_gemm(A, B)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        C = pd.mlp_tc_gemm(A, B)
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / args.steps
    err = (C.double() - A.double() @ B.double().T).abs().max().item()
    peaks = measured_peaks() or {}
    peak = peaks.get("bf16_tflops", 1900.0)
    tf = 2.0 * M * N * K / (ms * 1e-3) / 1e12
    print(json.dumps({"metric": "tcgen05 training product TFLOP/s", "value": round(tf, 3), "unit": "TFLOP/s",
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
                      "config": {"workload": "tc_gemm_4096x128x4096_bf16"}, "max_abs_err": err,
                      "roofline": {"bound": "tensor", "achieved": round(tf, 2), "peak": peak, "unit": "TFLOP/s",
                                   "frac": round(tf / peak, 4), "kernel": "k_tc_gemm<128>"}}))


def run_ceilings(args, local):
    """The on-chip ceilings alone (one JSON line): the denominators of the H·v's on-chip rooflines."""
    import torch
    torch.cuda.set_device(local)
    from paper_1707_03974_gb300.build import build
    build()
    import paper_1707_03974_gb300 as pd
    dev = torch.device("cuda", local)
    runs = [measure_ceilings(pd, torch, dev) for _ in range(max(1, args.steps))]
    best = {k: (min(r[k] for r in runs) if k.endswith("_clk") else max(r[k] for r in runs)) for k in runs[0]}
    print(json.dumps({"metric": "measured on-chip ceilings", "unit": "mixed (see keys)", "n_gpus": 1,
                      "runs": len(runs), "best": best, "all": runs,
                      "gpu": torch.cuda.get_device_name(dev)}))


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.workload == "ceilings" and args.impl == "ours":
        if rank == 0:
            run_ceilings(args, local)
        return
    if args.workload == "tcgemm" and args.impl == "ours":
        if rank == 0:
            run_tcgemm(args, local)
        return
    if args.workload == "learned4x4" and args.impl == "ours":
        if rank == 0:
            run_learned(args, world, rank, local)
        return
    if args.workload == "green4x4" and args.impl == "ours":
        if rank == 0:
            run_green(args, world, rank, local)
        return
    if args.workload == "start4x4" and args.impl == "ours":
        if rank == 0:
            run_start(args, world, rank, local)
        return
    if args.workload == "batch64" and args.impl == "ours":
        if rank == 0:
            run_batch(args, world, rank, local)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
