"""Writes tests/golden/oracle_energies.json: ground energies computed by the CPU oracle only.

Usage:  python tests/golden/make_oracle_energies.py [ring8] [square4x4] [batch64] [learned]

Every value comes from oracle/ (dense eigh for small D, the oracle's Lanczos with
its tensor-product operator otherwise); nothing is taken from the CUDA library.
Each record keeps its provenance (method, tolerance, iterations, residual).
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402
from oracle.basis import Basis  # noqa: E402
from oracle.build import build  # noqa: E402
from oracle.hamiltonian import KronOperator, Model, dense  # noqa: E402
from oracle.lanczos import lanczos, start_vector  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_energies.json")


def load():
    return json.load(open(OUT)) if os.path.exists(OUT) else {}


def save(d):
    tmp = OUT + ".tmp"
    json.dump(d, open(tmp, "w"), indent=1, sort_keys=True)
    os.replace(tmp, OUT)


def lanczos_record(cl, U, nu, nd, seed=0, tol=1e-11, maxit=3000):
    m = Model.from_cluster(cl, U, nu, nd)
    k = KronOperator(m)
    t0 = time.time()
    r = lanczos(k, start_vector(seed, k.D), maxit, reorth=False, tol=tol)
    return {"cluster": cl.name, "L": cl.L, "N_up": nu, "N_dn": nd, "U": U, "D": int(k.D),
            "E0": r.E0, "method": "oracle lanczos (3-term, tensor-product operator)", "seed": seed,
            "tol": tol, "iterations": r.iterations, "residual": r.residual, "converged": r.converged,
            "seconds": round(time.time() - t0, 1)}


def main(which):
    build()
    d = load()
    if "ring8" in which:
        cl = wl.ring(8)
        m = Model.from_cluster(cl, 4.0, 4, 4)
        ev = np.linalg.eigvalsh(dense(m, Basis(8, 4, 4)))
        d["ring8_U4_4_4"] = {"cluster": "ring8", "L": 8, "N_up": 4, "N_dn": 4, "U": 4.0, "D": 4900,
                             "E0": float(ev[0]), "E1": float(ev[1]), "method": "dense numpy.linalg.eigh"}
        save(d)
    if "square4x4" in which:
        d["square4x4_tp-0.3_U8_8_8"] = lanczos_record(wl.square_periodic(4, 1.0, -0.3), 8.0, 8, 8)
        save(d)
        print(d["square4x4_tp-0.3_U8_8_8"], flush=True)
    if "batch64" in which:
        recs = []
        for inst in wl.draw_batch_instances(64):
            rec = lanczos_record(inst.cluster, inst.U, inst.N_up, inst.N_dn, seed=inst.seed)
            rec["index"] = inst.index
            recs.append(rec)
            print(inst.index, rec["E0"], rec["iterations"], flush=True)
        d["batch64"] = recs
        save(d)
    if "learned" in which:
        cl = wl.square_periodic(4, 1.0, -0.3)
        for U, nu, nd in [(2.0, 8, 8), (4.0, 8, 8), (6.0, 8, 8), (10.0, 8, 8), (3.0, 8, 8), (5.0, 8, 8),
                          (12.0, 8, 8), (8.0, 7, 7)]:
            key = f"square4x4_tp-0.3_U{U:g}_{nu}_{nd}"
            if key in d:
                continue
            d[key] = lanczos_record(cl, U, nu, nd)
            save(d)
            print(key, d[key]["E0"], d[key]["iterations"], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["ring8", "square4x4", "batch64"])
