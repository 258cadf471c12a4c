"""Iteration counts of the CPU oracle on the 128^3 benchmark systems (test infrastructure).

For each 7-point Laplacian variant of the benchmark workload (n = 128^3,
x* ~ U[-1, 1] with seed 1, b = A x*, eps2 = 1e-10) this script runs the
oracle's Algorithm I for every candidate eps1 = 1e-2 .. 1e-7 (Sec. 2) and pure
FP64 CG, and stores N1, N2 and N_dp.  The benchmark's CPU-baseline legs use
these counts to scale live per-iteration timings of the oracle to whole
solves.  Only the oracle computes them.

    python -m oracle.workload_counts [--size 128] [--jobs 6]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))

import sys

sys.path.insert(0, os.path.dirname(HERE))
from synth import LAP3D_VARIANTS as VARIANTS  # noqa: E402  (name, eps, sigma)


def _one(args):
    size, name, eps, sigma = args
    import sys
    sys.path.insert(0, os.path.dirname(HERE))
    import oracle
    import synth
    A = synth.laplacian_3d(size, eps=eps, sigma=sigma)
    _, b = synth.rhs(A, seed=1)
    t0 = time.time()
    out = {"name": name, "eps": eps, "sigma": sigma, "n": A.n, "nnz": A.nnz, "sweep": {}}
    for t in range(2, 8):
        _, r = oracle.solve(A, b, eps1=float(f"1e-{t}"), eps2=1e-10)
        out["sweep"][str(t)] = {"n1": r["n1"], "n2": r["n2"], "status": r["status"],
                                "true_rel_resid": r["true_rel_resid"]}
    _, ndp, st = oracle.cg64(A, b, 1e-10)
    out["n_dp"] = ndp
    out["status_dp"] = st
    out["cpu_seconds"] = time.time() - t0
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--size", type=int, default=128)
    ap.add_argument("--jobs", type=int, default=len(VARIANTS))
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    out = a.out or os.path.join(HERE, "data", f"lap3d{a.size}_counts.json")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    import oracle
    oracle.build()
    with mp.get_context("spawn").Pool(a.jobs) as pool:
        res = pool.map(_one, [(a.size, nm, e, s) for nm, e, s in VARIANTS])
    with open(out, "w") as f:
        json.dump({"size": a.size, "eps2": 1e-10, "rhs": "x* ~ U[-1,1], seed 1, b = A x*",
                   "systems": res}, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
