"""Labelled kNN sample builder (Sec. 11.1) on the GPU path.

For every training matrix: the features chi = (n, m, l~, v) (Sec. 4) from
mpcg_features (or from a batched Algorithm II run, build_batched); N1 and N2 of Algorithm I for each candidate eps1 = 10^-t,
t = 2..7 (Sec. 2); N_dp of pure FP64 CG; and the matrix-specific
omega = t_sp / t_dp measured from the device clock marks of those runs
(Appendix C).  The label is the t minimising Eq. (4), omega N1 + N2, with
ties going to the smallest t.  All solver work runs in libmpcg.
"""
from __future__ import annotations

import json

import numpy as np
import torch

from . import mpcg

CLASSES = (2, 3, 4, 5, 6, 7)


def eps_of(t: int) -> float:
    return float(f"1e-{t}")


def sweep(dA: mpcg.DeviceCSR, db: torch.Tensor, ws=None, eps2: float = 1e-10, k0: int = 10,
          classes=CLASSES) -> dict:
    ws = mpcg.workspace(dA.n, dA.nnz) if ws is None else ws
    f = mpcg.features(dA, db, ws=ws, k0=k0)
    n1, n2, ms32, ms64, it32, it64 = [], [], 0.0, 0.0, 0, 0
    for t in classes:
        _, r = mpcg.solve(dA, db, ws=ws, eps1=eps_of(t), eps2=eps2)
        n1.append(r["n1"])
        n2.append(r["n2"])
        ms32 += r["ms_fp32"]
        ms64 += r["ms_fp64"]
        it32 += r["n1"]
        it64 += r["n2"]
    _, rd = mpcg.solve(dA, db, ws=ws, fp64_only=1, eps2=eps2)
    ms64 += rd["ms_fp64"]
    it64 += rd["n2"]
    t_sp = ms32 / max(it32, 1)
    t_dp = ms64 / max(it64, 1)
    return {"feat": [f["n"], f["m"], f["pdiam"], f["v"]], "k0_done": f["k0_done"],
            "n1": n1, "n2": n2, "n_dp": rd["n2"], "t_sp_ms": t_sp, "t_dp_ms": t_dp,
            "omega": t_sp / t_dp if t_dp > 0 else float("nan"), "classes": list(classes)}


def label(rec: dict, omega: float | None = None) -> int:
    """Eq. (4) argmin with the matrix's measured omega (or a given one)."""
    w = rec["omega"] if omega is None else omega
    best_t, best_I = None, np.inf
    for t, a, b in zip(rec["classes"], rec["n1"], rec["n2"]):
        I = w * a + b
        if I < best_I:
            best_t, best_I = t, I
    return best_t


def build(systems, omega: float | None = None, device="cuda"):
    """systems: iterable of (name, A (host CSR), b (host float64)).  Returns
    (feat [N,4], cls int8 [N], records)."""
    recs = []
    for name, A, b in systems:
        dA = mpcg.DeviceCSR.from_host(A, device)
        db = torch.from_numpy(np.ascontiguousarray(b)).to(device)
        rec = sweep(dA, db)
        rec["name"] = name
        recs.append(rec)
        del dA, db
    feat = np.array([r["feat"] for r in recs], dtype=np.float64)
    cls = np.array([label(r, omega) for r in recs], dtype=np.int8)
    return feat, cls, recs


def sweep_batched(mats, bs, device="cuda", eps2: float = 1e-10, k0: int = 10,
                  team_rows: int = 0, acc32: int = 0, tol_relative: int = 1,
                  classes=CLASSES) -> dict:
    """The same sweep for many matrices at once, as batched solves (the team
    kernels of mpcg_solve_batch): one Algorithm II batch for the features, one
    Algorithm I batch per candidate eps1, one pure-FP64 batch.  omega per
    matrix is t_sp / t_dp from the batches' clock marks: t_sp over the
    Algorithm I runs' single-precision stages, t_dp from the pure-FP64 run (a
    mixed batch runs its FP64 stages in a second launch, so their clock marks
    include the wait for the first launch to end).  mats: host CSR matrices;
    bs: host float64 right-hand sides."""
    dmats = [mpcg.DeviceCSR.from_host(A, device) for A in mats]
    dbs = [torch.from_numpy(np.ascontiguousarray(b)).to(device) for b in bs]
    xs = [torch.empty(A.n, dtype=torch.float64, device=device) for A in mats]
    ws = torch.empty(mpcg.batch_workspace_bytes(dmats), dtype=torch.uint8, device=device)
    res = mpcg.result_buffer(len(mats), device)
    N = len(mats)

    def run(opts, sample):
        mpcg.solve_batch_async(dmats, dbs, xs, opts, ws, res, sample)
        torch.cuda.synchronize()
        return mpcg.read_results(res, N)

    common = dict(eps2=eps2, k0=k0, team_rows=team_rows, acc32=acc32, tol_relative=tol_relative)
    # features (any sample: the label of this run is not used)
    dummy = mpcg.DeviceSample(np.ones((1, 4)), np.array([2], np.int8), device=device)
    rf = run(mpcg.options(**common), dummy)
    feat = np.array([[A.n, A.nnz, r["pdiam"], r["v"]] for A, r in zip(mats, rf)], dtype=np.float64)
    n1 = np.zeros((N, len(classes)), np.int64)
    n2 = np.zeros((N, len(classes)), np.int64)
    st = np.zeros((N, len(classes)), np.int64)
    ms32 = np.zeros(N)
    for j, t in enumerate(classes):
        for i, r in enumerate(run(mpcg.options(eps1=eps_of(t), **common), None)):
            n1[i, j], n2[i, j], st[i, j] = r["n1"], r["n2"], r["status"]
            ms32[i] += (r["t_fp32_ns"] - r["t_features_ns"]) / 1e6
    rd = run(mpcg.options(fp64_only=1, **common), None)
    ndp = np.array([r["n2"] for r in rd], np.int64)
    st_dp = np.array([r["status"] for r in rd], np.int64)
    ms64 = np.array([(r["t_fp64_ns"] - r["t_prep_ns"]) / 1e6 for r in rd])
    t_sp = ms32 / np.maximum(n1.sum(axis=1), 1)
    t_dp = ms64 / np.maximum(ndp, 1)
    return {"feat": feat, "n1": n1, "n2": n2, "status": st, "n_dp": ndp, "status_dp": st_dp,
            "omega": t_sp / t_dp, "classes": list(classes)}


def build_batched(systems, omega: float | None = None, device="cuda", team_rows: int = 0):
    """build() with the sweeps of sweep_batched: the labels then follow the
    cost of an iteration in the team kernels that batched and served solves
    run.  Matrices with a failed solve in the sweep are left out."""
    names = [s[0] for s in systems]
    rec = sweep_batched([s[1] for s in systems], [s[2] for s in systems], device,
                        team_rows=team_rows)
    ok = (rec["status"] >= 0).all(axis=1) & (rec["status_dp"] >= 0)
    w = rec["omega"] if omega is None else np.full(len(names), float(omega))
    cost = w[:, None] * rec["n1"] + rec["n2"]
    cls = np.array(rec["classes"], dtype=np.int8)[np.argmin(cost, axis=1)]  # ties: smallest t
    recs = [{"name": nm, "feat": rec["feat"][i].tolist(), "n1": rec["n1"][i].tolist(),
             "n2": rec["n2"][i].tolist(), "n_dp": int(rec["n_dp"][i]),
             "omega": float(rec["omega"][i]), "classes": rec["classes"]}
            for i, nm in enumerate(names) if ok[i]]
    return rec["feat"][ok], cls[ok], recs


def save(path: str, feat, cls, recs, meta: dict | None = None) -> None:
    with open(path, "w") as f:
        json.dump({"meta": meta or {}, "feat": np.asarray(feat).tolist(),
                   "cls": np.asarray(cls).tolist(), "records": recs}, f, indent=1)


def load(path: str):
    with open(path) as f:
        d = json.load(f)
    return np.array(d["feat"], dtype=np.float64), np.array(d["cls"], dtype=np.int8), d
