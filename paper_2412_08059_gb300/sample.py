"""Labelled kNN sample builder (Sec. 11.1) on the GPU path.

For every training matrix: the features chi = (n, m, l~, v) (Sec. 4) from
mpcg_features; N1 and N2 of Algorithm I for each candidate eps1 = 10^-t,
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


def save(path: str, feat, cls, recs, meta: dict | None = None) -> None:
    with open(path, "w") as f:
        json.dump({"meta": meta or {}, "feat": np.asarray(feat).tolist(),
                   "cls": np.asarray(cls).tolist(), "records": recs}, f, indent=1)


def load(path: str):
    with open(path) as f:
        d = json.load(f)
    return np.array(d["feat"], dtype=np.float64), np.array(d["cls"], dtype=np.int8), d
