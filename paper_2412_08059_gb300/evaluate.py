"""The paper's evaluation protocol for Algorithm II (Sec. 12, Appendices A-B).

Steps, in the paper's order:

1. General samples S_0 of the three generated matrix families (Appendix A):
   extended stars with random edges added, random sparse matrices (a random
   tree plus floor(c n) edges) and random banded matrices, with the
   diagonal a_ii = mu * sum_j |a_ij| for mu in {1.1, 3, 10}.
2. For every matrix: the features chi = (n, m, l~, v) (Sec. 4), N1 and N2 of
   Algorithm I for every eps1 = 10^-t, t = 2..7, N_dp of pure FP64 CG, and
   the matrix's measured omega = t_sp / t_dp (Appendix C: the mean time of a
   single-precision iteration over the sweep's stage-1 runs, over that of a
   double-precision iteration in the pure-FP64 run); its label is the
   t minimising Eq. (4) with omega = 1/3, ties to the smallest t.  The same
   labels serve both omega choices (Appendix C).
3. k_CG = mean N_dp; the training-set size N_S from Eq. (26) for each k.
4. Repeated random splits of S_0 into a training set S (N_S elements) and a
   test set T (the rest).  For every split and k: the weighted kNN vote on
   the 3-D features (m, l~, v) of Appendix B classifies T; kNN accuracy Acc,
   localization Loc (Sec. 11.4: the share of a query's k nearest neighbours
   in its own class) and the efficiencies E and E_opt of Eq. (27) for
   omega = 1/3 and the measured omega.  Means and standard deviations over
   the splits are reported, in percent.

All solver work -- the sweeps, the features, the vote for every test query --
runs in libmpcg (batched solves, mpcg_knn_batch).  This module builds the
inputs and keeps the books.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import mpcg

CLASSES = (2, 3, 4, 5, 6, 7)
MU = (1.1, 3.0, 10.0)

# (lc, nc) of the extended stars, n = 1 + nc * lc (Appendix A.1, Tables 7-9).
STAR_PAIRS = {
    301: [(1, 300), (2, 150), (5, 60), (10, 30), (15, 20), (20, 15), (30, 10), (60, 5), (150, 2),
          (300, 1)],
    501: [(1, 500), (2, 250), (4, 125), (5, 100), (10, 50), (20, 25), (25, 20), (50, 10),
          (100, 5), (125, 4), (250, 2), (500, 1)],
    1001: [(1, 1000), (2, 500), (4, 250), (5, 200), (8, 125), (10, 100), (20, 50), (25, 40),
           (40, 25), (50, 20), (100, 10), (125, 8), (200, 5), (250, 4), (500, 2), (1000, 1)],
}
RANDOM_C = (0.1, 0.5, 1.0, 2.0, 3.0, 5.0, 7.0, 10.0)   # Appendix A.2
BAND_MAX = {300: 29, 500: 51, 1000: 101}                  # Appendix A.3
BAND_P = (0.4, 0.6, 0.8)
# Matrices per parameter set in the paper: 100 per (lc, nc, mu) for stars
# (|S_0| = 3000, 3600, 4800), 200 per (c, mu) for random matrices (4800),
# 20 per (b, p) for banded ones.
PAPER_PER = {"xstar": 100, "random": 200, "banded": 20}
FAMILY_SIZES = {"xstar": (301, 501, 1001), "random": (300, 500, 1000), "banded": (300, 500, 1000)}


def general_sample(family: str, n: int, per: int | None = None, seed: int = 0) -> list[dict]:
    """Descriptors of S_0 for one family and size; `per` matrices per
    parameter set (the paper's count when None).  Banded matrices take mu in
    turn from {1.1, 3, 10} over their repetitions."""
    per = PAPER_PER[family] if per is None else per
    out = []
    if family == "xstar":
        for lc, nc in STAR_PAIRS[n]:
            for mu in MU:
                for r in range(per):
                    out.append({"family": family, "lc": lc, "nc": nc, "mu": mu})
    elif family == "random":
        for c in RANDOM_C:
            for mu in MU:
                for r in range(per):
                    out.append({"family": family, "n": n, "c": c, "mu": mu})
    elif family == "banded":
        for b in range(3, BAND_MAX[n] + 1):
            for p in BAND_P:
                for r in range(per):
                    out.append({"family": family, "n": n, "b": b, "p": p, "mu": MU[r % 3]})
    else:
        raise KeyError(family)
    for j, d in enumerate(out):
        d["seed"] = seed * 1_000_003 + j
    return out


def build(desc: dict):
    """The matrix of a descriptor (synth generators of the three families)."""
    import synth
    f = desc["family"]
    if f == "xstar":
        return synth.extended_star(desc["lc"], desc["nc"], desc["mu"], extra=None, seed=desc["seed"])
    if f == "random":
        return synth.random_tree_plus(desc["n"], desc["c"], desc["mu"], seed=desc["seed"])
    return synth.banded(desc["n"], desc["b"], desc["p"], desc["mu"], seed=desc["seed"])


def _batch_results(dmats, dbs, xs, ws, res, opts, sample):
    mpcg.solve_batch_async(dmats, dbs, xs, opts, ws, res, sample)
    torch.cuda.synchronize()
    return mpcg.read_results(res, len(dmats))


def sweep_records(descs: list[dict], device="cuda", eps2: float = 1e-10, k0: int = 10,
                  team_rows: int = 0) -> dict:
    """Step 2 for every descriptor, as batched solves on the GPU: one batch of
    Algorithm II for the features, one of Algorithm I per candidate eps1 and
    one pure-FP64 batch.  b = A x* with x* ~ U[-1, 1] (seeded per matrix)."""
    import synth
    t0 = time.time()
    mats = [build(d) for d in descs]
    bs = [synth.rhs(A, seed=d["seed"])[1] for A, d in zip(mats, descs)]
    t_gen = time.time() - t0
    dmats = [mpcg.DeviceCSR.from_host(A, device) for A in mats]
    dbs = [torch.from_numpy(np.ascontiguousarray(b)).to(device) for b in bs]
    xs = [torch.empty(A.n, dtype=torch.float64, device=device) for A in mats]
    ws = torch.empty(mpcg.batch_workspace_bytes(dmats), dtype=torch.uint8, device=device)
    res = mpcg.result_buffer(len(mats), device)
    N = len(mats)
    t1 = time.time()
    # features (any sample: the label of this run is not used)
    dummy = mpcg.DeviceSample(np.ones((1, 4)), np.array([2], np.int8), device=device)
    rf = _batch_results(dmats, dbs, xs, ws, res, mpcg.options(k0=k0, eps2=eps2, team_rows=team_rows),
                        dummy)
    feat = np.array([[A.n, A.nnz, r["pdiam"], r["v"]] for A, r in zip(mats, rf)], dtype=np.float64)
    n1 = np.zeros((N, len(CLASSES)), np.int64)
    n2 = np.zeros((N, len(CLASSES)), np.int64)
    st = np.zeros((N, len(CLASSES)), np.int64)
    ms32 = np.zeros(N)
    for j, t in enumerate(CLASSES):
        rr = _batch_results(dmats, dbs, xs, ws, res,
                            mpcg.options(eps1=float(f"1e-{t}"), eps2=eps2, k0=k0,
                                         team_rows=team_rows), None)
        for i, r in enumerate(rr):
            n1[i, j], n2[i, j], st[i, j] = r["n1"], r["n2"], r["status"]
            ms32[i] += (r["t_fp32_ns"] - r["t_features_ns"]) / 1e6
    rd = _batch_results(dmats, dbs, xs, ws, res,
                        mpcg.options(fp64_only=1, eps2=eps2, team_rows=team_rows), None)
    ndp = np.array([r["n2"] for r in rd], np.int64)
    st_dp = np.array([r["status"] for r in rd], np.int64)
    # t_sp from the single-precision stages of the Algorithm I runs; t_dp from
    # the pure-FP64 run (a mixed batch runs its FP64 stages in a second launch,
    # so their clock marks include the wait for the first launch to end)
    ms64 = np.array([(r["t_fp64_ns"] - r["t_prep_ns"]) / 1e6 for r in rd])
    t_sp = ms32 / np.maximum(n1.sum(axis=1), 1)
    t_dp = ms64 / np.maximum(ndp, 1)
    return {"descs": descs, "feat": feat, "n1": n1, "n2": n2, "status": st, "n_dp": ndp,
            "status_dp": st_dp, "omega": t_sp / t_dp, "seconds_generate": t_gen,
            "seconds_gpu": time.time() - t1}


def labels(n1: np.ndarray, n2: np.ndarray, omega: float = 1.0 / 3.0) -> np.ndarray:
    """Eq. (4) argmin per matrix (row), as a class t; ties to the smallest t."""
    cost = omega * n1 + n2
    return np.array(CLASSES)[np.argmin(cost, axis=1)]


def training_size(n: int, k: int, k_cg: float, c: float = 0.1, alpha: float = 0.01) -> int:
    """Eq. (26) with the parameters of Appendix B, rounded down."""
    return int(math.floor(alpha * 4.0 * (6.0 * c + 17.0) * n * k_cg / (44.0 + 3.0 * k)))


def gpu_classifier(device="cuda", weighted: int = 1, feat_mask: int = 0b1110):
    """kNN of the test set through mpcg_knn_batch: (pred, neighbour indices)."""
    def classify(tr_feat, tr_cls, te_feat, k):
        S = mpcg.DeviceSample(tr_feat, tr_cls, device=device)
        cls, nbr = mpcg.knn_batch(te_feat, S, neighbours=True, knn_k=k, weighted=weighted,
                                  feat_mask=feat_mask)
        return cls.cpu().numpy(), nbr.cpu().numpy()
    return classify


def protocol(rec: dict, classify, n: int, ks=(1, 5, 10, 15, 20), splits: int = 100,
             seed: int = 0) -> dict:
    """Steps 3-4 on the records of one general sample."""
    feat, n1, n2, ndp, om = rec["feat"], rec["n1"], rec["n2"], rec["n_dp"], rec["omega"]
    N = feat.shape[0]
    cls = labels(n1, n2)
    col = cls - CLASSES[0]
    k_cg = float(ndp.mean())
    P = [float(np.mean(cls == t) * 100.0) for t in CLASSES]
    rows = np.arange(N)
    out = {"N": N, "k_CG": k_cg, "P": dict(zip([f"1e-{t}" for t in CLASSES], P)), "k": {}}
    rng = np.random.default_rng(seed)
    for k in ks:
        ns = min(max(training_size(n, k, k_cg), k), N - 1)
        acc, loc, e13, eo13, em, eom = [], [], [], [], [], []
        for _ in range(splits):
            perm = rng.permutation(N)
            tr, te = perm[:ns], perm[ns:]
            pred, nbr = classify(feat[tr], cls[tr].astype(np.int8), feat[te], k)
            pred = np.asarray(pred)
            ok = pred >= CLASSES[0]
            acc.append(float(np.mean(pred == cls[te]) * 100.0))
            nb = np.asarray(nbr)[:, :min(k, ns)]
            loc.append(float(np.mean(cls[tr][nb] == cls[te][:, None]) * 100.0))
            pc = np.where(ok, pred - CLASSES[0], col[te])  # an invalid vote never occurs here
            r_te = rows[te]
            I_dp = float(ndp[te].sum())
            for w, E, Eo in ((np.full(te.size, 1.0 / 3.0), e13, eo13), (om[te], em, eom)):
                I = float(np.sum(w * n1[r_te, pc] + n2[r_te, pc]))
                Io = float(np.sum(w * n1[r_te, col[te]] + n2[r_te, col[te]]))
                E.append((1.0 - I / I_dp) * 100.0)
                Eo.append((1.0 - Io / I_dp) * 100.0)
        out["k"][k] = {"N_S": ns, "N_T": N - ns,
                       "Acc": [float(np.mean(acc)), float(np.std(acc))],
                       "Loc": [float(np.mean(loc)), float(np.std(loc))],
                       "E_omega_1_3": [float(np.mean(e13)), float(np.mean(eo13))],
                       "E_omega_measured": [float(np.mean(em)), float(np.mean(eom))]}
    return out


def run(families=("xstar", "random", "banded"), scale: float = 1.0, splits: int = 100,
        ks=(1, 5, 10, 15, 20), device="cuda", seed: int = 0, log=None) -> dict:
    """The whole protocol: every family and size, `scale` times the paper's
    matrices per parameter set (at least one)."""
    classify = gpu_classifier(device)
    out = {}
    for fam in families:
        for n in FAMILY_SIZES[fam]:
            per = max(1, int(round(PAPER_PER[fam] * scale)))
            descs = general_sample(fam, n, per, seed=seed + n)
            rec = sweep_records(descs, device)
            t = time.time()
            r = protocol(rec, classify, n, ks, splits, seed)
            r["seconds_generate"] = round(rec["seconds_generate"], 1)
            r["seconds_gpu_sweep"] = round(rec["seconds_gpu"], 1)
            r["seconds_protocol"] = round(time.time() - t, 1)
            r["omega_measured_mean"] = float(np.mean(rec["omega"]))
            r["failed_solves"] = int((rec["status"] < 0).sum() + (rec["status_dp"] < 0).sum())
            out[f"{fam}_{n}"] = r
            if log:
                log(f"{fam} n={n}: N={r['N']} k_CG={r['k_CG']:.1f} "
                    f"Acc(k=5)={r['k'].get(5, {}).get('Acc')}")
            del rec
            torch.cuda.empty_cache()
    return out
