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

from . import mpcg, sample

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
    """The matrix of a descriptor (synth generators of the three families, and
    the Laplacians of the condition-number study)."""
    import synth
    f = desc["family"]
    if f == "lap2d":
        return synth.laplacian_2d(desc["nx"], desc["ny"], sigma=desc["sigma"], cy=desc["c"])
    if f == "lap3d":
        return synth.laplacian_3d(desc["nx"], desc["ny"], desc["nz"], eps=desc["c"],
                                  sigma=desc["sigma"])
    if f == "xstar":
        return synth.extended_star(desc["lc"], desc["nc"], desc["mu"], extra=None, seed=desc["seed"])
    if f == "random":
        return synth.random_tree_plus(desc["n"], desc["c"], desc["mu"], seed=desc["seed"])
    return synth.banded(desc["n"], desc["b"], desc["p"], desc["mu"], seed=desc["seed"])


def sweep_records(descs: list[dict], device="cuda", eps2: float = 1e-10, k0: int = 10,
                  team_rows: int = 0, acc32: int = 0, tol_relative: int = 1) -> dict:
    """Step 2 for every descriptor, as batched solves on the GPU
    (sample.sweep_batched): one batch of Algorithm II for the features, one of
    Algorithm I per candidate eps1 and one pure-FP64 batch.  b = A x* with
    x* ~ U[-1, 1] (seeded per matrix).  acc32 = 1 sums the single-precision
    stage's inner products in float, and tol_relative = 0 stops on
    ||r|| <= eps as Sec. 3 prints it (the options of the same names)."""
    import synth
    t0 = time.time()
    mats = [build(d) for d in descs]
    bs = [synth.rhs(A, seed=d["seed"])[1] for A, d in zip(mats, descs)]
    t_gen = time.time() - t0
    t1 = time.time()
    rec = sample.sweep_batched(mats, bs, device, eps2=eps2, k0=k0, team_rows=team_rows,
                               acc32=acc32, tol_relative=tol_relative, classes=CLASSES)
    rec.update(descs=descs, seconds_generate=t_gen, seconds_gpu=time.time() - t1)
    return rec


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
        ks=(1, 5, 10, 15, 20), device="cuda", seed: int = 0, log=None, acc32: int = 0,
        tol_relative: int = 1) -> dict:
    """The whole protocol: every family and size, `scale` times the paper's
    matrices per parameter set (at least one); acc32 and tol_relative as in
    sweep_records."""
    classify = gpu_classifier(device)
    out = {}
    for fam in families:
        for n in FAMILY_SIZES[fam]:
            per = max(1, int(round(PAPER_PER[fam] * scale)))
            descs = general_sample(fam, n, per, seed=seed + n)
            rec = sweep_records(descs, device, acc32=acc32, tol_relative=tol_relative)
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


# Efficiency against the pseudo-diameter by condition-number class (Sec. 7,
# Tables 1-3) on Laplacians whose condition number has a closed form.
# ------------------------------------------------------------------------------

# The four classes of Sec. 7: kappa <= 10, 10 < kappa <= 100, 100 < kappa <= 1000,
# kappa > 1000 (upper bounds, inclusive).
KAPPA_BOUNDS = (10.0, 100.0, 1000.0)
KAPPA_NAMES = ("kappa<=10", "10<kappa<=100", "100<kappa<=1000", "kappa>1000")


def _tridiag_extremes(m: int) -> tuple[float, float]:
    """Smallest and largest eigenvalue of tridiag(-1, 2, -1) of order m:
    4 sin^2(k pi / (2 (m + 1))) for k = 1 and k = m."""
    return (4.0 * math.sin(math.pi / (2 * (m + 1))) ** 2,
            4.0 * math.sin(m * math.pi / (2 * (m + 1))) ** 2)


def kappa_closed_form(desc: dict) -> float:
    """Spectral condition number of a Laplacian descriptor.  The matrices are
    Kronecker sums of tridiag(-1, 2, -1) (weights 1, c) plus sigma I, so the
    extreme eigenvalues are sums of the factors' extreme eigenvalues."""
    if desc["family"] == "lap2d":
        dims, w = (desc["nx"], desc["ny"]), (1.0, desc["c"])
    elif desc["family"] == "lap3d":
        dims, w = (desc["nx"], desc["ny"], desc["nz"]), (1.0, 1.0, desc["c"])
    else:
        raise KeyError(desc["family"])
    lo = desc["sigma"] + sum(wk * _tridiag_extremes(m)[0] for m, wk in zip(dims, w))
    hi = desc["sigma"] + sum(wk * _tridiag_extremes(m)[1] for m, wk in zip(dims, w))
    return hi / lo


def grid_diameter(desc: dict) -> int:
    """Graph diameter of the grid: the sum over the axes of (points - 1)."""
    dims = [desc["nx"], desc["ny"]] + ([desc["nz"]] if desc["family"] == "lap3d" else [])
    return int(sum(m - 1 for m in dims))


def laplacian_sample(count: int, seed: int = 0, n_lo: float = 1e3, n_hi: float = 2.6e5) -> list[dict]:
    """Seeded 2-D (70 %) and 3-D 5/7-point Dirichlet Laplacians, n log-uniform
    in [n_lo, n_hi] before the grid sides are rounded.  The shape sets the diameter and, through its shortest
    side, the smallest eigenvalue, so the two vary apart: 2-D aspect ratios
    log-uniform in [1, 256], 3-D grids with the z side 1 to 64 times shorter.
    Coupling c (y in 2-D, z in 3-D) is 1, or 1e-2 in a quarter of the
    matrices; the shift sigma is 0 in a quarter, else log-uniform in
    [1e-5, 3], which moves kappa across the four classes."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        n = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        c = 1.0 if rng.random() < 0.75 else 1e-2
        sigma = 0.0 if rng.random() < 0.25 else float(10.0 ** rng.uniform(-5.0, math.log10(3.0)))
        if rng.random() < 0.7:
            a = math.exp(rng.uniform(0.0, math.log(256.0)))
            nx = max(2, int(round(math.sqrt(n * a))))
            ny = max(2, int(round(n / nx)))
            d = {"family": "lap2d", "nx": nx, "ny": ny}
        else:
            a = math.exp(rng.uniform(0.0, math.log(64.0)))
            nx = max(2, int(round((n * a) ** (1.0 / 3.0))))
            nz = max(2, int(round(n / (nx * nx))))
            d = {"family": "lap3d", "nx": nx, "ny": nx, "nz": nz}
        d.update(c=c, sigma=sigma, seed=seed * 1_000_003 + j)
        out.append(d)
    return out


def kappa_class(kappa: np.ndarray) -> np.ndarray:
    """Index 0..3 of the Sec. 7 class of each condition number."""
    return np.searchsorted(np.asarray(KAPPA_BOUNDS), np.asarray(kappa, float), side="left")


def optimal_efficiency(n1: np.ndarray, n2: np.ndarray, ndp: np.ndarray, omega) -> np.ndarray:
    """E(A) of Eq. (12) at the optimal eps1: Eq. (4) minimised over the
    candidates (ties to the smallest t), per matrix (rows of n1, n2)."""
    w = np.broadcast_to(np.asarray(omega, float).reshape(-1, 1) if np.ndim(omega) else omega,
                        n1.shape)
    cost = w * n1 + n2
    best = cost[np.arange(cost.shape[0]), np.argmin(cost, axis=1)]
    return (1.0 - best / ndp) * 100.0


def kappa_table(kappa, pdiam, E) -> list[dict]:
    """One row per condition-number class, as in Tables 1-3: the mean E, the
    mean pseudo-diameter and the count; then the mean pseudo-diameter and
    count of the matrices below the class's mean E, and of those at or above
    it (the two groups partition the class).  Empty classes give None."""
    kappa, pdiam, E = (np.asarray(v, float) for v in (kappa, pdiam, E))
    cls = kappa_class(kappa)
    rows = []
    for c, name in enumerate(KAPPA_NAMES):
        sel = cls == c
        N = int(sel.sum())
        if N == 0:
            rows.append({"kappa": name, "N": 0, "ME": None, "Ml": None, "worse": None,
                         "better": None})
            continue
        e, l = E[sel], pdiam[sel]
        me = float(e.mean())
        lo, hi = e < me, e >= me
        grp = lambda m: {"Ml": float(l[m].mean()) if m.any() else None, "N": int(m.sum())}
        rows.append({"kappa": name, "N": N, "ME": me, "Ml": float(l.mean()),
                     "worse": grp(lo), "better": grp(hi)})
    return rows


def kappa_study(count: int = 2400, seed: int = 0, device="cuda", chunk: int = 600,
                eps2: float = 1e-10, log=None) -> dict:
    """The Tables 1-3 analogue on laplacian_sample(count): GPU sweeps (chunks
    of `chunk` systems per batch), then kappa_table for omega = 1/3 and the
    matrix's measured omega.  Systems with a failed solve are left out and
    counted; the GPU pseudo-diameter is checked against the grid diameter."""
    descs = laplacian_sample(count, seed)
    kap, pd, n1, n2, ndp, om = [], [], [], [], [], []
    failed = pd_mismatch = 0
    t0 = time.time()
    for s in range(0, count, chunk):
        part = descs[s:s + chunk]
        rec = sweep_records(part, device, eps2=eps2)
        ok = (rec["status"] >= 0).all(axis=1) & (rec["status_dp"] >= 0)
        failed += int((~ok).sum())
        for i, d in enumerate(part):
            if not ok[i]:
                continue
            kap.append(kappa_closed_form(d))
            pd.append(float(rec["feat"][i, 2]))
            pd_mismatch += int(rec["feat"][i, 2] != grid_diameter(d))
            n1.append(rec["n1"][i])
            n2.append(rec["n2"][i])
            ndp.append(rec["n_dp"][i])
            om.append(rec["omega"][i])
        if log:
            log(f"kappa study: {min(s + chunk, count)}/{count} systems, {time.time() - t0:.0f} s")
        del rec
        torch.cuda.empty_cache()
    kap, pd, om = np.array(kap), np.array(pd), np.array(om)
    n1, n2, ndp = np.array(n1), np.array(n2), np.array(ndp, float)
    E13 = optimal_efficiency(n1, n2, ndp, 1.0 / 3.0)
    Em = optimal_efficiency(n1, n2, ndp, om)
    cls = kappa_class(kap)
    corr = {}
    for c, name in enumerate(KAPPA_NAMES):
        sel = cls == c
        if sel.sum() >= 3 and np.std(pd[sel]) > 0 and np.std(E13[sel]) > 0:
            corr[name] = float(np.corrcoef(np.log(pd[sel]), E13[sel])[0, 1])
    return {"systems": count, "used": int(kap.size), "failed": failed,
            "pdiam_not_grid_diameter": pd_mismatch, "omega_measured_mean": float(om.mean()),
            "table_omega_1_3": kappa_table(kap, pd, E13),
            "table_omega_measured": kappa_table(kap, pd, Em),
            "corr_E_log_pdiam_omega_1_3": corr, "seconds": round(time.time() - t0, 1)}
