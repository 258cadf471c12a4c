"""The condition-number study (Sec. 7, Tables 1-3 analogue) on CPU: the closed-form
kappa and grid diameter of its Laplacians against dense eigenvalues and the
oracle's 2BFS, the class boundaries of Sec. 7, and the table bookkeeping
against a recount through oracle/metrics.py on oracle sweeps of a small subset."""
import math

import numpy as np
import pytest

import oracle
from oracle import metrics
from paper_2412_08059_gb300 import evaluate as ev


SMALL = [
    {"family": "lap2d", "nx": 7, "ny": 5, "c": 1.0, "sigma": 0.0},
    {"family": "lap2d", "nx": 9, "ny": 4, "c": 1e-2, "sigma": 0.3},
    {"family": "lap2d", "nx": 31, "ny": 2, "c": 1.0, "sigma": 1e-4},
    {"family": "lap3d", "nx": 4, "ny": 4, "nz": 3, "c": 1e-2, "sigma": 1e-3},
    {"family": "lap3d", "nx": 5, "ny": 5, "nz": 5, "c": 1.0, "sigma": 0.0},
    {"family": "lap3d", "nx": 6, "ny": 6, "nz": 2, "c": 1.0, "sigma": 2.5},
]


@pytest.mark.parametrize("d", SMALL, ids=lambda d: f"{d['family']}-{d['nx']}")
def test_closed_form_kappa_and_diameter(d):
    A = ev.build(dict(d, seed=0))
    ev_ = np.linalg.eigvalsh(A.to_dense())
    assert ev.kappa_closed_form(d) == pytest.approx(ev_[-1] / ev_[0], rel=1e-10)
    assert oracle.pseudo_diameter(A) == ev.grid_diameter(d)


def test_kappa_class_bounds():
    k = np.array([1.0, 10.0, np.nextafter(10.0, 11.0), 100.0, 100.5, 1000.0, 1000.001, 1e9])
    assert ev.kappa_class(k).tolist() == [0, 0, 1, 1, 2, 2, 3, 3]


def test_sample_is_seeded_and_spans_the_classes():
    a, b = ev.laplacian_sample(400, seed=3), ev.laplacian_sample(400, seed=3)
    assert a == b
    assert a != ev.laplacian_sample(400, seed=4)
    cls = ev.kappa_class([ev.kappa_closed_form(d) for d in a])
    assert set(cls.tolist()) == {0, 1, 2, 3}
    n = [d["nx"] * d["ny"] * d.get("nz", 1) for d in a]
    assert 700 <= min(n) and max(n) <= 2.7e5  # shapes round n by up to ~15 %


def _recount(kappa, pdiam, n1s, n2s, ndp, omegas):
    """Tables 1-3 bookkeeping written with the paper's definitions, one matrix
    at a time: the Eq. (4) label through metrics.label, E of Eq. (12) through
    metrics.cost_I and metrics.efficiency, the classes of Sec. 7 by hand."""
    def which(k):
        if k <= 10:
            return 0
        if k <= 100:
            return 1
        if k <= 1000:
            return 2
        return 3

    per = {c: [] for c in range(4)}
    for k, l, a, b, dp, w in zip(kappa, pdiam, n1s, n2s, ndp, omegas):
        t = metrics.label(a, b, w)
        j = metrics.CLASSES.index(t)
        E = metrics.efficiency(metrics.cost_I(w, a[j], b[j]), dp)
        per[which(k)].append((E, l))
    rows = []
    for c in range(4):
        items = per[c]
        if not items:
            rows.append((0, None, None, None, None))
            continue
        me = sum(e for e, _ in items) / len(items)
        worse = [l for e, l in items if e < me]
        better = [l for e, l in items if not e < me]
        mean = lambda v: sum(v) / len(v) if v else None
        rows.append((len(items), me, mean([l for _, l in items]), (mean(worse), len(worse)),
                     (mean(better), len(better))))
    return rows


def _close(a, b):
    return (a is None and b is None) or (a is not None and b is not None
                                        and math.isclose(a, b, rel_tol=1e-12, abs_tol=1e-12))


def test_table_bookkeeping_equals_a_recount_on_oracle_sweeps():
    descs = ev.laplacian_sample(10, seed=11, n_lo=30, n_hi=400) + [
        {"family": "lap2d", "nx": 60, "ny": 60, "c": 1.0, "sigma": 0.0, "seed": 5},
        {"family": "lap2d", "nx": 40, "ny": 12, "c": 1.0, "sigma": 1.5, "seed": 6}]
    import synth
    kappa, pdiam, n1, n2, ndp = [], [], [], [], []
    for d in descs:
        A = ev.build(d)
        _, b = synth.rhs(A, seed=d["seed"])
        a1, a2, dp, st, st_dp = metrics.sweep(A, b, eps2=1e-10)
        assert all(s >= 0 for s in st) and st_dp >= 0
        kappa.append(ev.kappa_closed_form(d))
        pdiam.append(float(oracle.pseudo_diameter(A)))
        n1.append(a1)
        n2.append(a2)
        ndp.append(dp)
    assert len(set(ev.kappa_class(kappa).tolist())) >= 3
    n1, n2, ndp = np.array(n1), np.array(n2), np.array(ndp, float)
    omegas = 0.25 + 0.5 * np.random.default_rng(0).random(len(descs))  # a measured-omega stand-in
    for w in (np.full(len(descs), 1.0 / 3.0), omegas):
        E = ev.optimal_efficiency(n1, n2, ndp, w if not np.all(w == w[0]) else float(w[0]))
        got = ev.kappa_table(kappa, pdiam, E)
        want = _recount(kappa, pdiam, n1, n2, ndp, w)
        for g, (N, me, ml, worse, better) in zip(got, want):
            assert g["N"] == N
            if N == 0:
                continue
            assert _close(g["ME"], me) and _close(g["Ml"], ml)
            assert _close(g["worse"]["Ml"], worse[0]) and g["worse"]["N"] == worse[1]
            assert _close(g["better"]["Ml"], better[0]) and g["better"]["N"] == better[1]
            assert g["worse"]["N"] + g["better"]["N"] == N
