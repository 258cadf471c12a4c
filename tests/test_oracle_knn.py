"""Pins of the oracle's kNN (Sec. 11): selection, scaling and vote."""
import math

import numpy as np
import pytest

import oracle
import synth


def scaled(feat, lo, hi):
    out = np.zeros_like(feat, dtype=float)
    for c in range(4):
        if hi[c] > lo[c]:
            out[..., c] = (feat[..., c] - lo[c]) / (hi[c] - lo[c])
    return out


def brute_force(chi, feat, cls, k, weighted=1, mask=0xF, lo=None, hi=None):
    lo = feat.min(axis=0) if lo is None else lo
    hi = feat.max(axis=0) if hi is None else hi
    q = scaled(np.asarray(chi, float), lo, hi)
    P = scaled(feat, lo, hi)
    d2 = []
    for i in range(feat.shape[0]):
        s = 0.0
        for c in range(4):
            if mask >> c & 1:
                s = s + (q[c] - P[i, c]) ** 2
        d2.append((s, i))
    d2.sort()
    sel = d2[:min(k, len(d2))]
    score = {}
    if sel[0][0] == 0.0:
        for s, i in sel:
            if s == 0.0:
                score[int(cls[i])] = score.get(int(cls[i]), 0) + 1
    else:
        for s, i in sel:
            score[int(cls[i])] = score.get(int(cls[i]), 0.0) + (1 / math.sqrt(s) if weighted else 1)
    best = max(score.values())
    return min(t for t, v in score.items() if v == best), [i for _, i in sel]


def paper_procedure(dists, k):
    """The selection procedure of Sec. 11.2: keep the first k, then replace the
    farthest kept element when a later one is strictly closer.  Among equal
    farthest elements the most recently indexed one is replaced."""
    N = list(range(k))
    for i in range(k, len(dists)):
        far = max(N, key=lambda j: (dists[j], j))
        if dists[i] < dists[far]:
            N.remove(far)
            N.append(i)
    return sorted(N, key=lambda j: (dists[j], j))


@pytest.mark.parametrize("seed", range(6))
def test_selection_equals_paper_procedure(seed):
    rng = np.random.default_rng(seed)
    feat, cls = synth.random_sample(120, seed=seed)
    feat[::7] = feat[3]          # exact ties in distance
    chi = feat[rng.integers(0, 120)] * rng.uniform(0.8, 1.2, 4)
    lo, hi = feat.min(axis=0), feat.max(axis=0)
    q = scaled(chi, lo, hi)
    d = ((scaled(feat, lo, hi) - q) ** 2).sum(axis=1)
    for k in (1, 5, 10, 20):
        t, nbr, _ = oracle.knn(chi, (feat, cls), k=k, details=True)
        assert list(nbr) == paper_procedure(list(d), k)


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("weighted", [0, 1])
@pytest.mark.parametrize("mask", [0xF, 0xE, 0x5])
def test_knn_matches_brute_force(seed, weighted, mask):
    rng = np.random.default_rng(100 + seed)
    feat, cls = synth.random_sample(200, seed=seed)
    feat[10:20] = feat[30]
    chi = np.array([rng.uniform(1e3, 3e6), rng.uniform(5e3, 2e7), rng.uniform(1, 1e5),
                    rng.uniform(0, 1.2)])
    for k in (1, 3, 5, 15):
        t_ref, sel = brute_force(chi, feat, cls, k, weighted, mask)
        t, nbr, _ = oracle.knn(chi, (feat, cls), k=k, weighted=weighted, feat_mask=mask, details=True)
        assert t == t_ref and list(nbr) == sel


def test_hand_example_weighted_vs_unweighted():
    """Query at the origin (after scaling); one class-3 neighbour very close,
    two class-6 neighbours further away.  Weighted vote -> 3 (1/0.1 > 2/1),
    unweighted -> 6."""
    feat = np.array([[0.0, 0, 0, 0], [10, 10, 10, 10], [0.1 * 10, 0, 0, 0],
                     [0, 10 * 1.0, 0, 0], [0, 0, 10 * 1.0, 0], [10, 10, 10, 9]])
    cls = np.array([7, 2, 3, 6, 6, 2], np.int8)
    chi = np.array([0.0, 0, 0, 0]) + np.array([0, 0, 0, 1e-9])
    # exclude row 0 (it would be at distance ~0)
    feat, cls = feat[1:], cls[1:]
    lo, hi = np.zeros(4), np.full(4, 10.0)
    t_w = oracle.knn(chi, oracle.sample(feat, cls, lo, hi), k=3, weighted=1)
    t_u = oracle.knn(chi, oracle.sample(feat, cls, lo, hi), k=3, weighted=0)
    assert (t_w, t_u) == (3, 6)


def test_zero_distance_and_tie_rules():
    feat = np.array([[1.0, 1, 1, 1], [2, 2, 2, 2], [1, 1, 1, 1], [3, 3, 3, 3]])
    lo, hi = np.zeros(4), np.full(4, 4.0)
    # two zero-distance neighbours of classes 6 and 4 -> tie -> smaller t = 4
    t = oracle.knn(np.array([1.0, 1, 1, 1]), oracle.sample(feat, np.array([6, 2, 4, 2], np.int8), lo, hi), k=3)
    assert t == 4
    # equidistant neighbours with different classes -> smaller t
    t = oracle.knn(np.array([2.0, 2, 2, 2]), oracle.sample(feat[[0, 3]], np.array([7, 5], np.int8), lo, hi), k=2)
    assert t == 5


def test_scaling_constant_component_and_unclamped_query():
    feat = np.array([[5.0, 1, 1, 0.5], [5.0, 2, 2, 0.6], [5.0, 3, 9, 0.9]])
    cls = np.array([2, 3, 4], np.int8)
    chi = np.array([1e6, 10.0, 50.0, 0.9])   # outside the sample range on three components
    for w, expect in ((0, 3), (1, 4)):   # unweighted: 1-1 tie -> smaller t
        t_ref, sel = brute_force(chi, feat, cls, 2, w)
        t, nbr, _ = oracle.knn(chi, (feat, cls), k=2, weighted=w, details=True)
        assert t == t_ref == expect and list(nbr) == sel == [2, 1]


def test_k_larger_than_sample():
    feat, cls = synth.random_sample(4, seed=3)
    t, nbr, _ = oracle.knn(feat[0] * 1.01, (feat, cls), k=9, details=True)
    assert len(nbr) == 4 and t == brute_force(feat[0] * 1.01, feat, cls, 9)[0]
