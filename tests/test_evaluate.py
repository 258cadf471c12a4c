"""The evaluation protocol of Sec. 12 (paper_2412_08059_gb300/evaluate.py).

CPU: the general-sample grids of Appendix A, Eq. (26) and the Eq. (4)
labels against the oracle's formulas, and the protocol's bookkeeping (splits,
Acc, Loc, E and E_opt of Eq. (27)) recomputed independently with the
oracle's kNN and efficiency.  GPU: mpcg_knn_batch against the oracle's kNN
(classes and neighbour lists exact), and the sweep of a small general
sample against the oracle's sweep (N1, N2, N_dp within 2 %; l~ exact)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import metrics
from paper_2412_08059_gb300 import evaluate as ev

torch = pytest.importorskip("torch")


def test_general_sample_sizes_follow_appendix_a():
    # extended stars: (lc, nc) pairs x 3 mu x 100 = the paper's |S_0|
    assert [len(ev.general_sample("xstar", n)) for n in (301, 501, 1001)] == [3000, 3600, 4800]
    for n, pairs in ev.STAR_PAIRS.items():
        assert all(1 + lc * nc == n for lc, nc in pairs)
    # random sparse: 8 values of c x 3 mu x 200
    assert [len(ev.general_sample("random", n)) for n in (300, 500, 1000)] == [4800] * 3
    # banded: b = 3..b_max, 3 densities, 20 each
    assert [len(ev.general_sample("banded", n)) for n in (300, 500, 1000)] == \
        [27 * 60, 49 * 60, 99 * 60]
    d = ev.general_sample("xstar", 301, per=2, seed=5)
    assert len(d) == 60 and len({x["seed"] for x in d}) == 60
    A = ev.build(d[7])
    assert A.n == 301


def test_training_size_and_labels_match_the_formulas():
    for n, k, kcg in [(300, 1, 57.3), (1001, 5, 120.0), (1000, 20, 35.5)]:
        assert ev.training_size(n, k, kcg) == int(np.floor(metrics.sample_size(n, k, kcg)))
    rng = np.random.default_rng(3)
    n1 = rng.integers(1, 200, (50, 6))
    n2 = rng.integers(1, 300, (50, 6))
    n1[0], n2[0] = [3, 6, 9, 12, 15, 18], [20, 19, 18, 17, 16, 15]  # ties across t
    got = ev.labels(n1, n2)
    want = [metrics.label(a, b) for a, b in zip(n1, n2)]
    assert list(got) == want


def oracle_classifier(weighted=1, feat_mask=0b1110):
    def classify(tr_feat, tr_cls, te_feat, k):
        S = oracle.sample(tr_feat, tr_cls)
        kk = min(k, tr_feat.shape[0])
        pred, nbr = [], []
        for q in te_feat:
            t, nb, _ = oracle.knn(q, S, k=k, weighted=weighted, feat_mask=feat_mask, details=True)
            pred.append(t)
            nbr.append(list(nb) + [-1] * (k - kk))
        return np.array(pred), np.array(nbr, dtype=np.int64)
    return classify


def fake_records(N=80, seed=11):
    rng = np.random.default_rng(seed)
    feat = np.column_stack([np.full(N, 300.0), rng.integers(900, 3000, N), rng.integers(2, 60, N),
                            rng.uniform(0.2, 0.95, N)]).astype(np.float64)
    n1 = rng.integers(2, 120, (N, 6))
    n2 = rng.integers(10, 300, (N, 6))
    ndp = rng.integers(100, 400, N)
    return {"feat": feat, "n1": n1, "n2": n2, "n_dp": ndp, "omega": rng.uniform(0.3, 1.2, N)}


def test_protocol_bookkeeping_against_an_independent_recount():
    rec = fake_records()
    ks, splits, seed, n = (1, 5), 3, 4, 300
    out = ev.protocol(rec, oracle_classifier(), n, ks=ks, splits=splits, seed=seed)
    cls = np.array([metrics.label(a, b) for a, b in zip(rec["n1"], rec["n2"])])
    N = len(cls)
    k_cg = rec["n_dp"].mean()
    assert out["N"] == N and out["k_CG"] == k_cg
    assert abs(sum(out["P"].values()) - 100.0) < 1e-9
    rng = np.random.default_rng(seed)
    for k in ks:
        ns = min(max(int(np.floor(metrics.sample_size(n, k, k_cg))), k), N - 1)
        assert out["k"][k]["N_S"] == ns and out["k"][k]["N_T"] == N - ns
        acc, loc, e13, eo13, em, eom = [], [], [], [], [], []
        for _ in range(splits):
            perm = rng.permutation(N)
            tr, te = perm[:ns], perm[ns:]
            S = oracle.sample(rec["feat"][tr], cls[tr].astype(np.int8))
            hits, same = 0, []
            I13 = Io13 = Im = Iom = Idp = 0.0
            for i in te:
                t, nb, _ = oracle.knn(rec["feat"][i], S, k=k, weighted=1, feat_mask=0b1110,
                                      details=True)
                hits += t == cls[i]
                same.append(np.mean(cls[tr][nb] == cls[i]))
                p, o = t - 2, cls[i] - 2
                I13 += metrics.cost_I(1 / 3, rec["n1"][i, p], rec["n2"][i, p])
                Io13 += metrics.cost_I(1 / 3, rec["n1"][i, o], rec["n2"][i, o])
                Im += metrics.cost_I(rec["omega"][i], rec["n1"][i, p], rec["n2"][i, p])
                Iom += metrics.cost_I(rec["omega"][i], rec["n1"][i, o], rec["n2"][i, o])
                Idp += rec["n_dp"][i]
            acc.append(100.0 * hits / len(te))
            loc.append(100.0 * np.mean(same))
            e13.append(metrics.efficiency(I13, Idp))
            eo13.append(metrics.efficiency(Io13, Idp))
            em.append(metrics.efficiency(Im, Idp))
            eom.append(metrics.efficiency(Iom, Idp))
        r = out["k"][k]
        assert r["Acc"] == pytest.approx([np.mean(acc), np.std(acc)], abs=1e-9)
        assert r["Loc"] == pytest.approx([np.mean(loc), np.std(loc)], abs=1e-9)
        assert r["E_omega_1_3"] == pytest.approx([np.mean(e13), np.mean(eo13)], abs=1e-9)
        assert r["E_omega_measured"] == pytest.approx([np.mean(em), np.mean(eom)], abs=1e-9)


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_08059_gb300 import build, mpcg
    build.build()
    mpcg.load()
    return mpcg


@pytest.mark.gpu
@pytest.mark.parametrize("count,k,weighted,mask", [(1, 5, 1, 0xF), (7, 5, 1, 0xF), (300, 1, 1, 0xE),
                                                    (300, 20, 0, 0xE), (2000, 15, 1, 0xF),
                                                    (150, 64, 1, 0x7)])
def test_knn_batch_matches_oracle(mp, count, k, weighted, mask):
    feat, cls = synth.random_sample(count, seed=count + k)
    rng = np.random.default_rng(count)
    q = feat[rng.integers(0, count, 257)].copy()          # exact hits: zero distances
    q[::3] *= rng.uniform(0.7, 1.3, (q[::3].shape[0], 4))  # and off-sample points
    q[5, 2] = np.nan if mask & 0b100 else q[5, 2]          # an invalid query
    S = mp.DeviceSample(feat, cls)
    got, nbr = mp.knn_batch(q, S, neighbours=True, knn_k=k, weighted=weighted, feat_mask=mask)
    got, nbr = got.cpu().numpy(), nbr.cpu().numpy()
    Sh = oracle.sample(feat, cls)
    for i, qi in enumerate(q):
        t, nb, _ = oracle.knn(qi, Sh, k=k, weighted=weighted, feat_mask=mask, details=True)
        assert got[i] == t, (i, got[i], t)
        if t >= 0:
            kk = min(k, count)
            assert list(nbr[i, :kk]) == list(nb) and np.all(nbr[i, kk:] == -1)


@pytest.mark.gpu
def test_knn_batch_empty_query_and_small_sample(mp):
    feat, cls = synth.random_sample(3, seed=1)
    S = mp.DeviceSample(feat, cls)
    got, nbr = mp.knn_batch(np.zeros((0, 4)), S, neighbours=True, knn_k=5)
    assert got.numel() == 0 and tuple(nbr.shape) == (0, 5)
    got, nbr = mp.knn_batch(feat, S, neighbours=True, knn_k=5)   # k > sample size
    for i in range(3):
        t, nb, _ = oracle.knn(feat[i], oracle.sample(feat, cls), k=5, details=True)
        assert got[i].item() == t and list(nbr[i, :3].cpu().numpy()) == list(nb)
        assert np.all(nbr[i, 3:].cpu().numpy() == -1)


@pytest.mark.gpu
def test_sweep_of_a_small_general_sample_matches_oracle(mp):
    descs = ev.general_sample("xstar", 301, per=1, seed=9)[::3]   # 10 stars, one per (lc, nc)
    rec = ev.sweep_records(descs)
    assert np.all(rec["status"] >= 0) and np.all(rec["status_dp"] >= 0)
    for i in (0, 3, 6, 9):
        A = ev.build(descs[i])
        b = synth.rhs(A, seed=descs[i]["seed"])[1]
        n1, n2, ndp, _, _ = metrics.sweep(A, b)
        close = lambda a, c: abs(a - c) <= max(1, int(0.02 * max(a, c)))
        assert all(close(a, c) for a, c in zip(rec["n1"][i], n1)), (rec["n1"][i], n1)
        assert all(close(a, c) for a, c in zip(rec["n2"][i], n2)), (rec["n2"][i], n2)
        assert close(rec["n_dp"][i], ndp)
        assert rec["feat"][i][2] == oracle.pseudo_diameter(A)
    assert np.all(np.isfinite(rec["omega"])) and np.all(rec["omega"] > 0)
    # the protocol through the GPU kNN equals the protocol through the oracle's kNN
    a = ev.protocol(rec, ev.gpu_classifier(), 301, ks=(1, 5), splits=4, seed=2)
    b = ev.protocol(rec, oracle_classifier(), 301, ks=(1, 5), splits=4, seed=2)
    assert a == b


@pytest.mark.gpu
def test_batched_sample_builder_labels_by_eq4_with_the_team_omega(mp):
    """sample.build_batched: every label is the Eq. (4) argmin with the
    matrix's measured omega (a recount through oracle/metrics.py), and the
    features' pseudo-diameters are the oracle's."""
    from paper_2412_08059_gb300 import sample
    systems = []
    for i, d in enumerate(synth.batch_family(24, seed=31, n_lo=1e3, n_hi=4e4)):
        A = synth.build_desc(d)
        systems.append((f"s{i}", A, synth.rhs(A, seed=700 + i)[1]))
    feat, cls, recs = sample.build_batched(systems)
    assert len(recs) == len(systems) == feat.shape[0] == cls.size
    for (name, A, b), f, c, r in zip(systems, feat, cls, recs):
        assert r["name"] == name and r["omega"] > 0
        assert c == metrics.label(r["n1"], r["n2"], r["omega"])
        assert (f[0], f[1]) == (A.n, A.nnz)
        assert f[2] == oracle.pseudo_diameter(A)
