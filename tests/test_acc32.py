"""GPU tests of the option acc32 (the single-precision stage's inner products
summed in float, the other reading of Sec. 9, Remark 3).

- On a diagonal system built so that every float sum of b^T b equals its
  large term in any order, v of Eq. (13) after one iteration has a closed form
  under each reading: the single-system kernels (k_cg32 through mpcg_features,
  k_stage1 through Algorithm II) and the team kernels (batch) must give it
  bit for bit.
- Against the oracle with the same option (sequential float sums, where the
  GPU sums along its tree): statuses equal, N1 within 2 % or 2 iterations
  (see close_count; 10 % on the two order-sensitive systems), N2 within 10 %
  or 4 iterations (see n2_close),
  x within 1e-6, true residual <= eps2; labels from the kNN on the GPU's own
  features.
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_08059_gb300 import build, mpcg
    build.build()
    mpcg.load()
    return mpcg


def close_count(a, b):
    """2 %, or 2 iterations on short runs: the two sides round float sums in
    different orders (a tree against a sequential sum), which on a sensitive
    system moves N1 by 2 (the extended star below: 39 against 41 at eps1 =
    1e-5; the oracle's own two readings differ by 2 there too)."""
    return abs(a - b) <= max(2, int(0.02 * max(a, b)))


def absorbing_diagonal(m):
    n = m + 1
    A = synth.from_edges(n, np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0),
                         np.concatenate([[2.0], np.ones(m)]), "absorbing_diag")
    b = np.concatenate([[2.0 ** 12], np.full(m, 2.0 ** -13)])
    rr1 = m * 2.0 ** -28
    return (A, b, math.sqrt(rr1) / math.sqrt(2.0 ** 24 + m * 2.0 ** -26),
            math.sqrt(rr1) / math.sqrt(2.0 ** 24))


@pytest.mark.parametrize("m", [4000, 300000])
def test_v_closed_form_single_system(mp, m):
    A, b, v_double, v_float = absorbing_diagonal(m)
    dA = mp.DeviceCSR.from_host(A)
    db = torch.from_numpy(b).cuda()
    for acc32, want in ((0, v_double), (1, v_float)):
        f = mp.features(dA, db, k0=1, acc32=acc32)            # k_cg32, k0 phase
        assert f["status"] >= 0 and f["k0_done"] == 1
        assert f["v"] == want, (acc32, f["v"], want)
        S = mp.DeviceSample(np.array([[A.n, A.nnz, 0.0, want]]), np.array([4], np.int8))
        x, r = mp.solve(dA, db, S, k0=1, acc32=acc32)         # k_stage1
        assert r["status"] >= 0 and r["k0_done"] == 1
        assert r["v"] == want, (acc32, r["v"], want)
        assert r["true_rel_resid"] <= 1e-10


def test_v_closed_form_batch(mp):
    mats, bs, want = [], [], []
    for m in (4000, 70000):
        A, b, vd, vf = absorbing_diagonal(m)
        mats.append(A)
        bs.append(b)
        want.append((vd, vf))
    dmats = [mp.DeviceCSR.from_host(A) for A in mats]
    dbs = [torch.from_numpy(b).cuda() for b in bs]
    S = mp.DeviceSample(np.array([[1e4, 1e4, 0.0, 1e-6]]), np.array([4], np.int8))
    for acc32 in (0, 1):
        xs = [torch.empty(A.n, dtype=torch.float64, device="cuda") for A in mats]
        ws = torch.empty(mp.batch_workspace_bytes(dmats), dtype=torch.uint8, device="cuda")
        res = mp.result_buffer(len(mats))
        mp.solve_batch_async(dmats, dbs, xs, mp.options(k0=1, acc32=acc32, team_rows=16384),
                             ws, res, S)
        torch.cuda.synchronize()
        for r, w in zip(mp.read_results(res, len(mats)), want):
            assert r["status"] >= 0 and r["k0_done"] == 1
            assert r["v"] == w[acc32], (acc32, r["v"], w)


# Systems whose single-precision stage is sensitive to the order of its float
# sums: the GPU's tree and the oracle's sequential sum round differently, and
# the counts part by more than 2 % (measured: extended star N1 39 against 41,
# random tree 250 against 267 at eps1 = 1e-5).  For them the counts are held
# to 10 %; status, x and the final residual keep the full bar.
SENSITIVE = {"extended star", "random tree"}


def systems():
    return [("lap2d", synth.laplacian_2d(128, 128)),
            ("lap3d aniso", synth.laplacian_3d(40, eps=1e-2, sigma=1e-3)),
            ("random regular", synth.random_regular_laplacian(30000, 8, 1e-3, seed=4)),
            ("extended star", synth.extended_star(50, 200, 1.1, extra=None, seed=3)),
            ("random tree", synth.random_tree_plus(20000, 0.5, 1.1, seed=2)),
            ("banded", synth.banded(20000, 29, 0.6, 1.1, seed=7))]


def n2_close(a, b):
    """The FP64 stage starts from an x~ whose last bits depend on the order of
    the float sums, and its residual can plateau near eps2 (the banded system:
    2.0e-10 for four iterations from one x~, straight through 1e-10 from the
    other; N2 18 against 14), so N2 is held to 10 % or 4 iterations."""
    return abs(a - b) <= max(4, int(0.10 * max(a, b)))


def parity(r, ro, x, xo, name=""):
    assert r["status"] == ro["status"], (r, ro)
    if name in SENSITIVE:
        assert abs(r["n1"] - ro["n1"]) <= max(2, int(0.10 * max(r["n1"], ro["n1"]))), \
            (name, r["n1"], ro["n1"])
    else:
        assert close_count(r["n1"], ro["n1"]), (name, r["n1"], ro["n1"])
    assert n2_close(r["n2"], ro["n2"]), (name, r["n2"], ro["n2"])
    if ro["status"] >= 0:
        assert r["true_rel_resid"] <= 1e-10
        assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)


@pytest.mark.parametrize("eps1", [1e-5, 1e-7])
def test_algorithm_i_parity_single_and_batch(mp, eps1):
    names, mats = zip(*systems())
    bs = [synth.rhs(A, seed=90 + i)[1] for i, A in enumerate(mats)]
    dmats = [mp.DeviceCSR.from_host(A) for A in mats]
    dbs = [torch.from_numpy(b).cuda() for b in bs]
    xs = [torch.empty(A.n, dtype=torch.float64, device="cuda") for A in mats]
    ws = torch.empty(mp.batch_workspace_bytes(dmats), dtype=torch.uint8, device="cuda")
    res = mp.result_buffer(len(mats))
    mp.solve_batch_async(dmats, dbs, xs, mp.options(eps1=eps1, acc32=1, team_rows=16384), ws,
                         res, None)
    torch.cuda.synchronize()
    rb = mp.read_results(res, len(mats))
    for name, A, dA, db, b, xb, r_b in zip(names, mats, dmats, dbs, bs, xs, rb):
        xo, ro = oracle.solve(A, b, eps1=eps1, acc32=1)
        x1, r1 = mp.solve(dA, db, None, eps1=eps1, acc32=1)
        parity(r1, ro, x1.cpu().numpy(), xo, name)
        parity(r_b, ro, xb.cpu().numpy(), xo, name)


@pytest.mark.parametrize("kw", [dict(precond=1), dict(stop_true_residual=1)],
                         ids=["pcg", "true-residual"])
def test_algorithm_i_parity_with_options(mp, kw):
    # Not the random regular graph here: under Jacobi PCG its FP64 residual
    # falls to 6e-10, climbs back to 1e-8 and falls again, so the iteration
    # that first meets 1e-10 moves from 10 to 20 with the last bits of x~.
    sel = [systems()[k] for k in (0, 1, 5)]
    for i, (name, A) in enumerate(sel):
        b = synth.rhs(A, seed=120 + i)[1]
        xo, ro = oracle.solve(A, b, eps1=1e-6, acc32=1, **kw)
        x, r = mp.solve(mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda(), None, eps1=1e-6,
                        acc32=1, **kw)
        parity(r, ro, x.cpu().numpy(), xo, name)


def test_algorithm_ii_parity(mp):
    names, mats = zip(*systems())
    feat, cls = synth.random_sample(200, seed=9)
    ns = np.array([A.n for A in mats], float)
    feat[:, 0] = np.exp(np.linspace(np.log(0.5 * ns.min()), np.log(2 * ns.max()), 200))
    feat[:, 1] = feat[:, 0] * np.linspace(3.0, 9.0, 200)[::-1]
    S = mp.DeviceSample(feat, cls)
    for i, (name, A) in enumerate(zip(names, mats)):
        b = synth.rhs(A, seed=150 + i)[1]
        x, r = mp.solve(mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda(), S, acc32=1)
        xo, ro = oracle.solve(A, b, S=(feat, cls), acc32=1)
        assert r["pdiam"] == ro["pdiam"]
        # v rests on float sums of n squares, which the two sides round in
        # different orders: a relative spread of about sqrt(n) u (measured
        # 7.6e-6 on the 64000-row system).  On the extended star the first
        # iterations' norms are dominated by the hub, whose magnitude
        # swallows the small terms of a float sum: v moves with the order
        # (the oracle's own two readings give 0.884 and 0.722), so there only
        # the label is checked, against the kNN on the GPU's own features.
        if name not in SENSITIVE:
            assert abs(r["v"] - ro["v"]) <= 1e-4 * ro["v"]
        assert r["cls"] == oracle.knn([A.n, A.nnz, r["pdiam"], r["v"]], (feat, cls))
        if r["cls"] == ro["cls"]:
            parity(r, ro, x.cpu().numpy(), xo, name)
        else:  # a label across a decision boundary: the GPU's own label, run in the oracle
            xo2, ro2 = oracle.solve(A, b, eps1=r["eps1"], acc32=1)
            assert n2_close(r["n2"], ro2["n2"])
            assert r["true_rel_resid"] <= 1e-10
