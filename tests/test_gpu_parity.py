"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bars (from the method's definition and the readings in the sources):
* SpMV (single and double), BFS distances, 2BFS (l~, t), kNN labels on
  identical feature vectors: bit-exact.
* Iteration counts N1, N2 (and N_dp of pure FP64 CG): within 2 % (at least 1).
* Solution: ||x_gpu - x_oracle|| <= 1e-6 ||x_oracle||; true residual <= eps2.
"""
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
    return abs(a - b) <= max(1, int(0.02 * max(a, b)))


MATRICES = {
    "lap2d_37x29": lambda: synth.laplacian_2d(37, 29),            # ragged last slice
    "lap3d_13": lambda: synth.laplacian_3d(13, eps=1e-2, sigma=1e-3),
    "rreg_3000": lambda: synth.random_regular_laplacian(3000, 8, 1e-3, seed=4),
    "star_1001": lambda: synth.star(1001, 1.1),                    # one row of 1000 entries
    "xstar_20x50": lambda: synth.extended_star(20, 50, 1.1, extra=None, seed=3),
    "rtree_1000_c10": lambda: synth.random_tree_plus(1000, 10.0, 1.1, seed=2),
    "band_1000_b29": lambda: synth.banded(1000, 29, 0.6, 1.1, seed=7),
}


@pytest.mark.parametrize("name", sorted(MATRICES))
def test_spmv_bit_exact(mp, name):
    A = MATRICES[name]()
    dA = mp.DeviceCSR.from_host(A)
    rng = np.random.default_rng(11)
    x64 = rng.standard_normal(A.n)
    x32 = rng.standard_normal(A.n).astype(np.float32)
    y64 = mp.spmv(dA, torch.from_numpy(x64).cuda()).cpu().numpy()
    y32 = mp.spmv(dA, torch.from_numpy(x32).cuda()).cpu().numpy()
    assert np.array_equal(y64, oracle.spmv64(A, x64))
    assert np.array_equal(y32, oracle.spmv32(A, x32))


def disjoint(*mats):
    rp, cols, vals, off, base = [np.zeros(1, np.int64)], [], [], 0, 0
    for A in mats:
        rp.append(A.row_ptr[1:].astype(np.int64) + base)
        cols.append(A.col.astype(np.int64) + off)
        vals.append(A.val)
        off += A.n
        base += A.nnz
    return synth.CSR(np.concatenate(rp).astype(np.int32), np.concatenate(cols).astype(np.int32),
                     np.concatenate(vals))


def cycle(n):
    i = np.arange(n, dtype=np.int64)
    return synth.from_edges(n, i, (i + 1) % n, -np.ones(n), np.full(n, 2.2), f"cycle_{n}")


def caterpillar(spine, legs):
    """A path of `spine` vertices, each with `legs` leaves (numbered after the spine)."""
    i = list(range(spine - 1))
    j = list(range(1, spine))
    for v in range(spine):
        for k in range(legs):
            i.append(v)
            j.append(spine + v * legs + k)
    n = spine * (1 + legs)
    deg = np.bincount(np.concatenate([i, j]), minlength=n).astype(float)
    return synth.from_edges(n, np.array(i), np.array(j), -np.ones(len(i)), 1.1 * deg, "caterpillar")


def lollipop(k, tail):
    """A clique on k vertices with a path of `tail` vertices hanging off vertex k - 1."""
    i, j = [], []
    for a in range(k):
        for b in range(a + 1, k):
            i.append(a)
            j.append(b)
    for v in range(k - 1, k + tail - 1):
        i.append(v)
        j.append(v + 1)
    n = k + tail
    deg = np.bincount(np.concatenate([i, j]), minlength=n).astype(float)
    return synth.from_edges(n, np.array(i), np.array(j), -np.ones(len(i)), 1.1 * deg, "lollipop")


GRAPHS = dict(MATRICES)
GRAPHS.update({
    "path_2000": lambda: synth.path(2000),
    "band_p04_disconnected": lambda: synth.banded(3000, 3, 0.4, seed=1),
    "union": lambda: disjoint(synth.path(50), synth.star(40), synth.laplacian_2d(9, 7),
                              synth.from_edges(1, [], [], np.zeros(0), np.ones(1)),
                              synth.random_regular_laplacian(500, 4, seed=2)),
    "single": lambda: synth.from_edges(1, [], [], np.zeros(0), np.ones(1)),
    # narrow frontiers of the dual search (one warp, frontier tables): fronts that
    # meet at one level or at neighbouring levels, leaves off a path, a dense end
    "cycle_2001": lambda: cycle(2001),
    "cycle_2000": lambda: cycle(2000),
    "caterpillar": lambda: caterpillar(700, 3),
    "lollipop": lambda: lollipop(30, 900),
    "grid_37x300": lambda: synth.laplacian_2d(37, 300),
})


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_bfs_and_pseudo_diameter_bit_exact(mp, name):
    A = GRAPHS[name]()
    dA = mp.DeviceCSR.from_host(A)
    for src in sorted({0, A.n // 2, A.n - 1}):
        d_gpu = mp.bfs(dA, src).cpu().numpy()
        d_orc, _ = oracle.bfs(A, src)
        assert np.array_equal(d_gpu, d_orc), src
    assert mp.pseudo_diameter(dA) == oracle.pseudo_diameter(A, return_t=True)


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("weighted,mask", [(1, 0xF), (0, 0xF), (1, 0xE), (1, 0x9)])
def test_knn_labels_bit_exact_on_identical_features(mp, seed, weighted, mask):
    rng = np.random.default_rng(seed)
    feat, cls = synth.random_sample(300, seed=seed)
    feat[40:60] = feat[7]                    # duplicated rows: distance ties
    S = mp.DeviceSample(feat, cls)
    for q in range(25):
        if q % 5 == 0:
            chi = feat[rng.integers(0, 300)].copy()          # zero distance
        else:
            chi = np.array([rng.uniform(1e3, 3e6), rng.uniform(4e3, 2e7), rng.uniform(2, 8e4),
                            rng.uniform(0.1, 1.1)])
        for k in (1, 5, 20):
            eps, t = mp.choose_eps1(chi, S, knn_k=k, weighted=weighted, feat_mask=mask)
            t_orc = oracle.knn(chi, (feat, cls), k=k, weighted=weighted, feat_mask=mask)
            assert t == t_orc
            assert eps == float(f"1e-{t}")


def parity(r, ro, x, xo, eps2=1e-10):
    assert r["status"] == ro["status"], (r, ro)
    assert close_count(r["n1"], ro["n1"]), (r["n1"], ro["n1"])
    assert close_count(r["n2"], ro["n2"]), (r["n2"], ro["n2"])
    if ro["status"] >= 0:
        assert r["true_rel_resid"] <= eps2
        assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)


def test_config1_poisson64_algorithm_i(mp):
    """64x64 Poisson, x* ~ U[-1,1] seed 1, eps1 = 1e-4, eps2 = 1e-10."""
    A, xs, b = synth.poisson64()
    x, r = mp.solve(mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda(), eps1=1e-4, eps2=1e-10)
    xo, ro = oracle.solve(A, b, eps1=1e-4, eps2=1e-10)
    x = x.cpu().numpy()
    parity(r, ro, x, xo)
    assert r["n1"] == ro["n1"]  # single-precision stage follows the same trajectory
    err_o = np.linalg.norm(xo - xs) / np.linalg.norm(xs)
    err_g = np.linalg.norm(x - xs) / np.linalg.norm(xs)
    assert err_g <= 2 * err_o + 1e-12


@pytest.mark.parametrize("name", ["lap2d_37x29", "lap3d_13", "rreg_3000", "xstar_20x50",
                                  "rtree_1000_c10", "band_1000_b29"])
@pytest.mark.parametrize("eps1", [1e-2, 1e-4, 1e-6])
def test_algorithm_i_parity(mp, name, eps1):
    A = MATRICES[name]()
    xs, b = synth.rhs(A, seed=3)
    x, r = mp.solve(mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda(), eps1=eps1)
    xo, ro = oracle.solve(A, b, eps1=eps1)
    parity(r, ro, x.cpu().numpy(), xo)


@pytest.mark.parametrize("name", ["lap2d_37x29", "rreg_3000", "star_1001", "band_1000_b29"])
def test_pure_fp64_parity(mp, name):
    A = MATRICES[name]()
    xs, b = synth.rhs(A, seed=5)
    x, r = mp.solve(mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda(), fp64_only=1)
    xo, it, st = oracle.cg64(A, b, 1e-10)
    assert r["status"] == 0 and st == 0 and r["n1"] == 0
    assert close_count(r["n2"], it)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-6 * np.linalg.norm(xo)


@pytest.mark.parametrize("name", ["lap2d_37x29", "lap3d_13", "rreg_3000", "band_1000_b29",
                                  "xstar_20x50"])
def test_algorithm_ii_parity(mp, name):
    A = MATRICES[name]()
    xs, b = synth.rhs(A, seed=9)
    feat, cls = synth.random_sample(200, seed=1)
    # put the matrix's own (n, m) into the sample range so that every feature matters
    feat[:, 0] = np.linspace(0.5, 2.0, 200) * A.n
    feat[:, 1] = np.linspace(0.5, 2.0, 200)[::-1] * A.nnz
    S = mp.DeviceSample(feat, cls)
    dA = mp.DeviceCSR.from_host(A)
    db = torch.from_numpy(b).cuda()
    f = mp.features(dA, db)
    fo, k0d, _ = oracle.features(A, b)
    assert (f["n"], f["m"], f["pdiam"], f["k0_done"]) == (fo[0], fo[1], fo[2], k0d)
    assert abs(f["v"] - fo[3]) <= 1e-12 * max(1.0, abs(fo[3]))
    x, r = mp.solve(dA, db, S)
    xo, ro = oracle.solve(A, b, S=(feat, cls))
    # kNN on the GPU's own features must give the oracle's label (bit-exact)
    assert r["cls"] == oracle.knn([f["n"], f["m"], f["pdiam"], f["v"]], (feat, cls))
    assert r["pdiam"] == ro["pdiam"] and abs(r["v"] - ro["v"]) <= 1e-12
    assert r["cls"] == ro["cls"] and r["eps1"] == ro["eps1"]
    parity(r, ro, x.cpu().numpy(), xo)


def test_edge_cases(mp):
    A = synth.laplacian_2d(20, 10)
    dA = mp.DeviceCSR.from_host(A)
    # b = 0: x = 0 exactly
    x, r = mp.solve(dA, torch.zeros(A.n, dtype=torch.float64, device="cuda"), eps1=1e-4)
    assert r["status"] == 0 and not x.any().item() and r["n1"] == r["n2"] == 0
    # NaN in b
    b = np.ones(A.n)
    b[5] = np.nan
    _, r = mp.solve(dA, torch.from_numpy(b).cuda(), eps1=1e-4)
    assert r["status"] == mp.ERR_NAN
    # not SPD
    neg = mp.DeviceCSR.from_host(synth.CSR(A.row_ptr, A.col, -A.val))
    _, r = mp.solve(neg, torch.ones(A.n, dtype=torch.float64, device="cuda"), eps1=1e-4)
    _, ro = oracle.solve(synth.CSR(A.row_ptr, A.col, -A.val), np.ones(A.n), eps1=1e-4)
    assert r["status"] == ro["status"] == mp.ERR_BREAKDOWN
    # caps
    xs, b = synth.rhs(A, 2)
    db = torch.from_numpy(b).cuda()
    _, r = mp.solve(dA, db, eps1=1e-4, max_it_fp64=3)
    _, ro = oracle.solve(A, b, eps1=1e-4, max_it_fp64=3)
    assert r["status"] == ro["status"] == mp.ERR_NOT_CONVERGED and r["n2"] == 3
    x, r = mp.solve(dA, db, eps1=1e-4, max_it_fp32=4)
    xo, ro = oracle.solve(A, b, eps1=1e-4, max_it_fp32=4)
    assert r["status"] == ro["status"] == mp.WARN_EPS1_NOT_REACHED and r["n1"] == 4
    # n = 1
    one = synth.from_edges(1, [], [], np.zeros(0), np.full(1, 2.0))
    x, r = mp.solve(mp.DeviceCSR.from_host(one), torch.full((1,), 3.0, dtype=torch.float64,
                                                           device="cuda"), eps1=1e-4)
    assert r["status"] == 0 and abs(x.item() - 1.5) < 1e-15


def test_invalid_csr_is_reported_not_faulted(mp):
    A = synth.laplacian_2d(8, 8)
    b = torch.ones(A.n, dtype=torch.float64, device="cuda")
    bad_col = A.col.copy()
    bad_col[5] = A.n + 7                       # out of range
    _, r = mp.solve(mp.DeviceCSR(A.row_ptr, bad_col, A.val), b, eps1=1e-4)
    assert r["status"] == mp.ERR_INVALID_ARG
    unsorted = A.col.copy()
    unsorted[[0, 1]] = unsorted[[1, 0]]
    _, r = mp.solve(mp.DeviceCSR(A.row_ptr, unsorted, A.val), b, eps1=1e-4)
    assert r["status"] == mp.ERR_INVALID_ARG
    bad_rp = A.row_ptr.copy()
    bad_rp[3] = 10**6
    _, r = mp.solve(mp.DeviceCSR(bad_rp, A.col, A.val), b, eps1=1e-4)
    assert r["status"] == mp.ERR_INVALID_ARG


def test_workspace_errors_are_return_codes(mp):
    A = synth.laplacian_2d(8, 8)
    dA = mp.DeviceCSR.from_host(A)
    b = torch.ones(A.n, dtype=torch.float64, device="cuda")
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError, match="workspace"):
        mp.solve(dA, b, ws=small, eps1=1e-4)
    big = mp.workspace(A.n, A.nnz)
    with pytest.raises(RuntimeError, match="workspace"):
        mp.solve(dA, b, ws=big[1:], eps1=1e-4)   # misaligned base
    with pytest.raises(RuntimeError, match="invalid"):
        mp.solve(dA, b)                           # Algorithm II without a sample


def test_repeated_solves_reuse_workspace_identically(mp):
    A = synth.random_regular_laplacian(5000, 8, 1e-3, seed=1)
    xs, b = synth.rhs(A, 1)
    dA = mp.DeviceCSR.from_host(A)
    db = torch.from_numpy(b).cuda()
    ws = mp.workspace(A.n, A.nnz)
    x1, r1 = mp.solve(dA, db, ws=ws, eps1=1e-5)
    x2, r2 = mp.solve(dA, db, ws=ws, eps1=1e-5)
    assert torch.equal(x1, x2) and (r1["n1"], r1["n2"]) == (r2["n1"], r2["n2"])


@pytest.mark.slow
def test_full_size_128cubed_properties(mp):
    """128^3 7-point Laplacian (n = 2,097,152): sampled rows of the FP32 SpMV are
    bit-exact, the 2BFS value is 381 (exact, 3 (N-1)), the k0 decay rate matches
    the oracle's, and the solution meets eps2 in a residual computed on the host."""
    A = synth.laplacian_3d(128)
    xs, b = synth.rhs(A, seed=1)
    dA = mp.DeviceCSR.from_host(A)
    db = torch.from_numpy(b).cuda()
    rng = np.random.default_rng(0)
    x32 = rng.standard_normal(A.n).astype(np.float32)
    y32 = mp.spmv(dA, torch.from_numpy(x32).cuda()).cpu().numpy()
    rows = np.sort(rng.choice(A.n, 5000, replace=False))
    # the oracle's single-precision SpMV on the sub-matrix of the sampled rows
    lens = A.row_ptr[rows + 1] - A.row_ptr[rows]
    sub_rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    idx = np.concatenate([np.arange(A.row_ptr[i], A.row_ptr[i + 1]) for i in rows])
    y_ref = oracle.spmv32((sub_rp, A.col[idx], A.val[idx]), x32)
    assert np.array_equal(y32[rows], y_ref)
    assert mp.pseudo_diameter(dA)[0] == 381
    f = mp.features(dA, db)
    fo, k0d, _ = oracle.features(A, b)
    assert f["pdiam"] == fo[2] == 381 and k0d == f["k0_done"] == 10
    assert abs(f["v"] - fo[3]) <= 1e-12
    for kw in ({"eps1": 1e-4}, {"fp64_only": 1}):
        x, r = mp.solve(dA, db, **kw)
        assert r["status"] == 0
        xn = x.cpu().numpy()
        res = b - synth.spmv_input(A, xn)
        assert np.linalg.norm(res) / np.linalg.norm(b) <= 1e-10 * 1.01
        assert np.linalg.norm(xn - xs) / np.linalg.norm(xs) <= 6744 * 1e-10


@pytest.mark.parametrize("classes", [(0, 1, 9), (1, 9), (9,)])
def test_algorithm_ii_classes_outside_two_to_seven(mp, classes):
    """Labels whose eps1 = 10^-t is met at once (t = 0, 1) or never in single
    precision (t = 9: the stage stops at its cap with a warning), as the
    oracle does."""
    A = synth.laplacian_2d(37, 29)
    xs, b = synth.rhs(A, seed=12)
    feat, cls = synth.random_sample(200, seed=4, classes=classes)
    feat[:, 0] = np.linspace(0.5, 2.0, 200) * A.n
    feat[:, 1] = np.linspace(0.5, 2.0, 200)[::-1] * A.nnz
    S = mp.DeviceSample(feat, cls)
    x, r = mp.solve(mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda(), S)
    xo, ro = oracle.solve(A, b, S=(feat, cls))
    assert r["cls"] == ro["cls"] and r["eps1"] == ro["eps1"] and r["pdiam"] == ro["pdiam"]
    parity(r, ro, x.cpu().numpy(), xo)


@pytest.mark.parametrize("seed", [2, 10])
def test_algorithm_ii_more_classes_than_snapshots(mp, seed):
    """A sample with labels t = 0 .. 11 on a 5000-vertex path with a_ii = 2 deg:
    stage 1 meets the candidate eps1 within a few dozen iterations, long
    before the 2BFS of 4999 levels ends, and keeps only six snapshots of x~,
    so past the sixth crossing it waits for the label (here t = 8 and 10);
    label, eps1, l~ and the solve match the oracle."""
    A = synth.path(5000, 2.0)
    xs, b = synth.rhs(A, seed=13)
    feat, cls = synth.random_sample(240, seed=seed, classes=tuple(range(12)))
    feat[:, 0] = np.linspace(0.5, 2.0, 240) * A.n
    feat[:, 1] = np.linspace(0.5, 2.0, 240)[::-1] * A.nnz
    S = mp.DeviceSample(feat, cls)
    x, r = mp.solve(mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda(), S)
    xo, ro = oracle.solve(A, b, S=(feat, cls))
    assert r["cls"] == ro["cls"] and r["eps1"] == ro["eps1"] and r["pdiam"] == ro["pdiam"]
    parity(r, ro, x.cpu().numpy(), xo)


def _coupled_band(n, D, sigma=0.1):
    """Tridiagonal SPD matrix plus a symmetric coupling at column offset +-D:
    4 + sigma on the diagonal, -1 off it (strictly diagonally dominant)."""
    i = np.concatenate([np.arange(n - 1), np.arange(n - D)])
    j = np.concatenate([np.arange(1, n), np.arange(D, n)])
    return synth.from_edges(n, i, j, -np.ones(i.size), np.full(n, 4.0 + sigma), f"band+{D}")


@pytest.mark.parametrize("D", [32767, 32768])
def test_column_offset_format_boundary(mp, D):
    """The sliced layout stores int16 column offsets (column - row) when every
    kept entry's offset fits, int32 columns otherwise.  Offsets of +-32767 fit,
    +32768 does not: on either side the SpMV (single and double) is bit-exact
    against the oracle and Algorithm I takes the oracle's N1 and N2, the first
    slices' short rows and the last slice's padding rows included."""
    n = 70001
    A = _coupled_band(n, D)
    dA = mp.DeviceCSR.from_host(A)
    rng = np.random.default_rng(5)
    x64 = rng.standard_normal(n)
    x32 = rng.standard_normal(n).astype(np.float32)
    y64 = mp.spmv(dA, torch.from_numpy(x64).cuda()).cpu().numpy()
    y32 = mp.spmv(dA, torch.from_numpy(x32).cuda()).cpu().numpy()
    assert np.array_equal(y64, oracle.spmv64(A, x64))
    assert np.array_equal(y32, oracle.spmv32(A, x32))
    _, b = synth.rhs(A, seed=6)
    x, r = mp.solve(dA, torch.from_numpy(b).cuda(), eps1=1e-5)
    xo, ro = oracle.solve(A, b, eps1=1e-5)
    assert r["status"] == ro["status"] == 0
    assert r["n1"] == ro["n1"] and close_count(r["n2"], ro["n2"])
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-6 * np.linalg.norm(xo)
