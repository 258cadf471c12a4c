"""GPU parity of the batched solve (mpcg_solve_batch): every system of a batch
against the CPU oracle, with the bars of the single-system tests (labels,
l~ and statuses exact; N1, N2 within 2 %; x within 1e-6; true residual <= eps2),
across team sizes, queue stealing, a small grid and per-system failures."""
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


def parity(r, ro, x, xo, eps2=1e-10):
    assert r["status"] == ro["status"], (r, ro)
    assert close_count(r["n1"], ro["n1"]), (r["n1"], ro["n1"])
    assert close_count(r["n2"], ro["n2"]), (r["n2"], ro["n2"])
    if ro["status"] >= 0:
        assert r["true_rel_resid"] <= eps2
        assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)


def union(*mats):
    rp, cols, vals, off, base = [np.zeros(1, np.int64)], [], [], 0, 0
    for A in mats:
        rp.append(A.row_ptr[1:].astype(np.int64) + base)
        cols.append(A.col.astype(np.int64) + off)
        vals.append(A.val)
        off += A.n
        base += A.nnz
    return synth.CSR(np.concatenate(rp).astype(np.int32), np.concatenate(cols).astype(np.int32),
                     np.concatenate(vals))


def mixed_systems():
    """Small and medium systems of several families; the medium ones go to
    teams of 2, 4 and 8 blocks (16384 rows per block)."""
    return [
        synth.laplacian_2d(37, 29),
        synth.laplacian_3d(13, eps=1e-2, sigma=1e-3),
        synth.random_regular_laplacian(3000, 8, 1e-3, seed=4),
        synth.star(1001, 1.1),
        synth.extended_star(20, 50, 1.1, extra=None, seed=3),
        synth.random_tree_plus(1000, 10.0, 1.1, seed=2),
        synth.banded(1000, 29, 0.6, 1.1, seed=7),
        synth.path(700),
        synth.from_edges(1, [], [], np.zeros(0), np.full(1, 2.0)),
        synth.laplacian_2d(3, 2),
        union(synth.path(50), synth.star(40), synth.laplacian_2d(9, 7)),
        synth.laplacian_3d(32),                     # 32768 rows: team of 2
        synth.laplacian_2d(200, 200),               # 40000 rows: team of 4
        synth.laplacian_2d(300, 250, sigma=1e-4),   # 75000 rows: team of 8
    ]


def sample_over(mats, seed=1, count=200):
    """A sample whose (n, m) span the batch, so that every feature matters."""
    feat, cls = synth.random_sample(count, seed=seed)
    ns = np.array([A.n for A in mats], float)
    feat[:, 0] = np.exp(np.linspace(np.log(0.5 * ns.min()), np.log(2 * ns.max()), count))
    feat[:, 1] = feat[:, 0] * np.linspace(3.0, 9.0, count)[::-1]
    return feat, cls


def run_batch(mp, mats, bs, sample=None, **kw):
    dmats = [mp.DeviceCSR.from_host(A) for A in mats]
    dbs = [torch.from_numpy(np.ascontiguousarray(b)).cuda() for b in bs]
    xs = [torch.full((A.n,), np.nan, dtype=torch.float64, device="cuda") for A in mats]
    ws = torch.empty(mp.batch_workspace_bytes(dmats), dtype=torch.uint8, device="cuda")
    res = mp.result_buffer(len(mats))
    mp.solve_batch_async(dmats, dbs, xs, mp.options(**kw), ws, res, sample)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in xs], mp.read_results(res, len(mats))


def test_batch_algorithm_ii_parity(mp):
    mats = mixed_systems()
    bs = [synth.rhs(A, seed=20 + i)[1] for i, A in enumerate(mats)]
    feat, cls = sample_over(mats)
    S = mp.DeviceSample(feat, cls)
    xs, rs = run_batch(mp, mats, bs, S)
    for A, b, x, r in zip(mats, bs, xs, rs):
        xo, ro = oracle.solve(A, b, S=(feat, cls))
        assert r["pdiam"] == ro["pdiam"], (A.n, r["pdiam"], ro["pdiam"])
        assert abs(r["v"] - ro["v"]) <= 1e-12, (A.n, r["v"], ro["v"])
        assert r["k0_done"] == ro["k0_done"]
        # the kNN on the GPU's own features gives the oracle's label
        assert r["cls"] == oracle.knn([A.n, A.nnz, r["pdiam"], r["v"]], (feat, cls))
        assert r["cls"] == ro["cls"] and r["eps1"] == ro["eps1"]
        parity(r, ro, x, xo)


@pytest.mark.parametrize("eps1", [1e-3, 1e-6])
def test_batch_algorithm_i_parity(mp, eps1):
    mats = mixed_systems()
    bs = [synth.rhs(A, seed=40 + i)[1] for i, A in enumerate(mats)]
    xs, rs = run_batch(mp, mats, bs, None, eps1=eps1)
    for A, b, x, r in zip(mats, bs, xs, rs):
        xo, ro = oracle.solve(A, b, eps1=eps1)
        assert r["cls"] == -1 and r["eps1"] == eps1
        parity(r, ro, x, xo)


def test_batch_matches_single_solves(mp):
    mats = mixed_systems()[:8] + [synth.laplacian_2d(200, 200)]
    bs = [synth.rhs(A, seed=60 + i)[1] for i, A in enumerate(mats)]
    feat, cls = sample_over(mats, seed=3)
    S = mp.DeviceSample(feat, cls)
    xs, rs = run_batch(mp, mats, bs, S)
    for A, b, x, r in zip(mats, bs, xs, rs):
        x1, r1 = mp.solve(mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda(), S)
        assert (r["status"], r["cls"], r["pdiam"], r["k0_done"]) == \
            (r1["status"], r1["cls"], r1["pdiam"], r1["k0_done"])
        assert close_count(r["n1"], r1["n1"]) and close_count(r["n2"], r1["n2"])
        assert np.linalg.norm(x - x1.cpu().numpy()) <= 1e-6 * np.linalg.norm(x)


def test_batch_small_grid_and_failures(mp):
    """Eight blocks (the class of the 75000-row system is demoted), a system
    with b = 0, one with a NaN in b, one that is not SPD and one with a CSR
    error: each gets its own status, the others are unaffected."""
    good = [synth.laplacian_2d(300, 250, sigma=1e-4), synth.laplacian_2d(40, 30),
            synth.random_regular_laplacian(2000, 6, 1e-2, seed=9)]
    A0 = synth.laplacian_2d(20, 10)
    bad_col = A0.col.copy()
    bad_col[5] = A0.n + 7
    bad = synth.CSR(A0.row_ptr, bad_col, A0.val)
    neg = synth.CSR(A0.row_ptr, A0.col, -A0.val)
    mats = good + [A0, A0, neg, bad]
    bs = [synth.rhs(A, seed=80 + i)[1] for i, A in enumerate(good)]
    nan_b = np.ones(A0.n)
    nan_b[3] = np.nan
    bs += [np.zeros(A0.n), nan_b, np.ones(A0.n), np.ones(A0.n)]
    xs, rs = run_batch(mp, mats, bs, None, eps1=1e-4, grid_blocks=8)
    for A, b, x, r in zip(good, bs, xs, rs):
        xo, ro = oracle.solve(A, b, eps1=1e-4)
        parity(r, ro, x, xo)
    r_zero, r_nan, r_neg, r_bad = rs[3:]
    assert r_zero["status"] == 0 and not np.any(xs[3]) and r_zero["n1"] == r_zero["n2"] == 0
    assert r_nan["status"] == mp.ERR_NAN
    _, ro = oracle.solve(neg, np.ones(A0.n), eps1=1e-4)
    assert r_neg["status"] == ro["status"] == mp.ERR_BREAKDOWN
    assert r_bad["status"] == mp.ERR_INVALID_ARG


def test_batch_many_small_systems_steal(mp):
    """More systems than teams, of one size class, plus one large system:
    the large-team queue empties first and its team takes small systems."""
    mats = [synth.laplacian_2d(300, 300)] + [synth.laplacian_2d(10 + i % 7, 9 + i % 5)
                                            for i in range(300)]
    bs = [synth.rhs(A, seed=100 + i)[1] for i, A in enumerate(mats)]
    xs, rs = run_batch(mp, mats, bs, None, eps1=1e-5)
    for k in [0, 1, 2, 150, 299, 300]:
        xo, ro = oracle.solve(mats[k], bs[k], eps1=1e-5)
        parity(rs[k], ro, xs[k], xo)
    assert all(r["status"] in (0, 1) for r in rs)
    assert all(r["true_rel_resid"] <= 1e-10 for r in rs)


def test_batch_tune_picks_a_candidate_and_results_hold(mp):
    mats = mixed_systems()
    bs = [synth.rhs(A, seed=120 + i)[1] for i, A in enumerate(mats)]
    dmats = [mp.DeviceCSR.from_host(A) for A in mats]
    dbs = [torch.from_numpy(np.ascontiguousarray(b)).cuda() for b in bs]
    xs = [torch.empty(A.n, dtype=torch.float64, device="cuda") for A in mats]
    ws = torch.empty(mp.batch_workspace_bytes(dmats), dtype=torch.uint8, device="cuda")
    res = mp.result_buffer(len(mats))
    opts = mp.options(eps1=1e-4)
    best, ms = mp.batch_tune(dmats, dbs, xs, opts, ws, res, None)
    assert best in CANDIDATES
    assert len(ms) == 5 and all(t > 0 for t in ms[:4]) and ms[4] == -1
    assert ms[CANDIDATES.index(best)] == min(ms[:4])
    # a batch with the chosen granularity still matches the oracle
    xs2, rs = run_batch(mp, mats, bs, None, eps1=1e-4, team_rows=best)
    for A, b, x, r in zip(mats, bs, xs2, rs):
        xo, ro = oracle.solve(A, b, eps1=1e-4)
        parity(r, ro, x, xo)


CANDIDATES = (8192, 16384, 32768, 65536)


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_batch_tune_per_system_and_results_hold(mp, mode):
    """The per-system choice: every entry is a candidate; it is kept only if
    its own timed call beat the best uniform candidate (else every entry is
    that candidate); a batch run with it matches the oracle."""
    mats = mixed_systems()
    bs = [synth.rhs(A, seed=140 + i)[1] for i, A in enumerate(mats)]
    dmats = [mp.DeviceCSR.from_host(A) for A in mats]
    dbs = [torch.from_numpy(np.ascontiguousarray(b)).cuda() for b in bs]
    xs = [torch.empty(A.n, dtype=torch.float64, device="cuda") for A in mats]
    ws = torch.empty(mp.batch_workspace_bytes(dmats), dtype=torch.uint8, device="cuda")
    res = mp.result_buffer(len(mats))
    kw = dict(eps1=1e-5) if mode == "mixed" else dict(fp64_only=1)
    best, ms, rows = mp.batch_tune(dmats, dbs, xs, mp.options(**kw), ws, res, None,
                                   per_system=True)
    assert best in CANDIDATES and len(rows) == len(mats)
    assert all(int(r) in CANDIDATES for r in rows)
    assert ms[4] > 0
    if ms[4] >= ms[CANDIDATES.index(best)]:
        assert all(int(r) == best for r in rows)
    xs2, rs = run_batch(mp, mats, bs, None, team_rows=best, team_rows_sys=rows, **kw)
    for A, b, x, r in zip(mats, bs, xs2, rs):
        if mode == "mixed":
            xo, ro = oracle.solve(A, b, eps1=1e-5)
            parity(r, ro, x, xo)
        else:
            xo, it, st = oracle.cg64(A, b, 1e-10)
            assert st == 0 and r["status"] >= 0 and r["n1"] == 0 and close_count(r["n2"], it)
            assert r["true_rel_resid"] <= 1e-10
            assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)
        assert r["t_start_ns"] <= r["t_stage2_ns"] <= r["t_end_ns"]


def test_batch_per_system_team_sizes(mp):
    """Per-system rows per block that put neighbouring systems in teams of
    different sizes (1 to 8 blocks): every system still matches the oracle.
    A team of several blocks sums its partials in another order than one
    block, so x~ ends stage 1 with other last bits, and an FP64 stage that
    meets eps2 after a flat stretch of its residual moves by up to two
    iterations (the 37 x 29 grid on a 2-block team: N2 38 against the
    oracle's 40), below 2 % only from 100 iterations on: the counts are held
    to 2 % or 2 iterations here; status, x and the true residual keep the
    full bar."""
    mats = mixed_systems()
    bs = [synth.rhs(A, seed=160 + i)[1] for i, A in enumerate(mats)]
    rows = [CANDIDATES[i % 4] // 8 if i % 3 == 0 else CANDIDATES[i % 4] for i in range(len(mats))]
    xs, rs = run_batch(mp, mats, bs, None, eps1=1e-5, team_rows_sys=rows)
    # the planner's sizes on the grid the call used; a larger team may also take
    # a system from a smaller size's queue
    plan = mp.batch_plan([A.n for A in mats], [A.nnz for A in mats],
                         mp.options(eps1=1e-5, team_rows_sys=rows), 0)
    near = lambda a, c: abs(a - c) <= max(2, int(0.02 * max(a, c)))
    for A, b, x, r, z in zip(mats, bs, xs, rs, plan):
        assert r["team_blocks"] >= z and r["team_blocks"] & (r["team_blocks"] - 1) == 0, (A.n, r, z)
        xo, ro = oracle.solve(A, b, eps1=1e-5)
        assert r["status"] == ro["status"], (A.n, r, ro)
        assert near(r["n1"], ro["n1"]) and near(r["n2"], ro["n2"]), (A.n, r, ro)
        assert r["true_rel_resid"] <= 1e-10
        assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)


def test_batch_abort_reports_timeout_not_stale_records(mp):
    """A team barrier that times out aborts the launch.  The 2e5-vertex path
    is solved by a team of 32 blocks (8192 rows per block); its first block
    runs the block-local 2BFS (2e5 levels, tens of ms) while the other 31
    wait at the team barrier, past a 5 ms limit (the other systems are
    one-block teams, whose barriers cannot time out).  The records were first filled by a
    successful run, so a stale record would read as a success: every record
    must read either MPCG_ERR_TIMEOUT or a solve that matches the oracle.  The
    context stays usable."""
    mats = [synth.path(200000)] + [synth.laplacian_2d(30 + 3 * i, 20) for i in range(6)]
    bs = [synth.rhs(A, seed=140 + i)[1] for i, A in enumerate(mats)]
    feat, cls = sample_over(mats, seed=5)
    S = mp.DeviceSample(feat, cls)
    dmats = [mp.DeviceCSR.from_host(A) for A in mats]
    dbs = [torch.from_numpy(np.ascontiguousarray(b)).cuda() for b in bs]
    xs = [torch.empty(A.n, dtype=torch.float64, device="cuda") for A in mats]
    ws = torch.empty(mp.batch_workspace_bytes(dmats), dtype=torch.uint8, device="cuda")
    res = mp.result_buffer(len(mats))

    def run(**kw):
        mp.solve_batch_async(dmats, dbs, xs, mp.options(team_rows=8192, **kw), ws, res, S)
        torch.cuda.synchronize()
        return mp.read_results(res, len(mats))

    assert all(r["status"] >= 0 for r in run())
    rs = run(timeout_ms=5)
    assert rs[0]["status"] == mp.ERR_TIMEOUT
    for A, b, x, r in zip(mats, bs, xs, rs):
        assert r["status"] in (mp.ERR_TIMEOUT, mp.OK, mp.WARN_EPS1_NOT_REACHED), r["status"]
        if r["status"] >= 0:
            xo, ro = oracle.solve(A, b, S=(feat, cls))
            parity(r, ro, x.cpu().numpy(), xo)
    rs = run()  # same workspace, default limit
    assert all(r["status"] >= 0 and r["true_rel_resid"] <= 1e-10 for r in rs)


def test_batch_call_does_not_wait_for_earlier_stream_work(mp):
    """The descriptor tables travel inside kernel parameters: the call
    returns while a long kernel still runs ahead of it on the stream, and the
    batch still sees its tables (results equal the oracle's)."""
    import time
    mats = mixed_systems()[:6] + [synth.laplacian_2d(10 + i % 5, 9) for i in range(200)]
    bs = [synth.rhs(A, seed=500 + i)[1] for i, A in enumerate(mats)]
    dmats = [mp.DeviceCSR.from_host(A) for A in mats]
    dbs = [torch.from_numpy(np.ascontiguousarray(b)).cuda() for b in bs]
    xs = [torch.full((A.n,), np.nan, dtype=torch.float64, device="cuda") for A in mats]
    ws = torch.empty(mp.batch_workspace_bytes(dmats), dtype=torch.uint8, device="cuda")
    res = mp.result_buffer(len(mats))
    o = mp.options(eps1=1e-5)
    torch.cuda.synchronize()
    torch.cuda._sleep(1_000_000_000)  # about half a second of device time
    t0 = time.perf_counter()
    mp.solve_batch_async(dmats, dbs, xs, o, ws, res, None)
    t_call = time.perf_counter() - t0
    assert not torch.cuda.current_stream().query()  # the sleep is still running
    torch.cuda.synchronize()
    assert t_call < 0.2, t_call
    rs = mp.read_results(res, len(mats))
    for k in [0, 3, 5, 6, 205]:
        xo, ro = oracle.solve(mats[k], bs[k], eps1=1e-5)
        parity(rs[k], ro, xs[k].cpu().numpy(), xo)


def test_spmv_column_formats_give_identical_bits(mp):
    """Option spmv_variant: the sliced layout with 16-bit offsets from the row
    (chosen per system when every kept entry fits) and with 32-bit columns sum
    the same entries in the same order, so every result is bit-identical.
    Grids and a banded matrix fit; a random graph and a star past 32768 rows
    do not, and keep 32-bit columns under the default too.  A pure-FP64
    batch has no single-precision SpMV and reports 32."""
    mats = [synth.laplacian_3d(32), synth.laplacian_2d(200, 200),
            synth.banded(1000, 29, 0.6, 1.1, seed=7),
            synth.random_regular_laplacian(40000, 8, 1e-3, seed=5), synth.star(40001, 1.1)]
    fits = [True, True, True, False, False]
    bs = [synth.rhs(A, seed=300 + i)[1] for i, A in enumerate(mats)]
    feat, cls = sample_over(mats, seed=5)
    S = mp.DeviceSample(feat, cls)
    keys = ("status", "n1", "n2", "cls", "k0_done", "restarts", "eps1", "true_rel_resid",
            "pdiam", "v", "res_fp32", "res_fp64")
    # One system per call: in a batch of several, a larger team may take a
    # system from a smaller class's queue, and a team of another size sums in
    # another order; alone, a system always runs on a team of its own class.
    for kw in (dict(), dict(fp64_only=1), dict(eps1=1e-5)):
        s = None if kw else S
        for A, f, b in zip(mats, fits, bs):
            (x0,), (r0,) = run_batch(mp, [A], [b], s, **kw)
            (x1,), (r1,) = run_batch(mp, [A], [b], s, spmv_variant=1, **kw)
            assert r0["status"] >= 0, (A.n, r0)
            assert r0["team_blocks"] == r1["team_blocks"], (A.n, kw)
            narrow = f and "fp64_only" not in kw
            assert r0["spmv_cols"] == (16 if narrow else 32) and r1["spmv_cols"] == 32, (A.n, kw)
            assert np.array_equal(x0, x1), (A.n, kw)
            assert all(r0[k] == r1[k] for k in keys), (A.n, kw, r0, r1)
    for A, f, b in zip(mats, fits, bs):  # the single-system kernels
        dA, db = mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda()
        x0, r0 = mp.solve(dA, db, S)
        x1, r1 = mp.solve(dA, db, S, spmv_variant=1)
        assert r0["spmv_cols"] == (16 if f else 32) and r1["spmv_cols"] == 32, A.n
        assert torch.equal(x0, x1), A.n
        assert all(r0[k] == r1[k] for k in keys), (A.n, r0, r1)
