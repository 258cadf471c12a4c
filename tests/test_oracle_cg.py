"""Pins of the oracle's CG, Algorithm I and Algorithm II (CPU only).

Each pin comes from outside the oracle: a dense factorisation, a closed-form
spectrum, the convergence bound of Eq. (9), an exactly representable case.
"""
import math

import numpy as np
import pytest
import scipy.linalg
from scipy.sparse import csr_matrix, diags

import oracle
import oracle.metrics  # noqa: F401 (oracle.metrics.cg_iter_bound)
import synth


def random_spd(n, kappa, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.geomspace(1.0, kappa, n)
    M = (Q * ev) @ Q.T
    M = 0.5 * (M + M.T)
    rows, cols = np.nonzero(np.ones((n, n)))
    return synth.CSR(np.arange(0, n * n + 1, n, dtype=np.int32), cols.astype(np.int32),
                     M[rows, cols].copy(), f"dense_spd_{n}"), M


def star_laplacian(n, sigma):
    """L = D - Adj of the star K_{1,n-1} plus sigma I: eigenvalues sigma, 1+sigma, n+sigma."""
    i = np.zeros(n - 1, dtype=np.int64)
    j = np.arange(1, n, dtype=np.int64)
    deg = np.ones(n)
    deg[0] = n - 1
    return synth.from_edges(n, i, j, -np.ones(n - 1), deg + sigma, "starlap")


def test_spmv_matches_dense_product():
    A, M = random_spd(40, 100.0, 0)
    x = np.random.default_rng(1).standard_normal(40)
    np.testing.assert_allclose(oracle.spmv64(A, x), M @ x, rtol=1e-13, atol=1e-13)
    y32 = oracle.spmv32(A, x)
    M32 = M.astype(np.float32).astype(np.float64)
    ref = M32 @ x.astype(np.float32).astype(np.float64)
    assert np.all(np.abs(y32 - ref) <= 40 * 6e-8 * (np.abs(M32) @ np.abs(x)))


def test_fp32_dot_accumulates_in_double():
    """Remark 3 (Sec. 9): norms of the FP32 stage in double.  A float32
    accumulator would return exactly 1.0 here."""
    a = np.concatenate([[1.0], np.full(1000, 1e-4)]).astype(np.float32)
    exact = math.fsum(float(v) * float(v) for v in a)
    assert oracle.dot32(a, a) == pytest.approx(exact, rel=1e-14)
    assert oracle.dot32(a, a) > 1.0 + 9e-6


@pytest.mark.parametrize("n,kappa,seed", [(8, 10.0, 0), (32, 1e3, 1), (64, 1e4, 2)])
def test_cg64_matches_cholesky(n, kappa, seed):
    A, M = random_spd(n, kappa, seed)
    b = np.random.default_rng(seed + 10).standard_normal(n)
    xc = scipy.linalg.cho_solve(scipy.linalg.cho_factor(M), b)
    x, it, st = oracle.cg64(A, b, 1e-14, max_it=20 * n)
    assert st == oracle.OK
    assert np.linalg.norm(x - xc) / np.linalg.norm(xc) <= kappa * 1e-13


@pytest.mark.parametrize("n,seed", [(6, 0), (12, 1), (16, 2), (20, 3)])
def test_cg64_terminates_within_n_steps(n, seed):
    """n distinct eigenvalues in [1, 10]: the rate of Eq. (9) alone would need
    about 37 iterations for 1e-10, so stopping by n is finite termination."""
    A, M = random_spd(n, 10.0, seed)
    b = np.random.default_rng(seed).standard_normal(n)
    _, it, st = oracle.cg64(A, b, 1e-10, max_it=4 * n)
    assert st == oracle.OK and it <= n


@pytest.mark.parametrize("n,sigma", [(50, 0.5), (1001, 1e-2), (400, 1.0)])
def test_cg64_three_distinct_eigenvalues(n, sigma):
    A = star_laplacian(n, sigma)
    ev = np.unique(np.round(np.linalg.eigvalsh(A.to_dense()), 9))
    np.testing.assert_allclose(ev, [sigma, 1 + sigma, n + sigma], rtol=1e-9)
    b = np.random.default_rng(0).uniform(-1, 1, n)
    kappa = (n + sigma) / sigma
    x, it, st, h = oracle.cg64(A, b, 0.0, max_it=3, history=True)
    # the Krylov space is exhausted at step 3: the residual falls from O(1e-2)
    # to the rounding floor (a multiple of u * kappa)
    assert h.size == 4 and h[2] > 1e-3
    assert h[3] <= 1000 * kappa * 1.1e-16


def test_scaled_identity_one_iteration_and_v_zero():
    """A = 4I: alpha = 1/4 exactly, r1 = 0 exactly, so v over one ratio is 0."""
    n = 300
    A = synth.from_edges(n, np.zeros(0), np.zeros(0), np.zeros(0), np.full(n, 4.0))
    b = np.random.default_rng(2).uniform(1, 2, n)
    x, it, st = oracle.cg64(A, b, 1e-12)
    assert it == 1 and np.array_equal(x, b / 4)
    feat, k0d, st = oracle.features(A, b, k0=10)
    assert k0d == 1 and feat[3] == 0.0 and feat[2] == 0.0
    # Algorithm I: the FP32 stage ends at float32(b)/4; the FP64 restart sees
    # r0 = b - float32(b) != 0 and needs exactly one step, which lands on b/4.
    x, r = oracle.solve(A, b, eps1=1e-4, eps2=1e-10)
    assert (r["n1"], r["n2"]) == (1, 1) and np.array_equal(x, b / 4)


def test_residual_bound_eq9():
    """Eq. (9) in the residual norm: ||r_k|| / ||r_0|| <= 2 sqrt(kappa) rho^k."""
    nx, ny = 24, 17
    A = synth.laplacian_2d(nx, ny)
    ev = np.linalg.eigvalsh(A.to_dense())
    kappa = ev[-1] / ev[0]
    rho = (math.sqrt(kappa) - 1) / (math.sqrt(kappa) + 1)
    _, b = synth.rhs(A, 4)
    x, it, st, hist = oracle.cg64(A, b, 1e-12, history=True)
    assert st == oracle.OK
    rel = hist / hist[0]
    bound = 2 * math.sqrt(kappa) * rho ** np.arange(rel.size)
    assert np.all(rel <= bound * (1 + 1e-9))
    # and Eq. (9) bounds the iteration count through the A-norm error
    assert it <= oracle.metrics.cg_iter_bound(kappa, 1e-12 / math.sqrt(kappa)) + 1


def test_fp32_cg_follows_fp64_cg_on_the_rounded_matrix():
    """Before rounding errors dominate, the FP32 iterates track FP64 CG run on
    float32(A), float32(b)."""
    A = synth.laplacian_2d(30, 30)
    _, b = synth.rhs(A, 7)
    A32 = synth.CSR(A.row_ptr, A.col, A.val.astype(np.float32).astype(np.float64))
    b32 = b.astype(np.float32).astype(np.float64)
    _, _, _, h32 = oracle.cg32(A, b, 1e-5, history=True)
    _, _, _, h64 = oracle.cg64(A32, b32, 1e-5, history=True)
    k = min(h32.size, h64.size, 20)
    np.testing.assert_allclose(h32[:k], h64[:k], rtol=1e-4)
    assert abs(h32.size - h64.size) <= 2


def test_algorithm_i_stages_are_plain_cg_runs():
    """Algorithm I = FP32 CG to eps1, promote, FP64 CG to eps2 (Sec. 1)."""
    A, xs, b = synth.poisson64()
    x32, it32, _ = oracle.cg32(A, b, 1e-4)
    x64, it64, _ = oracle.cg64(A, b, 1e-10, x0=x32.astype(np.float64))
    x, r = oracle.solve(A, b, eps1=1e-4, eps2=1e-10)
    assert r["status"] == oracle.OK
    assert (r["n1"], r["n2"]) == (it32, it64)
    assert np.array_equal(x, x64)
    assert r["true_rel_resid"] <= 1e-10
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1711.7 * 1e-10 * 10
    assert r["true_rel_resid"] == pytest.approx(oracle.true_rel_resid(A, b, x), rel=1e-12)


def test_algorithm_ii_with_one_class_sample():
    """A sample whose every label is t = 5 must give eps1 = 1e-5; the k0
    iterations count toward N1 and the stage continues from iterate k0."""
    A, xs, b = synth.poisson64()
    feat, cls = synth.random_sample(30, seed=1)
    cls[:] = 5
    x, r = oracle.solve(A, b, S=(feat, cls), k0=10)
    assert r["cls"] == 5 and r["eps1"] == 1e-5 and r["k0_done"] == 10
    _, it32, _ = oracle.cg32(A, b, 1e-5)
    assert r["n1"] == it32          # continuing from k0 is the same FP32 trajectory
    assert r["pdiam"] == 126 and r["feat"][:3] == [4096.0, 20224.0, 126.0]
    _, _, _, h = oracle.cg32(A, b, 1e-5, history=True)
    v = np.mean(h[1:11] / h[0:10])
    assert r["v"] == pytest.approx(v, rel=1e-12)


def test_zero_rhs_and_nan_and_indefinite():
    A = synth.laplacian_2d(8, 8)
    x, r = oracle.solve(A, np.zeros(A.n), eps1=1e-4)
    assert r["status"] == oracle.OK and not x.any() and r["n1"] == r["n2"] == 0
    b = np.ones(A.n)
    b[3] = np.nan
    _, r = oracle.solve(A, b, eps1=1e-4)
    assert r["status"] == oracle.ERR_NAN
    neg = synth.CSR(A.row_ptr, A.col, -A.val)
    _, r = oracle.solve(neg, np.ones(A.n), eps1=1e-4)
    assert r["status"] == oracle.ERR_BREAKDOWN


def test_fp64_cap_reports_not_converged():
    A, xs, b = synth.poisson64()
    _, r = oracle.solve(A, b, eps1=1e-4, max_it_fp64=5)
    assert r["status"] == oracle.ERR_NOT_CONVERGED and r["n2"] == 5


def test_eps1_cap_warns_and_switches():
    A, xs, b = synth.poisson64()
    x, r = oracle.solve(A, b, eps1=1e-4, max_it_fp32=7)
    assert r["status"] == oracle.WARN_EPS1_NOT_REACHED and r["n1"] == 7
    assert r["true_rel_resid"] <= 1e-10


def test_decay_rate_v_closed_form_two_eigenvalues():
    """Eq. (13) with k0 = 1 on A = diag(l1 I, l2 I): the first CG step is a
    steepest-descent step, so ||r1||^2 = (1 - a l1)^2 |u|^2 + (1 - a l2)^2 |w|^2
    with a = (|u|^2 + |w|^2) / (l1 |u|^2 + l2 |w|^2), b = (u, w).  With k0 = 2
    the second ratio is ~0 (two eigenvalues: CG ends at step 2)."""
    n, l1, l2 = 64, 1.0, 16.0
    diag = np.where(np.arange(n) < n // 2, l1, l2)
    A = synth.from_edges(n, np.zeros(0), np.zeros(0), np.zeros(0), diag)
    b = np.random.default_rng(5).uniform(1, 2, n).astype(np.float32).astype(np.float64)
    u2 = float(np.sum(b[: n // 2] ** 2))
    w2 = float(np.sum(b[n // 2:] ** 2))
    a = (u2 + w2) / (l1 * u2 + l2 * w2)
    ratio1 = math.sqrt((1 - a * l1) ** 2 * u2 + (1 - a * l2) ** 2 * w2) / math.sqrt(u2 + w2)
    feat, k0d, _ = oracle.features(A, b, k0=1)
    assert k0d == 1 and feat[3] == pytest.approx(ratio1, rel=2e-6)
    feat, k0d, _ = oracle.features(A, b, k0=2, eps2=0.0)
    assert k0d == 2 and feat[3] == pytest.approx(ratio1 / 2, rel=1e-5)


# ---- Jacobi-preconditioned CG (the PCG form of Sec. 5), pinned by identities -------------

def _scaled(A):
    """D^-1/2 A D^-1/2 as a CSR, and the scaling vector D^-1/2."""
    M = csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n))
    s = 1.0 / np.sqrt(M.diagonal())
    S = (diags(s) @ M @ diags(s)).tocsr()
    S.sort_indices()
    return synth.CSR(S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data), s


def _varying_diagonal(n=300, seed=3):
    return synth.random_tree_plus(n, 2.0, 1.1, seed=seed)   # a_ii = 1.1 sum_j |a_ij|, uneven


def test_pcg_on_a_diagonal_matrix_takes_one_iteration():
    n = 50
    d = np.linspace(0.5, 40.0, n)
    A = synth.from_edges(n, [], [], np.zeros(0), d)
    b = np.random.default_rng(1).uniform(-1, 1, n)
    x, it, st = oracle.cg64(A, b, 1e-14, precond=1)
    assert st == 0 and it == 1 and np.allclose(x, b / d, rtol=1e-15, atol=0)
    x, it, st = oracle.cg64(A, b, 1e-10)                    # plain CG needs one per distinct value
    assert it > 10
    x32, it32, st32 = oracle.cg32(A, b, 1e-6, precond=1)
    assert st32 == 0 and it32 == 1


def test_pcg_with_a_power_of_two_diagonal_equals_cg_bit_for_bit():
    """z = r / 4 is exact, so every PCG quantity is CG's scaled by a power of two."""
    A = synth.laplacian_2d(23, 17)                            # a_ii = 4
    _, b = synth.rhs(A, seed=4)
    for k in (1, 3, 12):
        xc, ic, _ = oracle.cg64(A, b, 0.0, max_it=k)
        xp, ip, _ = oracle.cg64(A, b, 0.0, max_it=k, precond=1)
        assert ic == ip == k and np.array_equal(xc, xp)
        xc32, _, _ = oracle.cg32(A, b, 0.0, max_it=k)
        xp32, _, _ = oracle.cg32(A, b, 0.0, max_it=k, precond=1)
        assert np.array_equal(xc32, xp32)
    _, nc, _ = oracle.cg64(A, b, 1e-10)
    _, np_, _ = oracle.cg64(A, b, 1e-10, precond=1)
    assert nc == np_


def test_pcg_iterates_are_cg_iterates_of_the_scaled_system():
    """x_k(PCG on A) = D^-1/2 x^_k(CG on D^-1/2 A D^-1/2, b^ = D^-1/2 b) in exact
    arithmetic; both from x = 0 and for the first iterations they agree to rounding."""
    A = _varying_diagonal()
    _, b = synth.rhs(A, seed=5)
    As, s = _scaled(A)
    for k in (1, 2, 5, 10):
        xp, _, _ = oracle.cg64(A, b, 0.0, max_it=k, precond=1)
        xh, _, _ = oracle.cg64(As, s * b, 0.0, max_it=k)
        assert np.linalg.norm(xp - s * xh) <= 1e-11 * np.linalg.norm(xp), k


def test_pcg_helps_on_a_badly_scaled_system_and_rejects_a_zero_diagonal():
    n = 400
    rng = np.random.default_rng(2)
    i = np.arange(n - 1)
    j = i + 1
    off = -np.ones(n - 1)
    d = np.exp(rng.uniform(0, np.log(1e4), n)) + 2.0          # diagonals over four decades
    A = synth.from_edges(n, i, j, off, d)
    b = rng.uniform(-1, 1, n)
    _, nc, sc = oracle.cg64(A, b, 1e-10)
    _, np_, sp = oracle.cg64(A, b, 1e-10, precond=1)
    assert sc == sp == 0 and np_ * 4 < nc
    Z = synth.from_edges(3, [0], [1], np.array([1.0]), np.array([2.0, 0.0, 1.0]))
    assert oracle.cg64(Z, np.ones(3), 1e-10, precond=1)[2] == oracle.ERR_INVALID_ARG
    _, r = oracle.solve(Z, np.ones(3), eps1=1e-4, precond=1)
    assert r["status"] == oracle.ERR_INVALID_ARG


def test_mixed_pcg_reaches_eps2_and_its_features_follow_the_preconditioned_iterations():
    A = _varying_diagonal(500, seed=7)
    _, b = synth.rhs(A, seed=8)
    for eps1 in (1e-3, 1e-6):
        x, r = oracle.solve(A, b, eps1=eps1, precond=1)
        _, rp = oracle.solve(A, b, eps1=eps1)
        assert r["status"] >= 0 and r["true_rel_resid"] <= 1e-10
        assert r["n1"] + r["n2"] < rp["n1"] + rp["n2"]
    f_plain = oracle.features(A, b)[0]
    f_pc = oracle.features(A, b, precond=1)[0]
    assert np.array_equal(f_pc[:3], f_plain[:3]) and f_pc[3] != f_plain[3]  # v from PCG
    L = synth.laplacian_2d(20, 20)
    _, bl = synth.rhs(L, seed=2)
    assert oracle.features(L, bl, precond=1)[0][3] == oracle.features(L, bl)[0][3]


# ---- the stop test as printed: ||A x_i - b|| at the head of every iteration (Sec. 3) ----

def _csr_scipy(A, dtype):
    return csr_matrix((A.val.astype(dtype), A.col, A.row_ptr), shape=(A.n, A.n))


@pytest.mark.parametrize("A", [synth.laplacian_2d(40, 30), synth.path(401, 1.01),
                               synth.random_tree_plus(600, 3.0, 1.1, seed=2)],
                         ids=["lap2d", "path", "tree"])
def test_true_residual_stop_is_the_first_iterate_under_eps(A):
    """With true_res the run ends at the first iterate whose residual
    ||b - A x_k|| / ||b|| is at most eps.  The iterates themselves do not
    depend on the stop test, so x_k and x_{k-1} come from runs capped at k
    and k - 1 iterations, and their residuals are recomputed here with
    scipy (a different summation order; the eps are far from the rounding
    level, so the order does not decide)."""
    _, b = synth.rhs(A, seed=7)
    M64 = _csr_scipy(A, np.float64)
    bn = np.linalg.norm(b)
    for eps in (1e-6, 1e-8, 1e-10):
        _, k, st = oracle.cg64(A, b, eps, true_res=1)
        assert st == 0 and k > 0
        xk, _, _ = oracle.cg64(A, b, 0.0, max_it=k)
        xp, _, _ = oracle.cg64(A, b, 0.0, max_it=k - 1)
        assert np.linalg.norm(b - M64 @ xk) / bn <= eps * (1 + 1e-9)
        assert np.linalg.norm(b - M64 @ xp) / bn > eps * (1 - 1e-9)
    b32 = b.astype(np.float32).astype(np.float64)
    M32 = _csr_scipy(A, np.float32).astype(np.float64)   # float32(A), exact in double
    bn32 = np.linalg.norm(b32)
    for eps in (1e-3, 1e-4, 1e-5):
        _, k, st = oracle.cg32(A, b, eps, true_res=1)
        assert st == 0 and k > 0
        xk, _, _ = oracle.cg32(A, b, 0.0, max_it=k)
        xp, _, _ = oracle.cg32(A, b, 0.0, max_it=k - 1)
        rk = np.linalg.norm(b32 - M32 @ xk.astype(np.float64)) / bn32
        rp = np.linalg.norm(b32 - M32 @ xp.astype(np.float64)) / bn32
        assert rk <= eps * (1 + 1e-3) and rp > eps * (1 - 1e-3)


def test_true_residual_stop_shows_the_stagnation_of_fig2():
    """Sec. 7, Fig. 2: on the path with a_ii = 1.001 sum_j a_ij (n = 1001) the
    true residual of single-precision CG stops improving after a couple of
    hundred iterations (the paper: k = 176) near 1e-7 relative, and that of
    double precision hundreds of iterations later (the paper: k = 506) near
    1e-15, while the recursive residual keeps falling.  So with the stop test
    as printed, eps1 = 1e-7 cannot be met in single precision (as Table 5
    marks for the Jacobi method), whereas the recursive residual meets it.  The run ends once its
    recursive r has fallen 1e3 times below the true residual (the reading
    for a stagnated stage), well before its cap."""
    A = synth.path(1001, 1.001)
    _, b = synth.rhs(A, seed=1)
    _, _, _, h32 = oracle.cg32(A, b, 0.0, max_it=1200, history=True, true_res=1)
    _, _, _, r32 = oracle.cg32(A, b, 0.0, max_it=1200, history=True)
    _, _, _, h64 = oracle.cg64(A, b, 0.0, max_it=1200, history=True, true_res=1)

    def stagnation(h):  # first k whose running minimum is within 2x of the final one
        best = np.minimum.accumulate(h)
        return int(np.argmax(best <= 2 * best[-1])), best[-1]

    k32, f32 = stagnation(h32)
    k64, f64 = stagnation(h64)
    assert 120 <= k32 <= 300 and 1e-8 < f32 < 1e-5
    assert k64 > k32 + 200 and f64 < 1e-13
    assert r32.min() < 1e-20                     # the recursive residual does not stagnate
    _, k, st = oracle.cg32(A, b, 1e-7, max_it=3 * A.n, true_res=1)
    assert st == oracle.ERR_NOT_CONVERGED and k32 < k < 3 * A.n
    hk = r32[k] ** 2          # the recursive r^T r / ||b~||^2 where the run ended
    assert hk <= 1e-6 * h32[k] ** 2 and r32[k - 1] ** 2 > 1e-6 * h32[k - 1] ** 2
    _, k1, st = oracle.cg32(A, b, 1e-7, max_it=3 * A.n)
    assert st == 0 and k1 < k32 + 100
    # Algorithm I with eps1 = 1e-7: stage 1 ends at the stagnation and warns;
    # the FP64 stage then ends on the true residual, with no restart.
    x, r = oracle.solve(A, b, eps1=1e-7, stop_true_residual=1)
    assert r["status"] == oracle.WARN_EPS1_NOT_REACHED and r["n1"] == k
    assert r["true_rel_resid"] <= 1e-10
    x0, r0 = oracle.solve(A, b, eps1=1e-7)
    assert r0["status"] == 0 and r0["n1"] == k1


@pytest.mark.parametrize("name", ["lap2d", "xstar", "tree"])
def test_true_residual_stop_in_both_algorithms(name):
    """With the stop test as printed the FP64 stage ends on the true residual,
    so it never needs the restart of the recursive reading; Algorithm II's
    v (Eq. 13) still comes from the recursive r of the k0 iterations, so the
    features do not change."""
    A = {"lap2d": synth.laplacian_2d(50, 37),
         "xstar": synth.extended_star(20, 50, 3.0, extra=None, seed=6),
         "tree": synth.random_tree_plus(900, 2.0, 1.1, seed=4)}[name]
    _, b = synth.rhs(A, seed=5)
    for eps1 in (1e-3, 1e-5):
        x, r = oracle.solve(A, b, eps1=eps1, stop_true_residual=1)
        assert r["status"] in (0, oracle.WARN_EPS1_NOT_REACHED)
        assert r["true_rel_resid"] <= 1e-10
        assert oracle.true_rel_resid(A, b, x) == r["true_rel_resid"]
    feat, cls = synth.random_sample(50, seed=2)
    f0 = oracle.features(A, b)[0]
    f1 = oracle.features(A, b, stop_true_residual=1)[0]
    assert list(f0) == list(f1)
    _, r = oracle.solve(A, b, S=(feat, cls), stop_true_residual=1)
    assert r["v"] == f0[3] and r["true_rel_resid"] <= 1e-10


def test_true_residual_stop_with_the_absolute_test():
    """tol_relative = 0 (the paper's absolute ||A x_i - b|| > eps): the run ends
    at the first iterate whose unscaled residual is at most eps (rerun as in
    the relative case, residuals recomputed with scipy)."""
    A = synth.laplacian_2d(40, 30)
    _, b = synth.rhs(A, seed=7)
    M64 = _csr_scipy(A, np.float64)
    for eps in (1e-4, 1e-7):
        _, k, st = oracle.cg64(A, b, eps, tol_relative=0, true_res=1)
        assert st == 0 and k > 0
        xk, _, _ = oracle.cg64(A, b, 0.0, max_it=k)
        xp, _, _ = oracle.cg64(A, b, 0.0, max_it=k - 1)
        assert np.linalg.norm(b - M64 @ xk) <= eps * (1 + 1e-9)
        assert np.linalg.norm(b - M64 @ xp) > eps * (1 - 1e-9)


# ---- the true-residual restart of the FP64 stage (reading of Algorithm I) ----
# When the recursive residual meets eps2 and the true one does not, the FP64
# stage restarts from x (r = b - A x again), at most max_true_restarts times;
# if the last restart still misses eps2 the run ends NOT_CONVERGED.  The
# star with a_ii = 1.001 sum_j |a_ij| (n = 1001) shows the branch at eps2 near
# the rounding level: its first FP64 leg ends with the true residual a few
# times above 5e-16, one restart brings it several times below.

def _restart_legs(A, b, eps1, eps2, max_restarts):
    """Algorithm I composed from the separately pinned plain CG runs: FP32 CG
    from 0 to eps1, then FP64 CG legs from float64(x~), each to eps2 on its
    recursive residual (a leg starts with r = b - A x), restarting from the
    leg's x while the true residual -- recomputed here with scipy, not by the
    oracle -- misses eps2.  Returns x, N1, N2 (all legs), restarts, met."""
    M = _csr_scipy(A, np.float64)
    bn = np.linalg.norm(b)
    x32, n1, st1 = oracle.cg32(A, b, eps1)
    assert st1 == 0
    x = x32.astype(np.float64)
    n2 = restarts = 0
    legs = []
    while True:
        x, it, st = oracle.cg64(A, b, eps2, x0=x)
        assert st == 0
        n2 += it
        tr = np.linalg.norm(b - M @ x) / bn
        legs.append(tr)
        if tr <= eps2:
            return x, n1, n2, restarts, True, legs
        if restarts >= max_restarts:
            return x, n1, n2, restarts, False, legs
        restarts += 1


@pytest.mark.parametrize("seed", [3, 8])
def test_true_residual_restart_fires_and_succeeds(seed):
    """eps2 = 5e-16: the first leg's true residual misses it (checked with
    scipy, by a margin), a restart meets it; status, N2 = the sum of both legs,
    the restart count and x equal the composition of plain CG runs."""
    A = synth.star(1001, 1.001)
    _, b = synth.rhs(A, seed=seed)
    eps2 = 5e-16
    xc, n1c, n2c, rc, met, legs = _restart_legs(A, b, 1e-4, eps2, 2)
    assert legs[0] > 2 * eps2 and met and rc == 1 and legs[1] < eps2 / 2
    x, r = oracle.solve(A, b, eps1=1e-4, eps2=eps2, max_true_restarts=2)
    assert r["status"] == oracle.WARN_TRUE_RESID_RESTARTED
    assert (r["n1"], r["n2"], r["restarts"]) == (n1c, n2c, 1)
    assert np.array_equal(x, xc)
    M = _csr_scipy(A, np.float64)
    assert np.linalg.norm(b - M @ x) / np.linalg.norm(b) <= eps2
    assert r["true_rel_resid"] <= eps2


@pytest.mark.parametrize("max_restarts", [0, 2])
def test_true_residual_restart_exhausted_is_not_converged(max_restarts):
    """A tolerance below what the rounding allows (eps2 = 1e-19) is never met
    by the true residual: after max_true_restarts restarts (0 or 2) the run
    ends NOT_CONVERGED, not with a success status, and N2 counts every leg."""
    A = synth.star(1001, 1.001)
    _, b = synth.rhs(A, seed=3)
    eps2 = 1e-19
    xc, n1c, n2c, rc, met, legs = _restart_legs(A, b, 1e-4, eps2, max_restarts)
    assert not met and rc == max_restarts and len(legs) == max_restarts + 1
    assert min(legs) > 100 * eps2
    x, r = oracle.solve(A, b, eps1=1e-4, eps2=eps2, max_true_restarts=max_restarts)
    assert r["status"] == oracle.ERR_NOT_CONVERGED
    assert (r["n1"], r["n2"], r["restarts"]) == (n1c, n2c, max_restarts)
    assert np.array_equal(x, xc)
    M = _csr_scipy(A, np.float64)
    tr = np.linalg.norm(b - M @ x) / np.linalg.norm(b)
    assert tr > eps2 and abs(r["true_rel_resid"] - tr) <= 1e-3 * tr


def test_true_residual_restart_with_none_allowed_at_5e16():
    """The same star and eps2 = 5e-16 as the successful restart, but no
    restart allowed: the first leg's miss is reported as NOT_CONVERGED."""
    A = synth.star(1001, 1.001)
    _, b = synth.rhs(A, seed=3)
    x, r = oracle.solve(A, b, eps1=1e-4, eps2=5e-16, max_true_restarts=0)
    assert r["status"] == oracle.ERR_NOT_CONVERGED and r["restarts"] == 0
    assert r["true_rel_resid"] > 5e-16


# ---- the other reading of Sec. 9, Remark 3: single-precision sums (option acc32) ----

def test_float_sum_dot_exact_cases():
    """Cases whose float result follows from the rounding rule alone:
    1e8 + 1 rounds back to 1e8 (ulp 8), and 2^24 + 1 ties to the even 2^24."""
    one = np.ones(3, np.float32)
    a = np.float32([1e8, 1.0, -1e8])
    assert oracle.dot32(a, one, acc32=1) == 0.0
    assert oracle.dot32(a, one) == 1.0
    b = np.float32([2.0 ** 24, 1.0, 1.0])
    assert oracle.dot32(b, one, acc32=1) == 2.0 ** 24
    assert oracle.dot32(b, one) == 2.0 ** 24 + 2.0
    # the products round to float too: (1 + 2^-12)^2 = 1 + 2^-11 + 2^-24 -> 1 + 2^-11
    c = np.float32([1.0 + 2.0 ** -12])
    assert oracle.dot32(c, c, acc32=1) == 1.0 + 2.0 ** -11
    assert oracle.dot32(c, c) == (1.0 + 2.0 ** -12) ** 2


def test_float_sum_dot_is_the_sequential_float_sum():
    """numpy's accumulate is a sequential float32 running sum; the error of the
    float sum stays inside gamma_n sum |a_i b_i| and is far above the double
    sum's."""
    rng = np.random.default_rng(5)
    a = rng.uniform(-1, 1, 20000).astype(np.float32)
    b = rng.uniform(-1, 1, 20000).astype(np.float32)
    want = np.add.accumulate((a * b).astype(np.float32), dtype=np.float32)[-1]
    assert oracle.dot32(a, b, acc32=1) == float(want)
    exact = math.fsum(float(x) * float(y) for x, y in zip(a, b))
    u, n = 2.0 ** -24, a.size
    bound = n * u / (1 - n * u) * float(np.sum(np.abs(a.astype(np.float64) * b)))
    err32 = abs(oracle.dot32(a, b, acc32=1) - exact)
    assert 0 < err32 <= bound
    assert abs(oracle.dot32(a, b) - exact) < 1e-3 * err32


def test_float_sum_cg32_keeps_the_cg_invariants():
    """With float sums the FP32 CG still exhausts a 3-eigenvalue Krylov space
    in 3 steps (to the float rounding floor), solves a small SPD system like a
    dense solve to float accuracy, and its first stop measure is the float
    ||b~|| relative to itself."""
    A = star_laplacian(400, 1.0)
    b = np.random.default_rng(1).uniform(-1, 1, 400)
    _, it, st, h = oracle.cg32(A, b, 0.0, max_it=3, history=True, acc32=1)
    assert h.size == 4 and h[2] > 1e-3 and h[3] < 1e-4
    A2, M = random_spd(24, 50.0, 3)
    b2 = np.random.default_rng(4).uniform(-1, 1, 24)
    x, it, st = oracle.cg32(A2, b2, 1e-6, acc32=1)
    assert st == oracle.OK
    xs = scipy.linalg.solve(M, b2, assume_a="pos")
    assert np.linalg.norm(x - xs) <= 1e-4 * np.linalg.norm(xs)


def test_float_sum_reading_changes_stage_one_and_both_reach_eps2():
    """Algorithm I with either reading meets eps2; the float sums change the
    single-precision iteration count of a 128x128 Laplacian at eps1 = 1e-6 by
    a few iterations at most, and the FP64 stage is the same computation."""
    A = synth.laplacian_2d(128, 128)
    _, b = synth.rhs(A, 3)
    _, r0 = oracle.solve(A, b, eps1=1e-6)
    _, r1 = oracle.solve(A, b, eps1=1e-6, acc32=1)
    assert r0["status"] == r1["status"] == oracle.OK
    assert r0["true_rel_resid"] <= 1e-10 and r1["true_rel_resid"] <= 1e-10
    assert abs(r0["n1"] - r1["n1"]) <= max(3, 0.05 * r0["n1"])
    x32, it32, _ = oracle.cg32(A, b, 1e-6, acc32=1)
    assert it32 == r1["n1"]


def absorbing_diagonal(m=4000):
    """diag(2, 1, ..., 1) with b = (2^12, 2^-13, ..., 2^-13).  Every float sum
    of b^T b (and of b^T A b) equals its large term, in any order: the small
    terms add up to m 2^-26 < 1, below half an ulp of 2^24.  The double sums
    keep them exactly.  One CG step from 0 has alpha = 1/2 in float under both
    readings and leaves r_1 = (0, 2^-14, ...), whose r^T r = m 2^-28 is exact
    in any order; so v of Eq. (13) with k0 = 1 has a closed form per reading."""
    n = m + 1
    A = synth.from_edges(n, np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0),
                         np.concatenate([[2.0], np.ones(m)]), "absorbing_diag")
    b = np.concatenate([[2.0 ** 12], np.full(m, 2.0 ** -13)])
    rr1 = m * 2.0 ** -28
    v_double = math.sqrt(rr1) / math.sqrt(2.0 ** 24 + m * 2.0 ** -26)
    v_float = math.sqrt(rr1) / math.sqrt(2.0 ** 24)
    return A, b, v_double, v_float


def test_float_sum_reading_on_the_absorbing_diagonal():
    # (the oracle's per-component 2BFS is quadratic on n isolated vertices: keep m small)
    A, b, v_double, v_float = absorbing_diagonal()
    assert v_double != v_float
    feat0, k0d, st0 = oracle.features(A, b, k0=1)
    feat1, k0d1, st1 = oracle.features(A, b, k0=1, acc32=1)
    assert st0 == st1 == oracle.OK and k0d == k0d1 == 1
    assert feat0[3] == v_double
    assert feat1[3] == v_float
