"""Input generators: closed-form spectra and structure (CPU)."""
import math

import numpy as np
import pytest

import synth


def closed_form_2d(nx, ny, sigma=0.0, cy=1.0):
    tx = 4 * np.sin(np.arange(1, nx + 1) * np.pi / (2 * (nx + 1))) ** 2
    ty = 4 * np.sin(np.arange(1, ny + 1) * np.pi / (2 * (ny + 1))) ** 2
    return np.sort((tx[:, None] + cy * ty[None, :]).ravel() + sigma)


def closed_form_3d(nx, ny, nz, eps=1.0, sigma=0.0):
    t = lambda m: 4 * np.sin(np.arange(1, m + 1) * np.pi / (2 * (m + 1))) ** 2
    ev = t(nx)[:, None, None] + t(ny)[None, :, None] + eps * t(nz)[None, None, :]
    return np.sort(ev.ravel() + sigma)


def check_csr(A):
    assert A.row_ptr[0] == 0 and A.row_ptr[-1] == A.nnz
    assert np.all(np.diff(A.row_ptr) >= 1)
    rows = A.rows()
    # sorted, unique columns within each row; diagonal present
    key = rows.astype(np.int64) * A.n + A.col
    assert np.all(np.diff(key) > 0)
    assert np.count_nonzero(rows == A.col) == A.n
    D = A.to_dense() if A.n <= 2000 else None
    if D is not None:
        assert np.array_equal(D, D.T)


@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 5), (8, 8), (12, 7)])
def test_laplacian_2d_spectrum(nx, ny):
    A = synth.laplacian_2d(nx, ny)
    check_csr(A)
    assert A.nnz == 5 * nx * ny - 2 * nx - 2 * ny
    ev = np.linalg.eigvalsh(A.to_dense())
    np.testing.assert_allclose(ev, closed_form_2d(nx, ny), rtol=0, atol=1e-12)


@pytest.mark.parametrize("N,eps,sigma", [(4, 1.0, 0.0), (5, 1e-2, 0.0), (6, 1.0, 1e-2), (5, 1e-3, 1.0)])
def test_laplacian_3d_spectrum(N, eps, sigma):
    A = synth.laplacian_3d(N, eps=eps, sigma=sigma)
    check_csr(A)
    assert A.nnz == 7 * N**3 - 6 * N**2
    ev = np.linalg.eigvalsh(A.to_dense())
    np.testing.assert_allclose(ev, closed_form_3d(N, N, N, eps, sigma), rtol=0, atol=1e-12)


def test_condition_numbers_of_the_configurations():
    """Closed-form kappa of the benchmark matrices (extreme eigenvalues of the
    separable spectra), and the 64x64 value against an ARPACK estimate."""
    def kappa2(a, b):
        lo = 4 * math.sin(math.pi / (2 * (a + 1))) ** 2 + 4 * math.sin(math.pi / (2 * (b + 1))) ** 2
        hi = 4 * math.sin(a * math.pi / (2 * (a + 1))) ** 2 + 4 * math.sin(b * math.pi / (2 * (b + 1))) ** 2
        return hi / lo

    def kappa3(N, eps=1.0, sigma=0.0):
        s1 = 4 * math.sin(math.pi / (2 * (N + 1))) ** 2
        sN = 4 * math.sin(N * math.pi / (2 * (N + 1))) ** 2
        return ((2 + eps) * sN + sigma) / ((2 + eps) * s1 + sigma)

    assert kappa2(64, 64) == pytest.approx(1711.7, abs=0.1)
    assert kappa3(128) == pytest.approx(6744, abs=1)
    assert kappa3(128, sigma=1e-4) == pytest.approx(6385, abs=1)
    assert kappa3(128, sigma=1e-2) == pytest.approx(1019, abs=1)
    assert kappa3(128, sigma=1.0) == pytest.approx(12.98, abs=0.01)
    assert kappa2(65536, 16) == pytest.approx(233.9, abs=0.1)
    assert kappa2(4096, 256) == pytest.approx(53327, rel=1e-4)
    from scipy.sparse import csr_matrix
    from scipy.sparse.linalg import eigsh
    A = synth.laplacian_2d(64, 64)
    S = csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n))
    hi = eigsh(S, k=1, which="LA", return_eigenvectors=False)[0]
    lo = eigsh(S, k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
    assert hi / lo == pytest.approx(kappa2(64, 64), rel=1e-8)


def test_poisson64_shape():
    A, xs, b = synth.poisson64()
    assert (A.n, A.nnz) == (4096, 20224)
    assert xs.min() >= -1 and xs.max() <= 1
    np.testing.assert_allclose(b, A.to_dense() @ xs, rtol=0, atol=1e-12)


def test_random_regular_laplacian():
    A = synth.random_regular_laplacian(2000, 8, shift=1e-3, seed=3)
    check_csr(A)
    D = A.to_dense()
    np.testing.assert_allclose(D.sum(axis=1), 1e-3, atol=1e-12)  # Laplacian rows sum to 0
    off = D - np.diag(np.diag(D))
    assert set(np.unique(off)) <= {-1.0, 0.0}
    deg = -off.sum(axis=1)
    assert deg.max() <= 8 and deg.mean() > 7.5


@pytest.mark.parametrize("gen", [
    lambda: synth.star(50, 1.1), lambda: synth.path(50, 3.0),
    lambda: synth.extended_star(5, 6, 1.1, extra=None, seed=2),
    lambda: synth.random_tree_plus(60, 2.0, 1.1, seed=1),
    lambda: synth.banded(80, 9, 0.4, 1.1, seed=5)])
def test_paper_families_are_dominant_spd(gen):
    A = gen()
    check_csr(A)
    D = A.to_dense()
    off = np.abs(D - np.diag(np.diag(D))).sum(axis=1)
    mu = float(A.name.split("mu")[1].split("_")[0])
    has = off > 0
    np.testing.assert_allclose(np.diag(D)[has], mu * off[has], rtol=1e-14)
    assert np.all(np.diag(D)[~has] == 1.0)
    assert np.linalg.eigvalsh(D).min() > 0


def test_algorithm_iii_ranges():
    v = synth.algorithm_iii(20000, np.random.default_rng(0))
    mag = np.abs(v)
    assert np.all(((mag >= 0) & (mag <= 3)) | ((mag >= 7) & (mag <= 10)))
    assert abs(np.mean(mag <= 3) - 0.5) < 0.02 and abs(np.mean(v > 0) - 0.5) < 0.02


def test_extended_star_shape():
    A = synth.extended_star(10, 30, extra=0)
    assert A.n == 301 and A.nnz == 301 + 2 * 300


def test_batch_family_sizes():
    descs = synth.batch_family(64, seed=0)
    ns = []
    for fam, kw in descs:
        ns.append(kw["nx"] * kw.get("ny", kw["nx"]) if fam == "2d" else kw["nx"] ** 3)
    ns = np.array(ns)
    assert ns.min() >= 700 and ns.max() <= 3.2e5
