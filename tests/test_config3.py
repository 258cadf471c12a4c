"""GPU parity at the full sizes of the diameter sweep: thin 2-D grids
65536x16 and 4096x256 (large diameter) and a random 8-regular-like graph
Laplacian with n = 2^20 plus 1e-3 I (small diameter).

Pins: the 2BFS pseudo-diameter of an a x b grid is (a - 1) + (b - 1), reached
only at the corner opposite vertex 0 (t = n - 1); the random graph's l~ and t
come from the oracle's BFS.  SpMV is bit-exact against the oracle on every
row.  Algorithm II solves of the well-conditioned members match the oracle
(N1, N2 within 2 %; x within 1e-6; labels exact)."""
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


@pytest.fixture(scope="module")
def rreg():
    return synth.random_regular_laplacian(1 << 20, 8, 1e-3, seed=3)


def close_count(a, b):
    return abs(a - b) <= max(1, int(0.02 * max(a, b)))


@pytest.mark.parametrize("a,b", [(65536, 16), (4096, 256)])
def test_thin_grid_pseudo_diameter_and_spmv(mp, a, b):
    A = synth.laplacian_2d(a, b)
    assert A.nnz == 5 * a * b - 2 * a - 2 * b
    dA = mp.DeviceCSR.from_host(A)
    ell, t = mp.pseudo_diameter(dA)
    assert (ell, t) == ((a - 1) + (b - 1), A.n - 1)
    rng = np.random.default_rng(5)
    x64 = rng.standard_normal(A.n)
    x32 = rng.standard_normal(A.n).astype(np.float32)
    assert np.array_equal(mp.spmv(dA, torch.from_numpy(x64).cuda()).cpu().numpy(),
                          oracle.spmv64(A, x64))
    assert np.array_equal(mp.spmv(dA, torch.from_numpy(x32).cuda()).cpu().numpy(),
                          oracle.spmv32(A, x32))


def test_random_regular_pseudo_diameter_and_spmv(mp, rreg):
    A = rreg
    dA = mp.DeviceCSR.from_host(A)
    assert mp.pseudo_diameter(dA) == oracle.pseudo_diameter(A, return_t=True)
    rng = np.random.default_rng(6)
    x64 = rng.standard_normal(A.n)
    assert np.array_equal(mp.spmv(dA, torch.from_numpy(x64).cuda()).cpu().numpy(),
                          oracle.spmv64(A, x64))


def sample_for(mats, seed=8, count=200):
    feat, cls = synth.random_sample(count, seed=seed)
    ns = np.array([M.n for M in mats], float)
    feat[:, 0] = np.linspace(0.5, 2.0, count) * ns.mean()
    feat[:, 1] = np.linspace(0.5, 2.0, count)[::-1] * np.mean([M.nnz for M in mats])
    feat[:, 2] = np.exp(np.linspace(np.log(3.0), np.log(1.5e5), count))
    return feat, cls


@pytest.mark.parametrize("which", ["grid65536x16", "rreg"])
def test_algorithm_ii_full_size(mp, rreg, which):
    A = synth.laplacian_2d(65536, 16) if which == "grid65536x16" else rreg
    _, b = synth.rhs(A, seed=31)
    feat, cls = sample_for([synth.laplacian_2d(65536, 16), rreg])
    S = mp.DeviceSample(feat, cls)
    x, r = mp.solve(mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda(), S)
    xo, ro = oracle.solve(A, b, S=(feat, cls))
    assert r["pdiam"] == ro["pdiam"]
    assert abs(r["v"] - ro["v"]) <= 1e-12
    assert r["cls"] == oracle.knn([A.n, A.nnz, r["pdiam"], r["v"]], (feat, cls))
    assert r["cls"] == ro["cls"] and r["status"] == ro["status"]
    assert close_count(r["n1"], ro["n1"]) and close_count(r["n2"], ro["n2"])
    assert r["true_rel_resid"] <= 1e-10
    x = x.cpu().numpy()
    assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)
