"""GPU parity of Jacobi-preconditioned mixed CG (option precond; the PCG form
of Sec. 5) against the CPU oracle: Algorithm I, pure FP64 PCG and Algorithm
II (whose steps then run as separate launches in the paper's order), with
the bars of the plain-CG tests (statuses and labels exact; N1, N2 within
2 %; x within 1e-6; true residual <= eps2; v within 1e-12).  Matrices with
uneven diagonals, where the preconditioner changes the iteration, and a
constant diagonal, where it does not."""
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


def systems():
    return [synth.random_tree_plus(2000, 2.0, 1.1, seed=4),      # uneven diagonal
            synth.banded(3000, 21, 0.6, 1.1, seed=5),
            synth.extended_star(20, 50, 3.0, extra=None, seed=6),
            synth.random_tree_plus(300, 10.0, 10.0, seed=7),
            synth.laplacian_3d(24, sigma=1e-2),                   # constant diagonal
            synth.laplacian_2d(200, 150)]


def check(r, ro, x, xo, eps2=1e-10):
    assert r["status"] == ro["status"], (r["status"], ro["status"])
    assert close_count(r["n1"], ro["n1"]), (r["n1"], ro["n1"])
    assert close_count(r["n2"], ro["n2"]), (r["n2"], ro["n2"])
    assert r["true_rel_resid"] <= eps2
    assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)


@pytest.mark.parametrize("eps1", [1e-3, 1e-6])
def test_algorithm_i_pcg_matches_oracle(mp, eps1):
    for i, A in enumerate(systems()):
        _, b = synth.rhs(A, seed=10 + i)
        x, r = mp.solve(mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda(), eps1=eps1, precond=1)
        xo, ro = oracle.solve(A, b, eps1=eps1, precond=1)
        check(r, ro, x.cpu().numpy(), xo)


def test_fp64_pcg_matches_oracle_and_beats_cg_on_uneven_diagonals(mp):
    for i, A in enumerate(systems()):
        _, b = synth.rhs(A, seed=30 + i)
        dA, db = mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda()
        x, r = mp.solve(dA, db, fp64_only=1, precond=1)
        xo, it, st = oracle.cg64(A, b, 1e-10, precond=1)
        assert r["status"] == st == 0
        assert close_count(r["n2"], it), (r["n2"], it)
        assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-6 * np.linalg.norm(xo)
        _, rc = mp.solve(dA, db, fp64_only=1)
        if i < 4:
            assert r["n2"] < rc["n2"]
        else:  # constant diagonal: the same iteration
            assert close_count(r["n2"], rc["n2"])


def test_algorithm_ii_pcg_matches_oracle(mp):
    mats = systems()
    feat, cls = synth.random_sample(200, seed=9)
    ns = np.array([A.n for A in mats], float)
    feat[:, 0] = np.exp(np.linspace(np.log(0.5 * ns.min()), np.log(2 * ns.max()), 200))
    S = mp.DeviceSample(feat, cls)
    for i, A in enumerate(mats):
        _, b = synth.rhs(A, seed=50 + i)
        dA, db = mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda()
        x, r = mp.solve(dA, db, S, precond=1)
        xo, ro = oracle.solve(A, b, S=(feat, cls), precond=1)
        assert r["pdiam"] == ro["pdiam"] and r["k0_done"] == ro["k0_done"]
        assert abs(r["v"] - ro["v"]) <= 1e-12, (r["v"], ro["v"])
        assert r["cls"] == oracle.knn([A.n, A.nnz, r["pdiam"], r["v"]], (feat, cls))
        assert r["cls"] == ro["cls"] and r["eps1"] == ro["eps1"]
        check(r, ro, x.cpu().numpy(), xo)
        f = mp.features(dA, db, precond=1)
        fo, k0o, _ = oracle.features(A, b, precond=1)
        assert f["pdiam"] == fo[2] and abs(f["v"] - fo[3]) <= 1e-12 and f["k0_done"] == k0o


def test_pcg_errors_and_workspace(mp):
    Z = synth.from_edges(4, [0, 1], [1, 2], np.array([1.0, 1.0]), np.array([3.0, 0.0, 3.0, 1.0]))
    _, r = mp.solve(mp.DeviceCSR.from_host(Z), torch.ones(4, dtype=torch.float64).cuda(),
                    eps1=1e-4, precond=1)
    assert r["status"] == mp.ERR_INVALID_ARG
    n, nnz = 1000, 5000
    assert mp.workspace_bytes(n, nnz, mp.options(precond=1)) >= mp.workspace_bytes(n, nnz) + 16 * n
    A = synth.laplacian_2d(30, 20)
    dA = mp.DeviceCSR.from_host(A)
    db = torch.from_numpy(synth.rhs(A, seed=1)[1]).cuda()
    small = torch.empty(mp.workspace_bytes(A.n, A.nnz), dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError):  # a plain-CG workspace is too small for precond
        mp.solve_async(dA, db, torch.empty(A.n, dtype=torch.float64, device="cuda"),
                       mp.options(eps1=1e-4, precond=1), small, mp.result_buffer(1))
    xs = [torch.empty(A.n, dtype=torch.float64, device="cuda")]
    ws = torch.empty(mp.batch_workspace_bytes([dA]), dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError, match="unimplemented"):
        mp.solve_batch_async([dA], [db], xs, mp.options(eps1=1e-4, precond=1), ws,
                             mp.result_buffer(1), None)
