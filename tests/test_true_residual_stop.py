"""GPU parity of the stop test as the CG procedure of Sec. 3 prints it
(option stop_true_residual: every stop test on ||b - A x|| of the current
iterate) against the CPU oracle with the same option: Algorithm I, pure
FP64 CG and Algorithm II (whose steps then run as separate launches), with
the bars of the plain-CG tests (statuses and labels exact; N1, N2 within
2 %; x within 1e-6; true residual <= eps2; v within 1e-12).  The path of
Sec. 7 (Fig. 2) shows the difference: single precision cannot meet 1e-7 on
its true residual, so stage 1 ends at its stagnation (the recursive r 1e3
times below the true residual) and warns."""
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
    return [synth.laplacian_2d(200, 150),
            synth.random_tree_plus(2000, 2.0, 1.1, seed=4),
            synth.banded(3000, 21, 0.6, 1.1, seed=5),
            synth.extended_star(20, 50, 3.0, extra=None, seed=6),
            synth.laplacian_3d(24, sigma=1e-2)]


def check(r, ro, x, xo, eps2=1e-10):
    assert r["status"] == ro["status"], (r["status"], ro["status"])
    assert close_count(r["n1"], ro["n1"]), (r["n1"], ro["n1"])
    assert close_count(r["n2"], ro["n2"]), (r["n2"], ro["n2"])
    assert r["true_rel_resid"] <= eps2
    assert r["restarts"] == 0
    assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)


@pytest.mark.parametrize("eps1", [1e-3, 1e-5])
def test_algorithm_i_matches_oracle(mp, eps1):
    for i, A in enumerate(systems()):
        _, b = synth.rhs(A, seed=10 + i)
        x, r = mp.solve(mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda(), eps1=eps1,
                        stop_true_residual=1)
        xo, ro = oracle.solve(A, b, eps1=eps1, stop_true_residual=1)
        check(r, ro, x.cpu().numpy(), xo)


def test_fp64_matches_oracle(mp):
    for i, A in enumerate(systems()):
        _, b = synth.rhs(A, seed=30 + i)
        x, r = mp.solve(mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda(), fp64_only=1,
                        stop_true_residual=1)
        xo, it, st = oracle.cg64(A, b, 1e-10, true_res=1)
        assert r["status"] == st == 0 and r["restarts"] == 0
        assert close_count(r["n2"], it), (r["n2"], it)
        assert r["true_rel_resid"] <= 1e-10
        assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-6 * np.linalg.norm(xo)


def test_fig2_path_single_precision_cannot_meet_1e7(mp):
    A = synth.path(1001, 1.001)
    _, b = synth.rhs(A, seed=1)
    dA, db = mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda()
    x, r = mp.solve(dA, db, eps1=1e-7, stop_true_residual=1)
    xo, ro = oracle.solve(A, b, eps1=1e-7, stop_true_residual=1)
    assert r["status"] == ro["status"] == mp.WARN_EPS1_NOT_REACHED
    assert 200 < ro["n1"] < A.n    # ended at the stagnation, before the cap
    check(r, ro, x.cpu().numpy(), xo)
    _, r0 = mp.solve(dA, db, eps1=1e-7)   # the recursive r meets it
    assert r0["status"] == 0 and r0["n1"] < ro["n1"]
    # FP64 cannot meet 1e-16 either: not converged at its stagnation
    _, r = mp.solve(dA, db, fp64_only=1, eps2=1e-16, stop_true_residual=1)
    _, it, st = oracle.cg64(A, b, 1e-16, true_res=1)
    assert r["status"] == st == mp.ERR_NOT_CONVERGED and close_count(r["n2"], it)
    assert it < 10 * A.n


def test_algorithm_ii_and_features_match_oracle(mp):
    mats = systems()
    feat, cls = synth.random_sample(200, seed=9)
    ns = np.array([A.n for A in mats], float)
    feat[:, 0] = np.exp(np.linspace(np.log(0.5 * ns.min()), np.log(2 * ns.max()), 200))
    S = mp.DeviceSample(feat, cls)
    for i, A in enumerate(mats):
        _, b = synth.rhs(A, seed=50 + i)
        dA, db = mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda()
        x, r = mp.solve(dA, db, S, stop_true_residual=1)
        xo, ro = oracle.solve(A, b, S=(feat, cls), stop_true_residual=1)
        assert r["pdiam"] == ro["pdiam"] and r["k0_done"] == ro["k0_done"]
        assert abs(r["v"] - ro["v"]) <= 1e-12, (r["v"], ro["v"])
        assert r["cls"] == ro["cls"] and r["eps1"] == ro["eps1"]
        check(r, ro, x.cpu().numpy(), xo)
        f = mp.features(dA, db, stop_true_residual=1)
        fo, k0o, _ = oracle.features(A, b, stop_true_residual=1)
        assert f["pdiam"] == fo[2] and abs(f["v"] - fo[3]) <= 1e-12 and f["k0_done"] == k0o


def test_with_jacobi_preconditioning(mp):
    A = synth.random_tree_plus(2000, 2.0, 1.1, seed=4)
    _, b = synth.rhs(A, seed=3)
    x, r = mp.solve(mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda(), eps1=1e-4,
                    precond=1, stop_true_residual=1)
    xo, ro = oracle.solve(A, b, eps1=1e-4, precond=1, stop_true_residual=1)
    check(r, ro, x.cpu().numpy(), xo)


def test_refused_by_the_batch_and_the_server(mp):
    A = synth.laplacian_2d(30, 20)
    dA = mp.DeviceCSR.from_host(A)
    db = torch.from_numpy(synth.rhs(A, seed=1)[1]).cuda()
    xs = [torch.empty(A.n, dtype=torch.float64, device="cuda")]
    ws = torch.empty(mp.batch_workspace_bytes([dA]), dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError, match="unimplemented"):
        mp.solve_batch_async([dA], [db], xs, mp.options(eps1=1e-4, stop_true_residual=1), ws,
                             mp.result_buffer(1), None)
    with pytest.raises(RuntimeError, match="unimplemented"):
        mp.Server(4, 1 << 24, mp.options(eps1=1e-4, stop_true_residual=1))
    with pytest.raises(RuntimeError, match="invalid"):
        mp.solve(dA, db, eps1=1e-4, stop_true_residual=2)
