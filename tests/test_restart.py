"""GPU parity of the FP64 stage's restart on the true residual (the reading
of Algorithm I where the recursive residual meets eps2 and ||b - A x|| does
not: restart from x, at most max_true_restarts times, then NOT_CONVERGED),
in the single-system kernel (k_cg64) and the batched team kernel.

The case is the one the CPU pins use: the star with a_ii = 1.001 sum_j |a_ij|
(n = 1001), Algorithm I with eps1 = 1e-4.

* eps2 = 1e-19 lies three decades below what the rounding lets the true
  residual reach, on any summation order: both sides take every allowed
  restart and end NOT_CONVERGED; N1 exact, N2 within 2 %, x within 1e-6.
* eps2 = 5e-16 lies at the rounding level: whether the first FP64 leg's true
  residual misses it depends on the summation order of the dot products, so
  the GPU and the oracle may fall on different sides for a given right-hand
  side.  Over 15 right-hand sides the test checks, on each GPU path, that
  the branch follows that path's own first-leg residual (the run with no
  restart allowed reports it): a miss restarts (status
  WARN_TRUE_RESID_RESTARTED, final residual <= eps2, N2 counting every leg),
  a hit does not; that the branch is taken on several right-hand sides; and
  that wherever both sides' first legs fall on the same side of eps2 the GPU
  equals the oracle (status, restarts, N1, N2 within 2 %, x within 1e-6).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS1 = 1e-4
SEEDS = range(1, 16)


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_08059_gb300 import build, mpcg
    build.build()
    mpcg.load()
    return mpcg


@pytest.fixture(scope="module")
def star():
    return synth.star(1001, 1.001)


def close_count(a, b):
    return abs(a - b) <= max(1, int(0.02 * max(a, b)))


def gpu_single(mp, A, bs, **kw):
    dA = mp.DeviceCSR.from_host(A)
    out = []
    for b in bs:
        x, r = mp.solve(dA, torch.from_numpy(b).cuda(), eps1=EPS1, **kw)
        out.append((x.cpu().numpy(), r))
    return out


def gpu_batch(mp, A, bs, **kw):
    dA = mp.DeviceCSR.from_host(A)
    dmats = [dA] * len(bs)
    dbs = [torch.from_numpy(np.ascontiguousarray(b)).cuda() for b in bs]
    xs = [torch.full((A.n,), np.nan, dtype=torch.float64, device="cuda") for _ in bs]
    ws = torch.empty(mp.batch_workspace_bytes(dmats), dtype=torch.uint8, device="cuda")
    res = mp.result_buffer(len(bs))
    mp.solve_batch_async(dmats, dbs, xs, mp.options(eps1=EPS1, **kw), ws, res, None)
    torch.cuda.synchronize()
    return list(zip([x.cpu().numpy() for x in xs], mp.read_results(res, len(bs))))


PATHS = {"single": gpu_single, "batch": gpu_batch}


@pytest.mark.parametrize("path", list(PATHS))
def test_restarts_run_out_below_the_rounding_level(mp, star, path):
    eps2 = 1e-19
    bs = [synth.rhs(star, seed=s)[1] for s in (3, 8)]
    for maxr in (0, 2):
        got = PATHS[path](mp, star, bs, eps2=eps2, max_true_restarts=maxr)
        for b, (x, r) in zip(bs, got):
            xo, ro = oracle.solve(star, b, eps1=EPS1, eps2=eps2, max_true_restarts=maxr)
            assert ro["status"] == oracle.ERR_NOT_CONVERGED and ro["restarts"] == maxr
            assert r["status"] == mp.ERR_NOT_CONVERGED and r["restarts"] == maxr, r
            assert r["n1"] == ro["n1"] and close_count(r["n2"], ro["n2"]), (r, ro)
            assert r["true_rel_resid"] > 100 * eps2
            assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)


@pytest.mark.parametrize("path", list(PATHS))
def test_restart_at_the_rounding_level(mp, star, path):
    eps2 = 5e-16
    bs = [synth.rhs(star, seed=s)[1] for s in SEEDS]
    g0 = PATHS[path](mp, star, bs, eps2=eps2, max_true_restarts=0)
    g2 = PATHS[path](mp, star, bs, eps2=eps2, max_true_restarts=2)
    fired = compared = 0
    for b, (_, r0), (x, r) in zip(bs, g0, g2):
        leg1_missed = r0["true_rel_resid"] > eps2
        assert r0["status"] == (mp.ERR_NOT_CONVERGED if leg1_missed else mp.OK), r0
        assert r0["restarts"] == 0
        if leg1_missed:   # the branch: restart from x, N2 counts every leg
            fired += 1
            assert r["restarts"] >= 1 and r["n2"] > r0["n2"], (r0, r)
            if r["status"] == mp.WARN_TRUE_RESID_RESTARTED:
                assert r["true_rel_resid"] <= eps2
            else:
                assert r["status"] == mp.ERR_NOT_CONVERGED and r["restarts"] == 2, r
        else:             # no restart: the same run as with none allowed
            assert (r["status"], r["restarts"], r["n2"]) == (mp.OK, 0, r0["n2"])
            assert r["true_rel_resid"] <= eps2
        _, ro0 = oracle.solve(star, b, eps1=EPS1, eps2=eps2, max_true_restarts=0)
        if (ro0["true_rel_resid"] > eps2) == leg1_missed:
            compared += 1
            xo, ro = oracle.solve(star, b, eps1=EPS1, eps2=eps2, max_true_restarts=2)
            if ro["restarts"] == r["restarts"]:   # later legs at the rounding level too
                assert r["status"] == ro["status"], (r, ro)
                assert close_count(r["n2"], ro["n2"]), (r["n2"], ro["n2"])
            assert r["n1"] == ro["n1"]
            assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)
    assert fired >= 3, fired
    assert compared >= 5, compared
