"""GPU parity of the FP64 stage's restart on the true residual (the reading
of Algorithm I where the recursive residual meets eps2 and ||b - A x|| does
not: restart from x, at most max_true_restarts times, then NOT_CONVERGED).

The case is the one the CPU pins use: the star with a_ii = 1.001 sum_j |a_ij|
(n = 1001), Algorithm I with eps1 = 1e-4.  At eps2 = 5e-16 the first FP64
leg's true residual lies several times above eps2 and one restart brings it
several times below, on the oracle; the GPU, whose FP64 dot products are
summed in another order, must take the same branch: same status and restart
count, N1 and N2 within 2 % (here: exact or one apart), x within 1e-6 of the
oracle's.  At eps2 = 1e-19 no leg can meet it, and the restarts run out.
Both the single-system kernel (k_cg64) and the batched team kernel are
checked."""
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


CASES = [  # (seed, eps2, max_true_restarts, expected oracle status, expected restarts)
    (3, 5e-16, 2, oracle.WARN_TRUE_RESID_RESTARTED, 1),
    (8, 5e-16, 2, oracle.WARN_TRUE_RESID_RESTARTED, 1),
    (3, 5e-16, 0, oracle.ERR_NOT_CONVERGED, 0),
    (3, 1e-19, 2, oracle.ERR_NOT_CONVERGED, 2),
]


def _check(r, ro, x, xo, status, restarts, eps2):
    assert ro["status"] == status and ro["restarts"] == restarts, ro
    assert r["status"] == ro["status"], (r["status"], ro["status"])
    assert r["restarts"] == ro["restarts"], (r["restarts"], ro["restarts"])
    assert r["n1"] == ro["n1"], (r["n1"], ro["n1"])
    assert close_count(r["n2"], ro["n2"]), (r["n2"], ro["n2"])
    if status >= 0:
        assert r["true_rel_resid"] <= eps2
    else:
        assert r["true_rel_resid"] > eps2
    assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)


@pytest.mark.parametrize("seed,eps2,maxr,status,restarts", CASES)
def test_single_solve_restart_matches_oracle(mp, seed, eps2, maxr, status, restarts):
    A = synth.star(1001, 1.001)
    _, b = synth.rhs(A, seed=seed)
    x, r = mp.solve(mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda(), eps1=1e-4,
                    eps2=eps2, max_true_restarts=maxr)
    xo, ro = oracle.solve(A, b, eps1=1e-4, eps2=eps2, max_true_restarts=maxr)
    _check(r, ro, x.cpu().numpy(), xo, status, restarts, eps2)


@pytest.mark.parametrize("eps2,maxr,status,restarts",
                         [(5e-16, 2, oracle.WARN_TRUE_RESID_RESTARTED, 1),
                          (1e-19, 2, oracle.ERR_NOT_CONVERGED, 2)])
def test_batched_restart_matches_oracle(mp, eps2, maxr, status, restarts):
    """The team kernel's FP64 stage, two systems of the batch (seeds 3 and 8
    at 5e-16 both restart once; at 1e-19 both run out of restarts)."""
    A = synth.star(1001, 1.001)
    seeds = (3, 8) if status >= 0 else (3, 3)
    bs = [synth.rhs(A, seed=s)[1] for s in seeds]
    dA = mp.DeviceCSR.from_host(A)
    dmats = [dA, dA]
    dbs = [torch.from_numpy(np.ascontiguousarray(b)).cuda() for b in bs]
    xs = [torch.full((A.n,), np.nan, dtype=torch.float64, device="cuda") for _ in bs]
    ws = torch.empty(mp.batch_workspace_bytes(dmats), dtype=torch.uint8, device="cuda")
    res = mp.result_buffer(len(bs))
    mp.solve_batch_async(dmats, dbs, xs, mp.options(eps1=1e-4, eps2=eps2, max_true_restarts=maxr),
                         ws, res, None)
    torch.cuda.synchronize()
    rs = mp.read_results(res, len(bs))
    for b, x, r in zip(bs, xs, rs):
        xo, ro = oracle.solve(A, b, eps1=1e-4, eps2=eps2, max_true_restarts=maxr)
        _check(r, ro, x.cpu().numpy(), xo, status, restarts, eps2)
