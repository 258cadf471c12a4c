"""A single solve is stream-ordered and never synchronises the host, so it
can be captured in a CUDA graph: the replayed graph gives the eager call's
results bit for bit (Algorithm II's results do not depend on timing: the
fused stage 1 snapshots x~ at every candidate eps1)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("status", "n1", "n2", "cls", "k0_done", "restarts", "eps1", "true_rel_resid", "pdiam",
        "v", "res_fp32", "res_fp64")


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_08059_gb300 import build, mpcg
    build.build()
    mpcg.load()
    return mpcg


@pytest.mark.parametrize("kw", [{}, {"fp64_only": 1}, {"eps1": 1e-5}, {"precond": 1}],
                         ids=["algorithm_ii", "fp64", "algorithm_i", "pcg_algorithm_ii"])
def test_solve_replays_from_a_cuda_graph(mp, kw):
    A = synth.laplacian_2d(120, 90)
    _, b = synth.rhs(A, seed=2)
    dA, db = mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda()
    feat, cls = synth.random_sample(100, seed=3)
    feat[:, 0] = np.exp(np.linspace(np.log(0.5 * A.n), np.log(2 * A.n), 100))
    S = mp.DeviceSample(feat, cls)
    o = mp.options(**kw)
    ws = mp.workspace(A.n, A.nnz, opts=o)
    side = torch.cuda.Stream()
    x_e = torch.empty(A.n, dtype=torch.float64, device="cuda")
    res_e = mp.result_buffer(1)
    with torch.cuda.stream(side):  # eager call (also the warm-up before capture)
        mp.solve_async(dA, db, x_e, o, ws, res_e, S)
    torch.cuda.synchronize()
    r_e = mp.read_results(res_e)[0]
    assert r_e["status"] == 0 and r_e["true_rel_resid"] <= 1e-10

    x_g = torch.empty_like(x_e)
    res_g = mp.result_buffer(1)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        mp.solve_async(dA, db, x_g, o, ws, res_g, S)
    for _ in range(2):
        x_g.fill_(float("nan"))
        res_g.zero_()
        g.replay()
        torch.cuda.synchronize()
        r_g = mp.read_results(res_g)[0]
        assert torch.equal(x_g, x_e)
        assert {k: r_g[k] for k in KEYS} == {k: r_e[k] for k in KEYS}
