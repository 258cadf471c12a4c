"""Device-side waits end with a status, not a hang (GPU).

On the 65536 x 16 grid the single-precision iterations of Algorithm II meet
every candidate eps1 within a few milliseconds, while the 2BFS needs about
65,000 levels.  The consumers then wait for the kNN label.  With a 50 ms
limit that wait runs out: the solve must come back with MPCG_ERR_TIMEOUT
(every block leaves its loop, the later kernels see the status and return).
The context stays usable: the same solve with the default limit, and another
solve, succeed afterwards."""
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


def test_label_wait_times_out_and_context_survives(mp):
    A = synth.laplacian_2d(65536, 16)
    _, b = synth.rhs(A, seed=3)
    feat, cls = synth.random_sample(200, seed=2)
    S = mp.DeviceSample(feat, cls)
    dA = mp.DeviceCSR.from_host(A)
    db = torch.from_numpy(b).cuda()
    x, r = mp.solve(dA, db, S, timeout_ms=50)
    assert r["status"] == mp.ERR_TIMEOUT
    # same solve, default limit: completes
    x, r = mp.solve(dA, db, S)
    assert r["status"] in (mp.OK, mp.WARN_EPS1_NOT_REACHED)
    assert r["true_rel_resid"] <= 1e-10
    # another system on the same context
    B = synth.laplacian_2d(40, 30)
    _, bb = synth.rhs(B, seed=4)
    xb, rb = mp.solve(mp.DeviceCSR.from_host(B), torch.from_numpy(bb).cuda(), eps1=1e-4)
    xo, ro = oracle.solve(B, bb, eps1=1e-4)
    assert rb["status"] == ro["status"] == 0
    assert np.linalg.norm(xb.cpu().numpy() - xo) <= 1e-6 * np.linalg.norm(xo)
