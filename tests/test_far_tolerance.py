"""Stage 1 run far past the usual single-precision tolerances: where the
reading of the stage-1 inner products (Sec. 9, Remark 3: norms with double
accuracy) holds on the GPU and where it stops holding.

Both sides form the products of single-precision residuals; the oracle sums
them in double, the GPU as float-float sums of float products.  A float
product loses bits once |r_i| falls below about 1e-19 (its square below the
smallest normal float) and vanishes below about 2.6e-23 (its square below
half the smallest subnormal); a double product of the same floats does
neither.  On the grid below (||b|| = 98.6, n = 1024), measured on a GB300:

- down to eps1 = 1e-23 the GPU takes the oracle's steps: the same N1 and
  the same x bit for bit (the lost bits do not move alpha and beta, which are
  rounded to float);
- at iteration 78 every r_i^2 has vanished in float, the GPU's r^T r is 0 and
  its stage 1 ends there, where the oracle's double products go on (N1 80 at
  eps1 = 1e-25, 94 at 1e-30, 114 at 1e-36); the FP64 restart then gives the
  same x;
- under the option acc32 the oracle's float products vanish at the same
  iteration, and both sides end at 78.
"""
import numpy as np
import pytest

import oracle
import synth


def system():
    A = synth.laplacian_2d(32, 32, sigma=1.0)
    return A, synth.rhs(A, seed=17)[1]


def test_oracle_stage1_keeps_its_rate_far_past_float_underflow():
    """N1 grows by a steady number of iterations per decade of eps1 from 1e-13
    to 1e-36: the double products of the float residuals do not underflow."""
    A, b = system()
    eps = [1e-13, 1e-17, 1e-21, 1e-25, 1e-30, 1e-36]
    n1 = []
    for e in eps:
        _, ro = oracle.solve(A, b, eps1=e)
        assert ro["status"] == 0
        n1.append(ro["n1"])
    per_decade = np.diff(n1) / -np.diff(np.log10(eps))
    assert np.all(per_decade > 2.0) and np.all(per_decade < 5.0), (n1, per_decade)
    assert np.ptp(per_decade) < 1.5, per_decade


def test_oracle_float_sums_stop_where_the_float_products_vanish():
    """Under acc32 (float products summed in float) r^T r is exactly 0 once
    every r_i^2 underflows: stage 1 ends there for any smaller eps1, before
    the double-product reading does."""
    A, b = system()
    n1 = [oracle.solve(A, b, eps1=e, acc32=1)[1]["n1"] for e in (1e-25, 1e-30, 1e-36)]
    n1_double = oracle.solve(A, b, eps1=1e-36)[1]["n1"]
    assert n1[0] == n1[1] == n1[2] < n1_double, (n1, n1_double)


torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_08059_gb300 import build, mpcg
    build.build()
    mpcg.load()
    return mpcg


@pytest.mark.gpu
@pytest.mark.parametrize("eps1", [1e-13, 1e-17, 1e-21, 1e-23])
def test_stage1_matches_the_oracle_down_to_1e23(mp, eps1):
    A, b = system()
    x, r = mp.solve(mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda(), eps1=eps1)
    xo, ro = oracle.solve(A, b, eps1=eps1)
    assert r["status"] == ro["status"] == 0
    assert r["n1"] == ro["n1"] and abs(r["n2"] - ro["n2"]) <= 1, (r["n1"], ro["n1"], r["n2"], ro["n2"])
    assert r["true_rel_resid"] <= 1e-10
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-6 * np.linalg.norm(xo)


@pytest.mark.gpu
@pytest.mark.parametrize("eps1", [1e-25, 1e-30])
def test_stage1_where_the_float_products_vanish(mp, eps1):
    """The GPU's stage 1 ends when its r^T r is 0 (res_fp32 = 0), no later than
    the oracle's double-product reading and with the oracle's float-sum
    reading (acc32) exactly; the FP64 restart meets eps2 with the oracle's x."""
    A, b = system()
    dA, db = mp.DeviceCSR.from_host(A), torch.from_numpy(b).cuda()
    n1_23 = mp.solve(dA, db, eps1=1e-23)[1]["n1"]
    for acc32 in (0, 1):
        x, r = mp.solve(dA, db, eps1=eps1, acc32=acc32)
        xo, ro = oracle.solve(A, b, eps1=eps1, acc32=acc32)
        assert r["status"] == ro["status"] == 0
        assert r["res_fp32"] == 0.0 and n1_23 < r["n1"], (acc32, r["n1"], r["res_fp32"])
        if acc32:
            assert r["n1"] == ro["n1"], (r["n1"], ro["n1"])
        else:
            assert r["n1"] <= ro["n1"], (r["n1"], ro["n1"])
        assert r["true_rel_resid"] <= 1e-10
        assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-6 * np.linalg.norm(xo)
