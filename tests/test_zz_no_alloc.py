"""mpcg_solve_static (fixed scratch array, no allocation) against mpcg_solve.

The static variant runs the same kernels on a scratch array of the library
instead of a caller workspace, so its results must equal mpcg_solve's bit for
bit.  Two consecutive calls on different systems check that nothing carries
over from one call to the next through the shared array.  This file is
collected last so that the array is also exercised after every other GPU
test; it passes on its own as well.
"""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ("status", "n1", "n2", "cls", "k0_done", "restarts", "eps1", "true_rel_resid", "pdiam",
          "v", "res_fp32", "res_fp64")


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_08059_gb300 import build, mpcg
    build.build()
    mpcg.load()
    return mpcg


def _system(A, seed):
    _, b = synth.rhs(A, seed=seed)
    return A, torch.from_numpy(b).cuda()


CASES = [
    # (matrix, options): Algorithm II with the kNN, and Algorithm I with a fixed eps1
    (lambda: synth.laplacian_2d(60, 50), dict()),
    (lambda: synth.laplacian_3d(40, eps=1e-2, sigma=1e-3), dict(eps1=1e-4)),
]


def _reference(mp, dA, db, opts, S):
    x = torch.empty(dA.n, dtype=torch.float64, device="cuda")
    res = mp.result_buffer(1)
    mp.solve_async(dA, db, x, opts, mp.workspace(dA.n, dA.nnz), res, S)
    torch.cuda.synchronize()
    return x, mp.read_results(res)[0]


def _static(mp, dA, db, opts, S):
    x = torch.empty(dA.n, dtype=torch.float64, device="cuda")
    res = mp.result_buffer(1)
    before = torch.cuda.memory_allocated()
    st = mp.solve_static_async(dA, db, x, opts, res, S)
    assert torch.cuda.memory_allocated() == before  # nothing through torch's allocator
    torch.cuda.synchronize()
    assert st == mp.OK, mp.status_string(st)
    return x, mp.read_results(res)[0]


def test_static_matches_workspace_on_consecutive_calls(mp):
    feat, cls = synth.random_sample(200, seed=1)
    S = mp.DeviceSample(feat, cls)
    systems = []
    for k, (make, kw) in enumerate(CASES):
        A, db = _system(make(), seed=10 + k)
        dA = mp.DeviceCSR.from_host(A)
        assert mp.workspace_bytes(dA.n, dA.nnz) <= mp.STATIC_WS_BYTES
        systems.append((dA, db, mp.options(**kw)))
    refs = [_reference(mp, dA, db, o, S) for dA, db, o in systems]
    # two rounds of consecutive calls, alternating the systems
    for _ in range(2):
        for (dA, db, o), (xr, rr) in zip(systems, refs):
            xs, rs = _static(mp, dA, db, o, S)
            assert torch.equal(xs, xr)
            for f in FIELDS:
                a, b = rs[f], rr[f]
                assert a == b or (isinstance(a, float) and np.isnan(a) and np.isnan(b)), f
            assert rs["status"] in (mp.OK, mp.WARN_EPS1_NOT_REACHED)


def test_static_rejects_oversize_before_launch(mp):
    # The size check is on the host and reads only (n, nnz): a descriptor that
    # claims a system larger than the array is refused before any launch.
    # Its pointers still name real (small) device buffers.
    rp = torch.zeros(2, dtype=torch.int32, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    val = torch.ones(1, dtype=torch.float64, device="cuda")
    n, nnz = 4_000_000, 28_000_000
    assert mp.workspace_bytes(n, nnz) > mp.STATIC_WS_BYTES

    class Big:
        pass

    big = Big()
    big.n, big.nnz = n, nnz
    big.desc = mp.CsrDesc(n, nnz, rp.data_ptr(), col.data_ptr(), val.data_ptr())
    b = torch.ones(1, dtype=torch.float64, device="cuda")
    x = torch.empty(1, dtype=torch.float64, device="cuda")
    res = mp.result_buffer(1)
    st = mp.solve_static_async(big, b, x, mp.options(eps1=1e-4), res, None)
    torch.cuda.synchronize()
    assert st == mp.ERR_WORKSPACE
    assert bytes(res.cpu().numpy()) == bytes(C.sizeof(mp.Result))  # untouched


def test_static_then_workspace_call_still_agrees(mp):
    # A workspace call after static calls is unaffected by them.
    A, db = _system(synth.laplacian_2d(37, 29), seed=5)
    dA = mp.DeviceCSR.from_host(A)
    o = mp.options(eps1=1e-3)
    xs, rs = _static(mp, dA, db, o, None)
    xr, rr = _reference(mp, dA, db, o, None)
    assert torch.equal(xs, xr)
    assert (rs["n1"], rs["n2"], rs["status"]) == (rr["n1"], rr["n2"], rr["status"])
