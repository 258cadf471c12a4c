"""Cancellation through the options' cancel word (MPCG_ERR_CANCELLED).

The word lives in pinned host memory, which the GPU reads at the same
address.  On the 128^3 7-point Laplacian (sigma = 0, b = A x*), a solve that
runs tens of milliseconds is enqueued once with the word left at 0 (it ends
normally: that run bounds the case) and once with the host setting the word
a fifth of the way through: the result record then reports
MPCG_ERR_CANCELLED and the call ends well before the uncancelled one.  A
word already set when the call starts cancels it after at most one
iteration.  No GPU fault is involved: the kernels read a word and leave
through their error path."""
import time

import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_08059_gb300 import build, mpcg
    build.build()
    mpcg.load()
    return mpcg


@pytest.fixture(scope="module")
def system(mp):
    A = synth.laplacian_3d(128)
    _, b = synth.rhs(A, seed=1)
    dA = mp.DeviceCSR.from_host(A)
    return A, dA, torch.from_numpy(b).cuda(), mp.workspace(A.n, A.nnz)


KINDS = {  # the single-system kernels that poll the word: k_cg64, k_cg32, k_stage1
    "fp64": dict(fp64_only=1),
    "algorithm_i_stage1": dict(eps1=1e-7, stage1_only=1),
    "algorithm_ii": dict(),
}


def _sample(mp):
    feat, cls = synth.random_sample(50, seed=1, classes=(7,))
    return mp.DeviceSample(feat, cls)


def _run(mp, system, word, sample=None, delay=None, **kw):
    A, dA, db, ws = system
    o = mp.options(cancel=word.data_ptr(), **kw)
    x = torch.empty(dA.n, dtype=torch.float64, device="cuda")
    res = mp.result_buffer(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mp.solve_async(dA, db, x, o, ws, res, sample)
    if delay is not None:
        time.sleep(delay)
        word.numpy()[0] = 1
    torch.cuda.synchronize()
    return mp.read_results(res)[0], time.perf_counter() - t0


@pytest.mark.parametrize("kind", list(KINDS))
def test_cancel_while_running(mp, system, kind):
    S = _sample(mp) if kind == "algorithm_ii" else None
    word = torch.zeros(1, dtype=torch.int32, pin_memory=True)
    _run(mp, system, word, S, **KINDS[kind])                       # warm-up
    r_full, t_full = _run(mp, system, word, S, **KINDS[kind])
    assert r_full["status"] == 0, r_full
    r, t = _run(mp, system, word, S, delay=0.2 * t_full, **KINDS[kind])
    assert r["status"] == mp.ERR_CANCELLED, r
    assert t < 0.7 * t_full, (t, t_full)
    if kind == "fp64":
        assert 0 < r["n2"] < r_full["n2"]
    if kind == "algorithm_i_stage1":
        assert 0 < r["n1"] < r_full["n1"]
    print(f"{kind}: full run {t_full * 1e3:.1f} ms, cancelled run {t * 1e3:.1f} ms")


def test_word_already_set(mp, system):
    word = torch.ones(1, dtype=torch.int32, pin_memory=True)
    for kind, kw in KINDS.items():
        S = _sample(mp) if kind == "algorithm_ii" else None
        r, _ = _run(mp, system, word, S, **kw)
        assert r["status"] == mp.ERR_CANCELLED, (kind, r)
        assert r["n1"] <= 1 and r["n2"] <= 1, (kind, r)
    A, dA, db, ws = system
    f = mp.features(dA, db, ws=ws, cancel=word.data_ptr())
    assert f["status"] == mp.ERR_CANCELLED


def test_unset_word_changes_nothing(mp, system):
    A, dA, db, ws = system
    word = torch.zeros(1, dtype=torch.int32, pin_memory=True)
    x0, r0 = mp.solve(dA, db, ws=ws, eps1=1e-5)
    x1, r1 = mp.solve(dA, db, ws=ws, eps1=1e-5, cancel=word.data_ptr())
    assert torch.equal(x0, x1)
    assert (r0["n1"], r0["n2"], r0["status"]) == (r1["n1"], r1["n2"], 0)


def test_static_variant_polls_the_word(mp):
    A = synth.laplacian_3d(40)
    _, b = synth.rhs(A, seed=3)
    dA = mp.DeviceCSR.from_host(A)
    db = torch.from_numpy(b).cuda()
    word = torch.ones(1, dtype=torch.int32, pin_memory=True)
    x = torch.empty(A.n, dtype=torch.float64, device="cuda")
    res = mp.result_buffer(1)
    st = mp.solve_static_async(dA, db, x, mp.options(eps1=1e-5, cancel=word.data_ptr()), res, None)
    torch.cuda.synchronize()
    assert st == mp.OK and mp.read_results(res)[0]["status"] == mp.ERR_CANCELLED
