"""GPU tests of serving (mpcg_server_* and mpcg_batch_step): continuous
batching with staggered admission gives each request the result it gets
alone (within the stated tolerances: labels, l~ and statuses exact; N1, N2
within 2 %; x within 1e-6), every request matches the CPU oracle, requests
are admitted by pool footprint, and per-request eps2 is honoured."""
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


class Request:
    def __init__(self, mp, A, b, eps2=1e-10):
        self.A, self.b, self.eps2 = A, b, eps2
        self.dA = mp.DeviceCSR.from_host(A)
        self.db = torch.from_numpy(np.ascontiguousarray(b)).cuda()
        self.x = torch.full((A.n,), np.nan, dtype=torch.float64, device="cuda")
        self.res = mp.result_buffer(1)
        self.slot = None
        self.done = False

    def result(self, mp):
        return self.x.cpu().numpy(), mp.read_results(self.res)[0]


def requests(mp):
    mats = [synth.laplacian_2d(37, 29), synth.laplacian_3d(13, eps=1e-2, sigma=1e-3),
            synth.random_regular_laplacian(3000, 8, 1e-3, seed=4), synth.star(1001, 1.1),
            synth.banded(1000, 29, 0.6, 1.1, seed=7), synth.laplacian_2d(200, 200),
            synth.laplacian_3d(32, sigma=1e-2), synth.path(500),
            synth.laplacian_2d(60, 50, sigma=1e-4), synth.random_tree_plus(1000, 10.0, 1.1, seed=2)]
    return [Request(mp, A, synth.rhs(A, seed=300 + i)[1]) for i, A in enumerate(mats)]


def sample_over(mats, seed=5, count=200):
    feat, cls = synth.random_sample(count, seed=seed)
    ns = np.array([A.n for A in mats], float)
    feat[:, 0] = np.exp(np.linspace(np.log(0.5 * ns.min()), np.log(2 * ns.max()), count))
    feat[:, 1] = feat[:, 0] * np.linspace(3.0, 9.0, count)[::-1]
    return feat, cls


def serve(mp, srv, reqs, waves, max_iters, max_steps=100000):
    """Admit reqs in waves (one wave before each of the first steps), step
    until every admitted request is done, retire finished ones each step."""
    pending = list(waves)
    live = []
    for _ in range(max_steps):
        if pending:
            for r in pending.pop(0):
                r.slot = srv.admit(r.dA, r.db, r.x, r.eps2, r.res)
                assert r.slot is not None
                live.append(r)
        if not live and not pending:
            return
        srv.step(max_iters)
        torch.cuda.synchronize()
        ph = srv.phase.numpy()
        for r in list(live):
            if ph[r.slot] == mp.PHASE_DONE:
                srv.retire(r.slot)
                r.done = True
                live.remove(r)
    raise AssertionError("requests did not finish")


@pytest.mark.parametrize("kw", [dict(), dict(eps1=1e-4), dict(serve_split=1),
                                dict(eps1=1e-4, serve_split=1)],
                         ids=["alg2", "alg1", "alg2-split", "alg1-split"])
def test_serve_same_alone_and_in_mix(mp, kw):
    reqs_mix = requests(mp)
    reqs_alone = requests(mp)
    feat, cls = sample_over([r.A for r in reqs_mix])
    S = mp.DeviceSample(feat, cls)
    opts = mp.options(**kw)
    pool = 4 * sum(mp.workspace_bytes(r.A.n, r.A.nnz) for r in reqs_mix)
    alone = mp.Server(16, pool, opts, S)
    for r in reqs_alone:
        serve(mp, alone, [r], [[r]], max_iters=13)
    alone.close()
    mix = mp.Server(16, pool, opts, S)
    waves = [reqs_mix[0:4], [], reqs_mix[4:7], reqs_mix[7:10]]
    serve(mp, mix, reqs_mix, waves, max_iters=13)
    mix.close()
    for ra, rm in zip(reqs_alone, reqs_mix):
        xa, a = ra.result(mp)
        xm, m = rm.result(mp)
        assert (a["status"], a["cls"], a["pdiam"], a["k0_done"]) == \
            (m["status"], m["cls"], m["pdiam"], m["k0_done"])
        assert close_count(a["n1"], m["n1"]) and close_count(a["n2"], m["n2"])
        assert np.linalg.norm(xa - xm) <= 1e-6 * np.linalg.norm(xa)
        # and the oracle
        if "eps1" in kw:
            xo, ro = oracle.solve(rm.A, rm.b, eps1=kw["eps1"])
        else:
            xo, ro = oracle.solve(rm.A, rm.b, S=(feat, cls))
            assert m["cls"] == ro["cls"] and m["pdiam"] == ro["pdiam"]
        assert m["status"] == ro["status"]
        assert close_count(m["n1"], ro["n1"]) and close_count(m["n2"], ro["n2"])
        assert m["true_rel_resid"] <= 1e-10
        assert np.linalg.norm(xm - xo) <= 1e-6 * np.linalg.norm(xo)


def test_serve_admission_by_footprint(mp):
    """A pool that holds only part of the requests: admission fails with the
    pool full, succeeds again once finished requests are retired."""
    reqs = requests(mp)
    sizes = [mp.workspace_bytes(r.A.n, r.A.nnz) for r in reqs]
    pool = max(sizes) + sorted(sizes)[len(sizes) // 2] + 4096
    srv = mp.Server(8, pool, mp.options(eps1=1e-5))
    queue, live, refused = list(reqs), [], 0
    for _ in range(100000):
        while queue:
            r = queue[0]
            slot = srv.admit(r.dA, r.db, r.x, r.eps2, r.res)
            if slot is None:
                refused += 1
                break
            r.slot = slot
            live.append(queue.pop(0))
        if not live:
            break
        srv.step(20)
        torch.cuda.synchronize()
        ph = srv.phase.numpy()
        for r in list(live):
            if ph[r.slot] == mp.PHASE_DONE:
                srv.retire(r.slot)
                live.remove(r)
    srv.close()
    assert refused > 0 and not queue and not live
    for r in reqs:
        x, m = r.result(mp)
        xo, ro = oracle.solve(r.A, r.b, eps1=1e-5)
        assert m["status"] == ro["status"]
        assert close_count(m["n1"], ro["n1"]) and close_count(m["n2"], ro["n2"])
        assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)


def test_serve_per_request_eps2_and_fp64(mp):
    A = synth.laplacian_2d(80, 70)
    _, b = synth.rhs(A, seed=7)
    reqs = [Request(mp, A, b, eps2=1e-8), Request(mp, A, b, eps2=1e-10)]
    srv = mp.Server(4, 4 * mp.workspace_bytes(A.n, A.nnz), mp.options(fp64_only=1))
    serve(mp, srv, reqs, [reqs], max_iters=9)
    srv.close()
    for r in reqs:
        x, m = r.result(mp)
        xo, it, st = oracle.cg64(A, b, r.eps2)
        assert m["status"] == 0 and st == 0 and m["n1"] == 0
        assert close_count(m["n2"], it)
        assert m["true_rel_resid"] <= r.eps2
        assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)
    assert reqs[0].result(mp)[1]["n2"] < reqs[1].result(mp)[1]["n2"]


def test_serve_abort_ends_the_system_as_timed_out(mp):
    """A step that aborts (a team barrier timed out) ends the system its team
    was working on as MPCG_ERR_TIMEOUT, phase done, result written.  The
    2e5-vertex path goes to a team of 32 blocks (8192 rows per block); its
    first block runs the block-local 2BFS (2e5 levels, tens of ms) while the
    other 31 wait at the team barrier past a 5 ms limit.  Requests admitted
    after that step (one-block teams, whose barriers cannot time out) are
    served normally and match the oracle."""
    P = synth.path(200000)
    path = Request(mp, P, synth.rhs(P, seed=401)[1])
    later = requests(mp)[:4]
    feat, cls = sample_over([r.A for r in later] + [path.A])
    S = mp.DeviceSample(feat, cls)
    pool = 4 * sum(mp.workspace_bytes(r.A.n, r.A.nnz) for r in later + [path])
    srv = mp.Server(16, pool, mp.options(team_rows=8192, timeout_ms=5), S)
    serve(mp, srv, [path] + later, [[path], later], max_iters=13)
    srv.close()
    _, rp = path.result(mp)
    assert rp["status"] == mp.ERR_TIMEOUT
    for r in later:
        x, m = r.result(mp)
        xo, ro = oracle.solve(r.A, r.b, S=(feat, cls))
        assert m["status"] == ro["status"] and m["cls"] == ro["cls"]
        assert close_count(m["n1"], ro["n1"]) and close_count(m["n2"], ro["n2"])
        assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)


def test_serve_step_does_not_wait_for_earlier_stream_work(mp):
    """A step stages its slot tables inside kernel parameters and copies the
    phases to pinned memory: it returns while earlier work still runs."""
    import time
    reqs = requests(mp)[:4]
    o = mp.options(eps1=1e-4)
    pool = sum(mp.workspace_bytes(r.A.n, r.A.nnz) for r in reqs) + (1 << 20)
    srv = mp.Server(64, pool, o, None)
    for r in reqs:
        r.slot = srv.admit(r.dA, r.db, r.x, r.eps2, r.res)
        assert r.slot is not None
    torch.cuda.synchronize()
    torch.cuda._sleep(1_000_000_000)  # about half a second of device time
    t0 = time.perf_counter()
    srv.step(20)
    t_call = time.perf_counter() - t0
    assert not torch.cuda.current_stream().query()
    torch.cuda.synchronize()
    assert t_call < 0.2, t_call
    assert srv.launches_per_step() >= 3
    live = list(reqs)
    for _ in range(100000):  # finish the admitted requests
        ph = srv.phase.numpy()
        for r in list(live):
            if ph[r.slot] == mp.PHASE_DONE:
                srv.retire(r.slot)
                live.remove(r)
        if not live:
            break
        srv.step(20)
        torch.cuda.synchronize()
    assert not live
    for r in reqs:
        x, res = r.result(mp)
        xo, ro = oracle.solve(r.A, r.b, eps1=1e-4)
        assert res["status"] == ro["status"]
        assert close_count(res["n1"], ro["n1"]) and close_count(res["n2"], ro["n2"])
        assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)
    srv.close()
