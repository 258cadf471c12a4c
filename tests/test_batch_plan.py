"""The batch planner's team sizes (mpcg_batch_plan, host only; CPU): a system
goes to the smallest team of 1, 2, 4, ..., 128 blocks with at most its rows
per block (team_rows, or its own entry of team_rows_sys); while one team of
every size present does not fit in the grid, the largest size present is
halved.  The expected sizes are worked out here from that rule."""
import pytest

import synth


@pytest.fixture(scope="module")
def mp():
    from paper_2412_08059_gb300 import build, mpcg
    mpcg.load(build.build())
    return mpcg


def expected(ns, rows, grid):
    cls = []
    for n, r in zip(ns, rows):
        c = 0
        while c < 7 and n > r << c:
            c += 1
        cls.append(c)
    while True:
        need = sum(1 << c for c in set(cls))
        top = max(cls)
        if need <= grid or top == 0:
            break
        cls = [c - 1 if c == top else c for c in cls]
    return [1 << c for c in cls]


NS = [1000, 16384, 16385, 40000, 70000, 262144, 2_000_000, 5000]


def nnz_of(ns):
    return [7 * n for n in ns]


def test_uniform_granularity(mp):
    for rows in (8192, 16384, 65536):
        got = mp.batch_plan(NS, nnz_of(NS), mp.options(team_rows=rows), grid_blocks=152)
        assert got == expected(NS, [rows] * len(NS), 152), rows


def test_the_largest_size_is_halved_until_every_size_fits():
    # 2e6 rows at 16384 rows per block want 128 blocks; with the other sizes
    # present (1, 2, 4, 8, 16 blocks) that is 159 > 152, so the 2e6 system gets 64
    assert expected(NS, [16384] * len(NS), 152)[6] == 64


def test_small_grids(mp):
    for grid in (1, 3, 8, 20):
        got = mp.batch_plan(NS, nnz_of(NS), mp.options(team_rows=16384), grid_blocks=grid)
        assert got == expected(NS, [16384] * len(NS), grid), grid
        assert sum(set(got)) <= max(grid, 1)


def test_per_system_rows_per_block(mp):
    rows = [1024, 0, 8192, 65536, -1, 4096, 32768, 16384]
    base = 16384
    got = mp.batch_plan(NS, nnz_of(NS), mp.options(team_rows=base, team_rows_sys=rows),
                        grid_blocks=152)
    eff = [r if r > 0 else base for r in rows]
    assert got == expected(NS, eff, 152)
    # entries <= 0 take team_rows: the same plan as the uniform one there
    uni = mp.batch_plan(NS, nnz_of(NS), mp.options(team_rows=base), grid_blocks=152)
    assert got[1] == uni[1] and got[4] == uni[4]


def test_the_batch_family(mp):
    descs = synth.batch_family(512, seed=11)
    mats = [synth.build_desc(d) for d in descs[:64]]
    ns, nz = [A.n for A in mats], [A.nnz for A in mats]
    got = mp.batch_plan(ns, nz, mp.options(team_rows=32768), grid_blocks=152)
    assert got == expected(ns, [32768] * len(ns), 152)
    assert set(got) <= {1, 2, 4, 8}


def test_invalid_arguments(mp):
    from paper_2412_08059_gb300.mpcg import C, Options
    L = mp.load()
    o = mp.options()
    nv = (C.c_int32 * 2)(100, 200)
    mv = (C.c_int32 * 2)(500, 1000)
    out = (C.c_int32 * 2)()
    assert L.mpcg_batch_plan(0, nv, mv, C.byref(o), 152, out) == mp.ERR_INVALID_ARG
    assert L.mpcg_batch_plan(2, None, mv, C.byref(o), 152, out) == mp.ERR_INVALID_ARG
    assert L.mpcg_batch_plan(2, nv, mv, None, 152, out) == mp.ERR_INVALID_ARG
    assert L.mpcg_batch_plan(2, nv, mv, C.byref(o), -1, out) == mp.ERR_INVALID_ARG
    bad = (C.c_int32 * 2)(100, 0)
    assert L.mpcg_batch_plan(2, bad, mv, C.byref(o), 152, out) == mp.ERR_INVALID_ARG
