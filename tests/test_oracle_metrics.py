"""Pins of the cost model against numbers printed in the paper."""
import itertools

import pytest

from oracle import metrics
from conftest import read_golden


def test_eq4_reproduces_printed_I_of_tables_4_to_6():
    misprints = {("5", "path", "1e-5")}
    for table, graph, eps, I, n1, n2, marked in read_golden("tables_4_5_6_iterations.txt"):
        if (table, graph, eps) in misprints:
            continue
        val = metrics.cost_I(1.0 / 3.0, int(n1), int(n2))
        assert abs(val - float(I)) <= 0.05 + 1e-12, (table, graph, eps)


def test_label_tie_rule_picks_the_marked_rows():
    rows = read_golden("tables_4_5_6_iterations.txt")
    for (table, graph), grp in itertools.groupby(rows, key=lambda r: (r[0], r[1])):
        grp = list(grp)
        ts = [int(r[2].split("-")[1]) for r in grp]
        t = metrics.label([int(r[4]) for r in grp], [int(r[5]) for r in grp], 1.0 / 3.0, ts)
        marked = [int(r[2].split("-")[1]) for r in grp if r[6] == "1"]
        assert [t] == marked, (table, graph)


def test_eq26_reproduces_appendix_sample_sizes():
    misprints = {("26", 5)}
    checked = 0
    for table, n, kcg, *ns in read_golden("sample_sizes_eq26.txt"):
        for k, printed in zip((1, 5, 10, 15, 20), ns):
            if k == 15 or (table, k) in misprints:
                continue
            val = metrics.sample_size(int(n), k, float(kcg))
            assert abs(val - int(printed)) <= 1.0, (table, k, val, printed)
            checked += 1
    assert checked == 35


def test_efficiency_and_bound_formulas():
    assert metrics.efficiency(75.0, 100.0) == pytest.approx(25.0)
    assert metrics.efficiency(110.0, 100.0) == pytest.approx(-10.0)   # Remark 2: E can be < 0
    # Eq. (9): kappa = 100, eps = 1e-10 -> ceil(5 ln 2e10) = 119
    assert metrics.cg_iter_bound(100.0, 1e-10) == 119
