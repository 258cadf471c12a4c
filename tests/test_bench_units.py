"""The units behind bench.py's roofline figures (CPU): the algorithmic bytes
and flops per CG iteration and the derived FP64 peak, checked against values
worked out independently from the closed forms (nnz of the N^3 7-point
stencil = 7 N^3 - 6 N^2; the 2-D 5-point a x b stencil = 5ab - 2a - 2b)."""
import bench


def test_algorithmic_bytes_per_iteration():
    n, m = 128 ** 3, 7 * 128 ** 3 - 6 * 128 ** 2
    assert m == 14_581_760
    # the matrix once (value + column index), row offsets, x, r and d read and written once
    assert bench.algorithmic_bytes(n, m, 4) == 175_374_340
    assert bench.algorithmic_bytes(n, m, 8) == 284_033_028
    a, b = 65536, 16
    m2 = 5 * a * b - 2 * a - 2 * b
    assert m2 == 5_111_776
    assert round(bench.algorithmic_bytes(a * b, m2, 4) / 1e6, 1) == 70.3
    assert round(bench.algorithmic_bytes(a * b, m2, 8) / 1e6, 1) == 115.9
    assert bench.algorithmic_bytes(64 * 64, 20_224, 8) == 20_224 * 12 + 4 * 4097 + 48 * 4096
