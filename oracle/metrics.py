"""The paper's cost model and sample-size bound, written out (test infrastructure).

Each function restates one formula of Prolubnikov (arXiv 2412.08059):

* ``cost_I``        Eq. (4):  I(A, eps1) = omega * N1 + N2
* ``efficiency``    Eq. (12) / Eq. (27):  E = (1 - I / I_dp) * 100 %
* ``label``         Eq. (4) argmin over the candidate set of Sec. 2; ties go
                    to the smallest t (the larger eps1)
* ``sample_size``   Eq. (26) with the parameters of Appendix B
* ``cg_iter_bound`` Eq. (9):  k <= ceil(sqrt(kappa)/2 * ln(2/eps))
* ``sweep``         the labelling procedure of Sec. 11.1: for every
                    candidate eps1, Algorithm I gives N1 and N2; pure FP64 CG
                    gives I_dp
"""
from __future__ import annotations

import math

import numpy as np

# Candidate switching tolerances of Sec. 2: eps1 = 10^-t, t = 2..7.
CLASSES = (2, 3, 4, 5, 6, 7)
EPS1 = {t: float(f"1e-{t}") for t in CLASSES}


def cost_I(omega: float, n1: float, n2: float) -> float:
    """Eq. (4): iterations counted in equivalent double-precision iterations."""
    return omega * n1 + n2


def efficiency(I: float, I_dp: float) -> float:
    """Eq. (12) (one matrix) or Eq. (27) (sums over a test set), in percent."""
    return (1.0 - I / I_dp) * 100.0


def label(n1s, n2s, omega: float = 1.0 / 3.0, classes=CLASSES) -> int:
    """Class t of the eps1 minimising Eq. (4); the first (smallest t) on ties."""
    best_t, best_I = None, math.inf
    for t, a, b in zip(classes, n1s, n2s):
        I = cost_I(omega, a, b)
        if I < best_I:
            best_t, best_I = t, I
    return best_t


def sample_size(n: int, k: int, k_cg: float, c: float = 0.1, alpha: float = 0.01) -> float:
    """Eq. (26): N_S <= alpha * 4 (6c + 17) n k_CG / (44 + 3k)."""
    return alpha * 4.0 * (6.0 * c + 17.0) * n * k_cg / (44.0 + 3.0 * k)


def cg_iter_bound(kappa: float, eps: float) -> int:
    """Eq. (9): iterations that reduce the A-norm error by eps."""
    return math.ceil(0.5 * math.sqrt(kappa) * math.log(2.0 / eps))


def sweep(A, b, eps2: float = 1e-10, classes=CLASSES, **kw):
    """N1, N2 of Algorithm I for every candidate eps1, and N_dp of pure FP64 CG."""
    import oracle
    n1s, n2s, stats = [], [], []
    for t in classes:
        _, r = oracle.solve(A, b, eps1=EPS1[t], eps2=eps2, **kw)
        n1s.append(r["n1"])
        n2s.append(r["n2"])
        stats.append(r["status"])
    _, ndp, st = oracle.cg64(A, b, eps2)
    return np.array(n1s), np.array(n2s), ndp, stats, st
