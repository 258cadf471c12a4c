"""Pins of the oracle's BFS, components and 2BFS pseudo-diameter (Sec. 6)."""
from collections import deque

import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import connected_components, shortest_path

import oracle
import synth


def pattern(A):
    S = csr_matrix((np.ones(A.nnz), A.col, A.row_ptr), shape=(A.n, A.n))
    S.setdiag(0)
    S.eliminate_zeros()
    return S


def exact_diameter(A):
    D = shortest_path(pattern(A), unweighted=True, directed=False)
    D[np.isinf(D)] = -1
    return int(D.max())


def complete_graph(n):
    i, j = np.triu_indices(n, 1)
    return synth.from_edges(n, i, j, -np.ones(i.size), np.full(n, float(n)))


def disjoint(*mats):
    """Block-diagonal CSR of several matrices."""
    rp, cols, vals, off = [np.zeros(1, np.int64)], [], [], 0
    base = 0
    for A in mats:
        rp.append(A.row_ptr[1:].astype(np.int64) + base)
        cols.append(A.col.astype(np.int64) + off)
        vals.append(A.val)
        off += A.n
        base += A.nnz
    return synth.CSR(np.concatenate(rp).astype(np.int32), np.concatenate(cols).astype(np.int32),
                     np.concatenate(vals))


@pytest.mark.parametrize("seed", range(4))
def test_bfs_matches_library_shortest_paths(seed):
    A = synth.random_tree_plus(300, 0.5, seed=seed)
    ref = shortest_path(pattern(A), unweighted=True, directed=False, indices=[7])[0]
    dist, reached = oracle.bfs(A, 7)
    assert reached == A.n
    np.testing.assert_array_equal(dist, ref.astype(np.int32))


@pytest.mark.parametrize("make,ell", [
    (lambda: synth.path(1001), 1000),
    (lambda: synth.laplacian_2d(64, 64), 126),
    (lambda: synth.laplacian_2d(300, 7), 305),
    (lambda: synth.laplacian_3d(9), 24),
    (lambda: synth.laplacian_3d(6, 4, 11), 18),
    (lambda: synth.star(1001), 2),
    (lambda: synth.extended_star(25, 40, extra=0), 50),
    (lambda: synth.extended_star(1000, 1, extra=0), 1000),
    (lambda: complete_graph(30), 1),
])
def test_pseudo_diameter_exact_cases(make, ell):
    """2BFS is exact on paths, grids, stars, extended stars and complete graphs."""
    assert oracle.pseudo_diameter(make()) == ell


def test_farthest_vertex_tie_break_is_smallest_index():
    ell, t = oracle.pseudo_diameter(synth.star(50), return_t=True)
    assert (ell, t) == (2, 1)
    ell, t = oracle.pseudo_diameter(synth.laplacian_2d(10, 6), return_t=True)
    assert (ell, t) == (14, 59)


@pytest.mark.parametrize("seed", range(6))
def test_pseudo_diameter_exact_on_trees(seed):
    A = synth.random_tree_plus(400, 0.0, seed=seed)
    assert oracle.pseudo_diameter(A) == exact_diameter(A)


@pytest.mark.parametrize("seed,c", [(0, 0.1), (1, 0.5), (2, 1.0), (3, 2.0), (4, 0.3)])
def test_pseudo_diameter_bounds_on_random_graphs(seed, c):
    A = synth.random_tree_plus(250, c, seed=seed)
    ell = exact_diameter(A)
    est = oracle.pseudo_diameter(A)
    assert (ell + 1) // 2 <= est <= ell


def test_components_match_library_and_disconnected_rule():
    A = disjoint(synth.path(5), synth.path(9), synth.from_edges(1, [], [], np.zeros(0), np.ones(1)),
                 synth.star(6))
    lab, cnt = oracle.components(A)
    ncomp, ref = connected_components(pattern(A), directed=False)
    assert cnt == ncomp == 4
    # label = smallest vertex of each component
    np.testing.assert_array_equal(lab, [0] * 5 + [5] * 9 + [14] + [15] * 6)
    assert len(set(zip(lab, ref))) == 4
    assert oracle.pseudo_diameter(A) == 8


def test_banded_components():
    A = synth.banded(500, 3, 0.4, seed=1)
    lab, cnt = oracle.components(A)
    ncomp, _ = connected_components(pattern(A), directed=False)
    assert cnt == ncomp > 10
    # pseudo-diameter of a union of paths = longest path
    sizes = np.bincount(lab)
    assert oracle.pseudo_diameter(A) == sizes.max() - 1


def test_single_vertex():
    A = synth.from_edges(1, [], [], np.zeros(0), np.ones(1))
    assert oracle.pseudo_diameter(A) == 0


# ---- repeated 2BFS (remark of Sec. 6) ------------------------------------------------------

def _adj(A):
    return [[int(c) for c in A.col[A.row_ptr[i]:A.row_ptr[i + 1]] if c != i] for i in range(A.n)]


def _bfs_py(adj, s):
    d = [-1] * len(adj)
    d[s] = 0
    q = deque([s])
    while q:
        u = q.popleft()
        for w in adj[u]:
            if d[w] < 0:
                d[w] = d[u] + 1
                q.append(w)
    return d


def _two_bfs_py(adj, s):
    d = _bfs_py(adj, s)
    far = max(d)
    t = d.index(far)                      # smallest vertex at the largest distance
    return max(_bfs_py(adj, t))


def _repeated_py(A, R):
    """Run 0: per component from its smallest vertex; run r: 2BFS from floor(r n / R)."""
    adj = _adj(A)
    n = A.n
    ell, seen = 0, [False] * n
    for s in range(n):
        if not seen[s]:
            for v, dv in enumerate(_bfs_py(adj, s)):
                if dv >= 0:
                    seen[v] = True
            ell = max(ell, _two_bfs_py(adj, s))
    for r in range(1, R):
        ell = max(ell, _two_bfs_py(adj, (r * n) // R))
    return ell


def _diameter_py(A):
    adj = _adj(A)
    return max(max(_bfs_py(adj, s)) for s in range(A.n))


def _random_graph(n, m, seed):
    rng = np.random.default_rng(seed)
    pairs = set()
    while len(pairs) < m:
        a, b = rng.integers(0, n, 2)
        if a != b:
            pairs.add((int(min(a, b)), int(max(a, b))))
    i = np.array([p for p, _ in pairs])
    j = np.array([q for _, q in pairs])
    return synth.from_edges(n, i, j, -np.ones(i.size), np.full(n, 10.0))


def test_repeated_2bfs_matches_independent_bfs_and_bounds():
    for seed in range(40):
        n = 8 + seed % 9
        A = _random_graph(n, n + seed % 5, seed)        # often disconnected, often cyclic
        exact = _diameter_py(A)
        one = oracle.pseudo_diameter(A)
        prev, prev_R = one, 1
        for R in (1, 2, 3, 5, n):
            got = oracle.pseudo_diameter(A, starts=R)
            assert got == _repeated_py(A, R), (seed, R)
            assert one <= got <= exact
            assert got >= prev if R > 1 and R % prev_R == 0 else True
            prev, prev_R = got, R
        assert oracle.pseudo_diameter(A, starts=1) == one


def test_repeated_2bfs_can_beat_a_single_run():
    """Among small random connected graphs, some have a single-start 2BFS below the
    diameter; every start (R = n) then reaches at least as far, and strictly further on
    some of them."""
    better = 0
    for seed in range(300):
        n = 10 + seed % 7
        A = _random_graph(n, n + 2 + seed % 4, 1000 + seed)
        if oracle.components(A)[1] != 1:
            continue
        one, every = oracle.pseudo_diameter(A), oracle.pseudo_diameter(A, starts=n)
        assert one <= every <= _diameter_py(A)
        better += every > one
    assert better > 0


def test_repeated_2bfs_on_grids_and_paths_keeps_the_exact_value():
    for A, ell in ((synth.laplacian_2d(13, 7), 18), (synth.path(50), 49),
                   (synth.laplacian_3d(5), 12)):
        for R in (1, 4, 9):
            assert oracle.pseudo_diameter(A, starts=R) == ell
