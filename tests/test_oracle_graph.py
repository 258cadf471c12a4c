"""Pins of the oracle's BFS, components and 2BFS pseudo-diameter (Sec. 6)."""
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
