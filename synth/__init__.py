"""Seeded synthetic inputs for restarted mixed-precision CG.

This module only builds inputs: sparse SPD matrices in CSR form (int32
indices, float64 values, columns sorted within each row, diagonal stored)
and right-hand sides.  It holds none of the solver's arithmetic, and both the
CPU oracle and the CUDA library consume what it produces.

Families:

* Dirichlet Laplacians: 2-D 5-point and 3-D 7-point, with anisotropic
  coefficients (1, 1, eps) and shifts A + sigma*I.
* Random d-regular-like graph Laplacians: configuration model, with
  self-loops and multi-edges removed, plus shift*I.
* The paper's graph families (Sec. 12 and Appendix A), with diagonal
  a_ii = mu * sum_{j != i} |a_ij|:
  * star and path graphs (Sec. 7);
  * extended stars with added random edges;
  * random trees with floor(c n) added edges;
  * banded graphs.
  Random and banded graphs get values from Algorithm III.
* Right-hand sides: x* ~ U[lo, hi], b = A x*.  Sec. 2 uses U(1, 2); the
  Laplacian configurations use U[-1, 1].  The product A x* is part of
  building the input.

Every generator takes an explicit seed and uses numpy's PCG64 generator.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class CSR:
    row_ptr: np.ndarray  # int32[n+1]
    col: np.ndarray      # int32[nnz]
    val: np.ndarray      # float64[nnz]
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.row_ptr.size - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.size)

    def rows(self) -> np.ndarray:
        """Row index of every stored entry."""
        return np.repeat(np.arange(self.n, dtype=np.int32), np.diff(self.row_ptr))

    def to_dense(self) -> np.ndarray:
        A = np.zeros((self.n, self.n))
        A[self.rows(), self.col] = self.val
        return A

    def bytes(self) -> int:
        return self.row_ptr.nbytes + self.col.nbytes + self.val.nbytes


def _stencil_csr(cols: np.ndarray, vals: np.ndarray, mask: np.ndarray, name: str) -> CSR:
    """Rows given as fixed-width (n, w) tables whose masked entries are in column order."""
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(cols.shape[0] + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("nnz exceeds int32")
    return CSR(row_ptr.astype(np.int32), cols[mask].astype(np.int32), vals[mask].astype(np.float64), name)


def laplacian_2d(nx: int, ny: int, sigma: float = 0.0, cy: float = 1.0) -> CSR:
    """5-point Dirichlet Laplacian on an nx-by-ny interior grid, x fastest.

    A = T_nx (x) I + cy I (x) T_ny + sigma I with T = tridiag(-1, 2, -1).
    Row order: idx = y*nx + x.  Stored columns per row: y-1, x-1, self, x+1, y+1.
    """
    n = nx * ny
    idx = np.arange(n, dtype=np.int64)
    x = idx % nx
    y = idx // nx
    offs = np.array([-nx, -1, 0, 1, nx], dtype=np.int64)
    cols = idx[:, None] + offs[None, :]
    mask = np.stack([y > 0, x > 0, np.ones(n, bool), x < nx - 1, y < ny - 1], axis=1)
    diag = 2.0 + 2.0 * cy + sigma
    vals = np.broadcast_to(np.array([-cy, -1.0, diag, -1.0, -cy]), (n, 5))
    return _stencil_csr(np.where(mask, cols, 0), vals, mask, f"lap2d_{nx}x{ny}_s{sigma:g}")


def laplacian_3d(nx: int, ny: int | None = None, nz: int | None = None, eps: float = 1.0,
                 sigma: float = 0.0) -> CSR:
    """7-point Dirichlet Laplacian with coefficients (1, 1, eps) on (x, y, z), plus sigma I.

    Row order: idx = (z*ny + y)*nx + x.  Stored columns per row:
    z-1, y-1, x-1, self, x+1, y+1, z+1.
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    n = nx * ny * nz
    if 7 * n >= 2**31:
        raise ValueError("nnz exceeds int32")
    idx = np.arange(n, dtype=np.int64)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    pl = nx * ny
    offs = np.array([-pl, -nx, -1, 0, 1, nx, pl], dtype=np.int64)
    cols = (idx[:, None] + offs[None, :]).astype(np.int64)
    mask = np.stack([z > 0, y > 0, x > 0, np.ones(n, bool), x < nx - 1, y < ny - 1, z < nz - 1],
                    axis=1)
    diag = 4.0 + 2.0 * eps + sigma
    vals = np.broadcast_to(np.array([-eps, -1.0, -1.0, diag, -1.0, -1.0, -eps]), (n, 7))
    return _stencil_csr(np.where(mask, cols, 0), vals, mask,
                        f"lap3d_{nx}x{ny}x{nz}_e{eps:g}_s{sigma:g}")


def from_edges(n: int, i: np.ndarray, j: np.ndarray, offval: np.ndarray, diag: np.ndarray,
               name: str = "") -> CSR:
    """Symmetric CSR from an undirected edge list (i != j, no duplicates) and a diagonal."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    rows = np.concatenate([i, j, np.arange(n, dtype=np.int64)])
    cols = np.concatenate([j, i, np.arange(n, dtype=np.int64)])
    vals = np.concatenate([offval, offval, diag]).astype(np.float64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    return CSR(row_ptr.astype(np.int32), cols.astype(np.int32), vals, name)


def _dominant_diag(n: int, i, j, offval, mu: float) -> np.ndarray:
    """a_ii = mu * sum_{j != i} |a_ij| (Sec. 12); an isolated vertex gets a_ii = 1."""
    s = np.bincount(i, weights=np.abs(offval), minlength=n) + np.bincount(
        j, weights=np.abs(offval), minlength=n)
    d = mu * s
    d[s == 0] = 1.0
    return d


def random_regular_laplacian(n: int, degree: int = 8, shift: float = 1e-3, seed: int = 0) -> CSR:
    """Graph Laplacian of a configuration-model multigraph with self-loops and
    multi-edges removed (average degree just under `degree`), plus shift*I."""
    rng = np.random.default_rng(seed)
    stubs = rng.permutation(np.repeat(np.arange(n, dtype=np.int64), degree))
    if stubs.size % 2:
        stubs = stubs[:-1]
    a, b = stubs[0::2], stubs[1::2]
    keep = a != b
    a, b = a[keep], b[keep]
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    key = np.unique(lo * n + hi)
    i, j = key // n, key % n
    off = -np.ones(i.size)
    deg = np.bincount(i, minlength=n) + np.bincount(j, minlength=n)
    return from_edges(n, i, j, off, deg.astype(np.float64) + shift,
                      f"rreg{degree}_{n}_sh{shift:g}_seed{seed}")


# ----------------------------------------------------------------------------------------
# Paper families (Sec. 7, Sec. 12, Appendix A).
# ----------------------------------------------------------------------------------------

def star(n: int, mu: float = 1.1) -> CSR:
    """Star graph on n vertices (centre 0) with binary off-diagonals, a_ii = mu*deg (Sec. 7)."""
    i = np.zeros(n - 1, dtype=np.int64)
    j = np.arange(1, n, dtype=np.int64)
    off = np.ones(n - 1)
    return from_edges(n, i, j, off, _dominant_diag(n, i, j, off, mu), f"star_{n}_mu{mu:g}")


def path(n: int, mu: float = 1.1) -> CSR:
    """Path graph 0-1-...-(n-1) with binary off-diagonals, a_ii = mu*deg (Sec. 7)."""
    i = np.arange(n - 1, dtype=np.int64)
    j = i + 1
    off = np.ones(n - 1)
    return from_edges(n, i, j, off, _dominant_diag(n, i, j, off, mu), f"path_{n}_mu{mu:g}")


def _add_random_edges(n: int, existing: set, count: int, rng) -> tuple[list, list]:
    ai, aj = [], []
    while len(ai) < count:
        p, q = rng.integers(0, n, size=2)
        if p == q:
            continue
        p, q = (int(p), int(q)) if p < q else (int(q), int(p))
        if (p, q) in existing:
            continue
        existing.add((p, q))
        ai.append(p)
        aj.append(q)
    return ai, aj


def extended_star(lc: int, nc: int, mu: float = 1.1, extra: int | None = 0, seed: int = 0) -> CSR:
    """Extended star (Appendix A.1): centre 0 joined to nc rays, each a path of lc
    vertices; n = 1 + nc*lc.  `extra` random edges are added between uniformly
    chosen unordered pairs without duplicates (None: xi ~ U{0, ..., ceil(0.1 n)-1}).
    Binary off-diagonals, a_ii = mu * deg."""
    n = 1 + nc * lc
    rng = np.random.default_rng(seed)
    ii, jj = [], []
    for r in range(nc):
        first = 1 + r * lc
        ii.append(0)
        jj.append(first)
        for k in range(lc - 1):
            ii.append(first + k)
            jj.append(first + k + 1)
    if extra is None:
        extra = int(rng.integers(0, max(1, math.ceil(0.1 * n))))
    existing = set(zip(ii, jj))
    ai, aj = _add_random_edges(n, existing, extra, rng)
    i = np.array(ii + ai, dtype=np.int64)
    j = np.array(jj + aj, dtype=np.int64)
    off = np.ones(i.size)
    return from_edges(n, i, j, off, _dominant_diag(n, i, j, off, mu),
                      f"xstar_{lc}x{nc}_mu{mu:g}_seed{seed}")


def algorithm_iii(count: int, rng, a1=0.0, b1=3.0, a2=7.0, b2=10.0) -> np.ndarray:
    """Algorithm III (Appendix A.2): value of each upper-triangle entry.
    xi_d > 0.5 picks |a| ~ U(a1, b1), else U(a2, b2); xi_s > 0.5 picks +."""
    xi_d = rng.random(count)
    xi_s = rng.random(count)
    m1 = rng.uniform(a1, b1, count)
    m2 = rng.uniform(a2, b2, count)
    mag = np.where(xi_d > 0.5, m1, m2)
    return np.where(xi_s > 0.5, mag, -mag)


def random_tree_plus(n: int, c: float, mu: float = 1.1, seed: int = 0) -> CSR:
    """Random sparse matrix of Appendix A.2: a random tree on n vertices (each vertex
    of a random order attaches to a uniform earlier one) plus floor(c n) random
    edges; values by Algorithm III, a_ii = mu * sum |a_ij|."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    ii, jj = [], []
    for k in range(1, n):
        p = int(perm[int(rng.integers(0, k))])
        q = int(perm[k])
        ii.append(min(p, q))
        jj.append(max(p, q))
    existing = set(zip(ii, jj))
    extra = min(int(math.floor(c * n)), n * (n - 1) // 2 - len(existing))
    ai, aj = _add_random_edges(n, existing, extra, rng)
    pairs = sorted(zip(ii + ai, jj + aj))
    i = np.array([p for p, _ in pairs], dtype=np.int64)
    j = np.array([q for _, q in pairs], dtype=np.int64)
    off = algorithm_iii(i.size, rng)
    return from_edges(n, i, j, off, _dominant_diag(n, i, j, off, mu),
                      f"rtree_{n}_c{c:g}_mu{mu:g}_seed{seed}")


def banded(n: int, b: int, p: float, mu: float = 1.1, seed: int = 0) -> CSR:
    """Banded matrix of Appendix A.3: full bandwidth b (odd), every pair (i, j) with
    0 < j - i <= (b-1)/2 present with probability p; values by Algorithm III."""
    rng = np.random.default_rng(seed)
    h = (b - 1) // 2
    ii, jj = [], []
    for off in range(1, h + 1):
        i = np.arange(n - off, dtype=np.int64)
        keep = rng.random(i.size) < p
        ii.append(i[keep])
        jj.append(i[keep] + off)
    i = np.concatenate(ii) if ii else np.zeros(0, np.int64)
    j = np.concatenate(jj) if jj else np.zeros(0, np.int64)
    order = np.lexsort((j, i))
    i, j = i[order], j[order]
    off = algorithm_iii(i.size, rng)
    return from_edges(n, i, j, off, _dominant_diag(n, i, j, off, mu),
                      f"band_{n}_b{b}_p{p:g}_mu{mu:g}_seed{seed}")


# ----------------------------------------------------------------------------------------
# Right-hand sides.
# ----------------------------------------------------------------------------------------

def spmv_input(A: CSR, x: np.ndarray) -> np.ndarray:
    """b = A x in float64, used only to build right-hand sides."""
    return np.bincount(A.rows(), weights=A.val * x[A.col], minlength=A.n)


def rhs(A: CSR, seed: int = 1, lo: float = -1.0, hi: float = 1.0):
    """x* ~ U[lo, hi] (seeded), b = A x*.  Returns (x*, b)."""
    rng = np.random.default_rng(seed)
    xs = rng.uniform(lo, hi, A.n)
    return xs, spmv_input(A, xs)


# ----------------------------------------------------------------------------------------
# Workload recipes.
# ----------------------------------------------------------------------------------------

def poisson64(seed: int = 1):
    """64x64 5-point Dirichlet Laplacian (n = 4096, nnz = 20,224), x* ~ U[-1,1]."""
    A = laplacian_2d(64, 64)
    xs, b = rhs(A, seed)
    return A, xs, b


def batch_family(nsys: int, seed: int = 0, n_lo: float = 1e3, n_hi: float = 2.6e5):
    """Descriptors for a batch: n log-uniform in [n_lo, n_hi], family uniform over
    {2D, 3D, anisotropic 3D, shifted 3D}; grid sides rounded so that n is close to
    the drawn size.  Returns a list of (family, kwargs) usable by `build_desc`."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nsys):
        n = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        fam = ("2d", "3d", "aniso", "shift")[int(rng.integers(0, 4))]
        if fam == "2d":
            s = max(2, int(round(math.sqrt(n))))
            out.append(("2d", {"nx": s, "ny": s}))
        else:
            s = max(2, int(round(n ** (1.0 / 3.0))))
            if fam == "3d":
                out.append(("3d", {"nx": s}))
            elif fam == "aniso":
                out.append(("3d", {"nx": s, "eps": float(rng.choice([1e-2, 1e-3]))}))
            else:
                out.append(("3d", {"nx": s, "sigma": float(rng.choice([1e-4, 1e-2, 1.0]))}))
    return out


# The 3-D 7-point family of the benchmark: (name, anisotropy eps, shift sigma).
LAP3D_VARIANTS = (("sigma0", 1.0, 0.0), ("sigma1e-4", 1.0, 1e-4), ("sigma1e-2", 1.0, 1e-2),
                  ("sigma1", 1.0, 1.0), ("aniso1e-2", 1e-2, 0.0), ("aniso1e-3", 1e-3, 0.0))


def lap3d_workload(size: int = 128, seed: int = 1):
    """The benchmark systems: every LAP3D_VARIANTS matrix on a size^3 grid with
    x* ~ U[-1, 1] (seed) and b = A x*.  Yields (name, A, x*, b)."""
    for name, eps, sigma in LAP3D_VARIANTS:
        A = laplacian_3d(size, eps=eps, sigma=sigma)
        xs, b = rhs(A, seed)
        yield name, A, xs, b


def lap3d_training(seed: int = 7):
    """Training systems for a kNN sample of the 3-D family: other grid sizes and
    other shift / anisotropy values than the benchmark systems.
    Yields (name, A, b)."""
    rng = np.random.default_rng(seed)
    sizes = (72, 88, 104, 120, 136, 152)
    kinds = (("sigma", 0.0), ("sigma", 3e-4), ("sigma", 5e-3), ("sigma", 0.3), ("aniso", 3e-2),
             ("aniso", 3e-3))
    for s in sizes:
        for kind, p in kinds:
            A = laplacian_3d(s, eps=p if kind == "aniso" else 1.0, sigma=p if kind == "sigma" else 0.0)
            _, b = rhs(A, int(rng.integers(1, 1 << 30)))
            yield A.name, A, b


def build_desc(desc) -> CSR:
    fam, kw = desc
    if fam == "2d":
        return laplacian_2d(kw["nx"], kw["ny"], kw.get("sigma", 0.0))
    return laplacian_3d(kw["nx"], eps=kw.get("eps", 1.0), sigma=kw.get("sigma", 0.0))


def random_sample(count: int, seed: int = 0, classes=(2, 3, 4, 5, 6, 7)):
    """A synthetic labelled kNN sample: raw features (n, m, l~, v) drawn over
    ranges like those of the matrix families, and uniformly drawn classes.
    For testing classification mechanics, not for choosing eps1 in practice."""
    rng = np.random.default_rng(seed)
    n = np.exp(rng.uniform(math.log(1e3), math.log(2e6), count)).round()
    m = (n * rng.uniform(4.5, 9.0, count)).round()
    ell = np.exp(rng.uniform(math.log(3), math.log(7e4), count)).round()
    v = rng.uniform(0.2, 0.99, count)
    feat = np.stack([n, m, ell, v], axis=1)
    cls = rng.choice(np.array(classes, dtype=np.int8), count)
    return feat, cls
