"""Seeded synthetic workloads: P1 finite-element Poisson problems on triangulated squares.

This module only GENERATES INPUTS (matrix, node coordinates, right-hand sides). It holds none
of the multigrid method's arithmetic, so both the CUDA path and the CPU oracle may use it.

Workloads follow the paper's 2D experiments (Sec. 5, Example 1: -Laplace(u) = f on the unit
square, zero Dirichlet data, standard linear finite elements), on meshes synthesised here
because the paper's own meshes are only shown as (missing) figures:

* an ``n x n`` node grid on [0,1]^2, every cell split along its (i,j)-(i+1,j+1) diagonal;
* interior nodes jittered independently by U(-jitter*h, jitter*h) per coordinate
  (quasi-uniform grids), drawn from ``numpy.random.default_rng(seed)`` in lexicographic
  node order, x then y for each node;
* optionally graded by mapping x -> x^2, y -> y^2 after the jitter (shape-regular grids whose
  element size varies strongly towards the corner);
* optionally a piecewise-constant coefficient kappa, log10(kappa) ~ U(-1, 1), constant on
  each of 16 x 16 logical blocks of cells.

The stiffness matrix is assembled directly in its 7-point CSR layout (the topology of this
triangulation), with a fixed summation order, so the same seed gives the same bits on every
machine.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Problem:
    """A sparse SPD system with the geometry of its unknowns.

    rowptr/col/val: CSR (int32, int32, float64), columns ascending within each row.
    x, y: coordinates of each unknown (float64). b: right-hand side (float64).
    """

    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    x: np.ndarray
    y: np.ndarray
    b: np.ndarray
    name: str = ""
    z: np.ndarray | None = None  # third coordinate (3D problems only)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))


def _node_coords(n: int, jitter: float, graded: bool, rng: np.random.Generator):
    h = 1.0 / (n - 1)
    i = np.arange(n, dtype=np.float64)
    X = np.broadcast_to(i[None, :] * h, (n, n)).copy()  # X[j, i]
    Y = np.broadcast_to(i[:, None] * h, (n, n)).copy()
    if jitter > 0.0 and n > 2:
        m = n - 2
        d = rng.uniform(-jitter * h, jitter * h, size=(m * m, 2))  # node order, x then y
        X[1:-1, 1:-1] += d[:, 0].reshape(m, m)
        Y[1:-1, 1:-1] += d[:, 1].reshape(m, m)
    if graded:
        X = X * X
        Y = Y * Y
    return X, Y


def _triangle_terms(xa, ya, xb, yb, xc, yc, kap):
    """Area and the P1 stiffness entries of triangles (a, b, c) given counter-clockwise."""
    area2 = (xb - xa) * (yc - ya) - (xc - xa) * (yb - ya)  # twice the signed area
    if np.any(area2 <= 0.0):
        raise ValueError("mesh has a non-positive element area")
    # gradients of the barycentric functions times 2|T|
    gax, gay = yb - yc, xc - xb
    gbx, gby = yc - ya, xa - xc
    gcx, gcy = ya - yb, xb - xa
    s = kap / (2.0 * area2)  # kappa * |T| / (2|T|)^2
    k = {
        "aa": s * (gax * gax + gay * gay),
        "bb": s * (gbx * gbx + gby * gby),
        "cc": s * (gcx * gcx + gcy * gcy),
        "ab": s * (gax * gbx + gay * gby),
        "bc": s * (gbx * gcx + gby * gcy),
        "ac": s * (gax * gcx + gay * gcy),
    }
    return 0.5 * area2, k


def p1_poisson(n: int, jitter: float = 0.0, graded: bool = False, kappa_blocks: int = 0,
               seed: int = 0, rhs: str = "load", dirichlet: bool = True,
               name: str = "") -> Problem:
    """P1 stiffness matrix of -div(kappa grad u) on an ``n x n``-node triangulated unit square.

    ``dirichlet=True`` eliminates the boundary nodes (zero Dirichlet data): the unknowns are
    the ``(n-2)^2`` interior nodes in lexicographic order. ``dirichlet=False`` keeps every
    node (pure Neumann problem, singular, constants in the kernel).
    ``rhs``: "load" = load vector of f = 1 (sum of |T|/3 over the elements at each node),
    "normal" = N(0,1) entries from ``default_rng(seed + 1)``.
    """
    if n < 3:
        raise ValueError("need at least 3 nodes per side")
    rng = np.random.default_rng(seed)
    X, Y = _node_coords(n, jitter, graded, rng)
    kap = np.ones((n - 1, n - 1))
    if kappa_blocks:
        logk = rng.uniform(-1.0, 1.0, size=(kappa_blocks, kappa_blocks))
        cb = np.minimum((np.arange(n - 1) * kappa_blocks) // (n - 1), kappa_blocks - 1)
        kap = 10.0 ** logk[cb[:, None], cb[None, :]]  # kap[j, i] for cell (i, j)

    # cell (i, j): T1 = (i,j),(i+1,j),(i+1,j+1); T2 = (i,j),(i+1,j+1),(i,j+1)
    x00, y00 = X[:-1, :-1], Y[:-1, :-1]
    x10, y10 = X[:-1, 1:], Y[:-1, 1:]
    x11, y11 = X[1:, 1:], Y[1:, 1:]
    x01, y01 = X[1:, :-1], Y[1:, :-1]
    A1, k1 = _triangle_terms(x00, y00, x10, y10, x11, y11, kap)
    A2, k2 = _triangle_terms(x00, y00, x11, y11, x01, y01, kap)

    # edge couplings: E[j,i] = (i,j)-(i+1,j); N[j,i] = (i,j)-(i,j+1); D[j,i] = (i,j)-(i+1,j+1)
    E = np.zeros((n, n - 1))
    E[:-1, :] += k1["ab"]
    E[1:, :] += k2["bc"]  # T2 of cell (i, j-1): b=(i+1,j), c=(i,j) ... edge (i,j)-(i+1,j)
    Nn = np.zeros((n - 1, n))
    Nn[:, :-1] += k2["ac"]  # T2 of cell (i,j): a=(i,j), c=(i,j+1)
    Nn[:, 1:] += k1["bc"]  # T1 of cell (i-1,j): b=(i,j), c=(i,j+1)
    D = k1["ac"] + k2["ab"]  # both triangles share the diagonal (i,j)-(i+1,j+1)
    Dg = np.zeros((n, n))
    Dg[:-1, :-1] += k1["aa"]
    Dg[:-1, 1:] += k1["bb"]
    Dg[1:, 1:] += k1["cc"]
    Dg[:-1, :-1] += k2["aa"]
    Dg[1:, 1:] += k2["bb"]
    Dg[1:, :-1] += k2["cc"]
    load = np.zeros((n, n))
    for arr, sl in ((A1, (slice(0, -1), slice(0, -1))), (A1, (slice(0, -1), slice(1, None))),
                    (A1, (slice(1, None), slice(1, None))), (A2, (slice(0, -1), slice(0, -1))),
                    (A2, (slice(1, None), slice(1, None))), (A2, (slice(1, None), slice(0, -1)))):
        load[sl] += arr / 3.0

    if dirichlet:
        lo, hi = 1, n - 1
    else:
        lo, hi = 0, n
    m = hi - lo
    N = m * m
    jj, ii = np.meshgrid(np.arange(lo, hi), np.arange(lo, hi), indexing="ij")
    jj = jj.ravel()
    ii = ii.ravel()
    # the 7 couplings in ascending column order: SW, S, W, self, E, N, NE
    zeros = np.zeros(N)
    cand = [
        (ii - 1, jj - 1, lambda: D[np.clip(jj - 1, 0, n - 2), np.clip(ii - 1, 0, n - 2)]),
        (ii, jj - 1, lambda: Nn[np.clip(jj - 1, 0, n - 2), ii]),
        (ii - 1, jj, lambda: E[jj, np.clip(ii - 1, 0, n - 2)]),
        (ii, jj, lambda: Dg[jj, ii]),
        (ii + 1, jj, lambda: E[jj, np.clip(ii, 0, n - 2)]),
        (ii, jj + 1, lambda: Nn[np.clip(jj, 0, n - 2), ii]),
        (ii + 1, jj + 1, lambda: D[np.clip(jj, 0, n - 2), np.clip(ii, 0, n - 2)]),
    ]
    cols, vals, keep = [], [], []
    for ci, cj, getv in cand:
        ok = (ci >= lo) & (ci < hi) & (cj >= lo) & (cj < hi)
        cols.append(np.where(ok, (cj - lo) * m + (ci - lo), 0))
        vals.append(np.where(ok, getv(), zeros))
        keep.append(ok)
    cols = np.stack(cols, axis=1)
    vals = np.stack(vals, axis=1)
    keep = np.stack(keep, axis=1)
    counts = keep.sum(axis=1)
    rowptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    col = cols[keep].astype(np.int32)
    val = vals[keep].astype(np.float64)
    xs = X[lo:hi, lo:hi].ravel().copy()
    ys = Y[lo:hi, lo:hi].ravel().copy()
    if rhs == "load":
        b = load[lo:hi, lo:hi].ravel().copy()
    elif rhs == "normal":
        b = np.random.default_rng(seed + 1).standard_normal(N)
    elif rhs == "zero":
        b = np.zeros(N)
    else:
        raise ValueError(f"unknown rhs {rhs!r}")
    if rowptr[-1] >= 2**31:
        raise ValueError("matrix too large for int32 indices")
    return Problem(N, rowptr.astype(np.int32), col, val, xs, ys, b, name=name)


def five_point_grid(M: int, name: str = "") -> Problem:
    """5-point Laplacian [4,-1,-1,-1,-1] on an M x M grid (zero Dirichlet data outside).

    Unknown (i, j) sits at the cell centre ((i + 1/2)/M, (j + 1/2)/M), so with the auxiliary
    box fixed to [0,1]^2 and M = 2^(L+1) every level-L cell holds a 2 x 2 block of unknowns:
    the uniform-grid case in which the auxiliary-grid aggregation is geometric coarsening
    (Sec. 5, uniform grid).
    """
    N = M * M
    jj, ii = np.meshgrid(np.arange(M), np.arange(M), indexing="ij")
    jj = jj.ravel()
    ii = ii.ravel()
    cand = [(ii, jj - 1, -1.0), (ii - 1, jj, -1.0), (ii, jj, 4.0), (ii + 1, jj, -1.0),
            (ii, jj + 1, -1.0)]
    cols, vals, keep = [], [], []
    for ci, cj, v in cand:
        ok = (ci >= 0) & (ci < M) & (cj >= 0) & (cj < M)
        cols.append(np.where(ok, cj * M + ci, 0))
        vals.append(np.full(N, v))
        keep.append(ok)
    cols = np.stack(cols, 1)
    vals = np.stack(vals, 1)
    keep = np.stack(keep, 1)
    rowptr = np.zeros(N + 1, dtype=np.int32)
    np.cumsum(keep.sum(1), out=rowptr[1:])
    x = (ii + 0.5) / M
    y = (jj + 0.5) / M
    b = np.ones(N) / (M * M)
    return Problem(N, rowptr, cols[keep].astype(np.int32), vals[keep], x.astype(np.float64),
                   y.astype(np.float64), b, name=name)


# --- the named workloads -------------------------------------------------------------------

WORKLOADS = {
    # 65x65 nodes, jitter 0.2h, load vector of f=1, auxiliary grid 64x64 (L=6)
    "quasi_uniform_65": dict(n=65, jitter=0.2, seed=0, rhs="load", aux_level=6),
    # 1025x1025 nodes, jitter 0.2h, N(0,1) rhs, auxiliary grid 1024x1024 (L=10)
    "quasi_uniform_1025": dict(n=1025, jitter=0.2, seed=0, rhs="normal", aux_level=10),
    # 1449x1449 nodes graded x->x^2, y->y^2, jitter 0.1h, kappa on 16x16 blocks, L auto (=10)
    "graded_1449": dict(n=1449, jitter=0.1, graded=True, kappa_blocks=16, seed=0,
                        rhs="normal", aux_level=0),
    # disk of radius 0.5 cut from 1921x1921 nodes (jitter 0.2h): about 2.89M unknowns, the
    # size of the paper's smaller disk example; empty auxiliary cells in the corners; L auto
    "disk_1921": dict(disk=True, n=1921, jitter=0.2, seed=0, rhs="normal", aux_level=0),
    # 3D: 129^3-node Kuhn tetrahedral grid of the unit cube (jitter 0.15h), 2,048,383
    # unknowns, octree depth auto (= 6)
    "cube_129": dict(cube=True, n=129, seed=0, rhs="normal", aux_level=0),
}


def workload(name: str, **overrides) -> tuple[Problem, int]:
    """Return (problem, aux_level) for a named workload (aux_level 0 = automatic)."""
    spec = dict(WORKLOADS[name])
    spec.update(overrides)
    aux = spec.pop("aux_level")
    if spec.pop("disk", False):
        return disk_poisson(name=name, **spec), aux
    if spec.pop("cube", False):
        return p1_poisson_3d(name=name, **spec), aux
    return p1_poisson(name=name, **spec), aux


def batch_workload(count: int = 256, nmin: int = 45, nmax: int = 450, seed: int = 4,
                   jitter: float = 0.2) -> list[Problem]:
    """Independent jittered P1 Poisson systems of uneven sizes: system k has n_k x n_k nodes,
    n_k drawn log-uniform in [nmin, nmax] (so E[(n_k - 2)^2] is about 43k unknowns for the
    defaults), N(0,1) right-hand side; mesh seed `seed` + k + 1. The auxiliary level is chosen
    per system (aux_level 0)."""
    rng = np.random.default_rng(seed)
    sides = np.exp(rng.uniform(np.log(nmin), np.log(nmax), size=count))
    sides = np.clip(np.rint(sides).astype(int), nmin, nmax)
    return [p1_poisson(int(m), jitter=jitter, seed=seed + k + 1, rhs="normal",
                       name=f"batch_{k}_n{int(m)}") for k, m in enumerate(sides)]


def disk_poisson(n: int, jitter: float = 0.2, seed: int = 0, rhs: str = "normal",
                 radius: float = 0.5, name: str = "") -> Problem:
    """P1 Poisson on a disk cut from the jittered n x n triangulation of the unit square: the
    unknowns are the interior nodes at distance < radius from (0.5, 0.5), every other node is
    held at zero (Dirichlet), so the matrix is the principal submatrix of the square's on
    those nodes (SPD) and the domain is the union of elements with a node inside, a staircase
    approximation of the disk. The auxiliary grid over the nodes' bounding box then has empty
    cells in its four corners, as the paper's disk examples do. rhs: "normal" = N(0,1) from
    default_rng(seed + 1) over the kept unknowns, "load" = the square's load vector there."""
    sq = p1_poisson(n, jitter=jitter, seed=seed, rhs="load" if rhs == "load" else "zero")
    keep = np.flatnonzero((sq.x - 0.5) ** 2 + (sq.y - 0.5) ** 2 < radius * radius)
    if keep.size == 0:
        raise ValueError("no node inside the disk")
    newid = np.full(sq.n, -1, np.int64)
    newid[keep] = np.arange(keep.size)
    counts = np.diff(sq.rowptr.astype(np.int64))
    rows = np.repeat(np.arange(sq.n), counts)
    cnew = newid[sq.col]
    ok = (newid[rows] >= 0) & (cnew >= 0)
    r2, c2, v2 = newid[rows[ok]], cnew[ok], sq.val[ok]  # rows ascending, columns ascending
    rowptr = np.zeros(keep.size + 1, np.int64)
    np.add.at(rowptr, r2 + 1, 1)
    np.cumsum(rowptr, out=rowptr)
    if rhs == "normal":
        b = np.random.default_rng(seed + 1).standard_normal(keep.size)
    elif rhs == "load":
        b = sq.b[keep].copy()
    else:
        raise ValueError(f"unknown rhs {rhs!r}")
    return Problem(int(keep.size), rowptr.astype(np.int32), c2.astype(np.int32),
                   v2.astype(np.float64), sq.x[keep].copy(), sq.y[keep].copy(), b, name=name)


# Kuhn triangulation of the unit cube: one tetrahedron per ordering of the axes, the path
# (0,0,0) -> (0,0,0) + e_a -> ... + e_b -> (1,1,1); conforming across neighbouring cubes
_KUHN = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def p1_poisson_3d(n: int, jitter: float = 0.15, seed: int = 0, rhs: str = "normal",
                  name: str = "") -> Problem:
    """P1 stiffness matrix of -Laplace(u) on the unit cube, an ``n x n x n``-node grid with
    every cube split into the 6 tetrahedra of the Kuhn triangulation, interior nodes jittered
    by U(-jitter*h, jitter*h) per coordinate (default_rng(seed), lexicographic node order,
    x, y, z per node), zero Dirichlet data (the unknowns are the (n-2)^3 interior nodes,
    lexicographic with x fastest). rhs: "normal" = N(0,1) from default_rng(seed + 1), "load"
    = the load vector of f = 1 (|T|/4 per vertex). Assembled in stencil form (one array per
    node offset); the entries of one (row, column) pair are summed by tetrahedron type, then
    by local vertex pair, the same bits on every machine; the matrix is exactly symmetric. Tetrahedra are asserted
    non-degenerate."""
    if n < 3:
        raise ValueError("need at least 3 nodes per side")
    rng = np.random.default_rng(seed)
    h = 1.0 / (n - 1)
    g = np.arange(n) * h
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")  # [k, j, i]
    if jitter:
        d = rng.uniform(-jitter * h, jitter * h, size=(n, n, n, 3))
        inner = np.zeros((n, n, n), bool)
        inner[1:-1, 1:-1, 1:-1] = True
        X = X + np.where(inner, d[..., 0], 0.0)
        Y = Y + np.where(inner, d[..., 1], 0.0)
        Z = Z + np.where(inner, d[..., 2], 0.0)
    P = np.stack([X, Y, Z], axis=-1).reshape(-1, 3)  # node id = i + n j + n^2 k
    kk, jj, ii = np.meshgrid(np.arange(n - 1), np.arange(n - 1), np.arange(n - 1), indexing="ij")
    base = (ii + n * jj + n * n * kk).ravel()  # lowest node of each cube
    step = np.array([1, n, n * n])
    node_i = np.arange(n ** 3)
    ni, nj, nk = node_i % n, (node_i // n) % n, node_i // (n * n)
    inner = (ni > 0) & (ni < n - 1) & (nj > 0) & (nj < n - 1) & (nk > 0) & (nk < n - 1)
    # A in stencil form: entry (i, i + d) of every node i, one array per node offset d. Every
    # tetrahedron type puts its vertices at fixed offsets from the cube's base node, so a
    # (type, local pair) adds to one offset at distinct nodes. Contributions are added type by
    # type, and within a type by unordered local pair, so (i, j) and (j, i) add the same values
    # in the same order and A is exactly symmetric.
    stencil: dict = {}
    vols, tets = [], []
    for perm in _KUHN:
        off = np.cumsum([0] + [int(step[q]) for q in perm])  # vertex offsets from the base
        T = base[:, None] + off[None, :]
        V = P[T]  # [ne, 4, 3]
        E = V[:, 1:, :] - V[:, :1, :]  # edges from vertex 0
        det = np.linalg.det(E)
        if not np.all(np.abs(det) > 0):
            raise ValueError("degenerate tetrahedron")
        vol = np.abs(det) / 6.0
        # gradients of the barycentric functions: grad(lambda_a) = column a-1 of inv(E), a >= 1
        Ginv = np.linalg.inv(E)
        G = np.empty((T.shape[0], 4, 3))
        G[:, 1:, :] = np.transpose(Ginv, (0, 2, 1))
        G[:, 0, :] = -G[:, 1:, :].sum(axis=1)
        for a in range(4):
            for b in range(a, 4):
                kab = vol * np.einsum("ei,ei->e", G[:, a], G[:, b])
                for (s, t) in ((a, b),) if a == b else ((a, b), (b, a)):
                    d = int(off[t] - off[s])
                    acc = stencil.setdefault(d, np.zeros(n ** 3))
                    acc[T[:, s]] += kab  # distinct nodes within one (type, pair)
        vols.append(vol)
        tets.append(T)
    # unknowns: interior nodes; keep the entries whose column is interior too
    N = (n - 2) ** 3
    uid = np.full(n ** 3, -1, np.int64)
    uid[inner] = np.arange(N)
    rows_node = node_i[inner]
    ds = sorted(stencil)
    cols = np.stack([uid[np.clip(rows_node + d, 0, n ** 3 - 1)] for d in ds], axis=1)
    vals = np.stack([stencil[d][rows_node] for d in ds], axis=1)
    valid = np.stack([(rows_node + d >= 0) & (rows_node + d < n ** 3) for d in ds], axis=1)
    valid &= cols >= 0
    cnt = valid.sum(axis=1)
    indptr = np.zeros(N + 1, np.int64)
    indptr[1:] = np.cumsum(cnt)
    # offsets ascend, and so do the interior ids of i + d: each row comes out sorted
    indices, data = cols[valid], vals[valid]
    xs, ys, zs = P[inner, 0].copy(), P[inner, 1].copy(), P[inner, 2].copy()
    if rhs == "normal":
        b = np.random.default_rng(seed + 1).standard_normal(N)
    elif rhs == "load":
        load = np.zeros(n ** 3)
        for T, vol in zip(tets, vols):
            np.add.at(load, T.ravel(), np.repeat(vol / 4.0, 4))
        b = load[inner].copy()
    else:
        raise ValueError(f"unknown rhs {rhs!r}")
    return Problem(N, indptr.astype(np.int32), indices.astype(np.int32),
                   data.astype(np.float64), xs, ys, b, name=name, z=zs)
