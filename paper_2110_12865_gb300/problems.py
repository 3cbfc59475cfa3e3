"""Seeded synthetic workloads shared by the oracle tests, the CUDA path and the bench.

This module only *defines inputs*: mesh patterns, the incidence matrix A of
``K = A^T diag(w) A + shift*I``, per-element constant blocks ``K_e^0`` of the
element-sum form ``K = sum_e E_e K_e^0``, the fill-reducing permutation and
the per-instance values (w or E, shift, b).  It holds none of the assembly,
factorization or solve arithmetic.

The paper measures on meshes that are not available here (cloth, armadillo,
tet meshes; Sec. 5.3, 5.5, 5.6).  These generators stand in for them with the
same structure: 2D/3D meshes whose matrices come from mesh-derived weights
(cotangent weights as in Sec. 5.3, element blocks as the tagged dense blocks of
Sec. 4.2.4).

Conventions
-----------
* Nodes of a structured grid of shape ``dims`` are numbered in C order
  (last axis fastest).  Elasticity DOFs are ``3*node + component``.
* ``perm[new] = old``.  The permutation is an input to both the oracle and the
  library; it is produced here by geometric nested dissection.
* Every random number comes from ``numpy.random.default_rng(seed)`` (PCG64)
  with ``seed = 20211025 + 1000*cfg + instance``.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

SEED_BASE = 20211025

# pattern kinds, mirrored by SSCO_KIND_* in include/ssco.h
KIND_ATWA = 0
KIND_ELEM = 1
KIND_ELEM_BLOCKS = 2


def seed_for(cfg: int, instance: int) -> int:
    return SEED_BASE + 1000 * cfg + instance


# --------------------------------------------------------------------------
# orderings
# --------------------------------------------------------------------------
def nested_dissection(dims, leaf_max: int = 8) -> np.ndarray:
    """Geometric nested dissection of a structured node grid.

    The longest axis of a box (lowest axis index on ties) is split at
    ``mid = (lo+hi)//2`` (inclusive bounds); the separator is the node plane
    ``mid``.  Order: left box, right box, separator.  Boxes with at most
    ``leaf_max`` nodes, and separators, are listed in C order.  Valid for
    every stencil whose edges move at most one index per axis.
    Returns ``perm`` over nodes with ``perm[new] = old``.
    """
    dims = tuple(int(d) for d in dims)
    out: list[np.ndarray] = []

    def emit(lo, hi):
        rng = [np.arange(l, h + 1) for l, h in zip(lo, hi)]
        grids = np.meshgrid(*rng, indexing="ij")
        idx = np.ravel_multi_index(tuple(g.ravel() for g in grids), dims)
        out.append(idx.astype(np.int64))

    stack = [(tuple(0 for _ in dims), tuple(d - 1 for d in dims), 0)]
    # explicit stack emulating recursion: state 0 = visit, 1 = emit separator
    while stack:
        lo, hi, state = stack.pop()
        if any(h < l for l, h in zip(lo, hi)):
            continue
        if state == 1:
            emit(lo, hi)
            continue
        ext = [h - l + 1 for l, h in zip(lo, hi)]
        if int(np.prod(ext)) <= leaf_max:
            emit(lo, hi)
            continue
        ax = int(np.argmax(ext))
        mid = (lo[ax] + hi[ax]) // 2
        left_hi = list(hi)
        left_hi[ax] = mid - 1
        right_lo = list(lo)
        right_lo[ax] = mid + 1
        sep_lo = list(lo)
        sep_hi = list(hi)
        sep_lo[ax] = sep_hi[ax] = mid
        # pushed in reverse: left is processed first, separator last
        stack.append((tuple(sep_lo), tuple(sep_hi), 1))
        stack.append((tuple(right_lo), tuple(hi), 0))
        stack.append((tuple(lo), tuple(left_hi), 0))
    perm = np.concatenate(out) if out else np.zeros(0, np.int64)
    assert perm.size == int(np.prod(dims))
    return perm.astype(np.int32)


def expand_perm(node_perm: np.ndarray, k: int) -> np.ndarray:
    """Node permutation -> DOF permutation with ``k`` consecutive DOFs per node."""
    node_perm = np.asarray(node_perm, dtype=np.int64)
    return (node_perm[:, None] * k + np.arange(k)[None, :]).ravel().astype(np.int32)


# --------------------------------------------------------------------------
# graph patterns and incidence matrices
# --------------------------------------------------------------------------
def grid_edges(dims) -> np.ndarray:
    """Edges of the 2D 5-point / 3D 7-point stencil, (u, v) with u < v."""
    dims = tuple(dims)
    ids = np.arange(int(np.prod(dims))).reshape(dims)
    edges = []
    for ax in range(len(dims)):
        a = np.take(ids, np.arange(dims[ax] - 1), axis=ax).ravel()
        b = np.take(ids, np.arange(1, dims[ax]), axis=ax).ravel()
        edges.append(np.stack([a, b], 1))
    return np.concatenate(edges).astype(np.int64)


def trigrid_faces(nx: int, ny: int) -> np.ndarray:
    """Triangles of an nx x ny vertex grid (node id = i*ny + j), each cell
    split along its (i,j)-(i+1,j+1) diagonal."""
    ids = np.arange(nx * ny).reshape(nx, ny)
    a = ids[:-1, :-1].ravel()
    b = ids[1:, :-1].ravel()
    c = ids[1:, 1:].ravel()
    d = ids[:-1, 1:].ravel()
    t1 = np.stack([a, b, c], 1)
    t2 = np.stack([a, c, d], 1)
    return np.concatenate([t1, t2]).astype(np.int64)


def faces_to_edges(faces: np.ndarray):
    """Unique undirected edges of a triangle list, and for every face the
    edge id opposite each of its three corners."""
    f = faces
    half = np.concatenate([f[:, [1, 2]], f[:, [2, 0]], f[:, [0, 1]]])  # opp. corner 0,1,2
    lo = half.min(1)
    hi = half.max(1)
    key = lo * (int(f.max()) + 1) + hi
    uniq, inv = np.unique(key, return_inverse=True)
    nv = int(f.max()) + 1
    edges = np.stack([uniq // nv, uniq % nv], 1)
    opp = inv.reshape(3, -1).T  # [face, corner] -> edge id
    return edges.astype(np.int64), opp.astype(np.int64)


def incidence_csr(edges: np.ndarray, n: int):
    """Signed edge-vertex incidence: row e has +1 at u and -1 at v."""
    m = edges.shape[0]
    rowptr = np.arange(0, 2 * m + 1, 2, dtype=np.int64)
    colind = edges.reshape(-1).astype(np.int32)
    aval = np.tile(np.array([1.0, -1.0]), m)
    return rowptr, colind, aval


def path_incidence(n: int):
    """Incidence of a path graph plus one single-entry row at each end, so
    that ``A^T A = tridiag(-1, 2, -1)`` (rows with a single nonzero)."""
    rows = [[(0, 1.0)]]
    rows += [[(i, 1.0), (i + 1, -1.0)] for i in range(n - 1)]
    rows += [[(n - 1, 1.0)]]
    rowptr = np.zeros(len(rows) + 1, np.int64)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    colind = np.array([c for r in rows for c, _ in r], np.int32)
    aval = np.array([v for r in rows for _, v in r], np.float64)
    return rowptr, colind, aval


def cotan_weights(pos: np.ndarray, faces: np.ndarray, edges_opp):
    """Cotangent edge weights w_ij = 1/2 sum over adjacent triangles of the
    cotangent of the opposite angle (Sec. 5.3); cot = (u.v)/|u x v|."""
    edges, opp = edges_opp
    w = np.zeros(edges.shape[0])
    for c in range(3):
        k = faces[:, c]
        i = faces[:, (c + 1) % 3]
        j = faces[:, (c + 2) % 3]
        u = pos[i] - pos[k]
        v = pos[j] - pos[k]
        dot = (u * v).sum(1)
        cross = np.abs(u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0])
        np.add.at(w, opp[:, c], 0.5 * dot / cross)
    return w


# --------------------------------------------------------------------------
# linear elasticity on a Kuhn-split cube (tagged 12x12 element blocks)
# --------------------------------------------------------------------------
def kuhn_tets(k: int) -> np.ndarray:
    """6 tets per cell of a k^3-cell cube, split along the (0,0,0)-(1,1,1)
    diagonal: (v0, v0+e_p0, v0+e_p0+e_p1, v0+(1,1,1)) for every axis
    permutation p.  Nodes are numbered in C order on (k+1)^3."""
    dims = (k + 1,) * 3
    cells = np.stack(np.meshgrid(*[np.arange(k)] * 3, indexing="ij"), -1).reshape(-1, 3)
    tets = []
    for p in itertools.permutations(range(3)):
        e = np.eye(3, dtype=np.int64)
        c0 = cells
        c1 = c0 + e[p[0]]
        c2 = c1 + e[p[1]]
        c3 = c0 + 1
        tets.append(np.stack([np.ravel_multi_index(tuple(c.T), dims) for c in (c0, c1, c2, c3)], 1))
    # cell-major order: all 6 tets of a cell are consecutive
    t = np.stack(tets, 1).reshape(-1, 4)
    return t.astype(np.int64)


def lame_D(E: float = 1.0, nu: float = 0.3) -> np.ndarray:
    """Isotropic elasticity matrix, Voigt order (xx,yy,zz,yz,xz,xy), engineering shear."""
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[np.arange(3, 6), np.arange(3, 6)] = mu
    return D


def tet_stiffness(X: np.ndarray, D: np.ndarray) -> np.ndarray:
    """Element blocks K_e^0 = V_e B_e^T D B_e for linear tets.
    X: [n_tet, 4, 3] vertex positions.  Returns [n_tet, 12, 12]; local DOF
    order is 3*vertex + component."""
    nt = X.shape[0]
    M = np.ones((nt, 4, 4))
    M[:, :, 1:] = X
    Minv = np.linalg.inv(M)
    G = Minv[:, 1:, :]  # [nt, 3, 4]: d N_a / d x_c
    V = np.abs(np.linalg.det(M)) / 6.0
    B = np.zeros((nt, 6, 12))
    for a in range(4):
        gx, gy, gz = G[:, 0, a], G[:, 1, a], G[:, 2, a]
        B[:, 0, 3 * a + 0] = gx
        B[:, 1, 3 * a + 1] = gy
        B[:, 2, 3 * a + 2] = gz
        B[:, 3, 3 * a + 1] = gz
        B[:, 3, 3 * a + 2] = gy
        B[:, 4, 3 * a + 0] = gz
        B[:, 4, 3 * a + 2] = gx
        B[:, 5, 3 * a + 0] = gy
        B[:, 5, 3 * a + 1] = gx
    K = np.einsum("tki,kl,tlj->tij", B, D, B) * V[:, None, None]
    return 0.5 * (K + K.transpose(0, 2, 1))


def pack_lower(K: np.ndarray) -> np.ndarray:
    """[.., d, d] symmetric -> [.., d(d+1)/2], row-major lower (i >= j)."""
    d = K.shape[-1]
    ii, jj = np.tril_indices(d)
    return K[..., ii, jj]


# --------------------------------------------------------------------------
# problem assembly (inputs only)
# --------------------------------------------------------------------------
class Problem(dict):
    """Plain dict with attribute access.  Keys:
    kind, n, m, rowptr/colind/aval (ATWA) or elem_dim/elem_dofs/elem_K0
    (ELEM), perm, batch, vals [batch, m], shift [batch], b [batch, n],
    plus descriptive fields."""

    __getattr__ = dict.__getitem__


def _atwa(name, n, m, rowptr, colind, aval, perm, vals, shift, b, **extra):
    return Problem(kind=KIND_ATWA, name=name, n=int(n), m=int(m), rowptr=rowptr,
                   colind=colind, aval=aval, perm=np.ascontiguousarray(perm, np.int32),
                   batch=int(vals.shape[0]), vals=np.ascontiguousarray(vals),
                   shift=np.ascontiguousarray(shift, np.float64),
                   b=np.ascontiguousarray(b, np.float64), **extra)


def grid_problem(nx: int, ny: int, batch: int = 1, cfg: int = 1, shift: float = 1e-2,
                 w_dtype=np.float64, nd: bool = True):
    """2D 5-point grid Laplacian system, w ~ U[0.5, 2], b ~ N(0, 1)."""
    n = nx * ny
    edges = grid_edges((nx, ny))
    rowptr, colind, aval = incidence_csr(edges, n)
    m = edges.shape[0]
    vals = np.empty((batch, m), w_dtype)
    b = np.empty((batch, n))
    xstar = np.empty((batch, n))
    for i in range(batch):
        rng = np.random.default_rng(seed_for(cfg, i))
        vals[i] = rng.uniform(0.5, 2.0, m).astype(w_dtype)
        b[i] = rng.standard_normal(n)
        xstar[i] = rng.standard_normal(n)
    perm = nested_dissection((nx, ny)) if nd else np.arange(n, dtype=np.int32)
    return _atwa(f"grid{nx}x{ny}", n, m, rowptr, colind, aval, perm, vals,
                 np.full(batch, shift), b, dims=(nx, ny), edges=edges, xstar=xstar)


def trigrid_problem(s: int, batch: int = 1, cfg: int = 3, jitter: float = 0.3,
                    seed_offset: int = 0):
    """Triangulated s x s grid with cotangent weights from per-instance
    jittered vertices (+-jitter*h), shift ~ U[1e-3, 1e-1], b ~ N(0, 1)."""
    n = s * s
    faces = trigrid_faces(s, s)
    edges, opp = faces_to_edges(faces)
    rowptr, colind, aval = incidence_csr(edges, n)
    m = edges.shape[0]
    h = 1.0 / (s - 1)
    base = np.stack(np.meshgrid(np.arange(s), np.arange(s), indexing="ij"), -1).reshape(-1, 2) * h
    vals = np.empty((batch, m))
    shifts = np.empty(batch)
    b = np.empty((batch, n))
    positions = np.empty((batch, n, 2))
    for i in range(batch):
        rng = np.random.default_rng(seed_for(cfg, seed_offset + i))
        pos = base + rng.uniform(-jitter * h, jitter * h, base.shape)
        positions[i] = pos
        vals[i] = cotan_weights(pos, faces, (edges, opp))
        shifts[i] = rng.uniform(1e-3, 1e-1)
        b[i] = rng.standard_normal(n)
    perm = nested_dissection((s, s))
    return _atwa(f"trigrid{s}", n, m, rowptr, colind, aval, perm, vals, shifts, b,
                 dims=(s, s), edges=edges, faces=faces, opp=opp, positions=positions)


def uneven_trigrid_sides(count: int = 64, lo: int = 32, ratio: float = 8.0):
    return [int(round(lo * ratio ** (k / (count - 1)))) for k in range(count)]


def elasticity_problem(k: int, batch: int = 1, cfg: int = 2, jitter: float = 0.1,
                       nu: float = 0.3):
    """3D linear elasticity on a k^3 cube, 6 Kuhn tets per cell, nodes
    jittered by U[-jitter*h, jitter*h], bottom face (z = 0) fixed.
    Per-instance E_e = 10^U[3,5]; b ~ N(0, 1) on free DOFs, 0 on fixed.
    Geometry (hence K_e^0) comes from instance 0's seed and is shared."""
    dims = (k + 1,) * 3
    nn = int(np.prod(dims))
    n = 3 * nn
    h = 1.0 / k
    rng0 = np.random.default_rng(seed_for(cfg, 0))
    base = np.stack(np.meshgrid(*[np.arange(k + 1)] * 3, indexing="ij"), -1).reshape(-1, 3) * h
    pos = base + rng0.uniform(-jitter * h, jitter * h, base.shape)
    tets = kuhn_tets(k)
    Ke = tet_stiffness(pos[tets], lame_D(1.0, nu))
    node_fixed = np.isclose(base[:, 2], 0.0)
    dofs = (tets[:, :, None] * 3 + np.arange(3)[None, None, :]).reshape(-1, 12)
    dof_fixed = np.repeat(node_fixed, 3)
    elem_dofs = np.where(dof_fixed[dofs], -1, dofs).astype(np.int32)
    m = tets.shape[0]
    vals = np.empty((batch, m))
    b = np.empty((batch, n))
    for i in range(batch):
        rng = rng0 if i == 0 else np.random.default_rng(seed_for(cfg, i))
        vals[i] = 10.0 ** rng.uniform(3.0, 5.0, m)
        bi = rng.standard_normal(n)
        bi[dof_fixed] = 0.0
        b[i] = bi
    # Fixed DOFs are decoupled identity rows: numbering them first leaves the
    # fill unchanged and keeps every separator's free columns contiguous.
    dperm = expand_perm(nested_dissection(dims), 3)
    fixed_first = dof_fixed[dperm]
    perm = np.concatenate([dperm[fixed_first], dperm[~fixed_first]]).astype(np.int32)
    return Problem(kind=KIND_ELEM, name=f"elast{k}", n=n, m=m, elem_dim=12,
                   elem_dofs=np.ascontiguousarray(elem_dofs),
                   elem_K0=np.ascontiguousarray(pack_lower(Ke)), perm=perm,
                   batch=batch, vals=vals, shift=np.zeros(batch), b=b,
                   dims=dims, pos=pos, tets=tets, dof_fixed=dof_fixed, Ke=Ke)


def elasticity_geometry_problem(k: int, batch: int = 1, cfg: int = 6, jitter: float = 0.1,
                                nu: float = 0.3):
    """The k^3 Kuhn-tet elasticity mesh of elasticity_problem with the
    geometry itself varying per value set: instance i jitters the nodes by
    its own U[-jitter*h, jitter*h] draw and has its own E_e = 10^U[3,5].
    The pattern takes the element blocks per call (kind ELEM_BLOCKS), so the
    inputs are positions `pos` [batch][nodes][3], moduli `E` [batch][m] and
    `nu`; `vals` (the blocks) is left to the caller to build from them."""
    dims = (k + 1,) * 3
    nn = int(np.prod(dims))
    n = 3 * nn
    h = 1.0 / k
    base = np.stack(np.meshgrid(*[np.arange(k + 1)] * 3, indexing="ij"), -1).reshape(-1, 3) * h
    tets = kuhn_tets(k)
    node_fixed = np.isclose(base[:, 2], 0.0)
    dofs = (tets[:, :, None] * 3 + np.arange(3)[None, None, :]).reshape(-1, 12)
    dof_fixed = np.repeat(node_fixed, 3)
    elem_dofs = np.where(dof_fixed[dofs], -1, dofs).astype(np.int32)
    m = tets.shape[0]
    pos = np.empty((batch, nn, 3))
    E = np.empty((batch, m))
    b = np.empty((batch, n))
    for i in range(batch):
        rng = np.random.default_rng(seed_for(cfg, i))
        pos[i] = base + rng.uniform(-jitter * h, jitter * h, base.shape)
        E[i] = 10.0 ** rng.uniform(3.0, 5.0, m)
        bi = rng.standard_normal(n)
        bi[dof_fixed] = 0.0
        b[i] = bi
    dperm = expand_perm(nested_dissection(dims), 3)
    fixed_first = dof_fixed[dperm]
    perm = np.concatenate([dperm[fixed_first], dperm[~fixed_first]]).astype(np.int32)
    return Problem(kind=KIND_ELEM_BLOCKS, name=f"elastgeo{k}", n=n, m=m, elem_dim=12,
                   elem_dofs=np.ascontiguousarray(elem_dofs), elem_K0=None, perm=perm,
                   batch=batch, vals=None, shift=np.zeros(batch), b=b, dims=dims,
                   pos=pos, E=E, nu=float(nu), tets=np.ascontiguousarray(tets, np.int32),
                   dof_fixed=dof_fixed)


def laplacian_expression(p):
    """Expression nodes (structure only) of the weighted graph Laplacian of an
    ATWA problem, L = A^T (W A) with W = diag(w): leaves A (m x n, the
    incidence pattern) and W (m x m diagonal); node 4 is L.  Leaf values of
    value set b: A's entries then w_b."""
    m, n = p.m, p.n
    nodes = [("leaf", m, n, p.rowptr, p.colind), ("leaf", m, m, np.arange(m + 1), np.arange(m)),
             ("transpose", 0), ("mul", 1, 0), ("mul", 2, 3)]
    vals = np.stack([np.concatenate([p.aval, p.vals[b]]) for b in range(p.vals.shape[0])])
    return nodes, 4, vals


def symmetric_laplacian_leaf(p):
    """The weighted graph Laplacian of an ATWA problem as one leaf with shared
    values (structure only): the CSR pattern of L (neighbours and the vertex
    itself), and vmap sending (u, v) and (v, u) of edge e to value e and
    (u, u) to value m + u; n_vals = m + n.  The values themselves (-w_e off
    the diagonal, the sums on it) are the caller's."""
    m, n = p.m, p.n
    ends = np.asarray(p.colind).reshape(m, 2)
    u = np.concatenate([ends[:, 0], ends[:, 1], np.arange(n)])
    v = np.concatenate([ends[:, 1], ends[:, 0], np.arange(n)])
    val = np.concatenate([np.arange(m), np.arange(m), m + np.arange(n)])
    order = np.lexsort((v, u))
    u, v, val = u[order], v[order], val[order]
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, u + 1, 1)
    return np.cumsum(rowptr), v.astype(np.int32), val.astype(np.int64), m + n


def power_expression(rows, rowptr, colind, k: int = 3):
    """Nodes of M^k = (..(M M) M..) M for a square leaf M; the last node is M^k."""
    nodes = [("leaf", rows, rows, rowptr, colind), ("mul", 0, 0)]
    for _ in range(k - 2):
        nodes.append(("mul", len(nodes) - 1, 0))
    return nodes


def random_spd_pattern(n: int, extra_edges: int, rng, batch: int = 1):
    """Small random graph (a spanning path plus random edges) as an
    incidence matrix with w ~ U[0.5, 2] and shift 1e-1; random permutation."""
    e = [(i, i + 1) for i in range(n - 1)]
    for _ in range(extra_edges):
        u, v = rng.integers(0, n, 2)
        if u != v:
            e.append((min(u, v), max(u, v)))
    edges = np.unique(np.array(e, np.int64).reshape(-1, 2), axis=0) if e else np.zeros((0, 2), np.int64)
    rowptr, colind, aval = incidence_csr(edges, n)
    m = edges.shape[0]
    vals = rng.uniform(0.5, 2.0, (batch, m))
    shift = np.full(batch, 1e-1)
    b = rng.standard_normal((batch, n))
    perm = rng.permutation(n).astype(np.int32)
    return _atwa(f"rand{n}", n, m, rowptr, colind, aval, perm, vals, shift, b, edges=edges)


def workload(name: str, batch: int | None = None):
    """Named workloads (the five configurations of the hot path)."""
    if name == "grid32":
        return grid_problem(32, 32, batch or 1, cfg=1)
    if name == "elast24":
        return elasticity_problem(24, batch or 1, cfg=2)
    if name == "arap128":
        return trigrid_problem(128, batch or 256, cfg=3)
    if name == "grid256":
        return grid_problem(256, 256, batch or 1, cfg=4, w_dtype=np.float32)
    if name == "elast48":
        return elasticity_problem(48, batch or 16, cfg=5)
    if name.startswith("elast"):
        return elasticity_problem(int(name[5:]), batch or 1, cfg=2)
    if name.startswith("grid"):
        s = int(name[4:])
        return grid_problem(s, s, batch or 1, cfg=1)
    if name.startswith("trigrid"):
        s = int(name[7:])
        return trigrid_problem(s, batch or 1, cfg=3)
    raise KeyError(name)


def uneven_trigrids(count: int = 64):
    """Uneven-size triangulated grids, one value set each (sides from 32 to
    256, geometric)."""
    return [trigrid_problem(s, 1, cfg=3, seed_offset=10_000 + k)
            for k, s in enumerate(uneven_trigrid_sides(count))]
