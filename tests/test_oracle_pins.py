"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test checks one part of the oracle against a closed form, a library
routine used as a whole step (numpy dense Cholesky / solve / slogdet), brute
force on tiny inputs, or an invariant, chosen so that a dropped term, a wrong
sign, a wrong index or a transposed operand in the oracle fails at least one.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_12865_gb300 import problems as P


def dense_A(p):
    A = np.zeros((p.m, p.n))
    for e in range(p.m):
        s, t = p.rowptr[e], p.rowptr[e + 1]
        A[e, p.colind[s:t]] = p.aval[s:t]
    return A


def dense_K(p, inst=0):
    """K written out with numpy dense products (A^T W A + shift I), or the
    element blocks scattered with np.add.at; fixed DOFs become identity."""
    if p.kind == P.KIND_ATWA:
        A = dense_A(p)
        return A.T @ np.diag(np.asarray(p.vals[inst], np.float64)) @ A + p.shift[inst] * np.eye(p.n)
    K = np.zeros((p.n, p.n))
    E = p.vals[inst]
    d = p.elem_dim
    for e in range(p.m):
        full = np.zeros((d, d))
        ii, jj = np.tril_indices(d)
        full[ii, jj] = p.elem_K0[e]
        full[jj, ii] = p.elem_K0[e]
        dofs = p.elem_dofs[e]
        keep = dofs >= 0
        idx = dofs[keep]
        np.add.at(K, (idx[:, None], idx[None, :]), E[e] * full[np.ix_(keep, keep)])
    ref = np.zeros(p.n, bool)
    ref[p.elem_dofs[p.elem_dofs >= 0]] = True
    K[~ref, ~ref] = 1.0
    K[ref, ref] += p.shift[inst]
    return K


def permuted(Kd, perm):
    return Kd[np.ix_(perm, perm)]


def col_rel_err(L, Lref):
    num = np.linalg.norm(L - Lref, axis=0)
    den = np.linalg.norm(Lref, axis=0)
    return float(np.max(num / den))


# ----------------------------------------------------------------------------
# assembly
# ----------------------------------------------------------------------------
def test_assembly_grid_closed_form():
    """5-point grid: K_uu = sum_{e ni u} w_e + shift, K_uv = -w_e."""
    p = P.grid_problem(7, 5, cfg=1)
    K = O.assemble(p).dense()
    w = p.vals[0]
    ref = np.zeros((p.n, p.n))
    for e, (u, v) in enumerate(p.edges):
        ref[u, u] += w[e]
        ref[v, v] += w[e]
        ref[u, v] = ref[v, u] = -w[e]
    ref += p.shift[0] * np.eye(p.n)
    np.testing.assert_allclose(K, ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("maker", [lambda: P.grid_problem(16, 12, cfg=1),
                                   lambda: P.trigrid_problem(9, cfg=3),
                                   lambda: P.random_spd_pattern(60, 90, np.random.default_rng(3))])
def test_assembly_matches_dense_product(maker):
    p = maker()
    assert p.m <= 4096
    np.testing.assert_allclose(O.assemble(p).dense(), dense_K(p), rtol=1e-14, atol=1e-13)


def test_assembly_elem_matches_dense_scatter():
    p = P.elasticity_problem(2, cfg=2)
    p["shift"] = np.array([0.25])
    np.testing.assert_allclose(O.assemble(p).dense(), dense_K(p), rtol=1e-13, atol=1e-9)


def test_element_blocks_rigid_modes():
    """Each unconstrained K_e^0 is symmetric PSD with the 6 rigid-body modes
    (3 translations, 3 infinitesimal rotations) in its null space."""
    p = P.elasticity_problem(2, cfg=2)
    for e in range(0, p.m, 7):
        Ke = p.Ke[e]
        X = p.pos[p.tets[e]]
        modes = []
        for c in range(3):
            t = np.zeros((4, 3))
            t[:, c] = 1
            modes.append(t.ravel())
        for a, b in [(0, 1), (1, 2), (0, 2)]:
            r = np.zeros((4, 3))
            r[:, a] = -X[:, b]
            r[:, b] = X[:, a]
            modes.append(r.ravel())
        R = np.array(modes).T
        assert np.abs(Ke @ R).max() < 1e-10 * np.abs(Ke).max()
        ev = np.linalg.eigvalsh(Ke)
        assert ev.min() > -1e-12 * ev.max()
        assert np.sum(ev > 1e-8 * ev.max()) == 6


def test_permute_matches_dense():
    p = P.random_spd_pattern(40, 60, np.random.default_rng(5))
    Kp = O.permute(O.assemble(p), p.perm).dense()
    np.testing.assert_array_equal(Kp, permuted(O.assemble(p).dense(), p.perm))


# ----------------------------------------------------------------------------
# symbolic
# ----------------------------------------------------------------------------
def brute_symbolic(Kp_dense_bool):
    """Dense boolean elimination: returns pattern of L (lower incl. diagonal)."""
    n = Kp_dense_bool.shape[0]
    G = np.tril(Kp_dense_bool.copy()) | np.eye(n, dtype=bool)
    for k in range(n):
        rows = np.nonzero(G[k + 1:, k])[0] + k + 1
        for i in rows:
            G[i, rows[rows <= i]] = True
    return G


def levels_by_definition(parent):
    n = len(parent)
    lev = [0] * n
    for j in range(n):  # children precede parents
        if parent[j] >= 0:
            lev[parent[j]] = max(lev[parent[j]], lev[j] + 1)
    return np.array(lev)


@pytest.mark.parametrize("seed", range(6))
def test_symbolic_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(20, 300))
    p = P.random_spd_pattern(n, int(rng.integers(0, 2 * n)), rng)
    Kp = O.permute(O.assemble(p), p.perm)
    S = O.Symbolic(Kp)
    G = brute_symbolic(Kp.dense() != 0)
    Lpat = np.zeros((n, n), bool)
    for j in range(n):
        Lpat[S.Lrowind[S.Lcolptr[j]:S.Lcolptr[j + 1]], j] = True
    np.testing.assert_array_equal(Lpat, G)
    parent = np.array([np.nonzero(G[j + 1:, j])[0][0] + j + 1 if G[j + 1:, j].any() else -1
                       for j in range(n)])
    np.testing.assert_array_equal(S.parent, parent)
    np.testing.assert_array_equal(S.colcount, G.sum(0))
    np.testing.assert_array_equal(S.col_level, levels_by_definition(parent))
    # fundamental supernodes by definition
    nchild = np.bincount(parent[parent >= 0], minlength=n)
    cnt = G.sum(0)
    first = [j for j in range(n) if not (j > 0 and parent[j - 1] == j and nchild[j] == 1
                                         and cnt[j] == cnt[j - 1] - 1)]
    np.testing.assert_array_equal(S.snode_first[:-1], first)
    # supernodal tree levels by definition
    col2sn = np.repeat(np.arange(len(first)), np.diff(list(first) + [n]))
    snp = np.array([col2sn[parent[S.snode_first[k + 1] - 1]] if parent[S.snode_first[k + 1] - 1] >= 0
                    else -1 for k in range(len(first))])
    np.testing.assert_array_equal(S.sn_parent, snp)
    np.testing.assert_array_equal(S.sn_level, levels_by_definition(snp))


def test_symbolic_path_natural_order():
    """Path graph in natural order: zero fill, chain etree, n levels."""
    n = 50
    rowptr, colind, aval = P.path_incidence(n)
    p = P.Problem(kind=0, n=n, m=len(rowptr) - 1, rowptr=rowptr, colind=colind, aval=aval,
                  perm=np.arange(n, dtype=np.int32), vals=np.ones((1, len(rowptr) - 1)),
                  shift=np.zeros(1), b=np.ones((1, n)), batch=1)
    Kp = O.permute(O.assemble(p), p.perm)
    S = O.Symbolic(Kp)
    assert S.nnzL == Kp.nnz == 2 * n - 1
    np.testing.assert_array_equal(S.parent, list(range(1, n)) + [-1])
    np.testing.assert_array_equal(S.col_level, np.arange(n))


def test_symbolic_dense_is_one_supernode():
    n = 30
    edges = np.array([(i, j) for i in range(n) for j in range(i + 1, n)])
    rowptr, colind, aval = P.incidence_csr(edges, n)
    p = P.Problem(kind=0, n=n, m=len(edges), rowptr=rowptr, colind=colind, aval=aval,
                  perm=np.random.default_rng(0).permutation(n).astype(np.int32),
                  vals=np.ones((1, len(edges))), shift=np.ones(1), b=np.ones((1, n)), batch=1)
    S = O.Symbolic(O.permute(O.assemble(p), p.perm))
    assert S.n_snodes == 1 and S.nnzL == n * (n + 1) // 2


def test_symbolic_tree_leaf_first_zero_fill():
    """A tree whose vertices are numbered children-before-parent factors with
    no fill."""
    rng = np.random.default_rng(7)
    n = 200
    par = [int(rng.integers(i + 1, n)) for i in range(n - 1)]  # parent index > child
    edges = np.array([(i, par[i]) for i in range(n - 1)])
    rowptr, colind, aval = P.incidence_csr(edges, n)
    p = P.Problem(kind=0, n=n, m=n - 1, rowptr=rowptr, colind=colind, aval=aval,
                  perm=np.arange(n, dtype=np.int32), vals=np.ones((1, n - 1)),
                  shift=np.full(1, 0.5), b=np.ones((1, n)), batch=1)
    Kp = O.permute(O.assemble(p), p.perm)
    S = O.Symbolic(Kp)
    assert S.nnzL == Kp.nnz
    np.testing.assert_array_equal(S.parent, par + [-1])


# ----------------------------------------------------------------------------
# numeric factorization
# ----------------------------------------------------------------------------
def test_tridiagonal_closed_form():
    """A^T A of the path incidence with single-entry end rows is
    tridiag(-1, 2, -1); its factor is l_ii = sqrt((i+1)/i),
    l_{i+1,i} = -sqrt(i/(i+1)) (1-based)."""
    n = 64
    rowptr, colind, aval = P.path_incidence(n)
    p = P.Problem(kind=0, n=n, m=len(rowptr) - 1, rowptr=rowptr, colind=colind, aval=aval,
                  perm=np.arange(n, dtype=np.int32), vals=np.ones((1, len(rowptr) - 1)),
                  shift=np.zeros(1), b=np.ones((1, n)), batch=1)
    r = O.refactor_solve(p)
    assert r.bad == -1
    L = r.S.L_dense(r.L)
    i = np.arange(1, n + 1, dtype=np.float64)
    np.testing.assert_allclose(np.diag(L), np.sqrt((i + 1) / i), rtol=2e-16 * 8, atol=0)
    np.testing.assert_allclose(np.diag(L, -1), -np.sqrt(i[:-1] / (i[:-1] + 1)), rtol=2e-16 * 8, atol=0)


@pytest.mark.parametrize("seed", range(8))
def test_cholesky_matches_numpy_dense(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(2, 65))
    p = P.random_spd_pattern(n, int(rng.integers(0, 3 * n)), rng)
    r = O.refactor_solve(p)
    assert r.bad == -1
    Lref = np.linalg.cholesky(permuted(dense_K(p), p.perm))
    L = r.S.L_dense(r.L)
    assert col_rel_err(L, Lref) <= 1e-13
    assert np.all(np.triu(L, 1) == 0)


def own_dense_cholesky(A):
    """Textbook dense Cholesky-Crout in pure Python loops (a second pin,
    independent of numpy's LAPACK)."""
    n = len(A)
    L = [[0.0] * n for _ in range(n)]
    for j in range(n):
        s = A[j][j] - sum(L[j][k] * L[j][k] for k in range(j))
        L[j][j] = s ** 0.5
        for i in range(j + 1, n):
            L[i][j] = (A[i][j] - sum(L[i][k] * L[j][k] for k in range(j))) / L[j][j]
    return np.array(L)


def test_cholesky_matches_own_dense_routine():
    p = P.grid_problem(5, 4, cfg=1)
    r = O.refactor_solve(p)
    Kp = permuted(dense_K(p), p.perm)
    assert col_rel_err(r.S.L_dense(r.L), own_dense_cholesky(Kp.tolist())) <= 1e-14


@pytest.mark.parametrize("maker", [lambda: P.grid_problem(32, 32, cfg=1),
                                   lambda: P.trigrid_problem(20, cfg=3),
                                   lambda: P.elasticity_problem(4, cfg=2)])
def test_reconstruction(maker):
    p = maker()
    r = O.refactor_solve(p)
    Kp = r.Kp.dense()
    L = r.S.L_dense(r.L)
    assert np.linalg.norm(L @ L.T - Kp) / np.linalg.norm(Kp) < 1e-14


def test_not_spd_reports_first_failing_column():
    """Pivot j of Cholesky equals det(K~[:j+1,:j+1]) / det(K~[:j,:j]); the
    oracle must stop at the first j where it is not positive."""
    rng = np.random.default_rng(11)
    hits = 0
    for t in range(40):
        n = 30
        p = P.random_spd_pattern(n, 40, rng)
        p["vals"] = rng.uniform(-0.3, 2.0, (1, p.m))
        p["shift"] = np.array([-0.05])
        r = O.refactor_solve(p)
        Kp = permuted(dense_K(p), p.perm)
        first = -1
        prev = 0.0  # log|det| of the empty minor
        for j in range(n):
            sgn, ld = np.linalg.slogdet(Kp[: j + 1, : j + 1])
            if sgn <= 0:
                first = j
                break
        assert r.bad == first
        hits += first >= 0
    assert hits > 5


# ----------------------------------------------------------------------------
# solves
# ----------------------------------------------------------------------------
def test_solve_matches_numpy_dense():
    p = P.grid_problem(32, 32, cfg=1)
    r = O.refactor_solve(p)
    x = np.linalg.solve(dense_K(p), p.b[0])
    assert np.linalg.norm(r.x - x) / np.linalg.norm(x) < 1e-13


def test_solve_residual_elasticity():
    p = P.elasticity_problem(5, cfg=2)
    r = O.refactor_solve(p)
    res = O.symv(r.K, r.x) - p.b[0]
    assert np.linalg.norm(res) / np.linalg.norm(p.b[0]) < 1e-12
    assert np.all(r.x[p.dof_fixed] == 0.0)


def test_symv_matches_dense():
    p = P.trigrid_problem(10, cfg=3)
    K = O.assemble(p)
    x = np.random.default_rng(1).standard_normal(p.n)
    np.testing.assert_allclose(O.symv(K, x), dense_K(p) @ x, rtol=1e-13, atol=1e-12)


# ----------------------------------------------------------------------------
# adjoint
# ----------------------------------------------------------------------------
def loss_and_grad(p, inst=0):
    r = O.refactor_solve(p, inst)
    xs = p.xstar[inst]
    xbar = 2.0 * (r.x - xs)
    vbar, sbar, bbar = O.backward(p, r, xbar, inst)
    return float(np.sum((r.x - xs) ** 2)), vbar, sbar, bbar


def fd_loss(p, vals, shift, b, inst=0):
    r = O.refactor_solve(p, inst, vals=vals, shift=shift, b=b)
    return r.x


def fd_diff(p, xp, xm, inst=0):
    """loss(x+) - loss(x-) for loss = ||x - x*||^2, written as
    sum (x+ - x-)(x+ + x- - 2 x*) so the two large sums do not cancel."""
    return float(np.sum((xp - xm) * (xp + xm - 2.0 * p.xstar[inst])))


@pytest.mark.parametrize("shift", [1.0, 1e-2])
def test_gradient_central_differences(shift):
    """|g - g_FD| <= 1e-5 max(|g_FD|, 1e-3 ||g_FD||_inf) + floor, h = 1e-6.

    The central difference itself carries a rounding floor of about
    kappa(K) * u * ||x||_inf * ||xbar||_1 / h (the two perturbed solves round
    independently).  With shift 1 (kappa ~ 10) that floor is far below the
    1e-5 criterion and is set to 0; with shift 1e-2 (kappa ~ 1e3) it is added."""
    p = P.grid_problem(8, 8, cfg=4, shift=shift)
    _, vbar, sbar, bbar = loss_and_grad(p)
    rng = np.random.default_rng(3)
    h = 1e-6
    w0, s0, b0 = p.vals[0].astype(np.float64), float(p.shift[0]), p.b[0].copy()
    edges = rng.choice(p.m, 32, replace=False)
    g_fd = []
    for e in edges:
        wp, wm = w0.copy(), w0.copy()
        wp[e] += h
        wm[e] -= h
        g_fd.append(fd_diff(p, fd_loss(p, wp, s0, b0), fd_loss(p, wm, s0, b0)) / (2 * h))
    g_fd = np.array(g_fd)
    r = O.refactor_solve(p)
    ev = np.linalg.eigvalsh(dense_K(p))
    floor = 0.0 if shift >= 1.0 else (ev[-1] / ev[0]) * 2.2e-16 * np.abs(r.x).max() * \
        np.abs(2 * (r.x - p.xstar[0])).sum() / h
    tol = 1e-5 * np.maximum(np.abs(g_fd), 1e-3 * np.abs(g_fd).max()) + floor
    assert np.all(np.abs(vbar[edges] - g_fd) <= tol)
    fd_s = fd_diff(p, fd_loss(p, w0, s0 + h, b0), fd_loss(p, w0, s0 - h, b0)) / (2 * h)
    assert abs(sbar - fd_s) <= 1e-5 * abs(fd_s) + floor
    for i in rng.choice(p.n, 8, replace=False):
        bp, bm = b0.copy(), b0.copy()
        bp[i] += h
        bm[i] -= h
        fd_b = fd_diff(p, fd_loss(p, w0, s0, bp), fd_loss(p, w0, s0, bm)) / (2 * h)
        assert abs(bbar[i] - fd_b) <= 1e-5 * max(abs(fd_b), 1e-3 * np.abs(bbar).max()) + floor


def test_gradient_five_point_differences_ill_conditioned():
    """Shift 1e-2 (kappa ~ 1e3): the fourth-order central difference
    (8 (f(h) - f(-h)) - (f(2h) - f(-2h))) / (12 h) has a truncation error of
    order h^4 and a rounding floor of order kappa u / h.  At h = 1e-3 for the
    weights and right-hand side (entries of order 1) and h = 1e-3 * shift for
    the shift (which sets the smallest eigenvalue), both are far below the
    tolerances (2e-6 and 1e-8 relative).  So the adjoint's dloss/dw,
    dloss/dshift and dloss/db are pinned there without the floor that the
    two-point difference needs."""
    p = P.grid_problem(8, 8, cfg=4, shift=1e-2)
    _, vbar, sbar, bbar = loss_and_grad(p)
    rng = np.random.default_rng(5)
    h = 1e-3
    w0, s0, b0 = p.vals[0].astype(np.float64), float(p.shift[0]), p.b[0].copy()

    def five_point(solve_at, h=h):
        return (8.0 * fd_diff(p, solve_at(h), solve_at(-h)) - fd_diff(p, solve_at(2 * h), solve_at(-2 * h))) / (12 * h)

    def bump_w(e):
        def at(t):
            w = w0.copy()
            w[e] += t
            return fd_loss(p, w, s0, b0)
        return at

    def bump_b(i):
        def at(t):
            b = b0.copy()
            b[i] += t
            return fd_loss(p, w0, s0, b)
        return at

    scale_w = np.abs(vbar).max()
    for e in rng.choice(p.m, 24, replace=False):
        g = five_point(bump_w(e))
        assert abs(vbar[e] - g) <= 2e-6 * max(abs(g), 1e-3 * scale_w)
    g_s = five_point(lambda t: fd_loss(p, w0, s0 + t, b0), h=1e-3 * s0)
    assert abs(sbar - g_s) <= 1e-8 * abs(g_s)
    scale_b = np.abs(bbar).max()
    for i in rng.choice(p.n, 8, replace=False):
        g = five_point(bump_b(i))
        assert abs(bbar[i] - g) <= 2e-6 * max(abs(g), 1e-3 * scale_b)


def test_gradient_elasticity_central_differences():
    p = P.elasticity_problem(2, cfg=2)
    rng = np.random.default_rng(9)
    p["xstar"] = rng.standard_normal((1, p.n)) * 1e-4
    r = O.refactor_solve(p)
    xbar = 2.0 * (r.x - p.xstar[0])
    Ebar, _, _ = O.backward(p, r, xbar)
    E0 = p.vals[0].copy()
    for e in rng.choice(p.m, 6, replace=False):
        h = 1e-6 * E0[e]
        Ep, Em = E0.copy(), E0.copy()
        Ep[e] += h
        Em[e] -= h
        fd = fd_diff(p, fd_loss(p, Ep, 0.0, p.b[0]), fd_loss(p, Em, 0.0, p.b[0])) / (2 * h)
        assert abs(Ebar[e] - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(Ebar).max())


def test_gradient_scalar_closed_form():
    """n = 1: K = w + s, x = b/(w+s), loss (x - x*)^2:
    dl/dw = -2 (x - x*) b / (w+s)^2, dl/db = 2 (x - x*)/(w+s)."""
    w, s, b, xs = 1.7, 0.3, -0.8, 0.25
    p = P.Problem(kind=0, n=1, m=1, rowptr=np.array([0, 1], np.int64), colind=np.array([0], np.int32),
                  aval=np.array([1.0]), perm=np.array([0], np.int32), vals=np.array([[w]]),
                  shift=np.array([s]), b=np.array([[b]]), xstar=np.array([[xs]]), batch=1)
    _, vbar, sbar, bbar = loss_and_grad(p)
    x = b / (w + s)
    assert abs(vbar[0] - (-2 * (x - xs) * b / (w + s) ** 2)) < 1e-15
    assert abs(sbar - (-2 * (x - xs) * b / (w + s) ** 2)) < 1e-15
    assert abs(bbar[0] - 2 * (x - xs) / (w + s)) < 1e-15


def test_adjoint_symmetry():
    """<K^-1 u, v> = <u, K^-1 v> for the oracle's solve."""
    p = P.trigrid_problem(12, cfg=3)
    r = O.refactor_solve(p)
    rng = np.random.default_rng(4)
    u, v = rng.standard_normal(p.n), rng.standard_normal(p.n)
    a = np.dot(r.S.solve(r.L, p.perm, u), v)
    b = np.dot(u, r.S.solve(r.L, p.perm, v))
    assert abs(a - b) <= 1e-12 * max(abs(a), 1.0)


# ---------------------------------------------------------------------------
# Cotangent weights (value construction upstream of assembly, Sec. 5.3):
# pinned by closed-form triangles, similarity invariance and the linear
# precision of the cotangent Laplacian on planar meshes.
def _edges_of(faces):
    return P.faces_to_edges(np.asarray(faces, np.int64))


def test_cotan_right_isoceles_and_equilateral():
    # corner at the right angle: cot 90 = 0; the 45-degree corners: cot = 1
    w = O.cotan_weights([[0, 1, 2]], [[0, 1, 2]], [[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]], 3)
    assert np.array_equal(w, [0.0, 0.5, 0.5])
    h = np.sqrt(3.0) / 2
    w = O.cotan_weights([[0, 1, 2]], [[0, 1, 2]], [[0.0, 0.0], [1.0, 0.0], [0.5, h]], 3)
    assert np.allclose(w, 0.5 / np.sqrt(3.0), rtol=0, atol=1e-15)


def test_cotan_two_right_triangles_share_a_diagonal():
    faces = [[0, 1, 2], [0, 2, 3]]  # unit square split along (0,0)-(1,1)
    edges, opp = _edges_of(faces)
    xy = [[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]]
    w = O.cotan_weights(faces, opp, xy, edges.shape[0])
    diag = [e for e, (a, b) in enumerate(edges) if {int(a), int(b)} == {0, 2}][0]
    assert w[diag] == 0.0  # both opposite corners are right angles
    assert np.allclose(np.delete(w, diag), 0.5, rtol=0, atol=1e-15)


def test_cotan_similarity_invariance_and_linear_precision():
    s = 9
    faces = P.trigrid_faces(s, s)
    edges, opp = P.faces_to_edges(faces)
    rng = np.random.default_rng(7)
    base = np.stack(np.meshgrid(np.arange(s), np.arange(s), indexing="ij"), -1).reshape(-1, 2) / (s - 1.0)
    xy = base + rng.uniform(-0.3, 0.3, base.shape) / (s - 1.0)
    w = O.cotan_weights(faces, opp, xy, edges.shape[0])
    th, sc, tr = 0.7, 3.5, np.array([2.0, -1.0])
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    w2 = O.cotan_weights(faces, opp, sc * xy @ R.T + tr, edges.shape[0])
    assert np.allclose(w2, w, rtol=1e-12, atol=1e-12)
    # sum_j w_ij (p_j - p_i) = 0 at every interior vertex of a planar mesh
    acc = np.zeros_like(xy)
    for e, (a, b) in enumerate(edges):
        acc[a] += w[e] * (xy[b] - xy[a])
        acc[b] += w[e] * (xy[a] - xy[b])
    ij = np.stack(np.meshgrid(np.arange(s), np.arange(s), indexing="ij"), -1).reshape(-1, 2)
    interior = (ij.min(1) > 0) & (ij.max(1) < s - 1)
    assert np.abs(acc[interior]).max() <= 1e-12


def test_trigrid_problem_values_are_the_oracle_cotan_weights():
    p = P.trigrid_problem(12, batch=2, cfg=3)
    for i in range(2):
        w = O.cotan_weights(p.faces, p.opp, p.positions[i], p.m)
        assert np.array_equal(w, p.vals[i])


# element blocks from geometry (linear tetrahedra)
# ----------------------------------------------------------------------------
def _random_tets(rng, count):
    """Well-shaped random tets: a regular-ish reference tet, randomly
    stretched, rotated and moved; positive orientation not assumed."""
    ref = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    out = []
    for _ in range(count):
        A = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
        out.append(ref @ A.T + rng.standard_normal(3))
    return np.array(out)


def _oracle_block(X, E, nu):
    Kp, bad = O.tet_stiffness(np.arange(4, dtype=np.int32)[None], X, np.array([E]), nu)
    assert bad == 0
    K = np.zeros((12, 12))
    ii, jj = np.tril_indices(12)
    K[ii, jj] = Kp[0]
    K[jj, ii] = Kp[0]
    return K


def test_tet_block_matches_lame_index_formula():
    """The continuum derivation (energy mu eps:eps + lambda/2 (tr eps)^2,
    differentiated twice in the nodal displacements) gives
    K[3a+i][3b+j] = V (lambda g_a[i] g_b[j] + mu g_a[j] g_b[i] + mu d_ij g_a.g_b)
    with g_a the barycentric gradients from the inverse edge matrix.  The
    oracle builds K as V B^T D B instead; a transposed shear entry, a missing
    factor 2 or a wrong Voigt order fails here."""
    rng = np.random.default_rng(41)
    for X in _random_tets(rng, 12):
        E, nu = 10 ** rng.uniform(0, 3), rng.uniform(-0.5, 0.45)
        lam, mu = E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))
        J = (X[1:] - X[0]).T
        Gi = np.linalg.inv(J)                       # rows: grad of barycentric 1..3
        g = np.vstack([-Gi.sum(0), Gi])
        V = abs(np.linalg.det(J)) / 6
        Kl = np.zeros((12, 12))
        for a in range(4):
            for b in range(4):
                for i in range(3):
                    for j in range(3):
                        Kl[3 * a + i, 3 * b + j] = V * (lam * g[a, i] * g[b, j] + mu * g[a, j] * g[b, i]
                                                        + (mu * g[a] @ g[b] if i == j else 0.0))
        K = _oracle_block(X, E, nu)
        assert np.abs(K - Kl).max() <= 1e-12 * np.abs(Kl).max()


def test_tet_block_constant_strain_energy_and_rigid_modes():
    """An affine displacement u(x) = G x has the constant strain
    eps = (G + G^T)/2, so 1/2 u^T K u = V (mu eps:eps + lambda/2 (tr eps)^2)
    exactly; a rigid motion (G antisymmetric, or a translation) has none."""
    rng = np.random.default_rng(42)
    for X in _random_tets(rng, 8):
        E, nu = 2.5, 0.3
        lam, mu = E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))
        K = _oracle_block(X, E, nu)
        V = abs(np.linalg.det((X[1:] - X[0]).T)) / 6
        G = rng.standard_normal((3, 3))
        u = (X @ G.T).ravel()
        eps = 0.5 * (G + G.T)
        W = V * (mu * np.sum(eps * eps) + 0.5 * lam * np.trace(eps) ** 2)
        assert abs(0.5 * u @ K @ u - W) <= 1e-12 * W
        W_ = 0.5 * (G - G.T)
        for r in [(X @ W_.T).ravel(), np.tile(rng.standard_normal(3), 4)]:
            assert np.abs(K @ r).max() <= 1e-12 * np.abs(K).max() * np.abs(r).max()
        ev = np.linalg.eigvalsh(K)
        assert ev.min() > -1e-12 * ev.max() and np.sum(ev > 1e-9 * ev.max()) == 6


def test_tet_block_scaling_and_rotation_laws():
    """K(alpha X) = alpha K(X) (3D: volume ~ alpha^3, gradients ~ 1/alpha);
    K(X R^T) = Q K(X) Q^T with Q = diag(R, R, R, R) for a rotation R;
    K is linear in E; vertex order does not change the block up to the
    matching DOF permutation."""
    rng = np.random.default_rng(43)
    X = _random_tets(rng, 1)[0]
    K = _oracle_block(X, 1.0, 0.25)
    assert np.abs(_oracle_block(3.0 * X, 1.0, 0.25) - 3.0 * K).max() <= 1e-12 * np.abs(K).max()
    assert np.abs(_oracle_block(X, 7.0, 0.25) - 7.0 * K).max() <= 1e-12 * 7 * np.abs(K).max()
    R, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    Q = np.kron(np.eye(4), R)
    assert np.abs(_oracle_block(X @ R.T, 1.0, 0.25) - Q @ K @ Q.T).max() <= 1e-12 * np.abs(K).max()
    order = [2, 0, 3, 1]
    idx = np.array([3 * a + c for a in order for c in range(3)])
    assert np.abs(_oracle_block(X[order], 1.0, 0.25) - K[np.ix_(idx, idx)]).max() <= 1e-12 * np.abs(K).max()


def test_tet_block_degenerate_and_generator_consistency():
    """A flat tet is reported and gives a zero block; on the pattern geometry
    of the elasticity workloads the oracle reproduces the generator's K_e^0."""
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], float)
    Kp, bad = O.tet_stiffness(np.arange(4, dtype=np.int32)[None], X, None, 0.3)
    assert bad == 1 and np.all(Kp == 0)
    p = P.elasticity_problem(2, cfg=2)
    Kp, bad = O.tet_stiffness(p.tets, p.pos, None, 0.3)
    assert bad == 0
    np.testing.assert_allclose(Kp, p.elem_K0, rtol=0, atol=1e-12 * np.abs(p.elem_K0).max())


def test_element_blocks_pattern_assembles_as_the_element_sum():
    """A per-call element-block pattern whose blocks are E_e K_e^0 assembles
    to the same K as the modulus pattern of the same mesh."""
    p = P.elasticity_problem(2, batch=1, cfg=2)
    q = P.Problem(p)
    q.update(kind=P.KIND_ELEM_BLOCKS, elem_K0=None, vals=(p.vals[0][:, None] * p.elem_K0).reshape(1, -1))
    Kp, Kq = O.assemble(p).dense(), O.assemble(q).dense()
    assert np.abs(Kp - Kq).max() <= 1e-13 * np.abs(Kp).max()


def test_gradient_element_blocks_central_differences():
    """d loss / d (block entry) of a per-call element-block pattern against
    central differences of the oracle's solve: an off-diagonal entry moves
    K_uv and K_vu together, a diagonal entry K_uu alone."""
    g = P.elasticity_geometry_problem(2, batch=1, cfg=6)
    Kb = np.concatenate([O.tet_stiffness(g.tets, g.pos[0], g.E[0], g.nu)[0].ravel()])
    g["vals"] = Kb[None]
    rng = np.random.default_rng(11)
    g["xstar"] = rng.standard_normal((1, g.n)) * 1e-4
    r = O.refactor_solve(g)
    vbar, _, _ = O.backward(g, r, 2.0 * (r.x - g.xstar[0]))
    free = np.nonzero(np.all(g.elem_dofs >= 0, axis=1))[0]
    picks = [(e, q) for e in rng.choice(free, 3, replace=False) for q in (0, 4, 40, 77)]
    fixed_e = int(np.nonzero(np.any(g.elem_dofs < 0, axis=1))[0][0])
    for e, q in picks:
        h = 1e-6 * np.abs(Kb[e * 78: (e + 1) * 78]).max()
        vp, vm = Kb.copy(), Kb.copy()
        vp[e * 78 + q] += h
        vm[e * 78 + q] -= h
        fd = fd_diff(g, fd_loss(g, vp, 0.0, g.b[0]), fd_loss(g, vm, 0.0, g.b[0])) / (2 * h)
        assert abs(vbar[e * 78 + q] - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(vbar).max())
    dofs = g.elem_dofs[fixed_e]
    ii, jj = np.tril_indices(12)
    on_fixed = (dofs[ii] < 0) | (dofs[jj] < 0)
    assert np.all(vbar[fixed_e * 78: (fixed_e + 1) * 78][on_fixed] == 0)


# sparse matrix expressions
# ----------------------------------------------------------------------------
def _rand_csr(rng, rows, cols, per_row):
    rp, ci = [0], []
    for _ in range(rows):
        c = np.sort(rng.choice(cols, min(per_row, cols), replace=False))
        ci.extend(c.tolist())
        rp.append(len(ci))
    return np.array(rp, np.int64), np.array(ci, np.int32)


def _dense_eval(nodes, vals, outputs):
    """The same expressions with dense numpy matrices (values) and boolean
    matrices (structure) -- a different route to the same definitions."""
    D, Pm, off = [], [], 0
    for nd in nodes:
        if nd[0] == "leaf":
            _, r, c, rp, ci = nd
            M, Pb = np.zeros((r, c)), np.zeros((r, c), bool)
            for i in range(r):
                M[i, ci[rp[i]:rp[i + 1]]] = vals[off + rp[i]: off + rp[i + 1]]
                Pb[i, ci[rp[i]:rp[i + 1]]] = True
            off += rp[r]
            D.append(M), Pm.append(Pb)
        elif nd[0] == "add":
            D.append(D[nd[1]] + D[nd[2]]), Pm.append(Pm[nd[1]] | Pm[nd[2]])
        elif nd[0] == "scale":
            D.append(nd[2] * D[nd[1]]), Pm.append(Pm[nd[1]].copy())
        elif nd[0] == "transpose":
            D.append(D[nd[1]].T), Pm.append(Pm[nd[1]].T)
        else:
            D.append(D[nd[1]] @ D[nd[2]]), Pm.append((Pm[nd[1]].astype(int) @ Pm[nd[2]].astype(int)) > 0)
    return [(D[o], Pm[o]) for o in outputs]


def paper_expressions(n, rng, per_row=6):
    """(alpha A + B)^T (beta B^T + C), A B C and (A + B)(A B + C) on random
    n x n matrices with `per_row` entries per row (Sec. 5 sparse expressions)."""
    leaves = [("leaf", n, n, *_rand_csr(rng, n, n, per_row)) for _ in range(3)]
    nodes = list(leaves)  # 0 A, 1 B, 2 C

    def add(nd):
        nodes.append(nd)
        return len(nodes) - 1
    e1 = add(("mul", add(("transpose", add(("add", add(("scale", 0, 0.7)), 1)))),
              add(("add", add(("scale", add(("transpose", 1)), -1.3)), 2))))
    ab = add(("mul", 0, 1))
    e2 = add(("mul", ab, 2))
    e3 = add(("mul", add(("add", 0, 1)), add(("add", ab, 2))))
    nv = sum(int(l[3][-1]) for l in leaves)
    return nodes, [e1, e2, e3], nv


def test_expr_oracle_matches_dense_evaluation():
    rng = np.random.default_rng(51)
    nodes, outs, nv = paper_expressions(40, rng, per_row=4)
    vals = rng.standard_normal(nv)
    got = O.expr_eval(nodes, vals, outs)
    for (r, c, d), (M, Pb) in zip(got, _dense_eval(nodes, vals, outs)):
        assert set(d) == set(zip(*np.nonzero(Pb)))       # structural pattern
        G = np.zeros((r, c))
        for (i, j), v in d.items():
            G[i, j] = v
        assert np.abs(G - M).max() <= 1e-12 * np.abs(M).max()


def test_expr_oracle_tridiagonal_cube_closed_form():
    """T = tridiag(-1, 2, -1): T^3 has interior rows (-1, 6, -15, 20, -15, 6, -1)
    (the sixth finite difference, -(1 - x)^6 up to the shift)."""
    n = 12
    rp, ci, v = [0], [], []
    for i in range(n):
        for j, a in ((i - 1, -1.0), (i, 2.0), (i + 1, -1.0)):
            if 0 <= j < n:
                ci.append(j), v.append(a)
        rp.append(len(ci))
    nodes = [("leaf", n, n, np.array(rp), np.array(ci)), ("mul", 0, 0), ("mul", 1, 0)]
    (_, _, d), = O.expr_eval(nodes, np.array(v), [2])
    for i in range(3, n - 3):
        row = [d[(i, j)] for j in range(i - 3, i + 4)]
        assert row == [-1.0, 6.0, -15.0, 20.0, -15.0, 6.0, -1.0]
        assert all((i, j) not in d for j in range(n) if abs(i - j) > 3)


def test_expr_oracle_weighted_laplacian_of_a_path():
    """A^T (W A) for the incidence matrix A of a path and W = diag(w) is the
    weighted path Laplacian: L_ii = w_(i-1) + w_i, L_(i,i+1) = -w_i."""
    n, m = 6, 5
    w = np.array([0.5, 2.0, 1.5, 3.0, 0.25])
    A = ("leaf", m, n, np.arange(0, 2 * m + 1, 2), np.array([[e, e + 1] for e in range(m)]).ravel())
    W = ("leaf", m, m, np.arange(m + 1), np.arange(m))
    nodes = [A, W, ("transpose", 0), ("mul", 1, 0), ("mul", 2, 3)]
    vals = np.concatenate([np.tile([1.0, -1.0], m), w])
    (_, _, d), = O.expr_eval(nodes, vals, [4])
    for i in range(n):
        assert d[(i, i)] == (w[i - 1] if i > 0 else 0.0) + (w[i] if i < m else 0.0)
        if i < m:
            assert d[(i, i + 1)] == -w[i] and d[(i + 1, i)] == -w[i]


def test_expr_row_oracle_equals_full_oracle():
    """The lazy row evaluator gives the full evaluator's rows exactly (same
    definitions; transposes of leaves and of intermediates both covered)."""
    rng = np.random.default_rng(52)
    nodes, outs, nv = paper_expressions(30, rng, per_row=3)
    vals = rng.standard_normal(nv)
    for o in outs:
        (_, _, d), = O.expr_eval(nodes, vals, [o])
        rows = O.expr_eval_rows(nodes, vals, o, range(30))
        assert {(i, j): v for i, r in rows.items() for j, v in r.items()} == d


def test_expr_oracle_shared_values_equal_expanded_values():
    """A leaf whose entries share values (vmap) evaluates exactly like the
    same leaf given one value per entry, vals[vmap]; the lazy row evaluator
    agrees with the full one on shared leaves too."""
    rng = np.random.default_rng(53)
    n = 25
    rp, ci = _rand_csr(rng, n, n, 3)
    nnz = int(rp[-1])
    vm = rng.integers(0, 11, nnz)
    vals = rng.standard_normal(11)
    shared = [("leaf", n, n, rp, ci, vm, 11), ("transpose", 0), ("mul", 0, 1), ("add", 2, 0)]
    plain = [("leaf", n, n, rp, ci), ("transpose", 0), ("mul", 0, 1), ("add", 2, 0)]
    for o in (2, 3):
        (_, _, ds), = O.expr_eval(shared, vals, [o])
        (_, _, dp), = O.expr_eval(plain, vals[vm], [o])
        assert ds == dp
        rows = O.expr_eval_rows(shared, vals, o, range(n))
        assert {(i, j): v for i, r in rows.items() for j, v in r.items()} == ds
