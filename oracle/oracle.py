"""Python face of the FP64 oracle (``ssco_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The library path never imports it.
It shares nothing with the CUDA path except the seeded input generators.

Each wrapper names the definition it follows; the arithmetic itself is in the
C file (plain loops, FP64, ``-O2 -ffp-contract=off``), except the
sparse-expression evaluators at the end, which are plain Python dictionaries
of entries (FP64) written from the definitions of sum, scaling, transpose and
product.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ssco_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
# A test may point the wrapper at another build of this source, one with a
# planted mistake, to show that the pins fail on it (tests/test_oracle_mutants.py).
_BUILT_LIB = os.path.join(BUILD_DIR, "libssco_oracle.so")
_LIB_OVERRIDE = os.environ.get("SSCO_ORACLE_LIB")
LIB = _LIB_OVERRIDE or _BUILT_LIB

_lib = None
KIND_ELEM_BLOCKS = 2   # K = sum_e K_e, the element blocks are the per-set values

i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no fast-math, no FMA contraction)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_BUILT_LIB) or os.path.getmtime(_BUILT_LIB) < os.path.getmtime(SRC):
        tmp = _BUILT_LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-std=c11", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, _BUILT_LIB)
    return _BUILT_LIB


def lib():
    global _lib
    if _lib is None:
        if not _LIB_OVERRIDE:
            build()
        L = C.CDLL(LIB)
        L.or_atwa_cap.restype = C.c_int64
        L.or_atwa_cap.argtypes = [C.c_int32, C.c_int32, i64p]
        L.or_assemble_atwa.restype = C.c_int64
        L.or_assemble_atwa.argtypes = [C.c_int32, C.c_int32, i64p, i32p, f64p, f64p, C.c_double,
                                       i64p, i32p, f64p]
        L.or_elem_cap.restype = C.c_int64
        L.or_elem_cap.argtypes = [C.c_int32, C.c_int32, C.c_int32]
        L.or_assemble_elem.restype = C.c_int64
        L.or_assemble_elem.argtypes = [C.c_int32, C.c_int32, C.c_int32, i32p, f64p, f64p, C.c_double,
                                       i64p, i32p, f64p]
        L.or_permute.restype = None
        L.or_permute.argtypes = [C.c_int32, i64p, i32p, f64p, i32p, i64p, i32p, f64p]
        L.or_symbolic.restype = C.c_void_p
        L.or_symbolic.argtypes = [C.c_int32, i64p, i32p]
        L.or_symb_nnzL.restype = C.c_int64
        L.or_symb_nnzL.argtypes = [C.c_void_p]
        L.or_symb_nsnodes.restype = C.c_int32
        L.or_symb_nsnodes.argtypes = [C.c_void_p]
        L.or_symb_get.restype = None
        L.or_symb_get.argtypes = [C.c_void_p, i32p, i32p, i64p, i32p, i32p, i32p, i32p, i32p]
        L.or_symb_free.restype = None
        L.or_symb_free.argtypes = [C.c_void_p]
        L.or_numeric.restype = C.c_int32
        L.or_numeric.argtypes = [C.c_void_p, f64p, f64p]
        L.or_solve.restype = None
        L.or_solve.argtypes = [C.c_void_p, f64p, i32p, f64p, f64p]
        L.or_symv.restype = None
        L.or_symv.argtypes = [C.c_int32, i64p, i32p, f64p, f64p, f64p]
        L.or_grad_atwa.restype = None
        L.or_grad_atwa.argtypes = [C.c_int32, i64p, i32p, f64p, f64p, f64p, f64p]
        L.or_grad_elem.restype = None
        L.or_grad_elem.argtypes = [C.c_int32, C.c_int32, i32p, f64p, f64p, f64p, f64p]
        L.or_cotan_weights.restype = None
        L.or_cotan_weights.argtypes = [C.c_int64, i32p, i32p, f64p, C.c_int64, f64p]
        L.or_grad_blocks.restype = None
        L.or_grad_blocks.argtypes = [C.c_int32, C.c_int32, i32p, f64p, f64p, f64p]
        L.or_tet_stiffness.restype = C.c_int32
        L.or_tet_stiffness.argtypes = [C.c_int64, i32p, f64p, C.c_void_p, C.c_double, f64p]
        _lib = L
    return _lib


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class CSC:
    """Lower triangle of a symmetric matrix, compressed by columns."""

    def __init__(self, n, colptr, rowind, val):
        self.n, self.colptr, self.rowind, self.val = n, colptr, rowind, val

    @property
    def nnz(self):
        return int(self.colptr[-1])

    def dense(self):
        A = np.zeros((self.n, self.n))
        for j in range(self.n):
            s, e = self.colptr[j], self.colptr[j + 1]
            A[self.rowind[s:e], j] = self.val[s:e]
        return A + np.tril(A, -1).T


def assemble(p, inst: int = 0, vals=None, shift=None) -> CSC:
    """K in the original ordering: A^T diag(w) A + shift I, or sum_e E_e K_e^0."""
    L = lib()
    v = _c(p.vals[inst] if vals is None else vals, np.float64)
    s = float(p.shift[inst] if shift is None else shift)
    n, m = p.n, p.m
    colptr = np.zeros(n + 1, np.int64)
    if p.kind == 0:
        rowptr, colind, aval = _c(p.rowptr, np.int64), _c(p.colind, np.int32), _c(p.aval, np.float64)
        cap = L.or_atwa_cap(n, m, rowptr)
        rowind = np.zeros(max(cap, 1), np.int32)
        val = np.zeros(max(cap, 1))
        nz = L.or_assemble_atwa(n, m, rowptr, colind, aval, v, s, colptr, rowind, val)
    else:
        dofs = _c(p.elem_dofs, np.int32)
        if p.kind == KIND_ELEM_BLOCKS:
            # K = sum_e K_e with the blocks given per value set: the element
            # sum with unit moduli over those blocks
            K0 = _c(v, np.float64)
            v = np.ones(m)
        else:
            K0 = _c(p.elem_K0, np.float64)
        cap = L.or_elem_cap(n, m, p.elem_dim)
        rowind = np.zeros(max(cap, 1), np.int32)
        val = np.zeros(max(cap, 1))
        nz = L.or_assemble_elem(n, m, p.elem_dim, dofs, K0, v, s, colptr, rowind, val)
    return CSC(n, colptr, rowind[:nz].copy(), val[:nz].copy())


def permute(K: CSC, perm) -> CSC:
    """K~ = P K P^T, perm[new] = old."""
    L = lib()
    pc = np.zeros(K.n + 1, np.int64)
    pr = np.zeros(max(K.nnz, 1), np.int32)
    pv = np.zeros(max(K.nnz, 1))
    L.or_permute(K.n, K.colptr, _c(K.rowind, np.int32), _c(K.val, np.float64), _c(perm, np.int32),
                 pc, pr, pv)
    return CSC(K.n, pc, pr[:K.nnz], pv[:K.nnz])


class Symbolic:
    """Column-merge symbolic factorization of a permuted lower pattern."""

    def __init__(self, Kp: CSC):
        L = lib()
        self.n = Kp.n
        self._h = L.or_symbolic(Kp.n, Kp.colptr, _c(Kp.rowind, np.int32))
        n = self.n
        nzL = L.or_symb_nnzL(self._h)
        ns = L.or_symb_nsnodes(self._h)
        self.parent = np.zeros(n, np.int32)
        self.colcount = np.zeros(n, np.int32)
        self.Lcolptr = np.zeros(n + 1, np.int64)
        self.Lrowind = np.zeros(max(nzL, 1), np.int32)
        self.col_level = np.zeros(n, np.int32)
        self.snode_first = np.zeros(ns + 1, np.int32)
        self.sn_parent = np.zeros(max(ns, 1), np.int32)
        self.sn_level = np.zeros(max(ns, 1), np.int32)
        L.or_symb_get(self._h, self.parent, self.colcount, self.Lcolptr, self.Lrowind,
                      self.col_level, self.snode_first, self.sn_parent, self.sn_level)
        self.Lrowind = self.Lrowind[:nzL]
        self.sn_parent = self.sn_parent[:ns]
        self.sn_level = self.sn_level[:ns]
        self.nnzL = int(nzL)
        self.n_snodes = int(ns)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.or_symb_free(self._h)
            self._h = None

    def numeric(self, Kp: CSC):
        """Left-looking Cholesky values of L (CSC order of Lcolptr/Lrowind).
        Returns (Lval, bad) with bad = -1 or the first non-positive pivot."""
        Lval = np.zeros(max(self.nnzL, 1))
        bad = lib().or_numeric(self._h, _c(Kp.val, np.float64), Lval)
        return Lval[: self.nnzL], int(bad)

    def solve(self, Lval, perm, b):
        x = np.zeros(self.n)
        lib().or_solve(self._h, _c(Lval, np.float64), _c(perm, np.int32), _c(b, np.float64), x)
        return x

    def L_dense(self, Lval):
        A = np.zeros((self.n, self.n))
        for j in range(self.n):
            s, e = self.Lcolptr[j], self.Lcolptr[j + 1]
            A[self.Lrowind[s:e], j] = Lval[s:e]
        return A


def symv(K: CSC, x):
    y = np.zeros(K.n)
    lib().or_symv(K.n, K.colptr, _c(K.rowind, np.int32), _c(K.val, np.float64), _c(x, np.float64), y)
    return y


def grad_vals(p, mu, x):
    """d loss / d vals given the adjoint mu = K^-1 xbar (original ordering)."""
    if p.kind == KIND_ELEM_BLOCKS:
        d = p.elem_dim
        out = np.zeros(p.m * d * (d + 1) // 2)
        lib().or_grad_blocks(p.m, d, _c(p.elem_dofs, np.int32), _c(mu, np.float64), _c(x, np.float64), out)
        return out
    out = np.zeros(p.m)
    if p.kind == 0:
        lib().or_grad_atwa(p.m, _c(p.rowptr, np.int64), _c(p.colind, np.int32),
                           _c(p.aval, np.float64), _c(mu, np.float64), _c(x, np.float64), out)
    else:
        lib().or_grad_elem(p.m, p.elem_dim, _c(p.elem_dofs, np.int32), _c(p.elem_K0, np.float64),
                           _c(mu, np.float64), _c(x, np.float64), out)
    return out


def shifted_mask(p):
    """Diagonals that receive the shift (all for A^T W A; referenced DOFs for
    element sums)."""
    if p.kind == 0:
        return np.ones(p.n, bool)
    m = np.zeros(p.n, bool)
    d = p.elem_dofs[p.elem_dofs >= 0]
    m[d] = True
    return m


class Result(dict):
    __getattr__ = dict.__getitem__


def refactor_solve(p, inst: int = 0, vals=None, shift=None, b=None, symb: Symbolic | None = None):
    """The full FP64 pipeline for one value set: assemble, permute, symbolic
    (or a given one), numeric, solve.  Returns K, K~, symbolic, L values, x."""
    K = assemble(p, inst, vals, shift)
    Kp = permute(K, p.perm)
    S = symb if symb is not None else Symbolic(Kp)
    Lval, bad = S.numeric(Kp)
    bb = p.b[inst] if b is None else b
    x = S.solve(Lval, p.perm, bb) if bad < 0 else np.full(p.n, np.nan)
    return Result(K=K, Kp=Kp, S=S, L=Lval, bad=bad, x=x, b=np.asarray(bb, np.float64))


def backward(p, r: Result, xbar, inst: int = 0):
    """Adjoint of x = K^-1 b: mu = K^-1 xbar, then (vals_bar, shift_bar, b_bar)."""
    mu = r.S.solve(r.L, p.perm, xbar)
    vbar = grad_vals(p, mu, r.x)
    sbar = -float(np.dot(mu[shifted_mask(p)], r.x[shifted_mask(p)]))
    return vbar, sbar, mu


def cotan_weights(tri, tri_edge, xy, n_edge: int):
    """Cotangent edge weights of one value set (Sec. 5.3 mesh experiments):
    w_e = 1/2 sum over the triangles holding e of cot(angle opposite e),
    cot = (u . v)/|u x v|; tri / tri_edge [n_tri][3], xy [n_vert][2]."""
    tri = _c(tri, np.int32)
    te = _c(tri_edge, np.int32)
    w = np.empty(int(n_edge))
    lib().or_cotan_weights(tri.shape[0], tri, te, _c(xy, np.float64), int(n_edge), w)
    return w


def tet_stiffness(tets, xyz, E, nu: float):
    """Linear-tet stiffness blocks of one value set, V B^T D B (isotropic,
    Voigt order, engineering shear), packed lower triangles [n_tet][78];
    tets [n_tet][4], xyz [n_node][3], E [n_tet] or None (unit modulus).
    Returns (blocks, number of singular tets)."""
    tets = _c(tets, np.int32)
    xyz = _c(xyz, np.float64)
    out = np.empty((tets.shape[0], 78))
    Ec = None if E is None else _c(E, np.float64)
    bad = lib().or_tet_stiffness(tets.shape[0], tets, xyz, None if Ec is None else Ec.ctypes.data, float(nu), out)
    return out, int(bad)


# ---------------------------------------------------------------------------
# fixed-pattern sparse matrix expressions (Sec. 5 sparse-expression and
# structured-product experiments), by definition, in FP64
# ---------------------------------------------------------------------------
def expr_eval(nodes, leaf_vals, outputs, absolute: bool = False):
    """Evaluate a DAG of sparse matrices for one value set.

    nodes: ("leaf", rows, cols, rowptr, colind[, vmap, n_vals]) | ("add", a, b) |
    ("scale", a, alpha) | ("mul", a, b) | ("transpose", a), operands by
    earlier index.  leaf_vals: the leaves' values concatenated in node
    order (with vmap, entry q of a leaf is its value vmap[q] and the leaf
    holds n_vals values).  Entries are dictionaries {(i, j): value} holding every
    structurally present entry (a sum or product that happens to be zero
    included): A + B has the union of both patterns, A B every (i, j) with
    some k where A_ik and B_kj are present, summing A_ik B_kj over those k.
    With `absolute` every leaf value and every alpha enters by its absolute
    value (the scale of the rounding error of any evaluation order).
    Returns [(rows, cols, dict)] for the requested outputs."""
    mats, off = [], 0
    for nd in nodes:
        kind = nd[0]
        if kind == "leaf":
            r, c, rp, ci = nd[1:5]
            vm = nd[5] if len(nd) > 5 else None
            d = {}
            for i in range(r):
                for q in range(int(rp[i]), int(rp[i + 1])):
                    v = float(leaf_vals[off + (int(vm[q]) if vm is not None else q)])
                    d[(i, int(ci[q]))] = abs(v) if absolute else v
            off += int(nd[6]) if vm is not None else int(rp[r])
            mats.append((r, c, d))
        elif kind == "add":
            ra, ca, A = mats[nd[1]]
            B = mats[nd[2]][2]
            d = dict(A)
            for key, v in B.items():
                d[key] = d.get(key, 0.0) + v
            mats.append((ra, ca, d))
        elif kind == "scale":
            ra, ca, A = mats[nd[1]]
            al = abs(nd[2]) if absolute else nd[2]
            mats.append((ra, ca, {key: al * v for key, v in A.items()}))
        elif kind == "transpose":
            ra, ca, A = mats[nd[1]]
            mats.append((ca, ra, {(j, i): v for (i, j), v in A.items()}))
        elif kind == "mul":
            ra, _, A = mats[nd[1]]
            _, cb, B = mats[nd[2]]
            rows_b = {}
            for (k, j), v in B.items():
                rows_b.setdefault(k, []).append((j, v))
            d = {}
            for (i, k), a in A.items():
                for j, b in rows_b.get(k, ()):
                    d[(i, j)] = d.get((i, j), 0.0) + a * b
            mats.append((ra, cb, d))
        else:
            raise ValueError(kind)
    return [mats[o] for o in outputs]


def expr_eval_rows(nodes, leaf_vals, output, rows):
    """Selected rows of one node of the same DAG, by the same definitions as
    expr_eval, evaluated lazily: a row of a product needs one row of its left
    factor and the rows of its right factor that row touches; a row of a
    transposed leaf is a column of the leaf.  Returns {i: {j: value}}."""
    offs, off = [], 0
    for nd in nodes:
        offs.append(off)
        if nd[0] == "leaf":
            off += int(nd[6]) if len(nd) > 5 and nd[5] is not None else int(nd[3][nd[1]])
    cache, cols_of_leaf, full = {}, {}, {}

    def leaf_value(nid, q):
        nd = nodes[nid]
        vm = nd[5] if len(nd) > 5 else None
        return float(leaf_vals[offs[nid] + (int(vm[q]) if vm is not None else q)])

    def leaf_row(nid, i):
        rp, ci = nodes[nid][3], nodes[nid][4]
        return {int(ci[q]): leaf_value(nid, q) for q in range(int(rp[i]), int(rp[i + 1]))}

    def column(nid, j):
        if nodes[nid][0] == "leaf":
            if nid not in cols_of_leaf:
                r, rp, ci = nodes[nid][1], nodes[nid][3], nodes[nid][4]
                cl = {}
                for i in range(r):
                    for q in range(int(rp[i]), int(rp[i + 1])):
                        cl.setdefault(int(ci[q]), {})[i] = leaf_value(nid, q)
                cols_of_leaf[nid] = cl
            return dict(cols_of_leaf[nid].get(j, {}))
        if nid not in full:
            (_, _, d), = expr_eval(nodes, leaf_vals, [nid])
            cl = {}
            for (i, jj), v in d.items():
                cl.setdefault(jj, {})[i] = v
            full[nid] = cl
        return dict(full[nid].get(j, {}))

    def row(nid, i):
        key = (nid, i)
        if key in cache:
            return cache[key]
        nd = nodes[nid]
        if nd[0] == "leaf":
            r = leaf_row(nid, i)
        elif nd[0] == "add":
            r = dict(row(nd[1], i))
            for j, v in row(nd[2], i).items():
                r[j] = r.get(j, 0.0) + v
        elif nd[0] == "scale":
            r = {j: nd[2] * v for j, v in row(nd[1], i).items()}
        elif nd[0] == "transpose":
            r = column(nd[1], i)
        else:
            r = {}
            for k, a in row(nd[1], i).items():
                for j, b in row(nd[2], k).items():
                    r[j] = r.get(j, 0.0) + a * b
        cache[key] = r
        return r

    return {int(i): row(output, int(i)) for i in rows}
