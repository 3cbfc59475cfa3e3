"""Thin Python binding of the C ABI in ``include/ssco.h`` (libssco.so).

Argument marshalling only: every step of the numeric path runs in the
library's CUDA kernels; PyTorch provides device memory and streams.  If the
shared library is missing this module raises at import -- there is no
fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libssco.so")

SSCO_OK, SSCO_ERR_INVALID_ARG = 0, 1
KIND_ATWA, KIND_ELEM, KIND_ELEM_BLOCKS = 0, 1, 2
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "PATTERN", 3: "NOT_SPD", 4: "NONFINITE",
                5: "NO_CONVERGE", 6: "TIMEOUT", 7: "CUDA", 8: "OOM", 9: "UNSUPPORTED", 10: "STATE"}
FP64, FP32_REFINE = 0, 1
VALS_F64, VALS_F32 = 0, 1
(EXPORT_PERM, EXPORT_ETREE, EXPORT_COLCOUNT, EXPORT_L_COLPTR, EXPORT_L_ROWIND, EXPORT_COL_LEVEL,
 EXPORT_SNODE_FIRST, EXPORT_SN_PARENT, EXPORT_SN_LEVEL, EXPORT_K_COLPTR, EXPORT_K_ROWIND,
 EXPORT_GROUPS, EXPORT_GROUP_COEF, EXPORT_FRONT_FIRST, EXPORT_FRONT_LEVEL) = range(15)

EXPORTED_SYMBOLS = [
    "ssco_analyze", "ssco_plan_info", "ssco_plan_export", "ssco_bind", "ssco_numeric", "ssco_solve",
    "ssco_backward", "ssco_status_get", "ssco_export_L", "ssco_export_K", "ssco_refactor_solve_host",
    "ssco_last_launch_count", "ssco_last_error", "ssco_status_string", "ssco_plan_save", "ssco_plan_load",
    "ssco_destroy", "ssco_profile_enable", "ssco_profile_read", "ssco_kernel_name", "ssco_solve_noalloc", "ssco_profile_trace", "ssco_graph_run", "ssco_autotune",
    "ssco_cotan_weights", "ssco_tet_stiffness",
    "ssco_expr_compile", "ssco_expr_compile_opts", "ssco_expr_get_info", "ssco_expr_export", "ssco_expr_output_shape",
    "ssco_expr_output_pattern", "ssco_expr_bind", "ssco_expr_run", "ssco_expr_last_error", "ssco_expr_destroy",
    "ssco_expr_save", "ssco_expr_load", "ssco_set_flow", "ssco_graph_run_many", "ssco_autotune_many",
]
KERNEL_KINDS = ["assemble", "front_small", "big_init", "big_kscatter", "big_update", "big_potrf", "big_syrk",
                "fwd_solve", "bwd_solve", "resid", "check", "vector", "grad", "front_tiny", "big_trsm", "front_vec",
                "big_update_tc"]


class SscoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Pattern(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n", C.c_int32), ("m", C.c_int32),
                ("rowptr", C.c_void_p), ("colind", C.c_void_p), ("aval", C.c_void_p),
                ("elem_dim", C.c_int32), ("elem_dofs", C.c_void_p), ("elem_K0", C.c_void_p),
                ("perm", C.c_void_p)]


class Op(C.Structure):
    _fields_ = [("precision", C.c_int32), ("batch", C.c_int32), ("refine_tol", C.c_double),
                ("refine_max_iter", C.c_int32), ("small_front_max", C.c_int32),
                ("amalgamate", C.c_int32), ("tiny_front_max", C.c_int32), ("tensor_cores", C.c_int32),
                ("big_panel", C.c_int32), ("split_rows", C.c_int32),
                ("warp_front_max", C.c_int32), ("cluster_rows", C.c_int32),
                ("refine_mode", C.c_int32), ("gmres_restart", C.c_int32), ("vec2_max_cls", C.c_int32)]


class KernelStat(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("launches", C.c_int64), ("ms", C.c_double),
                ("flops", C.c_double), ("bytes", C.c_double)]


class Info(C.Structure):
    _fields_ = [(k, C.c_int64) for k in
                ["n", "n_pats", "batch", "n_systems", "m", "nnz_K", "nnz_L", "n_snodes", "n_fronts",
                 "n_levels", "max_col_level", "panel_entries", "update_entries", "max_front_rows",
                 "n_assembly_groups", "assembly_terms", "tables_bytes", "workspace_bytes"]] + \
              [("factor_flops", C.c_double), ("factor_flops_exact", C.c_double)] + \
              [(k, C.c_int64) for k in ["tune_warp_items", "tune_vec_max_cls", "tune_solve_threads_big", "tuned",
                                        "tune_use_tc", "tune_big_panel", "tune_split_rows",
                                        "tune_warp_front_max", "tune_cluster_rows", "tune_flow",
                                        "flow_fact_fronts", "flow_solve_fronts", "tune_vec2_max_cls"]]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ExprNode(C.Structure):
    _fields_ = [("op", C.c_int32), ("a", C.c_int32), ("b", C.c_int32), ("alpha", C.c_double),
                ("rows", C.c_int32), ("cols", C.c_int32), ("rowptr", C.c_void_p), ("colind", C.c_void_p),
                ("vmap", C.c_void_p), ("n_vals", C.c_int64)]


class ExprOpts(C.Structure):
    _fields_ = [(k, C.c_int32) for k in ["batch", "precision", "inline_terms", "algebraic", "factor_min",
                                        "t_ref", "t_compl", "reserved"]]


class ExprInfo(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ["n_leaf_vals", "n_out_vals", "n_slots", "n_ops", "n_terms",
                                        "n_unrolled"]] + \
              [(k, C.c_int32) for k in ["n_levels", "batch", "precision", "unit_coef"]] + \
              [("table_bytes", C.c_uint64), ("workspace_bytes", C.c_uint64)] + \
              [(k, C.c_int64) for k in ["n_alg_merged", "n_alg_zero", "n_factored", "n_inlined"]]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libssco.so (built by ``paper_2110_12865_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libssco.so not built ({path}); run paper_2110_12865_gb300.build.build()")
    L = C.CDLL(path)
    vp, i32, i64, dbl, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_size_t
    sig = {
        "ssco_analyze": (i32, [C.POINTER(C.POINTER(Pattern)), i32, C.POINTER(Op), C.POINTER(vp)]),
        "ssco_plan_info": (i32, [vp, C.POINTER(Info)]),
        "ssco_plan_export": (i32, [vp, i32, vp, sz]),
        "ssco_bind": (i32, [vp, vp, sz, vp, sz, vp]),
        "ssco_numeric": (i32, [vp, vp, i32, vp, vp]),
        "ssco_solve": (i32, [vp, vp, vp, vp]),
        "ssco_backward": (i32, [vp, vp, vp, vp, vp, vp, vp]),
        "ssco_status_get": (i32, [vp, vp, vp, vp, vp, vp]),
        "ssco_export_L": (i32, [vp, vp, vp]),
        "ssco_export_K": (i32, [vp, vp, vp]),
        "ssco_refactor_solve_host": (i32, [vp, vp, i32, vp, vp, vp, vp]),
        "ssco_last_launch_count": (i64, [vp]),
        "ssco_cotan_weights": (i32, [vp, vp, i64, i64, i64, i32, vp, vp, vp, vp]),
        "ssco_tet_stiffness": (i32, [vp, i64, i64, i32, vp, vp, C.c_double, vp, vp, vp]),
        "ssco_last_error": (C.c_char_p, [vp]),
        "ssco_status_string": (C.c_char_p, [i32]),
        "ssco_plan_save": (i32, [vp, C.c_char_p]),
        "ssco_plan_load": (i32, [C.c_char_p, C.POINTER(vp)]),
        "ssco_destroy": (None, [vp]),
        "ssco_profile_enable": (i32, [vp, i32]),
        "ssco_profile_read": (i32, [vp, C.POINTER(KernelStat)]),
        "ssco_kernel_name": (C.c_char_p, [i32]),
        "ssco_solve_noalloc": (i32, [vp, vp, vp, vp]),
        "ssco_profile_trace": (i32, [vp, vp, vp, vp, vp, i64, C.POINTER(i64)]),
        "ssco_graph_run": (i32, [vp, vp, i32, vp, vp, vp, vp]),
        "ssco_autotune": (i32, [vp, vp, i32, vp, vp, vp, i32, vp, C.POINTER(dbl)]),
        "ssco_expr_compile": (i32, [C.POINTER(ExprNode), i32, vp, i32, i32, i32, i32, C.POINTER(vp)]),
        "ssco_expr_compile_opts": (i32, [C.POINTER(ExprNode), i32, vp, i32, C.POINTER(ExprOpts), C.POINTER(vp)]),
        "ssco_expr_get_info": (i32, [vp, C.POINTER(ExprInfo)]),
        "ssco_expr_export": (i32, [vp, i32, vp, C.c_uint64]),
        "ssco_expr_output_shape": (i32, [vp, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i64)]),
        "ssco_expr_output_pattern": (i32, [vp, i32, vp, vp]),
        "ssco_expr_bind": (i32, [vp, vp, vp, vp]),
        "ssco_expr_run": (i32, [vp, vp, vp, vp]),
        "ssco_expr_last_error": (C.c_char_p, [vp]),
        "ssco_expr_save": (i32, [vp, C.c_char_p]),
        "ssco_expr_load": (i32, [C.c_char_p, C.POINTER(vp)]),
        "ssco_expr_destroy": (None, [vp]),
        "ssco_set_flow": (i32, [vp, i32, i64, i32]),
        "ssco_graph_run_many": (i32, [vp, i32, vp, vp, vp, vp, vp, vp]),
        "ssco_autotune_many": (i32, [vp, i32, vp, vp, vp, vp, vp, i32, vp, C.POINTER(dbl)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def atwa_pattern(n, rowptr, colind, aval, perm=None):
    """Pattern of K = A^T diag(w) A + shift I: A is m x n in CSR (rowptr
    [m+1], colind [nnz] in [0, n), aval [nnz] the constant entries); the
    per-call values are w [m].  perm[new] = old (None = natural order)."""
    rowptr = np.asarray(rowptr, np.int64)
    return {"kind": KIND_ATWA, "n": int(n), "m": int(rowptr.size - 1), "rowptr": rowptr,
            "colind": np.asarray(colind, np.int32), "aval": np.asarray(aval, np.float64), "perm": perm}


def elem_pattern(n, elem_dofs, elem_K0, perm=None):
    """Pattern of K = sum_e E_e K_e^0: elem_dofs [m][d] global DOFs (-1 =
    fixed), elem_K0 [m][d(d+1)/2] row-major packed lower triangles; the
    per-call values are E [m]."""
    dofs = np.asarray(elem_dofs, np.int32)
    return {"kind": KIND_ELEM, "n": int(n), "m": int(dofs.shape[0]), "elem_dim": int(dofs.shape[1]),
            "elem_dofs": dofs, "elem_K0": np.asarray(elem_K0, np.float64), "perm": perm}


def elem_blocks_pattern(n, elem_dofs, perm=None):
    """Pattern of K = sum_e K_e over m elements with the element blocks
    themselves as the per-call values ([m][d(d+1)/2] packed lower
    triangles per value set)."""
    dofs = np.asarray(elem_dofs, np.int32)
    return {"kind": KIND_ELEM_BLOCKS, "n": int(n), "m": int(dofs.shape[0]), "elem_dim": int(dofs.shape[1]),
            "elem_dofs": dofs, "perm": perm}


class Plan:
    """An analyzed fixed structure plus (after :meth:`bind`) its device memory.

    ``problems`` is one pattern or a list of them (several patterns
    concatenated, one value set each per instance).  A pattern is a mapping
    with the fields of ``ssco_pattern``: build one from arrays with
    :func:`atwa_pattern`, :func:`elem_pattern` or :func:`elem_blocks_pattern`
    (the seeded workload generators in ``problems.py`` return such mappings
    too, with their inputs attached).

    Options (the fields of ``ssco_op`` in ``ssco.h``; 0 = the default):
    ``precision`` FP64 or FP32_REFINE (FP32 factor, FP64 refinement to
    ``refine_tol`` within ``refine_max_iter`` corrections); ``batch`` value
    sets per pattern; ``small_front_max`` rows above which a front takes the
    multi-CTA path; ``amalgamate`` relaxed supernode merging (numeric
    partition only); ``tiny_front_max`` warp-per-subtree fronts (<= 32, -1
    off); ``tensor_cores`` 0 tcgen05 updates per tile, 2 persistent trailing
    updates, -1 SIMT only; ``big_panel`` columns per trailing update of a big
    front; ``split_rows`` / ``cluster_rows`` front sizes from which solves run
    as multi-launch splits / one CTA cluster per front (-1 never);
    ``warp_front_max`` small-front classes factored one warp per front;
    ``refine_mode`` 0 plain refinement, 1 GMRES-IR (FP64 GMRES preconditioned
    by the FP32 factor, ``gmres_restart`` Krylov vectors), 2 plain refinement
    then GMRES-IR for the systems where it stagnated; ``vec2_max_cls`` (FP32)
    larger small-front classes up to 128 or 160 rows factored two value sets
    per CTA.
    ``autotune`` re-chooses the launch-shape options on the caller's data."""

    def __init__(self, problems, precision=FP64, batch=None, refine_tol=1e-10, refine_max_iter=30,
                 small_front_max=0, amalgamate=1, tiny_front_max=0, tensor_cores=0, big_panel=0,
                 split_rows=0, warp_front_max=0, cluster_rows=0, refine_mode=0, gmres_restart=0, vec2_max_cls=0,
                 _handle=None):
        self.L = load_library()
        if _handle is not None:
            self._h = _handle
        else:
            probs = problems if isinstance(problems, (list, tuple)) else [problems]
            self._keep = []
            pats = []
            for p in probs:
                pat = Pattern()
                pat.kind, pat.n, pat.m = int(p["kind"]), int(p["n"]), int(p["m"])
                if pat.kind == KIND_ATWA:
                    rp = np.ascontiguousarray(p["rowptr"], np.int64)
                    ci = np.ascontiguousarray(p["colind"], np.int32)
                    av = np.ascontiguousarray(p["aval"], np.float64)
                    self._keep += [rp, ci, av]
                    pat.rowptr, pat.colind, pat.aval = rp.ctypes.data, ci.ctypes.data, av.ctypes.data
                elif pat.kind == KIND_ELEM:
                    dofs = np.ascontiguousarray(p["elem_dofs"], np.int32)
                    K0 = np.ascontiguousarray(p["elem_K0"], np.float64)
                    self._keep += [dofs, K0]
                    pat.elem_dim = int(p["elem_dim"])
                    pat.elem_dofs, pat.elem_K0 = dofs.ctypes.data, K0.ctypes.data
                elif pat.kind == KIND_ELEM_BLOCKS:   # element blocks given per call
                    dofs = np.ascontiguousarray(p["elem_dofs"], np.int32)
                    self._keep.append(dofs)
                    pat.elem_dim = int(p["elem_dim"])
                    pat.elem_dofs = dofs.ctypes.data
                if p.get("perm") is not None:
                    pm = np.ascontiguousarray(p["perm"], np.int32)
                    self._keep.append(pm)
                    pat.perm = pm.ctypes.data
                pats.append(pat)
            arr = (C.POINTER(Pattern) * len(pats))(*[C.pointer(q) for q in pats])
            op = Op()
            op.precision = precision
            op.batch = int(batch if batch is not None else probs[0].get("batch", 1))
            op.refine_tol = refine_tol
            op.refine_max_iter = refine_max_iter
            op.small_front_max = small_front_max
            op.amalgamate = amalgamate
            op.tiny_front_max = tiny_front_max
            op.tensor_cores = tensor_cores
            op.big_panel = big_panel
            op.split_rows = split_rows
            op.warp_front_max = warp_front_max
            op.cluster_rows = cluster_rows
            op.refine_mode = refine_mode
            op.gmres_restart = gmres_restart
            op.vec2_max_cls = vec2_max_cls
            h = C.c_void_p()
            st = self.L.ssco_analyze(arr, len(pats), C.byref(op), C.byref(h))
            if st != SSCO_OK:
                raise SscoError(st, self.L.ssco_last_error(None).decode())
            self._h = h
            self._keep = None
        inf = Info()
        self._check(self.L.ssco_plan_info(self._h, C.byref(inf)))
        self.info = inf.as_dict()
        self.n = self.info["n"]
        self.m = self.info["m"]
        self.batch = self.info["batch"]
        self.n_pats = self.info["n_pats"]
        self.n_systems = self.info["n_systems"]
        self.precision = precision
        self.tables = None
        self.ws = None
        self.device = None

    # -- plumbing -----------------------------------------------------------
    def _check(self, st):
        if st != SSCO_OK:
            raise SscoError(st, self.L.ssco_last_error(self._h).decode())

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.ssco_destroy(h)
            self._h = None

    # -- structure ------------------------------------------------------------
    _EXPORT_DTYPES = {EXPORT_PERM: np.int32, EXPORT_ETREE: np.int32, EXPORT_COLCOUNT: np.int32,
                      EXPORT_L_COLPTR: np.int64, EXPORT_L_ROWIND: np.int32, EXPORT_COL_LEVEL: np.int32,
                      EXPORT_SNODE_FIRST: np.int32, EXPORT_SN_PARENT: np.int32, EXPORT_SN_LEVEL: np.int32,
                      EXPORT_K_COLPTR: np.int64, EXPORT_K_ROWIND: np.int32, EXPORT_GROUPS: np.int64,
                      EXPORT_GROUP_COEF: np.float64, EXPORT_FRONT_FIRST: np.int32,
                      EXPORT_FRONT_LEVEL: np.int32}

    def export(self, what):
        i = self.info
        n = i["n"]
        sizes = {EXPORT_PERM: n, EXPORT_ETREE: n, EXPORT_COLCOUNT: n, EXPORT_L_COLPTR: n + 1,
                 EXPORT_L_ROWIND: i["nnz_L"], EXPORT_COL_LEVEL: n, EXPORT_SNODE_FIRST: i["n_snodes"] + 1,
                 EXPORT_SN_PARENT: i["n_snodes"], EXPORT_SN_LEVEL: i["n_snodes"], EXPORT_K_COLPTR: n + 1,
                 EXPORT_K_ROWIND: i["nnz_K"], EXPORT_GROUPS: 4 * i["n_assembly_groups"],
                 EXPORT_GROUP_COEF: i["n_assembly_groups"], EXPORT_FRONT_FIRST: i["n_fronts"] + 1,
                 EXPORT_FRONT_LEVEL: i["n_fronts"]}
        out = np.zeros(max(int(sizes[what]), 1), self._EXPORT_DTYPES[what])
        self._check(self.L.ssco_plan_export(self._h, what, out.ctypes.data, out.nbytes))
        out = out[: int(sizes[what])]
        return out.reshape(-1, 4) if what == EXPORT_GROUPS else out

    def save(self, path):
        self._check(self.L.ssco_plan_save(self._h, path.encode()))

    @classmethod
    def load(cls, path, precision=None):
        L = load_library()
        h = C.c_void_p()
        st = L.ssco_plan_load(path.encode(), C.byref(h))
        if st != SSCO_OK:
            raise SscoError(st, L.ssco_last_error(None).decode())
        return cls(None, precision=precision if precision is not None else FP64, _handle=h)

    # -- device ---------------------------------------------------------------
    def bind(self, device="cuda", stream=None):
        """Allocates the table buffer and workspace with torch and binds them."""
        self.device = torch.device(device)
        tb = int(self.info["tables_bytes"])
        wb = int(self.info["workspace_bytes"])
        self.tables = torch.empty(tb + 256, dtype=torch.uint8, device=self.device)
        self.ws = torch.empty(wb + 256, dtype=torch.uint8, device=self.device)
        t0 = (-self.tables.data_ptr()) % 256
        w0 = (-self.ws.data_ptr()) % 256
        self._check(self.L.ssco_bind(self._h, C.c_void_p(self.tables.data_ptr() + t0), tb,
                                     C.c_void_p(self.ws.data_ptr() + w0), wb, _stream_ptr(stream)))
        return self

    def numeric(self, vals: torch.Tensor, shift: torch.Tensor, stream=None):
        """vals: [B, m] float64/float32 on the device; shift: [n_systems] float64."""
        assert vals.is_cuda and vals.is_contiguous() and vals.numel() == self.batch * self.m
        assert shift.is_cuda and shift.dtype == torch.float64 and shift.numel() == self.n_systems
        dt = VALS_F64 if vals.dtype == torch.float64 else VALS_F32
        assert vals.dtype in (torch.float64, torch.float32)
        self._check(self.L.ssco_numeric(self._h, _ptr(vals), dt, _ptr(shift), _stream_ptr(stream)))

    def solve(self, b: torch.Tensor, x: torch.Tensor | None = None, stream=None):
        assert b.is_cuda and b.dtype == torch.float64 and b.is_contiguous()
        if x is None:
            x = torch.empty_like(b)
        self._check(self.L.ssco_solve(self._h, _ptr(b), _ptr(x), _stream_ptr(stream)))
        return x

    def solve_noalloc(self, b: torch.Tensor, x: torch.Tensor, stream=None):
        """ssco_solve_noalloc: FP64 direct solve whose scratch is a static
        device array (no allocation by the library or here; x is the caller's)."""
        assert b.is_cuda and b.dtype == torch.float64 and b.is_contiguous()
        assert x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()
        self._check(self.L.ssco_solve_noalloc(self._h, _ptr(b), _ptr(x), _stream_ptr(stream)))
        return x

    def autotune(self, vals: torch.Tensor, shift: torch.Tensor, b: torch.Tensor, x: torch.Tensor, reps: int = 3,
                 stream=None):
        """Times the launch-shape candidates on these inputs and keeps the
        fastest (see ssco_autotune); returns (best step ms, chosen knobs)."""
        dt = VALS_F64 if vals.dtype == torch.float64 else VALS_F32
        best = C.c_double(0.0)
        self._check(self.L.ssco_autotune(self._h, _ptr(vals), dt, _ptr(shift), _ptr(b), _ptr(x), int(reps),
                                         _stream_ptr(stream), C.byref(best)))
        inf = Info()
        self._check(self.L.ssco_plan_info(self._h, C.byref(inf)))
        self.info = inf.as_dict()
        return best.value, {k: self.info[k] for k in ("tune_warp_items", "tune_vec_max_cls",
                                                      "tune_solve_threads_big", "tune_use_tc",
                                                      "tune_big_panel", "tune_split_rows",
                                                      "tune_warp_front_max", "tune_cluster_rows", "tune_flow",
                                                      "tune_vec2_max_cls")}

    def graph_run(self, vals: torch.Tensor, shift: torch.Tensor, b: torch.Tensor, x: torch.Tensor, stream=None):
        """numeric + solve as one captured CUDA graph (re-captured when the
        pointers change)."""
        dt = VALS_F64 if vals.dtype == torch.float64 else VALS_F32
        self._check(self.L.ssco_graph_run(self._h, _ptr(vals), dt, _ptr(shift), _ptr(b), _ptr(x),
                                          _stream_ptr(stream)))
        return x

    def backward(self, x, xbar, stream=None, want_shift=True):
        vbar = torch.empty((self.batch, self.m), dtype=torch.float64, device=x.device)
        sbar = torch.empty(self.n_systems, dtype=torch.float64, device=x.device) if want_shift else None
        bbar = torch.empty_like(xbar)
        self._check(self.L.ssco_backward(self._h, _ptr(x), _ptr(xbar.contiguous()), _ptr(vbar), _ptr(sbar),
                                         _ptr(bbar), _stream_ptr(stream)))
        return vbar, sbar, bbar

    def status(self, stream=None):
        S = self.n_systems
        st = np.zeros(S, np.int32)
        it = np.zeros(S, np.int32)
        rs = np.zeros(S, np.float64)
        bc = np.zeros(S, np.int32)
        self.L.ssco_status_get(self._h, _stream_ptr(stream), st.ctypes.data, it.ctypes.data, rs.ctypes.data,
                               bc.ctypes.data)
        return {"status": st, "iters": it, "resid": rs, "bad_col": bc}

    def export_L(self, stream=None):
        out = np.zeros((self.batch, int(self.info["nnz_L"])))
        self._check(self.L.ssco_export_L(self._h, out.ctypes.data, _stream_ptr(stream)))
        return out

    def export_K(self, stream=None):
        out = np.zeros((self.batch, int(self.info["nnz_K"])))
        self._check(self.L.ssco_export_K(self._h, out.ctypes.data, _stream_ptr(stream)))
        return out

    def refactor_solve_host(self, vals: np.ndarray, shift: np.ndarray, b: np.ndarray, x: np.ndarray = None,
                            stream=None):
        """End-to-end call on host buffers (numpy or pinned torch CPU tensors)."""
        dt = VALS_F64 if vals.dtype in (np.float64, torch.float64) else VALS_F32
        if x is None:
            x = np.empty_like(b)
        self._check(self.L.ssco_refactor_solve_host(self._h, _ptr(vals), dt, _ptr(shift), _ptr(b), _ptr(x),
                                                    _stream_ptr(stream)))
        return x

    def set_flow(self, flow=3, max_polls=0, stall_item=-1):
        """Dataflow launches on (bit 0 solve sweeps, bit 1 factorization) or
        off, bit 2 the panel core for per-level small fronts, bit 3 big-front
        steps with the diagonal factor fused into the trsm launch; bound of
        every wait (0 = keep); test hook stall_item (see ssco_set_flow)."""
        self._check(self.L.ssco_set_flow(self._h, int(flow), int(max_polls), int(stall_item)))
        inf = Info()
        self._check(self.L.ssco_plan_info(self._h, C.byref(inf)))
        self.info = inf.as_dict()
        return self

    def last_launch_count(self):
        return int(self.L.ssco_last_launch_count(self._h))

    def profile_enable(self, max_launches: int):
        """Per-kernel CUDA-event timing of subsequent launches (0 = off)."""
        self._check(self.L.ssco_profile_enable(self._h, int(max_launches)))

    def profile_trace(self):
        """Per-launch records (kind name, ms, flops, bytes) in launch order."""
        n = C.c_int64(0)
        self._check(self.L.ssco_profile_trace(self._h, None, None, None, None, 0, C.byref(n)))
        k = np.zeros(n.value, np.int32)
        ms = np.zeros(n.value, np.float32)
        fl = np.zeros(n.value)
        by = np.zeros(n.value)
        self._check(self.L.ssco_profile_trace(self._h, k.ctypes.data, ms.ctypes.data, fl.ctypes.data,
                                              by.ctypes.data, n.value, C.byref(n)))
        return [(KERNEL_KINDS[int(a)], float(b), float(c), float(d)) for a, b, c, d in zip(k, ms, fl, by)]

    def profile_read(self):
        """{kernel kind: {launches, ms, flops, bytes}} summed since the last read."""
        arr = (KernelStat * len(KERNEL_KINDS))()
        self._check(self.L.ssco_profile_read(self._h, arr))
        return {self.L.ssco_kernel_name(a.kind).decode(): {"launches": a.launches, "ms": a.ms, "flops": a.flops,
                                                          "bytes": a.bytes} for a in arr}


class SscoSolve(torch.autograd.Function):
    """x = K(vals, shift)^-1 b with the hand-written adjoint (ssco_backward)."""

    @staticmethod
    def forward(ctx, plan: Plan, vals, shift, b):
        plan.numeric(vals.contiguous(), shift.contiguous())
        x = plan.solve(b.contiguous())
        ctx.plan = plan
        ctx.save_for_backward(x)
        ctx.vals_dtype = vals.dtype
        return x

    @staticmethod
    def backward(ctx, xbar):
        (x,) = ctx.saved_tensors
        vbar, sbar, bbar = ctx.plan.backward(x, xbar.contiguous())
        return None, vbar.to(ctx.vals_dtype), sbar, bbar


def graph_run_many(plans, vals, shifts, bs, xs, stream=None):
    """Several plans' numeric + solve as ONE captured CUDA graph (independent
    branches; see ssco_graph_run_many).  Lists with one entry per plan."""
    L = load_library()
    n = len(plans)
    arr = lambda ts: (C.c_void_p * n)(*[t.data_ptr() for t in ts])
    dts = (C.c_int32 * n)(*[VALS_F64 if v.dtype == torch.float64 else VALS_F32 for v in vals])
    hs = (C.c_void_p * n)(*[p._h.value if isinstance(p._h, C.c_void_p) else p._h for p in plans])
    st = L.ssco_graph_run_many(hs, n, arr(vals), dts, arr(shifts), arr(bs), arr(xs), _stream_ptr(stream))
    if st != SSCO_OK:
        raise SscoError(st, L.ssco_last_error(plans[0]._h).decode())
    return xs


def autotune_many(plans, vals, shifts, bs, xs, reps=3, stream=None):
    """ssco_autotune_many: the plans' dataflow choices (ssco_set_flow bits
    0..3, and the two-value-set classes of FP32 plans) tuned on their
    multi-plan graph.  Refreshes every plan's ``info`` (``tune_flow``,
    ``tune_vec2_max_cls``).  Returns (best step ms, tune_flow of every plan)."""
    L = load_library()
    n = len(plans)
    arr = lambda ts: (C.c_void_p * n)(*[t.data_ptr() for t in ts])
    dts = (C.c_int32 * n)(*[VALS_F64 if v.dtype == torch.float64 else VALS_F32 for v in vals])
    hs = (C.c_void_p * n)(*[p._h.value if isinstance(p._h, C.c_void_p) else p._h for p in plans])
    best = C.c_double(0.0)
    st = L.ssco_autotune_many(hs, n, arr(vals), dts, arr(shifts), arr(bs), arr(xs), int(reps), _stream_ptr(stream),
                              C.byref(best))
    if st != SSCO_OK:
        raise SscoError(st, L.ssco_last_error(plans[0]._h).decode())
    flows = []
    for p in plans:
        inf = Info()
        L.ssco_plan_info(p._h, C.byref(inf))
        p.info = inf.as_dict()
        flows.append(int(p.info["tune_flow"]))
    return best.value, flows


def ssco_solve(plan: Plan, vals, shift, b):
    return SscoSolve.apply(plan, vals, shift, b)


def tet_stiffness(tets: torch.Tensor, xyz: torch.Tensor, nu: float, E: torch.Tensor | None = None, stream=None,
                  out=None, check=True):
    """Linear-tet stiffness blocks [batch, n_tet, 78] (float64, device; packed
    lower triangles, local DOF 3*vertex + component) from vertex positions
    xyz [batch, n_node, 3] (float64, device), moduli E [batch, n_tet] (None =
    1) and Poisson ratio nu; tets [n_tet, 4] int32 device tensor.  The values
    of an ELEM_BLOCKS pattern over those tets.  See ssco_tet_stiffness in
    ssco.h.  With ``check`` the call synchronizes and raises if any tet had
    out-of-range ids or a degenerate shape (those blocks are zero)."""
    L = load_library()
    tets = tets.to(torch.int32).contiguous()
    xyz = xyz.to(torch.float64).contiguous()
    batch, n_node, n_tet = int(xyz.shape[0]), int(xyz.shape[1]), int(tets.shape[0])
    if E is not None:
        E = E.to(torch.float64).contiguous()
        assert tuple(E.shape) == (batch, n_tet)
    K = out if out is not None else torch.empty((batch, n_tet, 78), dtype=torch.float64, device=xyz.device)
    assert K.dtype == torch.float64 and K.is_contiguous() and K.numel() == batch * n_tet * 78
    nbad = torch.zeros(1, dtype=torch.int32, device=xyz.device) if check else None
    st = L.ssco_tet_stiffness(_ptr(tets), n_tet, n_node, batch, _ptr(xyz), _ptr(E) if E is not None else None,
                              float(nu), _ptr(K), _ptr(nbad) if check else None, _stream_ptr(stream))
    if st != SSCO_OK:
        raise SscoError(st, "ssco_tet_stiffness")
    if check and int(nbad.item()) > 0:
        raise SscoError(SSCO_ERR_INVALID_ARG, f"ssco_tet_stiffness: {int(nbad.item())} bad tets")
    return K


def cotan_weights(tri: torch.Tensor, tri_edge: torch.Tensor, xy: torch.Tensor, n_edge: int, stream=None, out=None,
                  check=True):
    """Cotangent edge weights [batch, n_edge] (float64, device) of a planar
    triangle mesh from vertex positions xy [batch, n_vert, 2] (float64,
    device); tri / tri_edge [n_tri, 3] int32 device tensors (vertex ids,
    edge opposite each corner).  See ssco_cotan_weights in ssco.h.  With
    ``check`` the call synchronizes and raises if any triangle carried an
    out-of-range id (those triangles are skipped on the device)."""
    L = load_library()
    tri = tri.to(torch.int32).contiguous()
    tri_edge = tri_edge.to(torch.int32).contiguous()
    xy = xy.to(torch.float64).contiguous()
    batch, n_vert = int(xy.shape[0]), int(xy.shape[1])
    w = out if out is not None else torch.empty((batch, int(n_edge)), dtype=torch.float64, device=xy.device)
    assert w.dtype == torch.float64 and w.is_contiguous() and tuple(w.shape) == (batch, int(n_edge))
    nbad = torch.zeros(1, dtype=torch.int32, device=xy.device) if check else None
    st = L.ssco_cotan_weights(_ptr(tri), _ptr(tri_edge), int(tri.shape[0]), n_vert, int(n_edge), batch, _ptr(xy),
                              _ptr(w), _ptr(nbad) if check else None, _stream_ptr(stream))
    if st != SSCO_OK:
        raise SscoError(st, "ssco_cotan_weights")
    if check and int(nbad.item()) > 0:
        raise SscoError(SSCO_ERR_INVALID_ARG, f"ssco_cotan_weights: {int(nbad.item())} triangles with out-of-range ids")
    return w


# ---------------------------------------------------------------------------
# fixed-pattern sparse matrix expressions
# ---------------------------------------------------------------------------
EXPR_LEAF, EXPR_ADD, EXPR_SCALE, EXPR_MUL, EXPR_TRANSPOSE = range(5)
(EXPR_EXPORT_LEVELS, EXPR_EXPORT_TERM_OFF, EXPR_EXPORT_F1, EXPR_EXPORT_F2, EXPR_EXPORT_COEF,
 EXPR_EXPORT_OUT_SLOT, EXPR_EXPORT_OUT_COEF) = range(7)


class Expr:
    """Builder of a sparse matrix expression DAG (see ssco_expr_compile in
    ssco.h).  Every method returns a node id.

        E = Expr()
        A = E.leaf(n, n, rowptr, colind); B = E.leaf(...)
        R = E.mul(E.add(E.scale(A, 2.0), B), E.transpose(B))
        prog = E.compile([R], batch=4).bind()
        out = prog.run(leaf_vals)        # [batch, n_leaf_vals] -> [batch, n_out_vals]
    """

    def __init__(self):
        self.nodes = []      # (op, a, b, alpha, rows, cols, rowptr, colind, vmap, n_vals)

    def _add(self, *nd):
        self.nodes.append(nd)
        return len(self.nodes) - 1

    def leaf(self, rows, cols, rowptr, colind, vmap=None, n_vals=None):
        """A leaf with a fixed CSR pattern; with ``vmap`` entry q takes value
        vmap[q] of the leaf's n_vals values (shared values, e.g. a symmetric
        matrix stored once)."""
        vm = None if vmap is None else np.ascontiguousarray(vmap, np.int64)
        nv = 0 if vm is None else int(n_vals if n_vals is not None else (vm.max() + 1 if vm.size else 0))
        return self._add(EXPR_LEAF, -1, -1, 0.0, int(rows), int(cols),
                         np.ascontiguousarray(rowptr, np.int64), np.ascontiguousarray(colind, np.int32), vm, nv)

    def add(self, a, b):
        return self._add(EXPR_ADD, a, b, 0.0, 0, 0, None, None, None, 0)

    def scale(self, a, alpha):
        return self._add(EXPR_SCALE, a, -1, float(alpha), 0, 0, None, None, None, 0)

    def mul(self, a, b):
        return self._add(EXPR_MUL, a, b, 0.0, 0, 0, None, None, None, 0)

    def transpose(self, a):
        return self._add(EXPR_TRANSPOSE, a, -1, 0.0, 0, 0, None, None, None, 0)

    def compile(self, outputs, batch=1, dtype=torch.float64, inline_terms=0, algebraic=False, factor_min=0,
                t_ref=0, t_compl=0):
        """inline_terms > 0 keeps sums of at most that many slot multiples
        local (expanded into their products) instead of storing them.  The
        optional steps of ssco_expr_compile_opts: ``algebraic`` hashing,
        factorization of slots shared by >= ``factor_min`` products, and the
        global decomposition thresholds ``t_ref`` / ``t_compl``."""
        opts = dict(inline_terms=int(inline_terms), algebraic=int(algebraic), factor_min=int(factor_min),
                    t_ref=int(t_ref), t_compl=int(t_compl))
        return ExprProgram(self, list(outputs), batch, dtype, opts)


class ExprProgram:
    """A compiled expression: host tables, then (after bind) device tables
    and slot workspace owned by this object as torch tensors."""

    def __init__(self, expr: Expr, outputs, batch, dtype, opts=None, _handle=None):
        self.L = load_library()
        if _handle is not None:
            self._adopt(_handle)
            return
        arr = (ExprNode * len(expr.nodes))()
        for i, (op, a, b, al, r, c, rp, ci, vm, nv) in enumerate(expr.nodes):
            arr[i].op, arr[i].a, arr[i].b, arr[i].alpha, arr[i].rows, arr[i].cols = op, a, b, al, r, c
            arr[i].rowptr = rp.ctypes.data if rp is not None else None
            arr[i].colind = ci.ctypes.data if ci is not None and ci.size else None
            arr[i].vmap = vm.ctypes.data if vm is not None and vm.size else None
            arr[i].n_vals = nv
        outs = np.ascontiguousarray(outputs, np.int32)
        self.dtype = dtype
        prec = VALS_F32 if dtype == torch.float32 else VALS_F64
        h = C.c_void_p()
        o = ExprOpts(batch=int(batch), precision=prec, **(opts or {}))
        st = self.L.ssco_expr_compile_opts(arr, len(expr.nodes), outs.ctypes.data, len(outs), C.byref(o), C.byref(h))
        if st != SSCO_OK:
            raise SscoError(st, self.L.ssco_expr_last_error(None).decode())
        self._adopt(h)

    def _adopt(self, h):
        self._h = h
        inf = ExprInfo()
        self.L.ssco_expr_get_info(h, C.byref(inf))
        self.info = inf.as_dict()
        self.batch = int(self.info["batch"])
        self.dtype = torch.float32 if self.info["precision"] == VALS_F32 else torch.float64
        r = C.c_int32()
        k = 0
        while self.L.ssco_expr_output_shape(h, k, C.byref(r), None, None) == SSCO_OK:
            k += 1
        self.n_out = k
        self._tab = self._ws = None

    def save(self, path):
        st = self.L.ssco_expr_save(self._h, path.encode())
        if st != SSCO_OK:
            raise SscoError(st, self.L.ssco_expr_last_error(None).decode())

    @classmethod
    def load(cls, path):
        L = load_library()
        h = C.c_void_p()
        st = L.ssco_expr_load(path.encode(), C.byref(h))
        if st != SSCO_OK:
            raise SscoError(st, L.ssco_expr_last_error(None).decode())
        return cls(None, None, None, None, _handle=h)

    def __del__(self):
        if getattr(self, "_h", None):
            self.L.ssco_expr_destroy(self._h)
            self._h = None

    def export(self, what):
        i = self.info
        n, dt = {EXPR_EXPORT_LEVELS: (i["n_levels"] + 1, np.int64), EXPR_EXPORT_TERM_OFF: (i["n_ops"] + 1, np.int64),
                 EXPR_EXPORT_F1: (i["n_terms"], np.int32), EXPR_EXPORT_F2: (i["n_terms"], np.int32),
                 EXPR_EXPORT_COEF: (i["n_terms"], np.float64), EXPR_EXPORT_OUT_SLOT: (i["n_out_vals"], np.int32),
                 EXPR_EXPORT_OUT_COEF: (i["n_out_vals"], np.float64)}[what]
        out = np.zeros(max(int(n), 1), dt)
        st = self.L.ssco_expr_export(self._h, what, out.ctypes.data, out.nbytes)
        if st != SSCO_OK:
            raise SscoError(st, "ssco_expr_export")
        return out[:int(n)]

    def output_pattern(self, k):
        r, c, nnz = C.c_int32(), C.c_int32(), C.c_int64()
        self.L.ssco_expr_output_shape(self._h, k, C.byref(r), C.byref(c), C.byref(nnz))
        rp = np.zeros(r.value + 1, np.int64)
        ci = np.zeros(max(nnz.value, 1), np.int32)
        self.L.ssco_expr_output_pattern(self._h, k, rp.ctypes.data, ci.ctypes.data)
        return r.value, c.value, rp, ci[:nnz.value]

    def bind(self, device="cuda", stream=None):
        i = self.info
        self._tab = torch.empty(max(int(i["table_bytes"]), 256), dtype=torch.uint8, device=device)
        self._ws = torch.empty(max(int(i["workspace_bytes"]), 256), dtype=torch.uint8, device=device)
        st = self.L.ssco_expr_bind(self._h, _ptr(self._tab), _ptr(self._ws), _stream_ptr(stream))
        if st != SSCO_OK:
            raise SscoError(st, "ssco_expr_bind")
        return self

    def run(self, leaf_vals: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        """leaf_vals [batch, n_leaf_vals] -> [batch, n_out_vals] (device, program dtype)."""
        i = self.info
        assert leaf_vals.is_cuda and leaf_vals.dtype == self.dtype and leaf_vals.is_contiguous()
        assert leaf_vals.numel() == self.batch * i["n_leaf_vals"]
        if out is None:
            out = torch.empty((self.batch, int(i["n_out_vals"])), dtype=self.dtype, device=leaf_vals.device)
        assert out.dtype == self.dtype and out.is_contiguous() and out.numel() == self.batch * i["n_out_vals"]
        st = self.L.ssco_expr_run(self._h, _ptr(leaf_vals), _ptr(out), _stream_ptr(stream))
        if st != SSCO_OK:
            raise SscoError(st, "ssco_expr_run: " + self.L.ssco_expr_last_error(self._h).decode())
        return out
