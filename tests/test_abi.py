"""Host-side checks of the C ABI (no GPU): the library loads, exports every
symbol the header declares, and its symbolic phase matches the oracle's
structures bit for bit."""
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_12865_gb300 import build as B
from paper_2110_12865_gb300 import problems as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def S():
    B.build()
    from paper_2110_12865_gb300 import ssco
    return ssco


def header_functions():
    src = open(os.path.join(ROOT, "include", "ssco.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ssco_[a-z_A-Z0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(S):
    import ctypes
    lib = ctypes.CDLL(S.LIB_PATH)
    names = header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(S.EXPORTED_SYMBOLS)


def symbolic_matches(S, p, **kw):
    pl = S.Plan(p, **kw)
    r = O.refactor_solve(p)
    Kp, Sy = r.Kp, r.S
    assert np.array_equal(pl.export(S.EXPORT_PERM), p.perm)
    assert np.array_equal(pl.export(S.EXPORT_K_COLPTR), Kp.colptr)
    assert np.array_equal(pl.export(S.EXPORT_K_ROWIND), Kp.rowind)
    assert np.array_equal(pl.export(S.EXPORT_ETREE), Sy.parent)
    assert np.array_equal(pl.export(S.EXPORT_COLCOUNT), Sy.colcount)
    assert np.array_equal(pl.export(S.EXPORT_L_COLPTR), Sy.Lcolptr)
    assert np.array_equal(pl.export(S.EXPORT_L_ROWIND), Sy.Lrowind)
    assert np.array_equal(pl.export(S.EXPORT_COL_LEVEL), Sy.col_level)
    assert np.array_equal(pl.export(S.EXPORT_SNODE_FIRST), Sy.snode_first)
    assert np.array_equal(pl.export(S.EXPORT_SN_PARENT), Sy.sn_parent)
    assert np.array_equal(pl.export(S.EXPORT_SN_LEVEL), Sy.sn_level)
    assert pl.info["nnz_L"] == Sy.nnzL and pl.info["nnz_K"] == Kp.nnz
    return pl


@pytest.mark.parametrize("name", ["grid32", "elast5", "trigrid24"])
@pytest.mark.parametrize("amalg", [0, 1])
def test_symbolic_parity_workloads(S, name, amalg):
    symbolic_matches(S, P.workload(name), amalgamate=amalg)


@pytest.mark.parametrize("seed", range(10))
def test_symbolic_parity_random(S, seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(1, 400))
    p = P.random_spd_pattern(n, int(rng.integers(0, 3 * n + 1)), rng)
    symbolic_matches(S, p)


def test_symbolic_parity_full_size_grid256(S):
    symbolic_matches(S, P.workload("grid256"))


def test_multi_pattern_concatenation(S):
    """Several patterns in one plan: the structures are the block-diagonal
    union of the per-pattern ones (offset by the preceding unknowns)."""
    probs = [P.trigrid_problem(s, 1, cfg=3, seed_offset=k) for k, s in enumerate([5, 9, 7])]
    probs.append(P.elasticity_problem(2, cfg=2))
    pl = S.Plan(probs)
    par = pl.export(S.EXPORT_ETREE)
    cc = pl.export(S.EXPORT_COLCOUNT)
    lev = pl.export(S.EXPORT_COL_LEVEL)
    off = 0
    for p in probs:
        r = O.refactor_solve(p)
        sl = slice(off, off + p.n)
        exp_par = np.where(r.S.parent >= 0, r.S.parent + off, -1)
        assert np.array_equal(par[sl], exp_par)
        assert np.array_equal(cc[sl], r.S.colcount)
        assert np.array_equal(lev[sl], r.S.col_level)
        off += p.n
    assert pl.info["n"] == off and pl.info["n_pats"] == 4


def test_fronts_partition_and_levels(S):
    """Numeric partition: contiguous fronts covering all columns; a front's
    level exceeds all its children's (members of one level are independent,
    Sec. 4.3)."""
    p = P.workload("elast5")
    pl = S.Plan(p, amalgamate=1)
    ff = pl.export(S.EXPORT_FRONT_FIRST)
    fl = pl.export(S.EXPORT_FRONT_LEVEL)
    et = pl.export(S.EXPORT_ETREE)
    assert ff[0] == 0 and ff[-1] == p.n and np.all(np.diff(ff) > 0)
    col2f = np.repeat(np.arange(len(fl)), np.diff(ff))
    for f in range(len(fl)):
        last = ff[f + 1] - 1
        # inside a front the etree is a chain
        assert np.all(et[ff[f]:last] == np.arange(ff[f] + 1, last + 1))
        if et[last] >= 0:
            assert fl[col2f[et[last]]] > fl[f]


def test_assembly_groups_leaf_tables(S):
    """Grouping by term count with uniform-constant folding (Sec. 4.3, 4.4,
    App. B): for an incidence matrix every coefficient is +1 (diagonal) or
    -1 (off-diagonal), so every group is uniform; diagonal term counts are
    the vertex degrees."""
    p = P.grid_problem(9, 7, cfg=1)
    pl = S.Plan(p)
    g = pl.export(S.EXPORT_GROUPS)
    c = pl.export(S.EXPORT_GROUP_COEF)
    assert g[:, 0].sum() == pl.info["nnz_K"]
    assert np.all(g[:, 2] == 1)
    deg = np.bincount(p.edges.ravel(), minlength=p.n)
    diag = g[g[:, 3] == 1]
    assert sorted(diag[:, 1]) == sorted(set(deg))
    assert dict(zip(diag[:, 1], diag[:, 0])) == {d: int(np.sum(deg == d)) for d in set(deg)}
    assert np.all(c[g[:, 3] == 1] == 1.0) and np.all(c[g[:, 3] == 0] == -1.0)
    assert (g[:, 0] * g[:, 1]).sum() == pl.info["assembly_terms"]
    pe = S.Plan(P.elasticity_problem(2, cfg=2))
    ge = pe.export(S.EXPORT_GROUPS)
    assert np.all(ge[ge[:, 1] > 0, 2] == 0)  # element blocks: varying constants


@pytest.mark.parametrize("bad", ["perm_dup", "col_range", "dup_col", "dofs_range", "bad_kind", "zero_n",
                                 "rowptr", "nan_aval"])
def test_invalid_patterns_rejected(S, bad):
    p = P.grid_problem(4, 4, cfg=1)
    if bad == "perm_dup":
        p["perm"] = p.perm.copy()
        p.perm[1] = p.perm[0]
    elif bad == "col_range":
        p["colind"] = p.colind.copy()
        p.colind[3] = p.n
    elif bad == "dup_col":
        p["colind"] = p.colind.copy()
        p.colind[1] = p.colind[0]
    elif bad == "bad_kind":
        p["kind"] = 7
    elif bad == "zero_n":
        p["n"] = 0
    elif bad == "rowptr":
        p["rowptr"] = p.rowptr.copy()
        p.rowptr[2] = p.rowptr[1] - 1
    elif bad == "nan_aval":
        p["aval"] = p.aval.copy()
        p.aval[0] = np.nan
    elif bad == "dofs_range":
        p = P.elasticity_problem(1, cfg=2)
        p["elem_dofs"] = p.elem_dofs.copy()
        p.elem_dofs[0, 0] = p.n
    with pytest.raises(S.SscoError) as ei:
        S.Plan(p)
    assert ei.value.status in (1, 2, 4)


def test_plan_save_load_roundtrip(S, tmp_path):
    p = P.workload("elast5")
    pl = S.Plan(p, precision=S.FP32_REFINE)
    f = str(tmp_path / "plan.bin")
    pl.save(f)
    q = S.Plan.load(f, precision=S.FP32_REFINE)
    assert q.info == pl.info
    for what in range(15):
        assert np.array_equal(q.export(what), pl.export(what))
    raw = open(f, "rb").read()
    bad = [b"garbage!" + raw[8:],                                       # magic
           raw[:len(raw) // 2] + bytes([raw[len(raw) // 2] ^ 0x10]) + raw[len(raw) // 2 + 1:],  # a table byte
           raw[:-1],                                                    # truncated digest
           raw + b"\0"]                                                 # trailing byte
    # 8 bytes of 0xff over each early field (counts and lengths included):
    # refused, never a huge allocation or a crash
    bad += [raw[:o] + b"\xff" * 8 + raw[o + 8:] for o in range(12, 400, 4)]
    for i, blob in enumerate(bad):
        g = str(tmp_path / f"bad{i}.bin")
        open(g, "wb").write(blob)
        with pytest.raises(S.SscoError) as ei:
            S.Plan.load(g)
        assert ei.value.status == 1


def _fnv1a64(data: bytes) -> int:
    h = 0xcbf29ce484222325
    for c in data:
        h = ((h ^ c) * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


def _find_solve_lists(raw: bytes, n_levels: int):
    """(offset, count) of the solve launch lists in a plan file: a u64 count N,
    then N 56-byte records (level, class, list offset, count, largest rows,
    width, three big-front maxima) whose level runs 0, 1, ..., whose class is
    0 and whose list offsets never decrease, then the plan's level count (the
    field the file writes next)."""
    import struct
    rec = 56
    for o in range(0, len(raw) - 12):
        n = struct.unpack_from("<Q", raw, o)[0]
        if not 1 <= n <= 4096 or o + 8 + n * rec + 4 > len(raw):
            continue
        base = o + 8
        recs = [struct.unpack_from("<iiqiii", raw, base + k * rec) for k in range(n)]
        if all(r[0] == k and r[1] == 0 and r[3] >= 0 for k, r in enumerate(recs)) and \
                all(recs[k][2] <= recs[k + 1][2] for k in range(n - 1)) and \
                struct.unpack_from("<i", raw, base + n * rec)[0] == n_levels:
            return base, n
    raise AssertionError("solve launch lists not found")


def test_plan_load_refuses_inconsistent_launch_lists(S, tmp_path):
    """A re-digested plan file whose launch list understates its largest front
    (which sizes shared memory), overstates its width, or reaches past the
    front list is refused with SSCO_ERR_INVALID_ARG; the untouched file, put
    through the same re-digest, loads."""
    import struct
    p = P.grid_problem(24, 24, cfg=1)
    pl = S.Plan(p, precision=S.FP32_REFINE)
    f = str(tmp_path / "plan.bin")
    pl.save(f)
    raw = open(f, "rb").read()
    body = bytearray(raw[:-8])
    base, n_lists = _find_solve_lists(bytes(body), int(pl.info["n_levels"]))
    # the first list with fronts
    k = next(k for k in range(n_lists) if struct.unpack_from("<i", body, base + k * 56 + 16)[0] > 0)
    o = base + k * 56
    count, rmax, wmax = struct.unpack_from("<iii", body, o + 16)
    assert count > 0 and rmax >= wmax >= 1

    def with_field(off, fmt, value):
        b = bytearray(body)
        struct.pack_into(fmt, b, off, value)
        return bytes(b) + struct.pack("<Q", _fnv1a64(bytes(b)))

    same = str(tmp_path / "same.bin")
    open(same, "wb").write(bytes(body) + struct.pack("<Q", _fnv1a64(bytes(body))))
    assert S.Plan.load(same, precision=S.FP32_REFINE).info == pl.info
    for i, blob in enumerate([with_field(o + 20, "<i", rmax - 1),       # largest rows understated
                              with_field(o + 24, "<i", wmax + 1),       # width overstated
                              with_field(o + 16, "<i", 1 << 30),        # count past the front list
                              with_field(o + 8, "<q", -1)]):            # negative list offset
        g = str(tmp_path / f"bad{i}.bin")
        open(g, "wb").write(blob)
        with pytest.raises(S.SscoError) as ei:
            S.Plan.load(g)
        assert ei.value.status == 1
    # a solve list out of its largest-first order: its fronts reversed in the
    # front list.  A level whose fronts all have one size stays in order, so
    # at least one of the reversed lists (not every one) must be refused.
    fl_base = _find_front_lists(bytes(body), base)
    refused = 0
    for k in range(n_lists):
        lo, cnt = struct.unpack_from("<qi", body, base + k * 56 + 8)
        if cnt < 2:
            continue
        ids = struct.unpack_from(f"<{cnt}i", body, fl_base + 4 * lo)
        assert len(set(ids)) == cnt and all(0 <= i < pl.info["n_fronts"] for i in ids)
        b = bytearray(body)
        struct.pack_into(f"<{cnt}i", b, fl_base + 4 * lo, *ids[::-1])
        g = str(tmp_path / f"order{k}.bin")
        open(g, "wb").write(bytes(b) + struct.pack("<Q", _fnv1a64(bytes(b))))
        try:
            S.Plan.load(g)
        except S.SscoError as e:
            assert e.status == 1
            refused += 1
    assert refused >= 1


def _find_front_lists(raw: bytes, solve_base: int) -> int:
    """Offset of the front-list entries (int32) in a plan file: the file
    writes the front list (u64 length, entries), then the factorization
    launch lists (u64 length, 56-byte records), then the solve lists."""
    import struct
    for n_fact in range(0, 1 << 16):
        fact_len_at = solve_base - 8 - 56 * n_fact - 8
        if fact_len_at < 8:
            break
        if struct.unpack_from("<Q", raw, fact_len_at)[0] != n_fact:
            continue
        for n_fl in range(1, (fact_len_at - 8) // 4 + 1):
            if struct.unpack_from("<Q", raw, fact_len_at - 4 * n_fl - 8)[0] == n_fl:
                return fact_len_at - 4 * n_fl
    raise AssertionError("front list not found")


def test_multi_plan_calls_refuse_bad_arguments(S):
    """ssco_graph_run_many and ssco_autotune_many refuse on the host, before
    any device work: no plans or more than 1024, a NULL plan array, a NULL
    plan, a plan given twice, a NULL per-plan pointer, an unknown dtype,
    reps < 1 (the tuner) and an unbound plan (SSCO_ERR_STATE)."""
    import ctypes as C
    L = S.load_library()
    a = S.Plan(P.grid_problem(6, 6, cfg=1), precision=S.FP32_REFINE)
    b = S.Plan(P.grid_problem(5, 7, cfg=1), precision=S.FP32_REFINE)

    def h(p):
        return p._h.value if isinstance(p._h, C.c_void_p) else p._h
    fake = 4096   # a per-plan device pointer that is never dereferenced

    def call(fn, hs, n=None, dtype=S.VALS_F32, ptr=fake, reps=3, plans_null=False):
        k = max(len(hs), 1)
        n = len(hs) if n is None else n
        H = None if plans_null else (C.c_void_p * k)(*hs)
        ptrs = (C.c_void_p * k)(*([ptr] * k))
        dts = (C.c_int32 * k)(*([dtype] * k))
        args = [H, n, ptrs, dts, ptrs, ptrs, ptrs]
        if fn == "many_tune":
            return L.ssco_autotune_many(*args, reps, None, None)
        return L.ssco_graph_run_many(*args, None)

    for fn in ("many_run", "many_tune"):
        assert call(fn, [h(a)], n=0) == 1
        assert call(fn, [h(a)], n=1025) == 1
        assert call(fn, [h(a)], plans_null=True) == 1
        assert call(fn, [h(a), None]) == 1
        assert call(fn, [h(a), h(a)]) == 1
        assert call(fn, [h(a), h(b)], ptr=None) == 1
        assert call(fn, [h(a), h(b)], dtype=7) == 1
        assert call(fn, [h(a), h(b)]) == 10          # neither plan is bound
    assert call("many_tune", [h(a), h(b)], reps=0) == 1


def test_fixed_dofs_are_identity_rows(S):
    p = P.elasticity_problem(3, cfg=2)
    pl = S.Plan(p)
    cc = pl.export(S.EXPORT_COLCOUNT)
    iperm = np.argsort(p.perm)
    fixed_new = iperm[np.nonzero(p.dof_fixed)[0]]
    assert np.all(cc[fixed_new] == 1)
    assert np.all(pl.export(S.EXPORT_ETREE)[fixed_new] == -1)


@pytest.mark.parametrize("opt", [{"big_panel": 48}, {"big_panel": 16}, {"big_panel": 2048}, {"split_rows": -2},
                                 {"warp_front_max": 65}, {"warp_front_max": -2}, {"cluster_rows": -5},
                                 {"batch": 0}, {"batch": 65536}])
def test_invalid_plan_options_rejected(S, opt):
    """Out-of-range launch-shape options are refused at analyze time with
    SSCO_ERR_INVALID_ARG (host only, no device work)."""
    with pytest.raises(S.SscoError) as ei:
        S.Plan(P.grid_problem(6, 6, cfg=1), **opt)
    assert ei.value.status == 1


@pytest.mark.parametrize("opt,key,want", [({"big_panel": 96}, "tune_big_panel", 96),
                                          ({"split_rows": -1}, "tune_split_rows", 1 << 30),
                                          ({"cluster_rows": 300}, "tune_cluster_rows", 300),
                                          ({"warp_front_max": 48}, "tune_warp_front_max", 48),
                                          ({"tensor_cores": -1}, "tune_use_tc", 0),
                                          ({"tensor_cores": 2}, "tune_use_tc", 2)])
def test_plan_options_reach_the_tunables(S, opt, key, want):
    pl = S.Plan(P.grid_problem(6, 6, cfg=1), precision=S.FP32_REFINE, **opt)
    assert pl.info[key] == want


def test_batch_dependent_solve_defaults(S):
    """Few value sets: CTA clusters for fronts >= 512 rows and split solves
    from 2048; many: no clusters, split from 1024."""
    one = S.Plan(P.grid_problem(6, 6, batch=1, cfg=1), precision=S.FP32_REFINE)
    many = S.Plan(P.grid_problem(6, 6, batch=16, cfg=1), precision=S.FP32_REFINE)
    assert (one.info["tune_cluster_rows"], one.info["tune_split_rows"]) == (512, 2048)
    assert (many.info["tune_cluster_rows"], many.info["tune_split_rows"]) == (1 << 30, 1024)


def test_cotan_weights_argument_checks(S):
    """ssco_cotan_weights refuses inconsistent sizes and null pointers before
    touching the device."""
    L = S.load_library()
    assert L.ssco_cotan_weights(None, None, 1, 3, 3, 1, None, None, None, None) == 1  # null tables
    assert L.ssco_cotan_weights(None, None, -1, 3, 3, 1, None, None, None, None) == 1  # negative count
    assert L.ssco_cotan_weights(None, None, 0, 3, 3, 0, None, None, None, None) == 1  # batch < 1


def test_tet_stiffness_argument_checks(S):
    """ssco_tet_stiffness refuses inconsistent sizes, an out-of-range Poisson
    ratio and null pointers before touching the device; no tets is a no-op."""
    L = S.load_library()
    assert L.ssco_tet_stiffness(None, 1, 4, 1, None, None, 0.3, None, None, None) == 1   # null tables
    assert L.ssco_tet_stiffness(None, -1, 4, 1, None, None, 0.3, None, None, None) == 1  # negative count
    assert L.ssco_tet_stiffness(None, 0, 4, 0, None, None, 0.3, None, None, None) == 1   # batch < 1
    assert L.ssco_tet_stiffness(None, 0, 4, 65536, None, None, 0.3, None, None, None) == 1
    for nu in (0.5, -1.0, 0.7, float("nan")):
        assert L.ssco_tet_stiffness(None, 0, 4, 1, None, None, nu, None, None, None) == 1
    assert L.ssco_tet_stiffness(None, 0, 4, 1, None, None, 0.3, None, None, None) == 0    # nothing to do


def test_element_blocks_pattern_structure(S, tmp_path):
    """A per-call element-block pattern has the structure of the modulus
    pattern on the same mesh (same K and L patterns, etree, fronts); only its
    value count grows to 78 per tet.  Its adjoint tables survive a plan file."""
    p = P.elasticity_problem(3, cfg=2)
    g = P.elasticity_geometry_problem(3, cfg=6)
    a, b = S.Plan(p), S.Plan(g)
    assert b.info["m"] == 78 * p.m and a.info["m"] == p.m
    for k in ("n", "nnz_K", "nnz_L", "n_snodes", "n_fronts"):
        assert a.info[k] == b.info[k], k
    for what in (S.EXPORT_ETREE, S.EXPORT_COLCOUNT, S.EXPORT_L_COLPTR, S.EXPORT_L_ROWIND, S.EXPORT_PERM):
        assert np.array_equal(a.export(what), b.export(what))
    f = str(tmp_path / "blocks.bin")
    b.save(f)
    c = S.Plan.load(f)
    assert c.info == b.info
    import ctypes as C
    pat = S.Pattern()
    pat.kind, pat.n, pat.m, pat.elem_dim = P.KIND_ELEM_BLOCKS, 12, 1, 12   # elem_dofs left NULL
    op = S.Op()
    op.batch = 1
    h = C.c_void_p()
    arr = (C.POINTER(S.Pattern) * 1)(C.pointer(pat))
    L = S.load_library()
    assert L.ssco_analyze(arr, 1, C.byref(op), C.byref(h)) == 1
    assert b"elem_dofs" in L.ssco_last_error(None)


def test_expr_abi_error_paths(S):
    """Host-side refusals of the expression ABI, all before any device call:
    run before bind, NULL or misaligned device buffers, a short export
    buffer, an output index out of range, every exported symbol present."""
    import ctypes as C
    L = S.load_library()
    E = S.Expr()
    A = E.leaf(3, 3, [0, 1, 2, 3], [0, 1, 2])
    prog = E.compile([E.mul(A, A)])
    h = prog._h
    assert L.ssco_expr_run(h, None, None, None) == 10                     # STATE: not bound
    assert L.ssco_expr_bind(h, None, None, None) == 1
    assert L.ssco_expr_bind(h, C.c_void_p(0x1001), C.c_void_p(0x2000), None) == 1   # misaligned
    buf = np.zeros(1, np.int64)
    assert L.ssco_expr_export(h, S.EXPR_EXPORT_TERM_OFF, buf.ctypes.data, 0) == 1    # too small
    assert L.ssco_expr_export(h, 99, buf.ctypes.data, 8) == 1                         # unknown table
    r = C.c_int32()
    assert L.ssco_expr_output_shape(h, 1, C.byref(r), None, None) == 1                # no output 1
    assert L.ssco_expr_output_shape(h, 0, C.byref(r), None, None) == 0 and r.value == 3
    assert L.ssco_expr_get_info(None, None) == 1
    assert prog.info["n_ops"] == 3 and prog.info["n_levels"] == 1   # diagonal squares: one term each


def test_plan_from_plain_arrays_matches_problem_dicts(S):
    """A plan built from plain CSR / element arrays (atwa_pattern,
    elem_pattern, elem_blocks_pattern) is the plan built from the workload
    generators' dicts: same perm, L pattern and assembly groups."""
    g = P.grid_problem(9, 7, batch=2, cfg=1)
    e = P.elasticity_problem(3, batch=1, cfg=2)
    eg = P.elasticity_geometry_problem(2, batch=1)
    pairs = [(g, S.atwa_pattern(g.n, g.rowptr, g.colind, g.aval, g.perm)),
             (e, S.elem_pattern(e.n, e.elem_dofs, e.elem_K0, e.perm)),
             (eg, S.elem_blocks_pattern(eg.n, eg.elem_dofs, eg.perm))]
    for prob, pat in pairs:
        a = S.Plan(prob, precision=S.FP64, batch=1)
        b = S.Plan(pat, precision=S.FP64, batch=1)
        assert a.info == b.info
        for what in (S.EXPORT_PERM, S.EXPORT_L_COLPTR, S.EXPORT_L_ROWIND, S.EXPORT_GROUPS):
            assert np.array_equal(a.export(what), b.export(what))
    both = S.Plan([pairs[0][1], pairs[1][1]], precision=S.FP32_REFINE, batch=1)
    assert both.info["n"] == g.n + e.n and both.info["n_pats"] == 2
