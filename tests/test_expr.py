"""Fixed-pattern sparse matrix expressions: the host compiler's tables
(interpreted on the CPU) and the device runner (GPU) against the oracle's
definitions; the paper's three random-matrix expressions and the cube of a
cotangent Laplacian (Sec. 5 sparse-expression and structured-product
experiments)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2110_12865_gb300 import problems as P


@pytest.fixture(scope="module")
def S():
    from paper_2110_12865_gb300 import build
    build.build()
    from paper_2110_12865_gb300 import ssco
    return ssco


def build_expr(S, nodes):
    """The same node tuples as the oracle, through the builder."""
    E = S.Expr()
    for nd in nodes:
        if nd[0] == "leaf":
            E.leaf(*nd[1:])
        elif nd[0] == "add":
            E.add(nd[1], nd[2])
        elif nd[0] == "scale":
            E.scale(nd[1], nd[2])
        elif nd[0] == "mul":
            E.mul(nd[1], nd[2])
        else:
            E.transpose(nd[1])
    return E


def interpret(S, prog, leaf_vals):
    """Runs the exported tables on the CPU, level by level (what the device
    runner does), in FP64; also checks that a level reads only earlier slots
    and that its expressions are ordered by term count."""
    i = prog.info
    lv = prog.export(S.EXPR_EXPORT_LEVELS)
    toff = prog.export(S.EXPR_EXPORT_TERM_OFF)
    f1, f2 = prog.export(S.EXPR_EXPORT_F1), prog.export(S.EXPR_EXPORT_F2)
    coef = prog.export(S.EXPR_EXPORT_COEF)
    L, base = i["n_leaf_vals"], 1 + i["n_leaf_vals"]
    B = leaf_vals.shape[0]
    slots = np.zeros((i["n_slots"], B))
    slots[0] = 1.0
    slots[1:1 + L] = leaf_vals.T
    for l in range(1, i["n_levels"] + 1):
        a, b = lv[l - 1], lv[l]
        q0, q1 = toff[a], toff[b]
        assert f1[q0:q1].max() < base + a and f2[q0:q1].max() < base + a   # only earlier slots
        assert np.all(f1[q0:q1] >= f2[q0:q1])
        counts = np.diff(toff[a:b + 1])
        assert np.all(np.diff(counts) >= 0)
        seg = np.repeat(np.arange(b - a), counts)
        acc = np.zeros((b - a, B))
        np.add.at(acc, seg, coef[q0:q1, None] * slots[f1[q0:q1]] * slots[f2[q0:q1]])
        slots[base + a: base + b] = acc
    os_, oc = prog.export(S.EXPR_EXPORT_OUT_SLOT), prog.export(S.EXPR_EXPORT_OUT_COEF)
    return (oc[:, None] * slots[os_]).T


def check_outputs(S, prog, nodes, outs, vals, got, rel):
    """Output patterns equal the oracle's structural patterns; values within
    rel x the absolute-value evaluation (the rounding scale)."""
    evals = [(O.expr_eval(nodes, vals[b], outs), O.expr_eval(nodes, vals[b], outs, absolute=True))
             for b in range(vals.shape[0])]
    col = 0
    for k in range(len(outs)):
        r, c, rp, ci = prog.output_pattern(k)
        nnz = int(rp[-1])
        keys = [(i, int(j)) for i in range(r) for j in ci[rp[i]:rp[i + 1]]]
        for b, (res, res_abs) in enumerate(evals):
            d, da = res[k][2], res_abs[k][2]
            assert keys == sorted(d), "pattern"
            ref = np.array([d[key] for key in keys])
            bound = np.array([da[key] for key in keys])
            assert np.all(np.abs(got[b, col:col + nnz] - ref) <= rel * bound + 1e-300)
        col += nnz


def random_expressions(n, seed, per_row=6):
    from tests.test_oracle_pins import paper_expressions
    return paper_expressions(n, np.random.default_rng(seed), per_row)


def cotan_laplacian_cube(p):
    """L = A^T (W A) from a triangulated grid's incidence matrix A and
    cotangent weights W = diag(w), then L^3, in one DAG; outputs L^3 and L."""
    nodes, l_id, _ = P.laplacian_expression(p)
    nodes = nodes + [("mul", l_id, l_id), ("mul", l_id + 1, l_id)]
    return nodes, [l_id + 2, l_id]


def cotan_leaf_vals(p, B):
    return P.laplacian_expression(p)[2][:B]


# ---------------------------------------------------------------------------
# host compiler (CPU)
# ---------------------------------------------------------------------------
def test_compiled_tables_match_oracle_random_expressions(S):
    nodes, outs, nv = random_expressions(60, 61)
    prog = build_expr(S, nodes).compile(outs, batch=3)
    vals = np.random.default_rng(62).standard_normal((3, nv))
    check_outputs(S, prog, nodes, outs, vals, interpret(S, prog, vals), 1e-13)


def test_compiled_tables_match_oracle_cotan_laplacian_cube(S):
    p = P.trigrid_problem(10, batch=2, cfg=3)
    nodes, outs = cotan_laplacian_cube(p)
    prog = build_expr(S, nodes).compile(outs, batch=2)
    vals = cotan_leaf_vals(p, 2)
    check_outputs(S, prog, nodes, outs, vals, interpret(S, prog, vals), 1e-13)
    assert prog.info["n_levels"] == 4   # W A, L, L^2, L^3: one level per product in the chain


def test_structural_hashing_merges_equal_expressions(S):
    """A B built twice is stored once; (A B) + (A B) and A + A become scaled
    relabellings (no new expression); A A^T stores each unordered pair of
    rows once, so only its lower triangle (with the diagonal) is computed."""
    rng = np.random.default_rng(63)
    from tests.test_oracle_pins import _rand_csr
    n = 50
    A = ("leaf", n, n, *_rand_csr(rng, n, n, 4))
    Bm = ("leaf", n, n, *_rand_csr(rng, n, n, 4))
    one = build_expr(S, [A, Bm, ("mul", 0, 1)]).compile([2])
    two = build_expr(S, [A, Bm, ("mul", 0, 1), ("mul", 0, 1), ("add", 2, 3), ("add", 0, 0)]).compile([4, 5])
    assert two.info["n_ops"] == one.info["n_ops"]
    oc = two.export(S.EXPR_EXPORT_OUT_COEF)
    assert np.all(oc == 2.0)
    aat = build_expr(S, [A, ("transpose", 0), ("mul", 0, 1)]).compile([2])
    r, c, rp, ci = aat.output_pattern(0)
    lower = sum(int(np.sum(ci[rp[i]:rp[i + 1]] <= i)) for i in range(r))
    assert aat.info["n_ops"] == lower and aat.info["n_unrolled"] == int(rp[-1])
    vals = rng.standard_normal((1, int(A[3][-1])))
    check_outputs(S, aat, [A, ("transpose", 0), ("mul", 0, 1)], [2], vals, interpret(S, aat, vals), 1e-13)


def test_compiled_tables_edge_cases(S):
    """Empty rows and an empty leaf, rectangular chains, a double transpose,
    a zero scale, exact cancellation A + (-1)A, a leaf and a repeated node as
    outputs, and a deep power chain: tables against the oracle, structure
    included."""
    rng = np.random.default_rng(67)
    from tests.test_oracle_pins import _rand_csr
    rp, ci = _rand_csr(rng, 7, 5, 2)
    rp[3:] -= rp[3] - rp[2]                                  # row 2 left empty
    ci = np.delete(ci, np.s_[2 * 2:2 * 3])
    A = ("leaf", 7, 5, rp, ci)                                # 7 x 5 with an empty row
    Bm = ("leaf", 5, 3, *_rand_csr(rng, 5, 3, 2))             # 5 x 3
    Z = ("leaf", 3, 3, np.zeros(4, np.int64), np.zeros(0, np.int32))   # no entries
    Sq = ("leaf", 6, 6, *_rand_csr(rng, 6, 6, 2))
    nodes = [A, Bm, Z, Sq,
             ("mul", 0, 1),                 # 4: 7 x 3
             ("transpose", 4), ("transpose", 5),   # 5, 6: (AB)^T, ((AB)^T)^T
             ("mul", 6, 2),                 # 7: (AB) Z -> no entries
             ("scale", 4, 0.0),             # 8: zero scale
             ("scale", 0, -1.0), ("add", 0, 9),    # 9, 10: A - A
             ("mul", 3, 3), ("mul", 11, 3), ("mul", 12, 3), ("mul", 13, 3), ("mul", 14, 3)]   # 11..15: Sq^2..Sq^6
    outs = [6, 7, 8, 10, 0, 15, 6]
    prog = build_expr(S, nodes).compile(outs, batch=2)
    nv = sum(int(nd[3][-1]) for nd in nodes if nd[0] == "leaf")
    vals = rng.standard_normal((2, nv))
    got = interpret(S, prog, vals)
    check_outputs(S, prog, nodes, outs, vals, got, 1e-13)
    assert prog.info["n_levels"] == 5                        # Sq^2 .. Sq^6
    r, c, rp7, _ = prog.output_pattern(1)
    assert (r, c, int(rp7[-1])) == (7, 3, 0)
    sizes = [int(prog.output_pattern(k)[2][-1]) for k in range(len(outs))]
    off = np.concatenate([[0], np.cumsum(sizes)])
    assert np.all(got[:, off[2]:off[4]] == 0.0)              # zero scale and A - A: exactly 0


@pytest.mark.parametrize("k", [1, 2, 4])
def test_inlined_sums_match_oracle_and_store_less(S, k):
    """Local sums (the paper's local expressions): with inline_terms = k a
    sum of at most k slot multiples is not stored; the products that use it
    expand over its terms.  Tables still match the oracle; for the paper's
    expressions with sums feeding products, fewer intermediates are stored
    and no more levels are needed; an inlined sum that is itself an output is
    stored at the end."""
    nodes, outs, nv = random_expressions(50, 68, per_row=4)
    nodes = nodes + [("add", 0, 1)]                  # a plain sum as an extra output
    outs = outs + [len(nodes) - 1]
    vals = np.random.default_rng(69).standard_normal((2, nv))
    base = build_expr(S, nodes).compile(outs, batch=2)
    prog = build_expr(S, nodes).compile(outs, batch=2, inline_terms=k)
    check_outputs(S, prog, nodes, outs, vals, interpret(S, prog, vals), 1e-13)
    if k >= 2:
        assert prog.info["n_ops"] < base.info["n_ops"] and prog.info["n_levels"] <= base.info["n_levels"]
    with pytest.raises(S.SscoError):
        build_expr(S, nodes).compile(outs, inline_terms=17)


def test_shared_leaf_values_halve_the_symmetric_square(S):
    """The cotangent Laplacian as one leaf whose (u, v) and (v, u) entries
    share a value (the paper's L is symmetric): structural hashing then finds
    (L L)_uv and (L L)_vu identical, so L^2 stores only its lower triangle;
    L^3 through the same leaf matches the oracle."""
    p = P.trigrid_problem(12, batch=2, cfg=3)
    rp, ci, vm, nv = P.symmetric_laplacian_leaf(p)
    n = p.n
    ends = np.asarray(p.colind).reshape(p.m, 2)
    vals = np.zeros((2, nv))
    for b in range(2):
        w = p.vals[b]
        d = np.zeros(n)
        np.add.at(d, ends[:, 0], w)
        np.add.at(d, ends[:, 1], w)
        vals[b] = np.concatenate([-w, d])
    leaf = ("leaf", n, n, rp, ci, vm, nv)
    sq = build_expr(S, [leaf, ("mul", 0, 0)]).compile([1], batch=2)
    r, c, rp2, ci2 = sq.output_pattern(0)
    lower = sum(int(np.sum(ci2[rp2[i]:rp2[i + 1]] <= i)) for i in range(r))
    assert sq.info["n_ops"] == lower and sq.info["n_leaf_vals"] == nv
    check_outputs(S, sq, [leaf, ("mul", 0, 0)], [1], vals, interpret(S, sq, vals), 1e-13)
    nodes = [leaf, ("mul", 0, 0), ("mul", 1, 0)]
    cube = build_expr(S, nodes).compile([2], batch=2)
    check_outputs(S, cube, nodes, [2], vals, interpret(S, cube, vals), 1e-13)
    plain = build_expr(S, [("leaf", n, n, rp, ci), ("mul", 0, 0), ("mul", 1, 0)]).compile([2])
    assert cube.info["n_ops"] < plain.info["n_ops"]
    with pytest.raises(S.SscoError):
        build_expr(S, [("leaf", n, n, rp, ci, vm, nv - 1)]).compile([0])   # vmap out of range


def test_expr_program_save_load(S, tmp_path):
    """A compiled program survives its file unchanged (info, every table,
    output patterns); damaged, truncated or padded files are refused."""
    nodes, outs, nv = random_expressions(40, 70, per_row=3)
    prog = build_expr(S, nodes).compile(outs, batch=3, dtype=torch.float32, inline_terms=2)
    f = str(tmp_path / "prog.bin")
    prog.save(f)
    q = S.ExprProgram.load(f)
    assert q.info == prog.info and q.n_out == prog.n_out == len(outs) and q.dtype == torch.float32
    for w in range(7):
        assert np.array_equal(q.export(w), prog.export(w))
    for k in range(len(outs)):
        for a, b in zip(q.output_pattern(k), prog.output_pattern(k)):
            assert np.array_equal(a, b)
    raw = open(f, "rb").read()
    mid = len(raw) // 2
    bad = [b"garbage!" + raw[8:], raw[:mid] + bytes([raw[mid] ^ 1]) + raw[mid + 1:], raw[:-3], raw + b"\0"]
    bad += [raw[:o] + b"\xff" * 8 + raw[o + 8:] for o in range(12, 120, 4)]
    for i, blob in enumerate(bad):
        g = str(tmp_path / f"bad{i}.bin")
        open(g, "wb").write(blob)
        with pytest.raises(S.SscoError) as ei:
            S.ExprProgram.load(g)
        assert ei.value.status == 1


def _fnv1a64(data: bytes) -> int:
    h = 0xcbf29ce484222325
    for c in data:
        h = ((h ^ c) * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


def _parse_program_file(raw: bytes):
    """Splits a program file into its header fields and tables (the layout
    written by ssco_expr_save) so that a test can change one field and
    re-digest the file, which the digest alone would otherwise refuse."""
    import struct
    off = 0
    hdr = {}
    for name, fmt in [("magic", "<Q"), ("ver", "<I"), ("B", "<i"), ("precision", "<i"), ("unit_coef", "<i"),
                      ("n_leaf_vals", "<q"), ("n_out_vals", "<q"), ("n_slots", "<q"), ("n_ops", "<q"),
                      ("n_terms", "<q"), ("n_unrolled", "<q")]:
        hdr[name] = struct.unpack_from(fmt, raw, off)[0]
        off += struct.calcsize(fmt)
    vecs = {}
    for name, dt in [("lvl_begin", np.int64), ("term_off", np.int64), ("f1", np.int32), ("f2", np.int32),
                     ("coef", np.float64), ("out_slot", np.int32), ("out_coef", np.float64)]:
        n = struct.unpack_from("<Q", raw, off)[0]
        off += 8
        vecs[name] = np.frombuffer(raw, dt, n, off).copy()
        off += n * np.dtype(dt).itemsize
    tail = raw[off:-8]     # output patterns, unchanged
    return hdr, vecs, tail


def _write_program_file(hdr, vecs, tail) -> bytes:
    import struct
    body = b"".join(struct.pack(fmt, hdr[name]) for name, fmt in [
        ("magic", "<Q"), ("ver", "<I"), ("B", "<i"), ("precision", "<i"), ("unit_coef", "<i"),
        ("n_leaf_vals", "<q"), ("n_out_vals", "<q"), ("n_slots", "<q"), ("n_ops", "<q"), ("n_terms", "<q"),
        ("n_unrolled", "<q")])
    for name in ["lvl_begin", "term_off", "f1", "f2", "coef", "out_slot", "out_coef"]:
        v = vecs[name]
        body += struct.pack("<Q", v.size) + v.tobytes()
    body += tail
    return body + struct.pack("<Q", _fnv1a64(body))


def test_expr_program_load_rejects_redigested_bad_tables(S, tmp_path):
    """The digest only detects damage: a file whose digest was recomputed
    after a field was changed must still be refused when its tables could
    make the runner read or write outside its buffers (negative counts or
    offsets, a level that reads its own or a later level's outputs)."""
    nodes, outs, nv = random_expressions(30, 50, per_row=3)
    prog = build_expr(S, nodes).compile(outs, batch=2)
    f = str(tmp_path / "prog.bin")
    prog.save(f)
    raw = open(f, "rb").read()
    hdr, vecs, tail = _parse_program_file(raw)
    assert _write_program_file(hdr, vecs, tail) == raw          # the parser reproduces the file
    assert hdr["n_ops"] > 0 and vecs["lvl_begin"].size >= 3

    def refused(h, v):
        g = str(tmp_path / "bad.bin")
        open(g, "wb").write(_write_program_file(h, v, tail))
        with pytest.raises(S.SscoError) as ei:
            S.ExprProgram.load(g)
        assert ei.value.status == 1

    def mod(**kw):
        h, v = dict(hdr), {k: a.copy() for k, a in vecs.items()}
        for k, val in kw.items():
            if k in h:
                h[k] = val
            else:
                v[k] = val
        return h, v

    # a negative leaf count with a slot count that still adds up
    refused(*mod(n_leaf_vals=-1, n_slots=hdr["n_ops"]))
    refused(*mod(n_out_vals=-1))
    # no ops and an empty term offset table (no .back() of an empty vector)
    refused(*mod(n_ops=-1, n_slots=hdr["n_leaf_vals"], term_off=np.zeros(0, np.int64),
                 lvl_begin=np.array([0, -1], np.int64)))
    refused(*mod(n_terms=-1))
    # level and term tables that start below zero
    lb = vecs["lvl_begin"].copy()
    lb[0] = -1
    refused(*mod(lvl_begin=lb))
    to = vecs["term_off"].copy()
    to[0] = -1
    refused(*mod(term_off=to))
    # a term of level 0 that reads an op slot (its own level's output)
    f1 = vecs["f1"].copy()
    f1[0] = 1 + hdr["n_leaf_vals"]
    refused(*mod(f1=f1))
    # a term of the last level that reads the last level's own first slot
    lvl = vecs["lvl_begin"]
    q_last = vecs["term_off"][lvl[-2]]
    f2 = vecs["f2"].copy()
    f2[q_last] = 1 + hdr["n_leaf_vals"] + lvl[-2]
    refused(*mod(f2=f2))


def test_expr_compile_rejects_malformed_nodes(S):
    rp, ci = np.array([0, 2, 3]), np.array([0, 1, 1])
    ok = ("leaf", 2, 2, rp, ci)
    cases = [
        ([("leaf", 2, 2, rp, np.array([1, 0, 1]))], [0], 2),          # columns not increasing
        ([("leaf", 2, 2, rp, np.array([0, 2, 1]))], [0], 2),          # column out of range
        ([ok, ("leaf", 3, 2, np.array([0, 1, 2, 3]), np.array([0, 1, 0])), ("add", 0, 1)], [2], 1),  # shapes
        ([ok, ("leaf", 3, 2, np.array([0, 1, 2, 3]), np.array([0, 1, 0])), ("mul", 0, 1)], [2], 1),
        ([ok, ("scale", 0, float("nan"))], [1], 4),
        ([ok], [1], 1),                                                # output id out of range
    ]
    for nodes, outs, status in cases:
        with pytest.raises(S.SscoError) as ei:
            build_expr(S, nodes).compile(outs)
        assert ei.value.status == status, nodes
    with pytest.raises(S.SscoError):
        build_expr(S, [ok]).compile([0], batch=0)


# ---------------------------------------------------------------------------
# device runner (GPU)
# ---------------------------------------------------------------------------
@pytest.mark.gpu
@pytest.mark.parametrize("dtype,B", [(torch.float64, 1), (torch.float64, 40), (torch.float32, 3)])
def test_expr_random_expressions_on_device(S, dtype, B):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nodes, outs, nv = random_expressions(1000, 64 + B)
    prog = build_expr(S, nodes).compile(outs, batch=B, dtype=dtype).bind()
    vals = np.random.default_rng(65).standard_normal((B, nv))
    if dtype == torch.float32:
        vals = vals.astype(np.float32).astype(np.float64)   # the oracle sees the same inputs
    got = prog.run(torch.tensor(vals, dtype=dtype, device="cuda")).double().cpu().numpy()
    sel = [0, B - 1] if B > 2 else list(range(B))
    check_outputs(S, prog, nodes, outs, vals[sel], got[sel], 1e-13 if dtype == torch.float64 else 3e-5)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_expr_cotan_laplacian_cube_on_device(S, dtype):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = P.trigrid_problem(24, batch=8, cfg=3)
    nodes, outs = cotan_laplacian_cube(p)
    prog = build_expr(S, nodes).compile(outs, batch=8, dtype=dtype).bind()
    vals = cotan_leaf_vals(p, 8)
    if dtype == torch.float32:
        vals = vals.astype(np.float32).astype(np.float64)
    got = prog.run(torch.tensor(vals, dtype=dtype, device="cuda")).double().cpu().numpy()
    check_outputs(S, prog, nodes, outs, vals[[0, 7]], got[[0, 7]], 1e-13 if dtype == torch.float64 else 3e-5)


@pytest.mark.gpu
def test_full_cotan_laplacian_cube_200k_sampled_rows(S):
    """L^3 of the cotangent Laplacian of a 448 x 448 triangulated grid
    (200,704 vertices; the paper's largest structured product), FP32, one
    value set, in the bench's form: a first program builds L = A^T (W A) on
    the device, the timed program takes L as its leaf and forms (L L) L.
    Sampled rows against the oracle's lazy row evaluation of the whole chain
    from A and w, and the zero row sums that every Laplacian power has."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = P.trigrid_problem(448, batch=1, cfg=3)
    lnodes, l_id, lvals = P.laplacian_expression(p)
    lvals = lvals[:1].astype(np.float32).astype(np.float64)
    lprog = build_expr(S, lnodes).compile([l_id], batch=1, dtype=torch.float32).bind()
    Ld = lprog.run(torch.tensor(lvals, dtype=torch.float32, device="cuda"))
    n, _, lrp, lci = lprog.output_pattern(0)
    cube = P.power_expression(n, lrp, lci, 3)
    prog = build_expr(S, cube).compile([len(cube) - 1], batch=1, dtype=torch.float32).bind()
    got = prog.run(Ld).double().cpu().numpy()[0]
    nodes, outs = cotan_laplacian_cube(p)
    vals = lvals
    r, c, rp, ci = prog.output_pattern(0)
    rows = np.random.default_rng(66).choice(r, 200, replace=False)
    ref = O.expr_eval_rows(nodes, vals[0], outs[0], rows)
    absvals = np.abs(vals[0])
    ref_abs = O.expr_eval_rows(nodes, absvals, outs[0], rows)
    for i in rows:
        cols = ci[rp[i]:rp[i + 1]]
        assert list(cols) == sorted(ref[i])
        want = np.array([ref[i][j] for j in cols])
        scale = np.array([ref_abs[i][j] for j in cols])
        assert np.all(np.abs(got[rp[i]:rp[i + 1]] - want) <= 3e-5 * scale)
    rs = np.add.reduceat(got, rp[:-1]) if got.size else got
    ra = np.add.reduceat(np.abs(got), rp[:-1])
    assert np.all(np.abs(rs) <= 1e-4 * ra)
