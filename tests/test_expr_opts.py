"""The optional steps of the sparse-expression compiler (ssco_expr_compile_opts):
algebraic hashing (Sec. 4.1.2, App. A), factorization and constant (zero)
expressions (App. D), and the global decomposition thresholds t_ref / t_compl
(Sec. 4.2.1).  Compiled tables are interpreted on the CPU and compared with
the oracle's evaluation by the definitions; the device runs them in the GPU
cases at the end."""
import numpy as np
import pytest
import torch

from paper_2110_12865_gb300 import problems as P
from tests.test_expr import build_expr, check_outputs, interpret, random_expressions


@pytest.fixture(scope="module")
def S():
    from paper_2110_12865_gb300 import build
    build.build()
    from paper_2110_12865_gb300 import ssco
    return ssco


def scalar_leaf():
    """A 1 x 1 leaf: a scalar variable of the paper's symbolic type."""
    return ("leaf", 1, 1, np.array([0, 1], np.int64), np.array([0], np.int32))


def rand_leaf(rng, r, c, per_row):
    from tests.test_oracle_pins import _rand_csr
    return ("leaf", r, c, *_rand_csr(rng, r, c, per_row))


def n_vals(nodes):
    return sum(int(nd[6]) if len(nd) > 5 and nd[5] is not None else int(nd[3][-1])
               for nd in nodes if nd[0] == "leaf")


def lower_count(prog, k):
    r, c, rp, ci = prog.output_pattern(k)
    return sum(int(np.sum(ci[rp[i]:rp[i + 1]] <= i)) for i in range(r))


# ---------------------------------------------------------------------------
# algebraic hashing
# ---------------------------------------------------------------------------
def test_algebraic_hash_equates_the_papers_example(S):
    """Sec. 4.1.2: 2 (x + y)(z + w) and 2xz + (2z + 2w) y + xw + wx have the
    same algebraic hash although their trees differ.  Built as 1 x 1
    matrices, the second is a chain of stored sums of stored products; with
    algebraic hashing its last sum is recognised as the first expression's
    product (factor 2), so both outputs read one slot with one factor.
    Without it they stay apart.  Values against the oracle either way."""
    x, y, z, w = 0, 1, 2, 3
    nodes = [scalar_leaf() for _ in range(4)] + [
        ("add", x, y), ("add", z, w), ("mul", 4, 5), ("scale", 6, 2.0),          # 4..7: E1
        ("scale", x, 2.0), ("mul", 8, z),                                         # 8, 9: 2x z
        ("scale", z, 2.0), ("scale", w, 2.0), ("add", 10, 11), ("mul", 12, y),    # 10..13: (2z + 2w) y
        ("mul", x, w), ("mul", w, x),                                             # 14, 15: xw, wx
        ("add", 9, 13), ("add", 16, 14), ("add", 17, 15)]                         # 16..18: E2
    outs = [7, 18]
    vals = np.random.default_rng(1).standard_normal((3, 4))
    plain = build_expr(S, nodes).compile(outs, batch=3)
    alg = build_expr(S, nodes).compile(outs, batch=3, algebraic=True)
    for prog in (plain, alg):
        check_outputs(S, prog, nodes, outs, vals, interpret(S, prog, vals), 1e-13)
    ps, pc = plain.export(S.EXPR_EXPORT_OUT_SLOT), plain.export(S.EXPR_EXPORT_OUT_COEF)
    s, c = alg.export(S.EXPR_EXPORT_OUT_SLOT), alg.export(S.EXPR_EXPORT_OUT_COEF)
    assert ps[0] != ps[1]
    assert s[0] == s[1] and c[0] == c[1] == 2.0
    # two merges: the last sum is 2 (x + y)(z + w), and 2z + 2w is 2 (z + w)
    assert alg.info["n_alg_merged"] == 2 and alg.info["n_ops"] == plain.info["n_ops"] - 2


def test_algebraic_hash_keeps_different_polynomials_apart(S):
    """(x + y)(z + w) and (x + y)(z - w), x y and x z, x^2 and x y: close in
    structure, different as polynomials -- no merge, values exact."""
    x, y, z, w = 0, 1, 2, 3
    nodes = [scalar_leaf() for _ in range(4)] + [
        ("add", x, y), ("add", z, w), ("scale", w, -1.0), ("add", z, 6),          # 4..7
        ("mul", 4, 5), ("mul", 4, 7), ("mul", x, y), ("mul", x, z), ("mul", x, x)]   # 8..12
    outs = [8, 9, 10, 11, 12]
    alg = build_expr(S, nodes).compile(outs, algebraic=True)
    plain = build_expr(S, nodes).compile(outs)
    assert alg.info["n_ops"] == plain.info["n_ops"] and alg.info["n_alg_merged"] == 0
    assert len(set(alg.export(S.EXPR_EXPORT_OUT_SLOT))) == len(outs)
    vals = np.random.default_rng(2).standard_normal((1, 4))
    check_outputs(S, alg, nodes, outs, vals, interpret(S, alg, vals), 1e-13)


def test_algebraic_hash_finds_multiples_negations_and_zeros(S):
    """On random sparse matrices: (2A)(B + C) equals 2 (AB + AC) and is
    stored once (factor 1 after the scale); (-A) B is -(AB); and
    (A + B) C - AC - BC is zero in every entry (no slot, exactly 0).
    Values against the oracle."""
    rng = np.random.default_rng(3)
    n = 30
    A, B, C = (rand_leaf(rng, n, n, 3) for _ in range(3))
    nodes = [A, B, C,
             ("scale", 0, 2.0), ("add", 1, 2), ("mul", 3, 4),                   # 3..5: (2A)(B + C)
             ("mul", 0, 1), ("mul", 0, 2), ("add", 6, 7), ("scale", 8, 2.0),    # 6..9: 2 (AB + AC)
             ("scale", 0, -1.0), ("mul", 10, 1),                                # 10, 11: (-A) B
             ("add", 0, 1), ("mul", 12, 2), ("mul", 1, 2),                      # 12..14: (A + B) C, BC
             ("scale", 7, -1.0), ("scale", 14, -1.0), ("add", 13, 15), ("add", 17, 16)]   # 15..18: (A+B)C - AC - BC
    outs = [5, 9, 11, 6, 18]
    vals = rng.standard_normal((2, n_vals(nodes)))
    alg = build_expr(S, nodes).compile(outs, batch=2, algebraic=True)
    got = interpret(S, alg, vals)
    check_outputs(S, alg, nodes, outs, vals, got, 1e-13)
    sl, co = alg.export(S.EXPR_EXPORT_OUT_SLOT), alg.export(S.EXPR_EXPORT_OUT_COEF)
    sizes = [int(alg.output_pattern(k)[2][-1]) for k in range(len(outs))]
    off = np.concatenate([[0], np.cumsum(sizes)])
    part = lambda a, k: a[off[k]:off[k + 1]]
    assert np.array_equal(part(sl, 0), part(sl, 1)) and np.array_equal(part(co, 0), part(co, 1))
    assert np.array_equal(part(sl, 2), part(sl, 3)) and np.all(part(co, 2) == -part(co, 3))
    assert sizes[4] > 0 and np.all(part(co, 4) == 0.0) and np.all(got[:, off[4]:off[5]] == 0.0)
    # the zeros come from merges ((A + B) C - AC is found equal to BC, and
    # BC - BC cancels); the plain tables store the difference
    assert alg.info["n_alg_merged"] > 0
    plain = build_expr(S, nodes).compile(outs, batch=2)
    assert alg.info["n_ops"] < plain.info["n_ops"]
    assert np.any(part(plain.export(S.EXPR_EXPORT_OUT_COEF), 4) != 0.0)


def test_algebraic_hash_stores_half_of_the_symmetric_cube(S):
    """The cotangent Laplacian as a symmetric leaf (one value per edge and
    per vertex): L^2 and L^3 are symmetric polynomials, so (L^3)_ij and
    (L^3)_ji -- structurally different sums -- get equal keys, and with
    algebraic hashing each unordered pair is stored once at both levels
    (structural hashing alone halves only L^2)."""
    p = P.trigrid_problem(12, batch=2, cfg=3)
    rp, ci, vm, nv = P.symmetric_laplacian_leaf(p)
    n = p.n
    leaf = ("leaf", n, n, rp, ci, vm, nv)
    nodes = [leaf, ("mul", 0, 0), ("mul", 1, 0)]
    vals = np.random.default_rng(4).standard_normal((2, nv))
    plain = build_expr(S, nodes).compile([1, 2], batch=2)
    alg = build_expr(S, nodes).compile([1, 2], batch=2, algebraic=True)
    check_outputs(S, alg, nodes, [1, 2], vals, interpret(S, alg, vals), 1e-13)
    assert plain.info["n_ops"] == lower_count(plain, 0) + int(plain.output_pattern(1)[2][-1])
    assert alg.info["n_ops"] == lower_count(alg, 0) + lower_count(alg, 1)


def test_algebraic_hash_on_random_expressions_matches_oracle(S):
    """The paper's three random-matrix expressions: algebraic hashing stores
    no more than structural hashing and the tables still match the oracle."""
    nodes, outs, nv = random_expressions(60, 5)
    vals = np.random.default_rng(6).standard_normal((2, nv))
    plain = build_expr(S, nodes).compile(outs, batch=2)
    alg = build_expr(S, nodes).compile(outs, batch=2, algebraic=True)
    assert alg.info["n_ops"] <= plain.info["n_ops"]
    check_outputs(S, alg, nodes, outs, vals, interpret(S, alg, vals), 1e-13)


def test_algebraic_zero_of_a_local_sum(S):
    """A sum that cancels only as a whole: with local sums (inline_terms) the
    chain (x + y)^2 - x^2 - 2xy - y^2 reaches the output as one linear
    combination of four stored products, which algebraic hashing finds to be
    zero (no slot; the entry is exactly 0).  Without it the combination is
    stored and evaluates to rounding noise."""
    x, y = 0, 1
    nodes = [scalar_leaf(), scalar_leaf(),
             ("add", x, y), ("mul", 2, 2),                                       # 2, 3: (x + y)^2
             ("mul", x, x), ("mul", x, y), ("mul", y, y),                        # 4..6
             ("scale", 4, -1.0), ("scale", 5, -2.0), ("scale", 6, -1.0),          # 7..9
             ("add", 3, 7), ("add", 10, 8), ("add", 11, 9)]                      # 10..12
    vals = np.random.default_rng(7).standard_normal((2, 2))
    alg = build_expr(S, nodes).compile([12], batch=2, inline_terms=16, algebraic=True)
    plain = build_expr(S, nodes).compile([12], batch=2, inline_terms=16)
    assert alg.info["n_alg_zero"] >= 1
    assert alg.export(S.EXPR_EXPORT_OUT_COEF)[0] == 0.0 and np.all(interpret(S, alg, vals) == 0.0)
    assert plain.info["n_ops"] == alg.info["n_ops"] + 1
    check_outputs(S, plain, nodes, [12], vals, interpret(S, plain, vals), 1e-13)


# ---------------------------------------------------------------------------
# factorization
# ---------------------------------------------------------------------------
def test_factorization_takes_a_shared_factor_out(S):
    """App. D on D B where each row of D shares one value (a leaf whose
    entries of row i all take value d_i): every product of entry (i, j) of
    D B has d_i as a factor, so factorization stores the partners' sum (the
    entries of B met by row i's pattern in column j) as a linear expression
    and leaves one product d_i s_ij per entry.  Products of two slots drop
    either way; the table shrinks when the partners' sums are shared --
    here when every row of D has one pattern, so s_ij depends on j alone
    and hashing stores it once for all rows.  With factor_min above the
    number of shared products nothing changes.  Values against the
    oracle."""
    rng = np.random.default_rng(8)
    n = 40
    from tests.test_oracle_pins import _rand_csr
    Bm = rand_leaf(rng, n, n, 4)
    rp, ci = _rand_csr(rng, n, n, 6)
    cols = np.sort(rng.choice(n, 30, replace=False)).astype(np.int32)
    for name, (drp, dci) in (("random rows", (rp, ci)),
                             ("one row pattern", (np.arange(n + 1, dtype=np.int64) * 30, np.tile(cols, n)))):
        row_of = np.repeat(np.arange(n), np.diff(drp)).astype(np.int64)
        D = ("leaf", n, n, drp, dci, row_of, n)
        nodes = [D, Bm, ("mul", 0, 1)]
        vals = rng.standard_normal((2, n_vals(nodes)))
        plain = build_expr(S, nodes).compile([2], batch=2)
        fac = build_expr(S, nodes).compile([2], batch=2, factor_min=2)
        check_outputs(S, fac, nodes, [2], vals, interpret(S, fac, vals), 1e-13)
        two = lambda prog: int(np.sum(prog.export(S.EXPR_EXPORT_F2) > 0))
        assert fac.info["n_factored"] > 0 and two(fac) < two(plain), name
        if name == "one row pattern":
            assert fac.info["n_terms"] < plain.info["n_terms"] // 2
        big = build_expr(S, nodes).compile([2], batch=2, factor_min=64)
        assert big.info["n_factored"] == 0 and big.info["n_terms"] == plain.info["n_terms"]


def test_factorization_regathers_inlined_sums(S):
    """With local sums, (A + B) C expands into a c + b c products per entry;
    factorization takes c out again and stores (a + b) once per entry of
    A + B, which gives the stored-sum tables' product count back.  Random
    expressions with both options against the oracle."""
    rng = np.random.default_rng(9)
    n = 40
    A, Bm, C = (rand_leaf(rng, n, n, 3) for _ in range(3))
    nodes = [A, Bm, C, ("add", 0, 1), ("mul", 3, 2)]
    vals = rng.standard_normal((1, n_vals(nodes)))
    stored = build_expr(S, nodes).compile([4])
    expanded = build_expr(S, nodes).compile([4], inline_terms=2)
    fac = build_expr(S, nodes).compile([4], inline_terms=2, factor_min=2)
    assert expanded.info["n_terms"] > stored.info["n_terms"]
    assert fac.info["n_terms"] == stored.info["n_terms"]
    check_outputs(S, fac, nodes, [4], vals, interpret(S, fac, vals), 1e-13)
    rn, routs, nv = random_expressions(50, 10, per_row=4)
    rv = np.random.default_rng(11).standard_normal((2, nv))
    both = build_expr(S, rn).compile(routs, batch=2, inline_terms=4, factor_min=2, algebraic=True)
    check_outputs(S, both, rn, routs, rv, interpret(S, both, rv), 1e-13)


# ---------------------------------------------------------------------------
# global decomposition (t_ref, t_compl)
# ---------------------------------------------------------------------------
def test_global_decomposition_inlines_small_and_single_use_sums(S):
    """Sec. 4.2.1: ((A + B) + C) + D feeding a product.  The inner sums are
    each referenced once, so with t_ref = 2 they are substituted into the
    next sum and only the full four-term sum is stored (one level instead of
    three before the product).  With t_compl = 8 the full sum (4 terms) is
    substituted into the product as well, which then has more products and
    no sum below it.  Outputs are never substituted.  Values against the
    oracle in every form."""
    rng = np.random.default_rng(12)
    n = 40
    A, Bm, C, Dm = (rand_leaf(rng, n, n, 12) for _ in range(4))   # dense enough to overlap four times
    E = rand_leaf(rng, n, n, 3)
    nodes = [A, Bm, C, Dm, E, ("add", 0, 1), ("add", 5, 2), ("add", 6, 3), ("mul", 7, 4)]
    outs = [8, 7]
    vals = rng.standard_normal((2, n_vals(nodes)))
    plain = build_expr(S, nodes).compile(outs, batch=2)
    ref2 = build_expr(S, nodes).compile(outs, batch=2, t_ref=2)
    cpl = build_expr(S, nodes).compile([8], batch=2, t_ref=2, t_compl=8)
    for prog, o in ((plain, outs), (ref2, outs), (cpl, [8])):
        check_outputs(S, prog, nodes, o, vals, interpret(S, prog, vals), 1e-13)
    assert plain.info["n_levels"] == 4 and ref2.info["n_levels"] == 2 and cpl.info["n_levels"] == 1
    assert ref2.info["n_inlined"] > 0 and ref2.info["n_ops"] < plain.info["n_ops"]
    # the products: the same expressions, more terms once the sum is substituted
    nl, nl_terms = nonlinear(S, ref2)
    assert cpl.info["n_ops"] == nl and cpl.info["n_terms"] > nl_terms
    assert nonlinear(S, cpl)[0] == cpl.info["n_ops"]          # no stored sum is left
    # ref2's sum output is still stored (an output is never substituted)
    assert ref2.info["n_ops"] - nl > 0


def nonlinear(S, prog):
    """(stored expressions with a product of two slots, their terms)."""
    toff = prog.export(S.EXPR_EXPORT_TERM_OFF)
    f2 = prog.export(S.EXPR_EXPORT_F2)
    seg = np.repeat(np.arange(len(toff) - 1), np.diff(toff))
    has = np.zeros(len(toff) - 1, bool)
    has[seg[f2 > 0]] = True
    return int(has.sum()), int(np.diff(toff)[has].sum())


def test_global_decomposition_keeps_shared_intermediates(S):
    """A sum referenced by many products (every entry of (A + B) is used by
    the whole row of the product) stays stored at t_ref = 2, t_compl = 2;
    the tables equal the plain ones.  The paper's random expressions with
    t_ref = 2 against the oracle."""
    rng = np.random.default_rng(13)
    n = 40
    A, Bm, C = (rand_leaf(rng, n, n, 4) for _ in range(3))
    nodes = [A, Bm, C, ("add", 0, 1), ("mul", 3, 2)]
    plain = build_expr(S, nodes).compile([4])
    dec = build_expr(S, nodes).compile([4], t_ref=2, t_compl=2)
    assert dec.info["n_inlined"] == 0
    for w in range(7):
        assert np.array_equal(dec.export(w), plain.export(w)), w
    rn, routs, nv = random_expressions(50, 14, per_row=4)
    rv = np.random.default_rng(15).standard_normal((2, nv))
    for opts in (dict(t_ref=2), dict(t_ref=2, t_compl=3, algebraic=True, factor_min=2)):
        prog = build_expr(S, rn).compile(routs, batch=2, **opts)
        check_outputs(S, prog, rn, routs, rv, interpret(S, prog, rv), 1e-13)


def test_compile_options_out_of_range_are_refused(S):
    rng = np.random.default_rng(16)
    nodes = [rand_leaf(rng, 5, 5, 2), ("mul", 0, 0)]
    for bad in (dict(algebraic=2), dict(factor_min=1), dict(factor_min=-1), dict(t_ref=-1), dict(t_compl=-2)):
        with pytest.raises(S.SscoError) as ei:
            build_expr(S, nodes).compile([1], **bad)
        assert ei.value.status == 1, bad


# ---------------------------------------------------------------------------
# device runner (GPU): the same tables format, so the same kernels
# ---------------------------------------------------------------------------
@pytest.mark.gpu
@pytest.mark.parametrize("dtype,B", [(torch.float64, 3), (torch.float32, 1)])
def test_expr_options_on_device(S, dtype, B):
    """The paper's random expressions compiled with every optional step
    (algebraic hashing, factorization, global decomposition, local sums) run
    on the device against the oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nodes, outs, nv = random_expressions(800, 17 + B, per_row=4)
    prog = build_expr(S, nodes).compile(outs, batch=B, dtype=dtype, inline_terms=2, algebraic=True,
                                        factor_min=2, t_ref=2, t_compl=3).bind()
    vals = np.random.default_rng(18).standard_normal((B, nv))
    if dtype == torch.float32:
        vals = vals.astype(np.float32).astype(np.float64)
    got = prog.run(torch.tensor(vals, dtype=dtype, device="cuda")).double().cpu().numpy()
    check_outputs(S, prog, nodes, outs, vals, got, 1e-13 if dtype == torch.float64 else 3e-5)


def symmetric_cube_inputs(S, side, dev):
    """L built on the device by the L = A^T (W A) program, then gathered into
    the symmetric leaf's values (one per edge and per vertex)."""
    p = P.trigrid_problem(side, batch=1, cfg=3)
    lnodes, l_id, lvals = P.laplacian_expression(p)
    lvals = lvals[:1].astype(np.float32).astype(np.float64)
    lprog = build_expr(S, lnodes).compile([l_id], batch=1, dtype=torch.float32).bind()
    Ld = lprog.run(torch.tensor(lvals, dtype=torch.float32, device=dev))
    n, _, lrp, lci = lprog.output_pattern(0)
    srp, sci, svm, snv = P.symmetric_laplacian_leaf(p)
    assert np.array_equal(srp, lrp) and np.array_equal(sci, lci)
    rep = np.zeros(snv, np.int64)
    rep[svm[::-1]] = np.arange(svm.size)[::-1]
    Ls = Ld[:, torch.tensor(rep, device=dev)].contiguous()
    return p, lvals, Ld, Ls, (n, srp, sci, svm, snv)


@pytest.mark.gpu
@pytest.mark.parametrize("side", [24, 448])
def test_symmetric_cube_with_algebraic_hashing_on_device(S, side):
    """L^3 of the cotangent Laplacian with L as a symmetric leaf and
    algebraic hashing (each mirror pair of L^2 and L^3 stored once), FP32,
    one value set: at 24 x 24 every entry against the oracle; at 448 x 448
    (200,704 vertices, the bench's size) 200 sampled rows against the
    oracle's lazy row evaluation of the whole chain from A and w, and every
    entry against the plain-leaf program's output."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import oracle as O
    from tests.test_expr import cotan_laplacian_cube
    p, lvals, Ld, Ls, (n, srp, sci, svm, snv) = symmetric_cube_inputs(S, side, "cuda")
    snodes = [("leaf", n, n, srp, sci, svm, snv), ("mul", 0, 0), ("mul", 1, 0)]
    prog = build_expr(S, snodes).compile([2], batch=1, dtype=torch.float32, algebraic=True).bind()
    assert prog.info["n_alg_merged"] > 0
    got = prog.run(Ls).double().cpu().numpy()[0]
    r, c, rp, ci = prog.output_pattern(0)
    if side <= 32:
        check_outputs(S, prog, snodes, [2], Ls.double().cpu().numpy(), got[None], 3e-5)
        return
    plain = build_expr(S, P.power_expression(n, srp, sci, 3)).compile([2], batch=1, dtype=torch.float32).bind()
    ref_dev = plain.run(Ld).double().cpu().numpy()[0]
    assert np.max(np.abs(got - ref_dev)) <= 1e-5 * np.max(np.abs(ref_dev))
    nodes, outs = cotan_laplacian_cube(p)
    rows = np.random.default_rng(19).choice(r, 200, replace=False)
    ref = O.expr_eval_rows(nodes, lvals[0], outs[0], rows)
    ref_abs = O.expr_eval_rows(nodes, np.abs(lvals[0]), outs[0], rows)
    for i in rows:
        cols = ci[rp[i]:rp[i + 1]]
        assert list(cols) == sorted(ref[i])
        want = np.array([ref[i][j] for j in cols])
        scale = np.array([ref_abs[i][j] for j in cols])
        assert np.all(np.abs(got[rp[i]:rp[i + 1]] - want) <= 3e-5 * scale)
