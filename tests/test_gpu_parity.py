"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (FP64 path): K entries 1e-14 relative to max|K|; L columns
||dL_j|| <= 1e-12 ||L_j||; relative residual ||b - K x|| / ||b|| <= 1e-10
with the oracle's K.  FP32 + refinement: the same residual bound; the error
against the oracle's FP64 solution is reported and bounded by
kappa-scaled limits.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2110_12865_gb300 import problems as P

pytestmark = pytest.mark.gpu

RESID_TOL = 1e-10


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_12865_gb300 import build
    build.build()
    from paper_2110_12865_gb300 import ssco
    return ssco


def run(S, probs, precision, batch=None, **kw):
    probs_l = probs if isinstance(probs, list) else [probs]
    B = batch if batch is not None else probs_l[0].batch
    pl = S.Plan(probs, precision=precision, batch=B, **kw).bind()
    vals = np.concatenate([np.asarray(p.vals[:B]) for p in probs_l], axis=1)
    shift = np.stack([np.asarray(p.shift[:B], np.float64) for p in probs_l], axis=1).reshape(-1)
    b = np.concatenate([p.b[:B] for p in probs_l], axis=1)
    vt = torch.tensor(vals, device="cuda")
    pl.numeric(vt, torch.tensor(shift, device="cuda"))
    x = pl.solve(torch.tensor(b, device="cuda")).cpu().numpy()
    st = pl.status()
    return pl, x, st, vals, shift, b


def check_against_oracle(S, pl, p, x, st, inst, sys_index, col_off=0, exact_L=True, check_K=True):
    r = O.refactor_solve(p, inst)
    n = p.n
    xi = x[inst, col_off:col_off + n] if x.ndim == 2 else x
    res = np.linalg.norm(O.symv(r.K, xi) - p.b[inst]) / np.linalg.norm(p.b[inst])
    assert st["status"][sys_index] == 0, (st, sys_index)
    assert res <= RESID_TOL, res
    assert st["resid"][sys_index] <= RESID_TOL
    err = np.linalg.norm(xi - r.x) / np.linalg.norm(r.x)
    return r, res, err


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kw", [{}, {"small_front_max": 32}, {"amalgamate": 0}, {"tiny_front_max": -1},
                                {"tiny_front_max": 8, "small_front_max": 40}])
def test_fp64_grid32_L_entries(S, kw):
    p = P.workload("grid32")
    pl, x, st, *_ = run(S, p, S.FP64, **kw)
    r, res, err = check_against_oracle(S, pl, p, x, st, 0, 0)
    K = pl.export_K()[0]
    assert np.max(np.abs(K - r.Kp.val)) <= 1e-14 * np.abs(r.Kp.val).max()
    L = pl.export_L()[0]
    Lc = r.S.Lcolptr
    for j in range(p.n):
        a, b = Lc[j], Lc[j + 1]
        assert np.linalg.norm(L[a:b] - r.L[a:b]) <= 1e-12 * np.linalg.norm(r.L[a:b]), j
    assert err < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kw", [{}, {"small_front_max": 32}, {"tiny_front_max": -1}])
def test_elasticity_small(S, prec, kw):
    p = P.elasticity_problem(6, cfg=2)
    precision = S.FP64 if prec == "fp64" else S.FP32_REFINE
    pl, x, st, *_ = run(S, p, precision, **kw)
    r, res, err = check_against_oracle(S, pl, p, x, st, 0, 0)
    K = pl.export_K()[0]
    assert np.max(np.abs(K - r.Kp.val)) <= 1e-14 * np.abs(r.Kp.val).max()
    if prec == "fp64":
        L = pl.export_L()[0]
        Lc = r.S.Lcolptr
        colerr = max(np.linalg.norm(L[Lc[j]:Lc[j + 1]] - r.L[Lc[j]:Lc[j + 1]]) /
                     np.linalg.norm(r.L[Lc[j]:Lc[j + 1]]) for j in range(p.n))
        assert colerr <= 1e-12
        assert err < 1e-10
    else:
        assert st["iters"][0] >= 1
        assert err < 1e-8


@pytest.mark.parametrize("tc", [0, 2, -1])
def test_fp32_factor_accuracy_big_fronts(S, tc):
    """FP32 factor through the multi-CTA path, updates on tcgen05 tensor
    cores (3xTF32; tc=0: one CTA per tile, tc=2: wide trailing updates in
    persistent CTAs with two TMEM accumulators) or SIMT FP32 (tc=-1): every
    column of L must
    agree with the FP64 oracle to FP32-level accuracy (plain TF32, ~1e-3,
    would fail), and the refined solution to the FP64 residual bound."""
    p = P.elasticity_problem(7, cfg=2)
    pl, x, st, *_ = run(S, p, S.FP32_REFINE, small_front_max=32, tensor_cores=tc)
    assert pl.info["tune_use_tc"] == {0: 1, 2: 2, -1: 0}[tc]
    r, res, err = check_against_oracle(S, pl, p, x, st, 0, 0)
    L = pl.export_L()[0]
    Lc = r.S.Lcolptr
    worst = max(np.linalg.norm(L[Lc[j]:Lc[j + 1]] - r.L[Lc[j]:Lc[j + 1]]) / np.linalg.norm(r.L[Lc[j]:Lc[j + 1]])
                for j in range(p.n))
    assert worst <= 2e-4, worst


def test_fp32_tensor_core_factor_entries_elast24(S):
    """The FP32 factor of the 24^3 elasticity system through the multi-CTA
    tcgen05 path at full size: fronts span many 128 x 128 tensor-core tiles
    in both dimensions (widths beyond 256 columns, so the narrow in-block
    updates and the wide trailing updates both run, with ragged tile edges),
    and every column of L agrees with the FP64 oracle to FP32-level
    accuracy (the same 2e-4 per-column bound as the small-case test)."""
    p = P.elasticity_problem(24, batch=1, cfg=2)
    pl, x, st, *_ = run(S, p, S.FP32_REFINE)
    widths = np.diff(pl.export(S.EXPORT_FRONT_FIRST))
    assert pl.info["tune_use_tc"] == 1 and widths.max() > 256 and pl.info["max_front_rows"] > 1024
    r, res, err = check_against_oracle(S, pl, p, x, st, 0, 0)
    L = pl.export_L()[0]
    Lc = r.S.Lcolptr
    num = np.sqrt(np.add.reduceat((L - r.L) ** 2, Lc[:-1]))
    den = np.sqrt(np.add.reduceat(r.L ** 2, Lc[:-1]))
    assert np.max(num / den) <= 2e-4, np.max(num / den)


@pytest.mark.parametrize("big_panel", [32, 96, 256])
def test_big_panel_blocks_fp64_L_entries(S, big_panel):
    """Multi-CTA fronts factored in panel blocks of 32, 96 or 256 columns
    (narrow in-block updates plus one trailing update per block): FP64
    entries of L within 1e-12 per column of the oracle's for every block
    width."""
    p = P.elasticity_problem(9, cfg=2)
    pl, x, st, *_ = run(S, p, S.FP64, small_front_max=32, big_panel=big_panel)
    assert pl.info["tune_big_panel"] == big_panel
    r, res, err = check_against_oracle(S, pl, p, x, st, 0, 0)
    L = pl.export_L()[0]
    Lc = r.S.Lcolptr
    colerr = max(np.linalg.norm(L[Lc[j]:Lc[j + 1]] - r.L[Lc[j]:Lc[j + 1]]) / np.linalg.norm(r.L[Lc[j]:Lc[j + 1]])
                 for j in range(p.n))
    assert colerr <= 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fused_big_front_steps_give_the_same_factor(S, prec):
    """Big fronts with the diagonal block of each 32-column step factored
    inside the trsm launch (ssco_set_flow bit 3): two patterns of different
    front widths, two value sets each, panel blocks of 96 columns -- the
    factor equals the separate-potrf factor bit for bit (same arithmetic),
    the solve meets the residual bound, and in FP64 L matches the oracle to
    1e-12 per column.  A non-positive pivot inside a fused step is reported
    at the same column as without fusion."""
    probs = [P.elasticity_problem(9, batch=2, cfg=2), P.elasticity_problem(6, batch=2, cfg=2)]
    precision = S.FP64 if prec == "fp64" else S.FP32_REFINE
    pl, x, st, vals, shift, b = run(S, probs, precision, small_front_max=32, big_panel=96)
    assert pl.info["tune_flow"] & 8 == 0 and pl.info["max_front_rows"] > 128
    L0 = pl.export_L()
    pl.set_flow(pl.info["tune_flow"] | 8)
    assert pl.info["tune_flow"] & 8
    pl.numeric(torch.tensor(vals, device="cuda"), torch.tensor(shift, device="cuda"))
    x1 = pl.solve(torch.tensor(b, device="cuda")).cpu().numpy()
    st1 = pl.status()
    assert np.array_equal(pl.export_L(), L0)
    assert np.array_equal(x1, x) and np.all(st1["status"] == 0)
    off = 0
    for k, p in enumerate(probs):
        for inst in range(2):
            r, *_ = check_against_oracle(S, pl, p, x1, st1, inst, inst * 2 + k, col_off=off)
            if prec == "fp64" and k == 0:
                Lc = r.S.Lcolptr
                L = pl.export_L()[inst]
                colerr = max(np.linalg.norm(L[Lc[j]:Lc[j + 1]] - r.L[Lc[j]:Lc[j + 1]])
                             / np.linalg.norm(r.L[Lc[j]:Lc[j + 1]]) for j in range(p.n))
                assert colerr <= 1e-12
        off += p.n
    # an indefinite shift for system 0: minus twice the Rayleigh quotient of
    # a smooth displacement (an upper bound of the smallest eigenvalue), so
    # K + shift I has a negative eigenvalue and the factorization must fail
    p0 = probs[0]
    K0 = O.refactor_solve(p0, 0).K
    v = np.tile([1.0, 0.0, 0.0], p0.n // 3) * np.linspace(1.0, 2.0, p0.n) * O.shifted_mask(p0)
    bad_shift = shift.copy()
    bad_shift[0] = shift[0] - 2.0 * float(v @ O.symv(K0, v)) / float(v @ v)
    ref = O.refactor_solve(p0, 0, shift=bad_shift[0])
    assert ref.bad >= 0
    got = []
    for flow in (pl.info["tune_flow"] | 8, pl.info["tune_flow"] & 7):
        pl.set_flow(flow)
        pl.numeric(torch.tensor(vals, device="cuda"), torch.tensor(bad_shift, device="cuda"))
        pl.solve(torch.tensor(b, device="cuda"))
        got.append(pl.status())
    for g in got:
        assert g["status"][0] == 3 and g["bad_col"][0] == ref.bad
        assert np.all(g["status"][1:] == 0)


def test_two_value_sets_per_cta_for_larger_classes(S):
    """FP32 small-front classes of 128 and 160 rows factored two value sets
    per CTA (vec2_max_cls = 160), with an odd batch so that the last CTA of
    every front holds one value set: the factor agrees with the
    one-value-set-per-CTA factor to FP32 rounding and the solves meet the
    residual bound against the oracle's K."""
    p = P.trigrid_problem(96, batch=5, cfg=3)
    pl0, x0, st0, *_ = run(S, p, S.FP32_REFINE)
    pl1, x1, st1, *_ = run(S, p, S.FP32_REFINE, vec2_max_cls=160)
    assert pl0.info["tune_vec2_max_cls"] == 0 and pl1.info["tune_vec2_max_cls"] == 160
    assert pl1.info["max_front_rows"] > 128
    L0, L1 = pl0.export_L(), pl1.export_L()
    assert np.max(np.abs(L1 - L0)) <= 1e-5 * np.max(np.abs(L0))
    for inst in (0, 3, 4):
        check_against_oracle(S, pl1, p, x1, st1, inst, inst)
    with pytest.raises(S.SscoError):
        S.Plan(p, precision=S.FP32_REFINE, vec2_max_cls=100)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_split_solves_uneven_patterns(S, prec):
    """Multi-CTA split solves (split_rows far below the largest fronts, so
    fronts of several widths, one with more than one 256-column block, share
    the split launches of a level) over three patterns of uneven size, two
    value sets each: every system meets the residual bound, and in FP64 the
    solution equals the one-CTA-per-front solve's to 1e-12."""
    probs = [P.elasticity_problem(10, batch=2), P.elasticity_problem(5, batch=2), P.grid_problem(24, 20, batch=2)]
    precision = S.FP64 if prec == "fp64" else S.FP32_REFINE
    pl, x, st, *_ = run(S, probs, precision, small_front_max=32, split_rows=40)
    assert pl.info["max_front_rows"] > 256
    off = 0
    for k, p in enumerate(probs):
        for inst in range(2):
            check_against_oracle(S, pl, p, x, st, inst, inst * 3 + k, col_off=off)
        off += p.n
    if prec == "fp64":
        _, x_ref, st_ref, *_ = run(S, probs, precision, small_front_max=32, split_rows=-1)
        assert np.all(st_ref["status"] == 0)
        assert np.max(np.abs(x - x_ref)) <= 1e-12 * np.max(np.abs(x_ref))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_warp_per_front_small_fronts(S, prec):
    """Warp-per-front factorization of the small-front classes (forced with
    warp_front_max on a 256 x 256 grid, whose lowest levels hold thousands
    of fronts): FP64 L entries within 1e-12 per column of the oracle's and
    the same solution as the one-CTA-per-front kernel; FP32 within the
    residual bound."""
    p = P.workload("grid256")
    precision = S.FP64 if prec == "fp64" else S.FP32_REFINE
    pl, x, st, *_ = run(S, p, precision, warp_front_max=64, tiny_front_max=8)
    assert pl.info["tune_warp_front_max"] == 64
    r, res, err = check_against_oracle(S, pl, p, x, st, 0, 0)
    if prec == "fp64":
        L = pl.export_L()[0]
        Lc = r.S.Lcolptr
        colerr = max(np.linalg.norm(L[Lc[j]:Lc[j + 1]] - r.L[Lc[j]:Lc[j + 1]]) /
                     np.linalg.norm(r.L[Lc[j]:Lc[j + 1]]) for j in range(p.n))
        assert colerr <= 1e-12
        _, x_ref, *_ = run(S, p, precision, tiny_front_max=8)
        assert np.max(np.abs(x - x_ref)) <= 1e-12 * np.max(np.abs(x_ref))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cluster_solves_uneven_patterns(S, prec):
    """Cluster solves (one 8-CTA cluster per front and value set, rows dealt
    to the CTAs in 32-row chunks, y and partial dot products exchanged
    through distributed shared memory) forced on every big front of three
    uneven patterns, two value sets each: the residual bound for every
    system, and in FP64 the one-CTA-per-front solve's solution to 1e-12."""
    probs = [P.elasticity_problem(10, batch=2), P.elasticity_problem(5, batch=2), P.grid_problem(24, 20, batch=2)]
    precision = S.FP64 if prec == "fp64" else S.FP32_REFINE
    pl, x, st, *_ = run(S, probs, precision, small_front_max=32, split_rows=-1, cluster_rows=40)
    assert pl.info["tune_cluster_rows"] == 40
    off = 0
    for k, p in enumerate(probs):
        for inst in range(2):
            check_against_oracle(S, pl, p, x, st, inst, inst * 3 + k, col_off=off)
        off += p.n
    if prec == "fp64":
        _, x_ref, st_ref, *_ = run(S, probs, precision, small_front_max=32, split_rows=-1, cluster_rows=-1)
        assert np.all(st_ref["status"] == 0)
        assert np.max(np.abs(x - x_ref)) <= 1e-12 * np.max(np.abs(x_ref))


def test_cotan_weights_on_device_match_oracle(S):
    """Cotangent weights built on the device from vertex positions (value
    construction upstream of assembly): bit-identical to the oracle's for
    every value set of a 128 x 128 ARAP pattern (plain IEEE operations, at
    most two terms per edge), and the refactor + solve they feed equals the
    one fed with host-built weights."""
    p = P.trigrid_problem(128, batch=4, cfg=3)
    tri = torch.tensor(p.faces, device="cuda")
    te = torch.tensor(p.opp, device="cuda")
    w = S.cotan_weights(tri, te, torch.tensor(p.positions, device="cuda"), p.m)
    wh = w.cpu().numpy()
    for i in range(4):
        assert np.array_equal(wh[i], O.cotan_weights(p.faces, p.opp, p.positions[i], p.m))
    pl = S.Plan(p, precision=S.FP32_REFINE, batch=4).bind()
    sh = torch.tensor(p.shift[:4], device="cuda")
    b = torch.tensor(p.b[:4], device="cuda")
    pl.numeric(w, sh)
    x1 = pl.solve(b).cpu().numpy()
    pl.numeric(torch.tensor(p.vals[:4], device="cuda"), sh)
    x2 = pl.solve(b).cpu().numpy()
    assert np.array_equal(x1, x2)
    assert np.all(pl.status()["status"] == 0)
    # out-of-range ids are skipped on the device (never dereferenced) and reported
    bad = te.clone()
    bad[5, 1] = p.m + 7
    with pytest.raises(S.SscoError):
        S.cotan_weights(tri, bad, torch.tensor(p.positions, device="cuda"), p.m)


@pytest.mark.parametrize("seed", range(6))
def test_fp64_random_patterns(S, seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(1, 500))
    p = P.random_spd_pattern(n, int(rng.integers(0, 4 * n + 1)), rng, batch=2)
    pl, x, st, *_ = run(S, p, S.FP64, small_front_max=int(rng.choice([0, 32, 64])))
    for inst in range(2):
        r, res, err = check_against_oracle(S, pl, p, x, st, inst, inst)
        L = pl.export_L()[inst]
        Lc = r.S.Lcolptr
        for j in range(n):
            a, b = Lc[j], Lc[j + 1]
            assert np.linalg.norm(L[a:b] - r.L[a:b]) <= 1e-12 * np.linalg.norm(r.L[a:b])


def test_fp32_batched_trigrid(S):
    p = P.trigrid_problem(24, batch=8, cfg=3)
    pl, x, st, *_ = run(S, p, S.FP32_REFINE)
    for inst in range(8):
        check_against_oracle(S, pl, p, x, st, inst, inst)
    assert np.all(st["iters"] >= 1)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_warp_per_item_solves(S, prec):
    """B = 64 value sets: the low levels take the warp-per-item solve kernels,
    the top levels the CTA kernels; both must agree with the oracle."""
    p = P.trigrid_problem(40, batch=64, cfg=3)
    precision = S.FP64 if prec == "fp64" else S.FP32_REFINE
    pl, x, st, *_ = run(S, p, precision)
    assert np.all(st["status"] == 0)
    for inst in (0, 31, 63):
        r, res, err = check_against_oracle(S, pl, p, x, st, inst, inst)
        assert err < (1e-12 if prec == "fp64" else 1e-8)


@pytest.mark.parametrize("prec,B", [("fp64", 5), ("fp32", 7)])
def test_instance_vectorized_fronts_ragged_batch(S, prec, B):
    """Small fronts are factored V value sets per CTA (V = 2 FP64, 4 FP32);
    a batch that is not a multiple of V leaves a partial group."""
    p = P.trigrid_problem(24, batch=B, cfg=3)
    precision = S.FP64 if prec == "fp64" else S.FP32_REFINE
    pl, x, st, *_ = run(S, p, precision)
    assert np.all(st["status"] == 0)
    L = pl.export_L() if prec == "fp64" else None
    for inst in range(B):
        r, res, err = check_against_oracle(S, pl, p, x, st, inst, inst)
        if L is not None:
            Lc = r.S.Lcolptr
            for j in range(0, p.n, 7):
                a, b = Lc[j], Lc[j + 1]
                assert np.linalg.norm(L[inst, a:b] - r.L[a:b]) <= 1e-12 * np.linalg.norm(r.L[a:b])


def test_multi_pattern_uneven(S):
    probs = [P.trigrid_problem(s, 1, cfg=3, seed_offset=100 + k) for k, s in enumerate([5, 11, 17, 23, 30, 9])]
    pl, x, st, *_ = run(S, probs, S.FP32_REFINE, batch=1)
    off = 0
    for k, p in enumerate(probs):
        check_against_oracle(S, pl, p, x, st, 0, k, col_off=off)
        off += p.n


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_many_big_fronts_one_plan(S, prec):
    """Many concurrent multi-CTA fronts (24 large grids in one plan): every
    CTA of a launch must read only what no other CTA of it writes."""
    sides = list(range(170, 257, 4))
    probs = [P.trigrid_problem(s, 1, cfg=3, seed_offset=300 + k) for k, s in enumerate(sides)]
    precision = S.FP64 if prec == "fp64" else S.FP32_REFINE
    pl, x, st, *_ = run(S, probs, precision, batch=1, small_front_max=96)
    assert np.all(st["status"] == 0), st
    assert np.all(st["resid"] <= RESID_TOL)
    off = 0
    for k, p in enumerate(probs):
        if k in (0, len(probs) - 1):
            check_against_oracle(S, pl, p, x, st, 0, k, col_off=off)
        off += p.n


def test_batch_and_patterns_combined(S):
    probs = [P.grid_problem(6, 5, batch=3, cfg=1), P.elasticity_problem(2, batch=3, cfg=2)]
    pl, x, st, *_ = run(S, probs, S.FP64, batch=3)
    for inst in range(3):
        off = 0
        for k, p in enumerate(probs):
            check_against_oracle(S, pl, p, x, st, inst, inst * 2 + k, col_off=off)
            off += p.n


def test_not_spd_reports_first_column(S):
    rng = np.random.default_rng(21)
    found = 0
    for t in range(10):
        p = P.random_spd_pattern(60, 80, rng, batch=1)
        p["vals"] = rng.uniform(-0.3, 2.0, (1, p.m))
        p["shift"] = np.array([-0.05])
        r = O.refactor_solve(p)
        pl, x, st, *_ = run(S, p, S.FP64)
        if r.bad >= 0:
            found += 1
            assert st["status"][0] == 3 and st["bad_col"][0] == r.bad
        else:
            assert st["bad_col"][0] == -1
    assert found >= 3


def test_nonfinite_values_flagged(S):
    p = P.grid_problem(8, 8, batch=2, cfg=1)
    p["vals"] = p.vals.copy()
    p.vals[1, 5] = np.nan
    pl, x, st, *_ = run(S, p, S.FP32_REFINE)
    assert st["status"][0] == 0
    assert st["status"][1] != 0


def test_deterministic_and_host_e2e(S):
    p = P.trigrid_problem(20, batch=3, cfg=3)
    pl, x1, st, vals, shift, b = run(S, p, S.FP32_REFINE)
    pl.numeric(torch.tensor(vals, device="cuda"), torch.tensor(shift, device="cuda"))
    x2 = pl.solve(torch.tensor(b, device="cuda")).cpu().numpy()
    assert np.array_equal(x1, x2)
    x3 = pl.refactor_solve_host(np.ascontiguousarray(vals), np.ascontiguousarray(shift), np.ascontiguousarray(b))
    assert np.array_equal(x1, x3)
    assert pl.last_launch_count() > 0


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_graph_run_matches_eager(S, prec):
    """ssco_graph_run (numeric + solve captured once, refinement loop as a
    conditional WHILE node) gives bit-identical results to the eager calls,
    replays correctly, and re-captures when the pointers change."""
    probs = [P.trigrid_problem(20, batch=3, cfg=3), P.grid_problem(9, 7, batch=3, cfg=1)]
    precision = S.FP64 if prec == "fp64" else S.FP32_REFINE
    pl, x_eager, st_e, vals, shift, b = run(S, probs, precision, batch=3)
    v = torch.tensor(vals, device="cuda")
    sh = torch.tensor(shift, device="cuda")
    bt = torch.tensor(b, device="cuda")
    x = torch.empty_like(bt)
    for _ in range(3):
        x.fill_(float("nan"))
        pl.graph_run(v, sh, bt, x)
        assert np.array_equal(x.cpu().numpy(), x_eager)
    st = pl.status()
    assert np.array_equal(st["iters"], st_e["iters"]) and np.all(st["status"] == 0)
    # new right-hand side in a new buffer: re-capture
    b2 = torch.tensor(np.random.default_rng(5).standard_normal(b.shape), device="cuda")
    x2 = torch.empty_like(b2)
    pl.graph_run(v, sh, b2, x2)
    ref = pl.solve(b2)
    assert np.array_equal(x2.cpu().numpy(), ref.cpu().numpy())
    off = 0
    xh = x2.cpu().numpy()
    for k, p in enumerate(probs):
        K = O.assemble(p, 1)
        res = np.linalg.norm(O.symv(K, xh[1, off:off + p.n]) - b2.cpu().numpy()[1, off:off + p.n])
        assert res <= RESID_TOL * np.linalg.norm(b2.cpu().numpy()[1, off:off + p.n])
        off += p.n


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_graph_run_many_matches_single_graphs(S, prec):
    """Several plans as ONE captured graph (ssco_graph_run_many: a batched
    pattern and a plan of uneven patterns, each with its own refinement loop
    as a branch) give bit-identical results to each plan's own graph and to
    the eager calls, replay correctly, and re-capture when a pointer changes
    or a plan's knobs change."""
    precision = S.FP64 if prec == "fp64" else S.FP32_REFINE
    items = [(P.trigrid_problem(20, batch=6, cfg=3), 6),
             ([P.trigrid_problem(s, 1, cfg=3, seed_offset=k) for k, s in enumerate([9, 14, 21])], 1)]
    plans, ins, ref = [], [], []
    for item, B in items:
        pl, x_eager, st, vals, shift, b = run(S, item, precision, batch=B)
        plans.append(pl)
        ins.append([torch.tensor(a, device="cuda") for a in (vals, shift, b)] +
                   [torch.empty((B, pl.n), dtype=torch.float64, device="cuda")])
        ref.append((x_eager, st["iters"]))
    for rep in range(3):
        for t in ins:
            t[3].fill_(float("nan"))
        S.graph_run_many(plans, [t[0] for t in ins], [t[1] for t in ins], [t[2] for t in ins], [t[3] for t in ins])
        for pl, t, (xe, it) in zip(plans, ins, ref):
            assert np.array_equal(t[3].cpu().numpy(), xe)
            st = pl.status()
            assert np.all(st["status"] == 0) and np.array_equal(st["iters"], it)
    # a plan's knobs change (its graphs are released): the group re-captures
    plans[1].set_flow(0)
    S.graph_run_many(plans, [t[0] for t in ins], [t[1] for t in ins], [t[2] for t in ins], [t[3] for t in ins])
    xs = [t[3].cpu().numpy() for t in ins]
    for pl, t, x in zip(plans, ins, xs):
        single = torch.empty_like(t[3])
        pl.graph_run(t[0], t[1], t[2], single)
        assert np.array_equal(single.cpu().numpy(), x)
    with pytest.raises(S.SscoError):
        S.graph_run_many([plans[0], plans[0]], [ins[0][0]] * 2, [ins[0][1]] * 2, [ins[0][2]] * 2,
                         [ins[0][3], ins[0][3].clone()])
    # the dataflow choices tuned on the multi-plan graph (ssco_autotune_many):
    # every plan keeps valid settings and the tuned graph solves every system
    ms, flows = S.autotune_many(plans, [t[0] for t in ins], [t[1] for t in ins], [t[2] for t in ins],
                                [t[3] for t in ins], reps=2)
    assert ms > 0 and len(flows) == 2 and all(0 <= f < 16 for f in flows)
    for t in ins:
        t[3].fill_(float("nan"))
    S.graph_run_many(plans, [t[0] for t in ins], [t[1] for t in ins], [t[2] for t in ins], [t[3] for t in ins])
    for pl, t, (xe, it) in zip(plans, ins, ref):
        st = pl.status()
        assert np.all(st["status"] == 0) and np.all(st["resid"] <= RESID_TOL)
        assert np.max(np.abs(t[3].cpu().numpy() - xe)) <= 1e-9 * np.max(np.abs(xe))
    with pytest.raises(S.SscoError):
        S.autotune_many(plans, [t[0] for t in ins], [t[1] for t in ins], [t[2] for t in ins],
                        [t[3] for t in ins], reps=0)


def test_autotune_keeps_parity_and_persists(S, tmp_path):
    p = P.trigrid_problem(24, batch=16, cfg=3)
    pl, x0, st0, vals, shift, b = run(S, p, S.FP32_REFINE)
    v, sh, bt = (torch.tensor(a, device="cuda") for a in (vals, shift, b))
    x = torch.empty_like(bt)
    ms, knobs = pl.autotune(v, sh, bt, x, reps=2)
    assert ms > 0 and pl.info["tuned"] == 1
    assert knobs["tune_vec_max_cls"] in (0, 64, 96) and knobs["tune_solve_threads_big"] in (256, 512)
    assert knobs["tune_vec2_max_cls"] in (0, 128, 160)
    pl.graph_run(v, sh, bt, x)
    st = pl.status()
    xh = x.cpu().numpy()
    for inst in (0, 15):
        check_against_oracle(S, pl, p, xh, st, inst, inst)
    f = str(tmp_path / "tuned.bin")
    pl.save(f)
    q = S.Plan.load(f, precision=S.FP32_REFINE)
    assert all(q.info[k] == pl.info[k] for k in knobs) and q.info["tuned"] == 1


def test_plan_file_roundtrip_runs(S, tmp_path):
    p = P.elasticity_problem(4, cfg=2)
    pl0 = S.Plan(p, precision=S.FP32_REFINE)
    f = str(tmp_path / "p.bin")
    pl0.save(f)
    pl = S.Plan.load(f, precision=S.FP32_REFINE).bind()
    pl.numeric(torch.tensor(p.vals, device="cuda"), torch.tensor(p.shift, device="cuda"))
    x = pl.solve(torch.tensor(p.b, device="cuda")).cpu().numpy()
    check_against_oracle(S, pl, p, x, pl.status(), 0, 0)


# ---------------------------------------------------------------------------
# adjoint
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_gradient_matches_oracle(S, prec):
    p = P.grid_problem(16, 16, batch=2, cfg=4)
    precision = S.FP64 if prec == "fp64" else S.FP32_REFINE
    pl, x, st, vals, shift, b = run(S, p, precision)
    xt = torch.tensor(x, device="cuda")
    xbar = 2.0 * (xt - torch.tensor(p.xstar, device="cuda"))
    vbar, sbar, bbar = pl.backward(xt, xbar)
    vbar, sbar, bbar = vbar.cpu().numpy(), sbar.cpu().numpy(), bbar.cpu().numpy()
    for inst in range(2):
        r = O.refactor_solve(p, inst)
        gv, gs, gb = O.backward(p, r, 2.0 * (r.x - p.xstar[inst]), inst)
        tol = 1e-9 if prec == "fp64" else 1e-7
        assert np.max(np.abs(vbar[inst] - gv)) <= tol * np.abs(gv).max()
        assert abs(sbar[inst] - gs) <= tol * abs(gs)
        assert np.max(np.abs(bbar[inst] - gb)) <= tol * np.abs(gb).max()


def test_gradient_elasticity(S):
    p = P.elasticity_problem(3, cfg=2)
    p["xstar"] = np.random.default_rng(2).standard_normal((1, p.n)) * 1e-4
    pl, x, st, *_ = run(S, p, S.FP64)
    xt = torch.tensor(x, device="cuda")
    xbar = 2.0 * (xt - torch.tensor(p.xstar, device="cuda"))
    vbar, _, _ = pl.backward(xt, xbar)
    r = O.refactor_solve(p)
    gv, _, _ = O.backward(p, r, 2.0 * (r.x - p.xstar[0]))
    assert np.max(np.abs(vbar.cpu().numpy()[0] - gv)) <= 1e-9 * np.abs(gv).max()


def test_autograd_function(S):
    p = P.grid_problem(12, 10, batch=1, cfg=4)
    pl = S.Plan(p, precision=S.FP64).bind()
    w = torch.tensor(p.vals, device="cuda", requires_grad=True)
    s = torch.tensor(p.shift, device="cuda", requires_grad=True)
    b = torch.tensor(p.b, device="cuda", requires_grad=True)
    x = S.ssco_solve(pl, w, s, b)
    loss = ((x - torch.tensor(p.xstar, device="cuda")) ** 2).sum()
    loss.backward()
    r = O.refactor_solve(p)
    gv, gs, gb = O.backward(p, r, 2.0 * (r.x - p.xstar[0]))
    assert np.max(np.abs(w.grad.cpu().numpy()[0] - gv)) <= 1e-9 * np.abs(gv).max()
    assert abs(s.grad.item() - gs) <= 1e-9 * abs(gs)
    assert np.max(np.abs(b.grad.cpu().numpy()[0] - gb)) <= 1e-9 * np.abs(gb).max()


# ---------------------------------------------------------------------------
# full-size configurations (the bench's launch configuration)
# ---------------------------------------------------------------------------
def test_full_grid32_fp64(S):
    p = P.workload("grid32")
    pl, x, st, *_ = run(S, p, S.FP64)
    check_against_oracle(S, pl, p, x, st, 0, 0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_elast24(S, prec):
    p = P.workload("elast24")
    precision = S.FP64 if prec == "fp64" else S.FP32_REFINE
    pl, x, st, *_ = run(S, p, precision)
    r, res, err = check_against_oracle(S, pl, p, x, st, 0, 0)
    if prec == "fp64":
        L = pl.export_L()[0]
        rng = np.random.default_rng(0)
        Lc = r.S.Lcolptr
        for j in rng.choice(p.n, 2000, replace=False):
            a, b = Lc[j], Lc[j + 1]
            assert np.linalg.norm(L[a:b] - r.L[a:b]) <= 1e-12 * np.linalg.norm(r.L[a:b])


def test_full_arap128_batch256(S):
    p = P.workload("arap128")
    pl, x, st, *_ = run(S, p, S.FP32_REFINE)
    assert np.all(st["status"] == 0) and np.all(st["resid"] <= RESID_TOL)
    for inst in [0, 77, 255]:
        K = O.assemble(p, inst)
        res = np.linalg.norm(O.symv(K, x[inst]) - p.b[inst]) / np.linalg.norm(p.b[inst])
        assert res <= RESID_TOL


def test_full_grid256_gradient(S):
    p = P.workload("grid256")
    pl, x, st, *_ = run(S, p, S.FP64)
    r, res, err = check_against_oracle(S, pl, p, x, st, 0, 0)
    xt = torch.tensor(x, device="cuda")
    xbar = 2.0 * (xt - torch.tensor(p.xstar, device="cuda"))
    vbar, sbar, bbar = pl.backward(xt, xbar)
    gv, gs, gb = O.backward(p, r, 2.0 * (r.x - p.xstar[0]))
    vb = vbar.cpu().numpy()[0]
    assert np.max(np.abs(vb - gv)) <= 1e-8 * np.abs(gv).max()


def test_full_uneven64_one_plan(S):
    """The 64 uneven triangulated grids (sides 32..256) of the batched
    workload, one plan, FP32 factor + refinement: every system converges and
    sampled systems meet the residual bound with the oracle's K."""
    ps = P.uneven_trigrids(64)
    pl, x, st, *_ = run(S, ps, S.FP32_REFINE, batch=1)
    assert np.all(st["status"] == 0) and np.all(st["resid"] <= RESID_TOL)
    offs = np.concatenate([[0], np.cumsum([q.n for q in ps])])
    for k in [0, 21, 42, 63]:
        q = ps[k]
        xk = x[0, offs[k]:offs[k + 1]]
        res = np.linalg.norm(O.symv(O.assemble(q, 0), xk) - q.b[0]) / np.linalg.norm(q.b[0])
        assert res <= RESID_TOL, (k, res)


def test_full_elast48_batch16_with_gradient(S):
    """48^3 Kuhn tets x 16 Young's-modulus fields, FP32 factor (tensor-core
    panel updates) + refinement, then the adjoint for every instance.  The
    oracle factor is out of reach at this size, so the checks are properties
    that hold at any size, with the oracle's own assembly: the solution and
    adjoint residuals, and the element gradient -mu_e^T K_e^0 x_e and the
    shift gradient recomputed by the oracle from the device's mu and x."""
    p = P.workload("elast48")
    pl, x, st, *_ = run(S, p, S.FP32_REFINE)
    assert np.all(st["status"] == 0) and np.all(st["resid"] <= RESID_TOL)
    xbar = np.random.default_rng(48).standard_normal(x.shape)
    vbar, sbar, mu = pl.backward(torch.tensor(x, device="cuda"), torch.tensor(xbar, device="cuda"))
    vbar, sbar, mu = vbar.cpu().numpy(), sbar.cpu().numpy(), mu.cpu().numpy()
    mask = O.shifted_mask(p)
    for inst in [0, 15]:
        K = O.assemble(p, inst)
        res = np.linalg.norm(O.symv(K, x[inst]) - p.b[inst]) / np.linalg.norm(p.b[inst])
        assert res <= RESID_TOL, (inst, res)
        res_mu = np.linalg.norm(O.symv(K, mu[inst]) - xbar[inst]) / np.linalg.norm(xbar[inst])
        assert res_mu <= RESID_TOL, (inst, res_mu)
        gv = O.grad_vals(p, mu[inst], x[inst])
        assert np.max(np.abs(vbar[inst] - gv)) <= 1e-11 * np.abs(gv).max()
        gs = -float(np.dot(mu[inst][mask], x[inst][mask]))
        assert abs(sbar[inst] - gs) <= 1e-12 * np.linalg.norm(mu[inst]) * np.linalg.norm(x[inst])


# ---------------------------------------------------------------------------
# element blocks from geometry (ELEM_BLOCKS patterns, ssco_tet_stiffness)
# ---------------------------------------------------------------------------
def _blocks_close(Kd, Ko, rel=1e-12):
    """Per tet: max |device - oracle| <= rel * max |oracle block|."""
    Kd, Ko = Kd.reshape(-1, 78), Ko.reshape(-1, 78)
    return bool(np.all(np.abs(Kd - Ko).max(axis=1) <= rel * np.abs(Ko).max(axis=1)))


def test_tet_stiffness_on_device_match_oracle(S):
    g = P.elasticity_geometry_problem(6, batch=3, cfg=6)
    tets = torch.tensor(g.tets, device="cuda")
    xyz = torch.tensor(g.pos, device="cuda")
    K = S.tet_stiffness(tets, xyz, g.nu, torch.tensor(g.E, device="cuda")).cpu().numpy()
    for i in range(3):
        Ko, bad = O.tet_stiffness(g.tets, g.pos[i], g.E[i], g.nu)
        assert bad == 0 and _blocks_close(K[i], Ko)
    K1 = S.tet_stiffness(tets, xyz[:1], g.nu).cpu().numpy()[0]   # E omitted: unit moduli
    assert _blocks_close(K1, O.tet_stiffness(g.tets, g.pos[0], None, g.nu)[0])
    # an out-of-range vertex id (counted once) and a flat tet (once per value
    # set): reported, their blocks zero, the others untouched
    bt = g.tets[:5].copy()
    bt[1, 2] = g.pos.shape[1]
    bt[3, 3] = bt[3, 0]
    btd = torch.tensor(bt, device="cuda")
    with pytest.raises(S.SscoError) as ei:
        S.tet_stiffness(btd, xyz, g.nu)
    assert "4 bad tets" in str(ei.value)
    Kb = S.tet_stiffness(btd, xyz, g.nu, check=False).cpu().numpy()
    assert np.all(Kb[:, [1, 3]] == 0)
    good = [0, 2, 4]
    for i in range(3):
        assert _blocks_close(Kb[i, good], O.tet_stiffness(bt[good], g.pos[i], None, g.nu)[0])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_element_blocks_pattern_solve_and_gradient(S, prec):
    """An ELEM_BLOCKS plan fed the oracle's blocks: solutions meet the
    residual bound with the oracle's K and the per-entry gradient matches the
    oracle's adjoint; then the device chain geometry -> blocks -> solve gives
    the same solutions (the blocks' layout is the plan's value order)."""
    g = P.elasticity_geometry_problem(4, batch=3, cfg=6)
    B = 3
    precision = S.FP64 if prec == "fp64" else S.FP32_REFINE
    Ko = np.stack([O.tet_stiffness(g.tets, g.pos[i], g.E[i], g.nu)[0].ravel() for i in range(B)])
    pl = S.Plan(g, precision=precision, batch=B).bind()
    zero = torch.zeros(B, dtype=torch.float64, device="cuda")
    bt = torch.tensor(g.b, device="cuda")
    pl.numeric(torch.tensor(Ko, device="cuda"), zero)
    x = pl.solve(bt)
    st = pl.status()
    assert np.all(st["status"] == 0) and np.all(st["resid"] <= RESID_TOL)
    xbar = torch.tensor(np.random.default_rng(5).standard_normal((B, g.n)), device="cuda")
    vbar, sbar, mu = pl.backward(x, xbar)
    xh, vbar = x.cpu().numpy(), vbar.cpu().numpy()
    tol = 1e-9 if prec == "fp64" else 1e-7
    for i in range(B):
        r = O.refactor_solve(g, i, vals=Ko[i], shift=0.0)
        res = np.linalg.norm(O.symv(r.K, xh[i]) - g.b[i]) / np.linalg.norm(g.b[i])
        assert res <= RESID_TOL, (i, res)
        gv, _, _ = O.backward(g, r, xbar[i].cpu().numpy(), i)
        assert np.max(np.abs(vbar[i] - gv)) <= tol * np.abs(gv).max()
    Kd = S.tet_stiffness(torch.tensor(g.tets, device="cuda"), torch.tensor(g.pos, device="cuda"), g.nu,
                         torch.tensor(g.E, device="cuda"))
    pl.numeric(Kd.reshape(B, -1), zero)
    x2 = pl.solve(bt).cpu().numpy()
    st = pl.status()
    assert np.all(st["status"] == 0) and np.all(st["resid"] <= RESID_TOL)
    assert np.linalg.norm(x2 - xh) <= 1e-6 * np.linalg.norm(xh)


def test_full_elastgeo24_blocks_and_refine(S):
    """Full 24^3 mesh (82,944 tets), geometry per call: device blocks against
    the oracle on sampled tets, then FP32 factor + refinement on them."""
    g = P.elasticity_geometry_problem(24, batch=1, cfg=6)
    Kd = S.tet_stiffness(torch.tensor(g.tets, device="cuda"), torch.tensor(g.pos, device="cuda"), g.nu,
                         torch.tensor(g.E, device="cuda"))
    Kh = Kd.cpu().numpy()[0]
    pick = np.random.default_rng(24).choice(g.m, 2000, replace=False)
    Ko, bad = O.tet_stiffness(g.tets[pick], g.pos[0], g.E[0][pick], g.nu)
    assert bad == 0 and _blocks_close(Kh[pick], Ko)
    pl = S.Plan(g, precision=S.FP32_REFINE, batch=1).bind()
    pl.numeric(Kd.reshape(1, -1), torch.zeros(1, dtype=torch.float64, device="cuda"))
    pl.solve(torch.tensor(g.b, device="cuda"))
    st = pl.status()
    assert np.all(st["status"] == 0) and np.all(st["resid"] <= RESID_TOL)


# ---------------------------------------------------------------------------
# dataflow launches (persistent grids walking all levels, per-item done flags)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["uneven_trigrids", "elast_big_fronts", "trigrid_batch"])
def test_dataflow_matches_level_launches(S, prec, case):
    """The default schedule (one persistent launch per factorization size
    group and per solve sweep, items waiting on their children's or parent's
    done flags) against one launch per level and size class (flow=0): the
    factors agree to rounding (per column; blocked panels reorder the sums)
    and both solutions meet the residual bound with the oracle's K."""
    precision = S.FP64 if prec == "fp64" else S.FP32_REFINE
    if case == "uneven_trigrids":
        probs = [P.trigrid_problem(s, 1, cfg=3, seed_offset=k) for k, s in enumerate([9, 17, 23, 31, 40])]
        B, kw = 1, {}
    elif case == "elast_big_fronts":
        probs = [P.elasticity_problem(8, batch=2, cfg=2)]
        B, kw = 2, {"small_front_max": 96}
    else:
        probs = [P.trigrid_problem(20, batch=7, cfg=3)]
        B, kw = 7, {}
    item = probs if len(probs) > 1 else probs[0]
    pl = S.Plan(item, precision=precision, batch=B, **kw).bind()
    assert pl.info["tune_flow"] == 3 and pl.info["flow_fact_fronts"] > 0 and pl.info["flow_solve_fronts"] > 0
    vals = np.concatenate([np.asarray(p.vals[:B]) for p in probs], axis=1)
    shift = np.stack([np.asarray(p.shift[:B], np.float64) for p in probs], axis=1).reshape(-1)
    b = np.concatenate([p.b[:B] for p in probs], axis=1)
    vt, st_, bt = (torch.tensor(a, device="cuda") for a in (vals, shift, b))
    res = {}
    for flow in (0, 3, 4):
        pl.set_flow(flow)
        pl.numeric(vt, st_)
        x = pl.solve(bt).cpu().numpy()
        st = pl.status()
        assert np.all(st["status"] == 0), (flow, st)
        res[flow] = (pl.export_L(), x)
    L0 = res[0][0]
    tol = 1e-12 if prec == "fp64" else 2e-5
    Lc = np.concatenate([[0], np.cumsum(pl.export(S.EXPORT_COLCOUNT))])
    for flow in (3, 4):   # 4: per-level launches with the dataflow kernel's panel core
        off = 0
        for k, p in enumerate(probs):
            for i in range(B):
                xi = res[flow][1][i, off:off + p.n]
                assert np.linalg.norm(O.symv(O.assemble(p, i), xi) - p.b[i]) <= RESID_TOL * np.linalg.norm(p.b[i])
            off += p.n
        # per column of the concatenated factor (exported in CSC order of L)
        Lf = res[flow][0]
        num = np.sqrt(np.add.reduceat((Lf - L0) ** 2, Lc[:-1], axis=1))
        den = np.sqrt(np.add.reduceat(L0 ** 2, Lc[:-1], axis=1))
        assert np.max(num / den) <= tol, (flow, np.max(num / den))


def test_dataflow_wait_timeout_reports_status(S):
    """Bounded waits: with the test hook one item of the first dataflow
    launch waits on a flag that nothing sets; after max_polls polls it gives
    up, the launches end early and every system reports SSCO_ERR_TIMEOUT
    (the device stays usable).  The next call without the hook is correct."""
    p = P.trigrid_problem(24, batch=8, cfg=3)
    pl = S.Plan(p, precision=S.FP32_REFINE).bind()
    vt, st_, bt = (torch.tensor(a, device="cuda") for a in (p.vals, p.shift, p.b))
    for stall in (0, 5):
        pl.set_flow(3, max_polls=2000, stall_item=stall)
        pl.numeric(vt, st_)
        pl.solve(bt)
        st = pl.status()
        assert np.all(st["status"] == 6), st["status"]
    pl.set_flow(3, max_polls=1 << 22, stall_item=-1)
    pl.numeric(vt, st_)
    x = pl.solve(bt).cpu().numpy()
    st = pl.status()
    assert np.all(st["status"] == 0)
    for i in range(p.batch):
        r = O.refactor_solve(p, i)
        assert np.linalg.norm(O.symv(r.K, x[i]) - p.b[i]) <= RESID_TOL * np.linalg.norm(p.b[i])


# ---------------------------------------------------------------------------
# GMRES-IR (refine_mode 1 / 2)
def _ill_conditioned_grid(batch=2):
    """A 16x16 5-point grid Laplacian with the tiny shift 2e-9 (kappa ~ 5e9,
    so kappa * u32 > 1) and right-hand sides b = K x* with seeded x* ~ N(0,1):
    in FP32 the last pivot (about n * shift = 5e-7) is below the rounding
    noise of the elimination, so the FP32 factor is at best a perturbed one
    and plain refinement cannot reach 1e-10 with it (it stagnates, or the
    pivot comes out non-positive), while the FP64 residual floor of this b
    stays near 1e-16."""
    p = P.grid_problem(16, 16, batch=batch, cfg=1, shift=2e-9)
    rng = np.random.default_rng(P.seed_for(7, 0))
    xs = rng.standard_normal((batch, p.n))
    p["b"] = np.stack([O.symv(O.assemble(p, i), xs[i]) for i in range(batch)])
    return p


@pytest.mark.parametrize("mode", [1, 2])
def test_gmres_ir_converges_where_plain_refinement_stagnates(S, mode):
    """Plain refinement fails on the ill-conditioned grid (NO_CONVERGE, or
    NOT_SPD when the FP32 last pivot comes out non-positive); GMRES-IR (every
    correction by FP64 GMRES preconditioned with the FP32 factor, or as the
    fallback after plain refinement stagnated) reaches the 1e-10 residual
    with the oracle's K, and its solution agrees with the oracle's FP64
    solution within the forward-error bound that kappa allows."""
    p = _ill_conditioned_grid()
    vt, st_, bt = (torch.tensor(a, device="cuda") for a in (p.vals, p.shift, p.b))
    plain = S.Plan(p, precision=S.FP32_REFINE).bind()
    plain.numeric(vt, st_)
    plain.solve(bt)
    st0 = plain.status()
    assert np.all((st0["status"] == 5) | (st0["status"] == 3)), st0
    assert np.all(st0["resid"] > 1e-10)
    pl = S.Plan(p, precision=S.FP32_REFINE, refine_mode=mode).bind()
    pl.numeric(vt, st_)
    x = pl.solve(bt).cpu().numpy()
    st = pl.status()
    assert np.all(st["status"] == 0), st
    for i in range(p.batch):
        r = O.refactor_solve(p, i)
        assert np.linalg.norm(O.symv(r.K, x[i]) - p.b[i]) <= RESID_TOL * np.linalg.norm(p.b[i])
        # forward error: at most kappa (~5e9) times the 1e-10 residual; here
        # it sits in the near-null constant mode, far inside that bound
        assert np.linalg.norm(x[i] - r.x) <= 1e-2 * np.linalg.norm(r.x)
    # the graph entry point runs the same (eager) calls for these plans
    x2 = torch.empty_like(bt)
    pl.graph_run(vt, st_, bt, x2)
    assert np.all(pl.status()["status"] == 0)


def test_gmres_ir_on_well_conditioned_batch_matches_plain(S):
    """On an ordinary batched plan GMRES-IR needs at most as many corrections
    as plain refinement and meets the same residual bound."""
    p = P.trigrid_problem(20, batch=5, cfg=3)
    vt, st_, bt = (torch.tensor(a, device="cuda") for a in (p.vals, p.shift, p.b))
    its = {}
    for mode in (0, 1):
        pl = S.Plan(p, precision=S.FP32_REFINE, refine_mode=mode, gmres_restart=8).bind()
        pl.numeric(vt, st_)
        x = pl.solve(bt).cpu().numpy()
        st = pl.status()
        assert np.all(st["status"] == 0)
        its[mode] = st["iters"]
        for i in range(p.batch):
            r = O.refactor_solve(p, i)
            assert np.linalg.norm(O.symv(r.K, x[i]) - p.b[i]) <= RESID_TOL * np.linalg.norm(p.b[i])
    assert np.all(its[1] <= its[0])


def test_fp32_solve_graph_matches_eager_and_recaptures(S):
    """ssco_solve of an FP32 plan runs its refinement loop as a captured
    graph (no host round trip): the result and the per-system iteration
    counts are bit-identical to the host-driven loop (forced here by
    per-launch profiling), for two right-hand-side buffers in turn (the two
    cached graphs) and for a third (a re-capture), the same with graphs
    switched off (ssco_set_flow bit 4), and the adjoint through its own
    cached graph matches its host-driven form."""
    p = P.trigrid_problem(16, batch=4, cfg=3)
    pl = S.Plan(p, precision=S.FP32_REFINE).bind()
    vt, st_ = torch.tensor(p.vals, device="cuda"), torch.tensor(p.shift, device="cuda")
    pl.numeric(vt, st_)
    rng = np.random.default_rng(11)
    bs = [torch.tensor(rng.standard_normal(p.b.shape), device="cuda") for _ in range(3)]
    graph_x, eager_x = [], []
    for rep in range(2):
        for b in bs:
            graph_x.append((pl.solve(b).cpu().numpy(), pl.status()["iters"].copy()))
    pl.profile_enable(1000)
    for b in bs:
        eager_x.append((pl.solve(b).cpu().numpy(), pl.status()["iters"].copy()))
    pl.profile_enable(0)
    for k, (x, it) in enumerate(graph_x):
        xe, ite = eager_x[k % 3]
        assert np.array_equal(x, xe) and np.array_equal(it, ite)
    # ssco_set_flow bit 4: eager launches without profiling, same results
    flow = pl.info["tune_flow"]
    pl.set_flow(flow | 16)
    assert pl.info["tune_flow"] & 16
    for k, b in enumerate(bs):
        assert np.array_equal(pl.solve(b).cpu().numpy(), eager_x[k][0])
        assert pl.last_launch_count() > 3
    pl.set_flow(flow)
    x = pl.solve(bs[0])
    xbar = 2.0 * (x - torch.tensor(rng.standard_normal(p.b.shape), device="cuda"))
    g1 = [t.cpu().numpy() for t in pl.backward(x, xbar)]
    pl.profile_enable(1000)
    g2 = [t.cpu().numpy() for t in pl.backward(x, xbar)]
    pl.profile_enable(0)
    for a, c in zip(g1, g2):
        assert np.array_equal(a, c)
