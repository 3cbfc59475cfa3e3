"""Host-side arithmetic of the bench (no GPU): the step roofline's
algorithmic bytes, checked against a count written out by hand."""
import numpy as np
import pytest

from paper_2110_12865_gb300 import build as B
from paper_2110_12865_gb300 import problems as P


@pytest.fixture(scope="module")
def S():
    B.build()
    from paper_2110_12865_gb300 import ssco
    return ssco


def test_step_bytes_of_the_arap_pattern_match_a_hand_count(S):
    """The 128 x 128 triangulated grid (the batched workload's main pattern):
    n = 16,384, m = 48,641 weights, z_K = 65,025, z_L = 502,242.  At one
    correction (I = 1), FP64 weights and an FP32 factor, one value set moves
    48,641*8 + 2*65,025*8 + 502,242*4 + 2*2*502,242*4 + 65,025*8 + 7*16,384*8
    = 12,912,072 bytes.  The bytes beyond that are the update matrices
    (written and read) and the dense panels' explicit zeros."""
    import bench
    pl = S.Plan(P.trigrid_problem(128, batch=2, cfg=3), precision=S.FP32_REFINE, batch=2)
    i = pl.info
    assert (i["n"], i["m"], i["nnz_K"], i["nnz_L"]) == (16384, 48641, 65025, 502242)
    per_set = 48641 * 8 + 2 * 65025 * 8 + 502242 * 4 + 2 * 2 * 502242 * 4 + 65025 * 8 + 7 * 16384 * 8
    assert per_set == 12_912_072
    alg, upd, pad, imean = bench.step_bytes([pl], [{"iters": np.ones(2, np.int32)}], 8)
    assert alg == 2 * per_set and imean == 1.0
    assert upd == 2 * 2 * i["update_entries"] * 4
    assert pad == 2 * (i["panel_entries"] - i["nnz_L"]) * 4
    # linear in the corrections: 0 and 2 for the two value sets move what
    # 1 and 1 do; 2 and 2 add one SpMV, two sweeps and three vectors per set
    alg02, _, _, _ = bench.step_bytes([pl], [{"iters": np.array([0, 2], np.int32)}], 8)
    assert alg02 == alg
    alg22, _, _, imean2 = bench.step_bytes([pl], [{"iters": np.array([2, 2], np.int32)}], 8)
    assert imean2 == 2.0
    assert alg22 - alg == 2 * (2 * 502242 * 4 + 65025 * 8 + 3 * 16384 * 8)
