"""ssco_solve_noalloc: the allocation-free solve for callers that must not
allocate device memory per call (an application whose memory manager owns
all device memory, or a latency-critical loop where cudaMalloc/cudaFree would
synchronize the device).  Its scratch is a static 64 MiB device array; this
file is collected last so that a failure here leaves every other test run.
The result must match ssco_solve (same factor, FP64 direct solve) within the
FP64 parity tolerance on two calls in a row, whether this file runs alone in
a fresh process or after the rest of the suite."""
import numpy as np
import pytest
import torch

from paper_2110_12865_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_12865_gb300 import build
    build.build()
    from paper_2110_12865_gb300 import ssco
    return ssco


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("case", ["grid32", "elast10_big_fronts"])
def test_noalloc_matches_oracle_two_calls(S, case):
    """The allocation-free solve against the FP64 oracle's solution (same
    1e-12 relative bound as the direct FP64 parity tests), on a grid plan of
    small fronts and on an elasticity plan whose fronts above 32 rows take
    the multi-CTA path (small_front_max=32): the allocation-free solve runs
    its own fixed-shape launches over those large fronts, which ssco_solve
    would split or cluster.  Two right-hand sides in a row."""
    from oracle import oracle as O
    if case == "grid32":
        p = P.grid_problem(32, 32, batch=3, cfg=1)
        kw = {}
    else:
        p = P.elasticity_problem(10, batch=2, cfg=2)
        kw = {"small_front_max": 32, "split_rows": 64, "cluster_rows": 48}
    pl = S.Plan(p, precision=S.FP64, **kw).bind()
    if kw:
        assert pl.info["max_front_rows"] > 4 * 32      # several 32-column blocks per big front
    pl.numeric(torch.tensor(p.vals, device="cuda"), torch.tensor(p.shift, device="cuda"))
    rng = np.random.default_rng(P.seed_for(9, 0))
    b2h = rng.standard_normal(p.b.shape)
    if case != "grid32":
        b2h[:, p.dof_fixed] = 0.0
    for bh in (np.asarray(p.b), b2h):
        x = torch.full((p.batch, p.n), float("nan"), dtype=torch.float64, device="cuda")
        pl.solve_noalloc(torch.tensor(bh, device="cuda"), x)
        torch.cuda.synchronize()
        xh = x.cpu().numpy()
        for i in range(p.batch):
            r = O.refactor_solve(p, i, b=bh[i])
            assert np.linalg.norm(xh[i] - r.x) <= 1e-12 * np.linalg.norm(r.x), (case, i)


def test_noalloc_matches_solve_two_calls(S):
    p = P.grid_problem(32, 32, batch=3, cfg=1)
    pl = S.Plan(p, precision=S.FP64).bind()
    pl.numeric(torch.tensor(p.vals, device="cuda"), torch.tensor(p.shift, device="cuda"))
    b1 = torch.tensor(p.b, device="cuda")
    b2 = torch.tensor(p.xstar, device="cuda")
    ref1 = pl.solve(b1)
    ref2 = pl.solve(b2)
    x1 = torch.full_like(b1, float("nan"))
    x2 = torch.full_like(b2, float("nan"))
    pl.solve_noalloc(b1, x1)
    pl.solve_noalloc(b2, x2)
    torch.cuda.synchronize()
    assert rel(x1, ref1) <= 1e-12
    assert rel(x2, ref2) <= 1e-12
    # the second call reused the array the first one left behind
    pl.solve_noalloc(b1, x2)
    torch.cuda.synchronize()
    assert rel(x2, ref1) <= 1e-12


def test_noalloc_rejects_oversize_and_fp32(S):
    big = P.grid_problem(64, 64, batch=600, cfg=1)   # 2*B*n doubles > 64 MiB
    pl = S.Plan(big, precision=S.FP64)
    d = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(S.SscoError) as ei:
        pl.solve_noalloc(d, d.clone())
    assert ei.value.status == 9 and "64 MiB" not in str(ei.value) and "bytes" in str(ei.value)
    small = S.Plan(P.grid_problem(8, 8, cfg=1), precision=S.FP32_REFINE)
    with pytest.raises(S.SscoError) as ei:
        small.solve_noalloc(d, d.clone())
    assert ei.value.status == 9
