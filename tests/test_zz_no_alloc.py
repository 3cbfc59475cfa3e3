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
