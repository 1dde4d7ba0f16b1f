"""Full-size parity at the 4096 x 4096 order-3 clumped-disk workload (64 Gaussian clumps,
seed 3, the one bench.py times): every precision form against the FP64 oracle's full-grid
FFT solve, element by element over all 16.8 million cells.  Tolerances: relative L2 of the
pair (F^x, F^y) <= 1e-5 for FP32 and FP32_TC16, <= 1e-12 for FP64; and the largest
elementwise error at most 1e-5 (1e-12) of the largest force magnitude."""
import numpy as np
import pytest

from gpu_common import TOL_FP32, TOL_FP64, library, rel_l2_pair, to_np
from workloads import synthetic as syn

pytestmark = pytest.mark.gpu

N = 4096


@pytest.fixture(scope="module")
def oracle_forces():
    import os
    from oracle.convolution import Solver
    library()
    sigma = syn.clumps(N, N, seed=3)
    rx, ry = Solver(N, N, 3, 1.0 / N, 1.0 / N).forces(sigma, workers=os.cpu_count() or 1)
    return sigma, rx, ry


@pytest.mark.parametrize("form,tol", [("fp32", TOL_FP32), ("fp32_tc16", TOL_FP32), ("fp64", TOL_FP64)])
def test_4096_every_form_vs_oracle_full_grid(oracle_forces, form, tol):
    import torch
    from paper_1904_07400_gb300.api import Plan
    sigma, rx, ry = oracle_forces
    plan = Plan(N, N, 3, 1.0 / N, 1.0 / N, precision=form)
    s = torch.as_tensor(sigma, dtype=plan.dtype, device=plan.device)
    fx, fy = plan.forces(s)
    torch.cuda.synchronize()
    assert plan.device_error() == 0
    fx, fy = to_np(fx), to_np(fy)
    assert rel_l2_pair(fx, fy, rx, ry) <= tol
    scale = max(np.abs(rx).max(), np.abs(ry).max())
    assert max(np.abs(fx - rx).max(), np.abs(fy - ry).max()) <= tol * scale
    plan.close()
