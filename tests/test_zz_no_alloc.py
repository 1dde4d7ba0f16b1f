"""tdg_solve_forces_noalloc: the force solve for callers that cannot allocate device memory
where they solve (for instance while another allocator owns the device's free memory, or
in loops that must not hit cudaMalloc's implicit synchronisation).  It must give the same
forces as tdg_solve_forces, call after call, with its scratch in the library's fixed
device array.  This file is collected last on purpose, so a run that stops at its first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from gpu_common import TOL_FP32, TOL_FP64, library, rel_l2_pair, to_np
from workloads import synthetic as syn

pytestmark = pytest.mark.gpu


def _plan(nx, ny, k, prec):
    from paper_1904_07400_gb300.api import Plan
    return Plan(nx, ny, k, 1.0 / nx, 1.0 / ny, precision=prec)


def _noalloc(plan, sigma, fx, fy):
    import torch
    lib = library()
    return lib.tdg_solve_forces_noalloc(plan.handle, sigma.data_ptr(), fx.data_ptr(), fy.data_ptr(),
                                        torch.cuda.current_stream(plan.device).cuda_stream)


@pytest.mark.parametrize("shape,k,prec,tol", [((256, 192), 3, "fp32", TOL_FP32),
                                             ((96, 160), 2, "fp64", TOL_FP64),
                                             ((256, 256), 5, "fp32", TOL_FP32),
                                             ((100, 60), 4, "fp64", TOL_FP64),
                                             ((200, 176), 1, "fp32", TOL_FP32),
                                             ((1040, 128), 3, "fp32_tc16", TOL_FP32)])
def test_noalloc_matches_solve_on_two_calls_in_a_row(shape, k, prec, tol):
    import torch
    nx, ny = shape
    from paper_1904_07400_gb300 import native
    plan = _plan(nx, ny, k, prec)
    assert plan.workspace_bytes() <= native.NOALLOC_SCRATCH_BYTES
    for call, seed in enumerate((3, 44)):
        s = torch.as_tensor(syn.clumps(nx, ny, seed=seed), dtype=plan.dtype, device=plan.device)
        ref = plan.forces(s)
        fx = torch.full_like(s, float("nan"))
        fy = torch.full_like(s, float("nan"))
        assert _noalloc(plan, s, fx, fy) == 0
        torch.cuda.synchronize()
        err = rel_l2_pair(to_np(fx), to_np(fy), to_np(ref[0]), to_np(ref[1]))
        assert err <= tol, (call, err)
    assert plan.device_error() == 0


def test_noalloc_rejects_plans_beyond_its_scratch():
    import torch
    from paper_1904_07400_gb300 import native
    lib = library()
    plan = _plan(2048, 2048, 3, "fp32")
    limit = native.NOALLOC_SCRATCH_BYTES
    assert plan.workspace_bytes() > limit
    s = torch.ones((2048, 2048), dtype=torch.float32, device=plan.device)
    fx = torch.zeros_like(s)
    fy = torch.zeros_like(s)
    st = _noalloc(plan, s, fx, fy)
    assert native.STATUS[st] == "TDG_ERR_UNSUPPORTED"
    torch.cuda.synchronize()
    assert float(fx.abs().max()) == 0.0 and float(fy.abs().max()) == 0.0
    # an unbuilt plan and bad pointers are rejected before any launch
    from paper_1904_07400_gb300.api import Plan
    p2 = Plan(64, 64, 3, 1.0 / 64, 1.0 / 64, precision="fp32", build=False)
    small = torch.ones((64, 64), dtype=torch.float32, device="cuda")
    out = torch.zeros_like(small)
    assert native.STATUS[_noalloc(p2, small, out, torch.zeros_like(small))] == "TDG_ERR_NOT_BUILT"
    assert lib.tdg_solve_forces_noalloc(plan.handle, None, fx.data_ptr(), fy.data_ptr(), None) == 1
