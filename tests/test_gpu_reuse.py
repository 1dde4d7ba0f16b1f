"""In-simulation reuse: plans rebuilt from kept kernel tables, and repeated solves inside a
captured time-stepping graph.

A plan built from saved FP64 tables computes the same spectra from the same numbers, so
its forces equal those of the original plan bit for bit.  The kernels are deterministic
(no atomics on the data path), so a CUDA graph of several time steps replays to the same
bits as the same steps run eagerly.
"""
import numpy as np
import pytest

from gpu_common import library, to_np
from workloads import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    library()


def _forces(plan, sigma):
    import torch
    s = torch.as_tensor(sigma, dtype=plan.dtype, device=plan.device)
    fx, fy = plan.forces(s)
    torch.cuda.synchronize()
    assert plan.device_error() == 0
    return to_np(fx), to_np(fy)


@pytest.mark.parametrize("shape,k,prec", [((1024, 1024), 3, "fp32"), ((384, 512), 2, "fp32"),
                                          ((96, 80), 3, "fp64"), ((130, 66), 1, "fp32")])
def test_plan_from_saved_tables_is_bit_identical(tmp_path, shape, k, prec):
    from paper_1904_07400_gb300.api import Plan
    nx, ny = shape
    dx, dy = 1.0 / nx, 0.9 / ny
    a = Plan(nx, ny, k, dx, dy, precision=prec)
    path = str(tmp_path / "tables.npz")
    a.save_tables(path)
    b = Plan(nx, ny, k, dx, dy, precision=prec, tables=path)
    sigma = syn.clumps(nx, ny, seed=nx + k)
    fa, fb = _forces(a, sigma), _forces(b, sigma)
    assert np.array_equal(fa[0], fb[0]) and np.array_equal(fa[1], fb[1])
    wa, wb = a.kernel_tables(), b.kernel_tables()
    assert np.array_equal(wa[0], wb[0]) and np.array_equal(wa[1], wb[1])


def test_tables_cross_precision_and_mismatch(tmp_path):
    from paper_1904_07400_gb300 import native
    from paper_1904_07400_gb300.api import Plan
    nx = ny = 256
    d = 1.0 / nx
    p64 = Plan(nx, ny, 3, d, d, precision="fp64")
    path = str(tmp_path / "t.npz")
    p64.save_tables(path)
    # FP64 tables serve an FP32 plan of the same grid
    ref = Plan(nx, ny, 3, d, d, precision="fp32")
    got = Plan(nx, ny, 3, d, d, precision="fp32", tables=path)
    sigma = syn.clumps(nx, ny, seed=11)
    fr, fg = _forces(ref, sigma), _forces(got, sigma)
    assert np.array_equal(fr[0], fg[0]) and np.array_equal(fr[1], fg[1])
    # another order: refused by the parameter check, and by the library's spot check
    with pytest.raises(ValueError):
        Plan(nx, ny, 2, d, d, precision="fp32", tables=path)
    other = Plan(nx, ny, 2, d, d, precision="fp32", build=False)
    wx, wy = p64.kernel_tables()
    st = native.load().tdg_build_kernel_tables_from(other.handle, wx.ctypes.data, wy.ctypes.data, None)
    assert native.STATUS[st] == "TDG_ERR_INVALID_ARG"


def test_time_stepping_graph_replays_eager_steps():
    # a toy evolution step: forces from sigma, then sigma nudged by them (torch element-
    # wise ops); K steps captured once in a CUDA graph replay to the eager result
    import torch
    from paper_1904_07400_gb300.api import Plan
    nx = ny = 512
    d = 1.0 / nx
    plan = Plan(nx, ny, 3, d, d, precision="fp32")
    s0 = torch.as_tensor(syn.clumps(nx, ny, seed=21), dtype=torch.float32, device=plan.device)
    fx = torch.empty_like(s0)
    fy = torch.empty_like(s0)
    K, dt = 4, 1e-4

    def step(s):
        plan.forces(s, out=(fx, fy))
        s.add_(dt * (fx * fx + fy * fy).sqrt() - dt * s)

    eager = s0.clone()
    for _ in range(K):
        step(eager)
    torch.cuda.synchronize()

    state = s0.clone()
    step(state.clone())  # first call outside the capture (workspace, kernel attributes)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            for _ in range(K):
                step(state)
    torch.cuda.current_stream().wait_stream(side)
    state.copy_(s0)
    g.replay()
    torch.cuda.synchronize()
    assert plan.device_error() == 0
    assert torch.equal(state, eager)
    # a second replay continues from where the first left off
    again = eager.clone()
    for _ in range(K):
        step(again)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(state, again)
