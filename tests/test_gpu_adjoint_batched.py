"""GPU adjoint (hand-written backward), autograd wrapper, batched solves and error paths.

Tolerances: FP64 relative L2 <= 1e-12, FP32 <= 1e-5; finite differences on the FP32 path
within 1e-3 of rms(dL/dsigma) (L is linear in sigma, so only rounding remains).
"""
import numpy as np
import pytest

from gpu_common import TOL_FP32, TOL_FP64, library, oracle_solver, to_np
from workloads import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    library()


def _plan(nx, ny, k, dx, dy, prec, **kw):
    from paper_1904_07400_gb300.api import Plan
    return Plan(nx, ny, k, dx, dy, precision=prec, **kw)


def _t(a, plan):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=plan.dtype, device=plan.device)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("shape,k", [((5, 7), 3), ((17, 33), 2), ((64, 48), 3), ((96, 96), 1)])
def test_adjoint_vs_oracle(shape, k):
    nx, ny = shape
    dx, dy = 1.0 / nx, 1.0 / ny
    rng = np.random.default_rng(nx + ny)
    gx, gy = rng.standard_normal((nx, ny)), rng.standard_normal((nx, ny))
    ref = oracle_solver(nx, ny, k, dx, dy).adjoint(gx, gy)
    for prec, tol in (("fp64", TOL_FP64), ("fp32", TOL_FP32)):
        p = _plan(nx, ny, k, dx, dy, prec)
        got = to_np(p.adjoint(_t(gx, p), _t(gy, p)))
        assert _rel(got, ref) <= tol, prec


@pytest.mark.parametrize("k", [1, 2, 3])
def test_adjoint_on_half_warp_lines_vs_oracle(k):
    # sides up to 256 run the adjoint on the 256-point network, two lines per 32-thread
    # block (columns, then rows with the y solve)
    nx, ny = 160, 224
    dx, dy = 1.0 / nx, 1.0 / ny
    rng = np.random.default_rng(40 + k)
    gx, gy = rng.standard_normal((nx, ny)), rng.standard_normal((nx, ny))
    ref = oracle_solver(nx, ny, k, dx, dy).adjoint(gx, gy)
    p = _plan(nx, ny, k, dx, dy, "fp32")
    assert p.path() == 2
    got = to_np(p.adjoint(_t(gx, p), _t(gy, p)))
    assert _rel(got, ref) <= TOL_FP32


def test_adjoint_dot_product_identity_fp64():
    import torch
    N, k = 256, 3
    p = _plan(N, N, k, 1.0 / N, 1.0 / N, "fp64")
    s = torch.randn((N, N), dtype=torch.float64, device=p.device)
    gx = torch.randn_like(s)
    gy = torch.randn_like(s)
    fx, fy = p.forces(s)
    gs = p.adjoint(gx, gy)
    lhs = float((gx * fx).sum() + (gy * fy).sum())
    rhs = float((gs * s).sum())
    assert abs(lhs - rhs) <= 1e-12 * float((gs.abs() * s.abs()).sum())


def test_config5_adjoint_2048_fd_and_oracle():
    import torch
    N, k = 2048, 3
    _, _, dx, dy = syn.grid(N, N)
    sigma = syn.clumps(N, N, seed=5)
    gxn, gyn = syn.adjoint_weights(N, N, seed=6)
    p = _plan(N, N, k, dx, dy, "fp32")
    s, gx, gy = _t(sigma, p), _t(gxn, p), _t(gyn, p)
    gs = to_np(p.adjoint(gx, gy))
    # against the oracle's FP64 adjoint (whole grid)
    ref = oracle_solver(N, N, k, dx, dy).adjoint(gxn, gyn)
    assert _rel(gs, ref) <= TOL_FP32
    # central finite differences at the 32 seeded probe cells; L accumulated in FP64
    h = float(sigma.max())
    rms = float(np.sqrt(np.mean(gs ** 2)))
    gx64, gy64 = gx.double(), gy.double()
    for (i, j) in syn.fd_points(N, N, seed=7):
        sp = s.clone()
        sp[i, j] += h
        sm = s.clone()
        sm[i, j] -= h
        px, py = p.forces(sp)
        mx, my = p.forces(sm)
        lp = float((gx64 * px.double()).sum() + (gy64 * py.double()).sum())
        lm = float((gx64 * mx.double()).sum() + (gy64 * my.double()).sum())
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gs[i, j]) <= 1e-3 * rms, (i, j, fd, gs[i, j])


def test_autograd_function_uses_adjoint():
    import torch
    from paper_1904_07400_gb300.api import ThinDiskForces
    N, k = 48, 3
    p = _plan(N, N, k, 1.0 / N, 1.0 / N, "fp64")
    s = torch.randn((N, N), dtype=torch.float64, device=p.device, requires_grad=True)
    wx = torch.randn((N, N), dtype=torch.float64, device=p.device)
    wy = torch.randn_like(wx)
    fx, fy = ThinDiskForces.apply(p, s)
    loss = (wx * fx).sum() + (wy * fy).sum()
    loss.backward()
    ref = p.adjoint(wx, wy)
    assert float((s.grad - ref).abs().max()) == 0.0


def test_batched_equals_individual_solves():
    import torch
    from paper_1904_07400_gb300.api import forces_batched
    specs = [(128, 192, 1), (256, 128, 3), (192, 192, 2), (64, 384, 3), (9, 5, 2)]
    plans, sigmas, refs = [], [], []
    for (nx, ny, k) in specs:
        p = _plan(nx, ny, k, 1.0 / nx, 1.0 / ny, "fp32")
        s = _t(syn.clumps(nx, ny, seed=nx + ny), p)
        plans.append(p)
        sigmas.append(s)
        refs.append(p.forces(s))
    outs = forces_batched(plans, sigmas)
    torch.cuda.synchronize()
    # the batched kernel runs the transforms with another thread layout: equal to rounding
    for (ax, ay), (bx, by) in zip(outs, refs):
        num = float(((ax - bx) ** 2).sum() + ((ay - by) ** 2).sum()) ** 0.5
        den = float((bx ** 2).sum() + (by ** 2).sum()) ** 0.5
        assert num <= TOL_FP32 * den


def test_error_paths():
    import torch
    from paper_1904_07400_gb300 import native
    from paper_1904_07400_gb300.api import Plan
    p = Plan(32, 32, 3, 0.1, 0.1, precision="fp32", build=False)
    s = torch.zeros((32, 32), dtype=torch.float32, device="cuda")
    with pytest.raises(native.TdgError) as e:
        p.forces(s)
    assert e.value.status == 3  # NOT_BUILT
    p.build()
    buf = torch.zeros(32 * 32 + 1, dtype=torch.float32, device="cuda")
    lib = native.load()
    fx = torch.empty_like(s)
    fy = torch.empty_like(s)
    # misaligned and aliased pointers are rejected before any launch
    assert lib.tdg_solve_forces(p.handle, buf.data_ptr() + 4, fx.data_ptr(), fy.data_ptr(), None) == 1
    assert lib.tdg_solve_forces(p.handle, s.data_ptr(), fx.data_ptr(), fx.data_ptr(), None) == 1
    # a caller-owned workspace is used and kept
    ws = torch.empty(p.workspace_bytes() // 4 + 64, dtype=torch.float32, device="cuda")
    p.set_workspace(ws)
    a = p.forces(torch.randn_like(s))
    torch.cuda.synchronize()
    assert torch.isfinite(a[0]).all()
    assert p.device_error() == 0
