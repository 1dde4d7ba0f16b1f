"""B-spline orders 4 and 5 on the GPU against the FP64 oracle, through the C ABI.

The same construction as orders 1-3 with the wider interpolation stencils (1, 4, 1)/6 and
(1, 76, 230, 76, 1)/384 (truncated banded solves along y and x) and tables of the wider
splines.  Tolerances: FP64 relative L2 <= 1e-12, FP32 <= 1e-5 (written below).
"""
import numpy as np
import pytest

from gpu_common import TOL_FP32, TOL_FP64, library, oracle_solver, rel_l2_pair, to_np
from workloads import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    library()


def _plan(nx, ny, k, dx, dy, prec, G=1.0):
    from paper_1904_07400_gb300.api import Plan
    return Plan(nx, ny, k, dx, dy, G=G, precision=prec)


def _solve(plan, sigma):
    import torch
    s = torch.as_tensor(sigma, dtype=plan.dtype, device=plan.device).contiguous()
    fx, fy = plan.forces(s)
    torch.cuda.synchronize()
    assert plan.device_error() == 0
    return to_np(fx), to_np(fy)


# square cells (the oracle's near-field entries are shared across sizes), ragged sides
SMALL = [(1, 1), (2, 3), (5, 7), (17, 33), (27, 9), (64, 48), (130, 66)]


@pytest.mark.parametrize("shape", SMALL)
@pytest.mark.parametrize("k", [4, 5])
def test_small_and_ragged_vs_oracle(shape, k):
    nx, ny = shape
    d = 1.0 / max(nx, ny)
    rng = np.random.default_rng(nx * 100 + ny + k)
    sigma = rng.standard_normal((nx, ny))
    S = oracle_solver(nx, ny, k, d, d)
    rx, ry = S.forces(sigma, method="direct" if nx * ny <= 4096 else "fft")
    for prec, tol in (("fp64", TOL_FP64), ("fp32", TOL_FP32)):
        fx, fy = _solve(_plan(nx, ny, k, d, d, prec), sigma)
        if not (np.any(rx) or np.any(ry)):
            assert not (np.any(fx) or np.any(fy)), (prec, fx, fy)
            continue
        err = rel_l2_pair(fx, fy, rx, ry)
        assert err <= tol, (prec, err)


@pytest.mark.parametrize("k", [4, 5])
def test_tables_match_oracle_orders_4_5(k):
    from oracle import kernel_tables as kt
    cases = [(40, 40, 0.025, 0.025)]
    if k == 5:
        cases.append((24, 20, 1.0 / 24, 0.5 / 24))  # thin cells (dy/dx = 1/2)
    for nx, ny, dx, dy in cases:
        plan = _plan(nx, ny, k, dx, dy, "fp64")
        wx, wy = plan.kernel_tables()
        qx = kt.kernel_table_quarter(k, nx, ny, dx, dy, "x")
        qy = kt.kernel_table_quarter(k, nx, ny, dx, dy, "y")
        for got, ref in ((wx, qx), (wy, qy)):
            nz = ref != 0.0
            assert np.array_equal(got == 0.0, ~nz)
            assert np.max(np.abs(got[nz] - ref[nz]) / np.abs(ref[nz])) < 2e-14


@pytest.mark.parametrize("k", [4, 5])
def test_512_disk_orders_4_5(k):
    N = 512
    _, _, dx, dy = syn.grid(N, N)
    sigma = syn.perturbed_disk(3, N, seed=2)
    S = oracle_solver(N, N, k, dx, dy)
    rx, ry = S.forces(sigma)
    assert rel_l2_pair(*_solve(_plan(N, N, k, dx, dy, "fp64"), sigma), rx, ry) <= TOL_FP64
    assert rel_l2_pair(*_solve(_plan(N, N, k, dx, dy, "fp32"), sigma), rx, ry) <= TOL_FP32


@pytest.mark.parametrize("k", [4, 5])
def test_2048_sampled_and_4096_fp32_vs_fp64(k):
    # 2048^2: both forms against the oracle at sampled cells (each its own literal sum);
    # 4096^2: FP32 against FP64 over the whole grid
    N = 2048
    _, _, dx, dy = syn.grid(N, N)
    sigma = syn.clumps(N, N, seed=3 + k)
    pts = syn.sample_points(N, N, 8, seed=40 + k)
    rx, ry = oracle_solver(N, N, k, dx, dy).forces_at(sigma, pts)
    idx = tuple(np.array(pts).T)
    scale = np.sqrt(np.sum(rx ** 2 + ry ** 2))
    for prec, tol in (("fp64", TOL_FP64), ("fp32", TOL_FP32)):
        fx, fy = _solve(_plan(N, N, k, dx, dy, prec), sigma)
        e = np.sqrt(np.sum((fx[idx] - rx) ** 2 + (fy[idx] - ry) ** 2)) / scale
        assert e <= tol, (prec, e)
    N = 4096
    _, _, dx, dy = syn.grid(N, N)
    sigma = syn.clumps(N, N, seed=9 + k)
    f64 = _solve(_plan(N, N, k, dx, dy, "fp64"), sigma)
    f32 = _solve(_plan(N, N, k, dx, dy, "fp32"), sigma)
    assert rel_l2_pair(f32[0], f32[1], f64[0], f64[1]) <= TOL_FP32


@pytest.mark.parametrize("shape,k", [((5, 7), 5), ((17, 33), 4), ((64, 48), 5)])
def test_adjoint_orders_4_5(shape, k):
    import torch
    nx, ny = shape
    d = 1.0 / max(nx, ny)
    rng = np.random.default_rng(nx + ny + k)
    gx, gy = rng.standard_normal((nx, ny)), rng.standard_normal((nx, ny))
    ref = oracle_solver(nx, ny, k, d, d).adjoint(gx, gy)
    for prec, tol in (("fp64", TOL_FP64), ("fp32", TOL_FP32)):
        p = _plan(nx, ny, k, d, d, prec)
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=p.dtype, device=p.device)
        got = to_np(p.adjoint(t(gx), t(gy)))
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= tol, prec


def test_batch_mixing_all_orders_equals_individual_solves():
    import torch
    from paper_1904_07400_gb300.api import Batch
    specs = [(96, 64, 1), (70, 70, 2), (128, 40, 3), (64, 96, 4), (100, 52, 5), (33, 17, 5)]
    plans, sigmas, ref = [], [], []
    for i, (nx, ny, k) in enumerate(specs):
        p = _plan(nx, ny, k, 1.0 / nx, 1.0 / nx, "fp32")
        s = torch.as_tensor(syn.clumps(nx, ny, seed=i), dtype=torch.float32, device=p.device)
        plans.append(p)
        sigmas.append(s)
        ref.append(tuple(t.clone() for t in p.forces(s)))
    for streams in (0, 4):
        b = Batch(plans, sigmas)
        b.set_streams(streams)
        b.launch()
        torch.cuda.synchronize()
        assert b.error() == 0
        for (fx, fy), (rx, ry) in zip(b.outs, ref):
            assert rel_l2_pair(to_np(fx), to_np(fy), to_np(rx), to_np(ry)) <= 1e-6


@pytest.mark.parametrize("shape", [(128, 144), (256, 192), (1024, 1008)])
@pytest.mark.parametrize("k", [4, 5])
def test_network_path_orders_4_5(shape, k):
    # FP32 sides that are multiples of 16 from 128 to 4096 run the one-barrier transform
    # network with its chunked register solves (tridiagonal for 4, pentadiagonal for 5)
    import torch
    nx, ny = shape
    d = 1.0 / max(nx, ny)
    sigma = syn.clumps(nx, ny, seed=nx + k)
    p32 = _plan(nx, ny, k, d, d, "fp32")
    assert p32.path() == 2
    f32 = _solve(p32, sigma)
    f64 = _solve(_plan(nx, ny, k, d, d, "fp64"), sigma)
    assert rel_l2_pair(*f32, *f64) <= TOL_FP32
    if nx * ny <= 256 * 192:
        rx, ry = oracle_solver(nx, ny, k, d, d).forces(sigma)
        assert rel_l2_pair(*f64, rx, ry) <= TOL_FP64
        assert rel_l2_pair(*f32, rx, ry) <= TOL_FP32
    # adjoint on the same path
    rng = np.random.default_rng(k)
    gx, gy = rng.standard_normal((nx, ny)), rng.standard_normal((nx, ny))
    t = lambda a, p: torch.as_tensor(a, dtype=p.dtype, device=p.device)
    p64 = _plan(nx, ny, k, d, d, "fp64")
    a32 = to_np(p32.adjoint(t(gx, p32), t(gy, p32)))
    a64 = to_np(p64.adjoint(t(gx, p64), t(gy, p64)))
    assert np.linalg.norm(a32 - a64) / np.linalg.norm(a64) <= TOL_FP32


@pytest.mark.parametrize("k", [3, 4, 5])
def test_network_path_nonsquare_cells(k):
    # cells with dy = 0.7 dx on the network path against the FP64 generic form
    nx, ny = 384, 256
    dx = 1.0 / nx
    dy = 0.7 * dx
    sigma = syn.clumps(nx, ny, seed=50 + k)
    p32 = _plan(nx, ny, k, dx, dy, "fp32")
    assert p32.path() == 2
    f32 = _solve(p32, sigma)
    f64 = _solve(_plan(nx, ny, k, dx, dy, "fp64"), sigma)
    assert rel_l2_pair(*f32, *f64) <= TOL_FP32
