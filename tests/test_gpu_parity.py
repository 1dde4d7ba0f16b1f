"""GPU parity of the force solve against the FP64 oracle, through the C ABI.

Every solve here runs in the library's CUDA kernels (paper_1904_07400_gb300.api -> ctypes
-> libtdgrav.so).  Tolerances: FP64 relative L2 <= 1e-12, FP32 <= 1e-5 (written below).
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


SMALL = [(1, 1), (1, 4), (4, 1), (2, 3), (5, 7), (17, 33), (33, 17), (12, 20), (27, 9)]


@pytest.mark.parametrize("shape", SMALL)
@pytest.mark.parametrize("k", [1, 2, 3])
def test_small_and_ragged_vs_direct_sum(shape, k):
    nx, ny = shape
    dx, dy = 1.0 / nx, 1.3 / ny
    rng = np.random.default_rng(nx * 100 + ny + k)
    sigma = rng.standard_normal((nx, ny))
    S = oracle_solver(nx, ny, k, dx, dy)
    rx, ry = S.forces(sigma, method="direct")
    for prec, tol in (("fp64", TOL_FP64), ("fp32", TOL_FP32)):
        fx, fy = _solve(_plan(nx, ny, k, dx, dy, prec), sigma)
        if not (np.any(rx) or np.any(ry)):
            # a single cell exerts no force on itself: exactly zero
            assert not (np.any(fx) or np.any(fy)), (prec, fx, fy)
            continue
        err = rel_l2_pair(fx, fy, rx, ry)
        assert err <= tol, (prec, err)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_tables_match_oracle(k):
    # kernel-table construction (FP64, on the device) against the oracle's tables
    from oracle import kernel_tables as kt
    for nx, ny, dx, dy in ((40, 40, 0.025, 0.025), (24, 56, 1.0 / 24, 1.0 / 56), (64, 8, 0.01, 0.08)):
        plan = _plan(nx, ny, k, dx, dy, "fp64")
        wx, wy = plan.kernel_tables()
        qx = kt.kernel_table_quarter(k, nx, ny, dx, dy, "x")
        qy = kt.kernel_table_quarter(k, nx, ny, dx, dy, "y")
        for got, ref in ((wx, qx), (wy, qy)):
            nz = ref != 0.0
            assert np.array_equal(got == 0.0, ~nz)
            assert np.max(np.abs(got[nz] - ref[nz]) / np.abs(ref[nz])) < 1e-14


def test_config1_plain_fp64_64():
    # 64 x 64 on [-0.5, 0.5]^2, order 2, G = 1, D2 disk (exponent 3/2, R = 0.4)
    from oracle.analytic import cartesian_force
    N = 64
    x, y, dx, dy = syn.grid(N, N)
    sigma = syn.maclaurin_density(2, x, y, 0.4)
    S = oracle_solver(N, N, 2, dx, dy)
    rx, ry = S.forces(sigma, method="direct")
    fx, fy = _solve(_plan(N, N, 2, dx, dy, "fp64"), sigma)
    assert rel_l2_pair(fx, fy, rx, ry) <= TOL_FP64
    X, Y = np.meshgrid(x, y, indexing="ij")
    ax, ay, _ = cartesian_force(2, X, Y, 0.4)
    # second-order method on a grid of 64: a few 1e-3 relative to the analytic force
    assert rel_l2_pair(fx, fy, ax, ay) < 2e-2


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("disk", [2, 3])
def test_config2_512(k, disk):
    N = 512
    _, _, dx, dy = syn.grid(N, N)
    sigma = syn.perturbed_disk(disk, N, seed=2)
    S = oracle_solver(N, N, k, dx, dy)
    rx, ry = S.forces(sigma)
    f64 = _solve(_plan(N, N, k, dx, dy, "fp64"), sigma)
    f32 = _solve(_plan(N, N, k, dx, dy, "fp32"), sigma)
    assert rel_l2_pair(*f64, rx, ry) <= TOL_FP64
    assert rel_l2_pair(*f32, rx, ry) <= TOL_FP32


def test_nonsquare_cells_and_G():
    nx, ny, k = 96, 40, 3
    dx, dy = 1.0 / 96, 0.7 / 40
    rng = np.random.default_rng(11)
    sigma = rng.random((nx, ny))
    S = oracle_solver(nx, ny, k, dx, dy, 6.674e-3)
    rx, ry = S.forces(sigma)
    fx, fy = _solve(_plan(nx, ny, k, dx, dy, "fp64", G=6.674e-3), sigma)
    assert rel_l2_pair(fx, fy, rx, ry) <= TOL_FP64


def test_invariants_on_gpu_output():
    # reflection of sigma in x: F^x odd, F^y even (exact in exact arithmetic)
    N, k = 128, 3
    dx = 1.0 / N
    rng = np.random.default_rng(5)
    s = rng.random((N, N))
    s = s + s[::-1, :]
    fx, fy = _solve(_plan(N, N, k, dx, dx, "fp64"), s)
    assert np.abs(fx + fx[::-1, :]).max() < 1e-12 * np.abs(fx).max()
    assert np.abs(fy - fy[::-1, :]).max() < 1e-12 * np.abs(fy).max()
    # x <-> y symmetric sigma on a square grid: F^y = (F^x)^T
    s2 = s + s.T
    gx, gy = _solve(_plan(N, N, k, dx, dx, "fp64"), s2)
    assert np.abs(gy - gx.T).max() < 1e-12 * np.abs(gx).max()


def test_config3_4096_sampled():
    # full size of the timed workload: FP64 and FP32 GPU forms against the oracle at
    # sampled cells (each computed by its own literal sum), and FP32 against FP64 over
    # the whole grid
    N, k = 4096, 3
    _, _, dx, dy = syn.grid(N, N)
    sigma = syn.clumps(N, N, seed=3)
    pts = syn.sample_points(N, N, 12, seed=33)
    S = oracle_solver(N, N, k, dx, dy)
    rx, ry = S.forces_at(sigma, pts)
    f64 = _solve(_plan(N, N, k, dx, dy, "fp64"), sigma)
    f32 = _solve(_plan(N, N, k, dx, dy, "fp32"), sigma)
    idx = tuple(np.array(pts).T)
    scale = np.sqrt(np.sum(rx ** 2 + ry ** 2))
    e64 = np.sqrt(np.sum((f64[0][idx] - rx) ** 2 + (f64[1][idx] - ry) ** 2)) / scale
    e32 = np.sqrt(np.sum((f32[0][idx] - rx) ** 2 + (f32[1][idx] - ry) ** 2)) / scale
    assert e64 <= TOL_FP64, e64
    assert e32 <= TOL_FP32, e32
    assert rel_l2_pair(f32[0], f32[1], f64[0], f64[1]) <= TOL_FP32


def test_linearity_and_zero_input():
    import torch
    N, k = 64, 3
    plan = _plan(N, N, k, 1.0 / N, 1.0 / N, "fp64")
    z = torch.zeros((N, N), dtype=torch.float64, device=plan.device)
    fx, fy = plan.forces(z)
    assert float(fx.abs().max()) == 0.0 and float(fy.abs().max()) == 0.0
    a = torch.randn((N, N), dtype=torch.float64, device=plan.device)
    b = torch.randn((N, N), dtype=torch.float64, device=plan.device)
    ax, ay = plan.forces(a)
    bx, by = plan.forces(b)
    cx, cy = plan.forces(2 * a - b)
    assert float((cx - (2 * ax - bx)).abs().max()) < 1e-12 * float(cx.abs().max())
