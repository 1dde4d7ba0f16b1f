"""Parity of the FP32 and FP32_TC16 forms on the transform-network path (sides that are
multiples of 16 from 128 to 4096 cells).

The FP32 forms of these grids run the network kernels; the FP64 form runs the generic ones,
so the comparison also cross-checks two independent kernel sets.  Tolerance: FP32
relative L2 <= 1e-5 against the FP64 oracle (and against the FP64 GPU form, itself within
1e-12 of the oracle).
"""
import numpy as np
import pytest

from gpu_common import TOL_FP32, library, oracle_solver, rel_l2_pair, to_np
from workloads import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    library()


def _forces(nx, ny, k, dx, dy, prec, sigma):
    import torch
    from paper_1904_07400_gb300.api import Plan
    p = Plan(nx, ny, k, dx, dy, precision=prec)
    s = torch.as_tensor(sigma, dtype=p.dtype, device=p.device)
    fx, fy = p.forces(s)
    torch.cuda.synchronize()
    assert p.device_error() == 0
    return to_np(fx), to_np(fy)


@pytest.mark.parametrize("shape", [(1024, 1024), (1024, 2048), (2048, 1024), (4096, 1024), (1024, 4096)])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_fast_path_vs_fp64_gpu(shape, k):
    nx, ny = shape
    dx, dy = 1.0 / nx, 1.0 / ny
    sigma = syn.clumps(nx, ny, seed=nx + 7 * ny + k)
    f32 = _forces(nx, ny, k, dx, dy, "fp32", sigma)
    f64 = _forces(nx, ny, k, dx, dy, "fp64", sigma)
    assert rel_l2_pair(*f32, *f64) <= TOL_FP32


@pytest.mark.parametrize("shape", [(528, 2064), (1040, 1040), (272, 4080)])
@pytest.mark.parametrize("k", [2, 3, 5])
def test_row_pairs_with_rows_off_the_128_byte_pieces(shape, k):
    # rows of 2048 and 4096 transform points run in pairs; rows whose length is not a
    # multiple of 32 cells are loaded without the row TMA (their last 16 cells would not
    # fill a 128-byte piece), the others by it
    nx, ny = shape
    dx, dy = 1.0 / nx, 1.0 / ny
    sigma = syn.clumps(nx, ny, seed=nx + 3 * ny + k)
    f32 = _forces(nx, ny, k, dx, dy, "fp32", sigma)
    f64 = _forces(nx, ny, k, dx, dy, "fp64", sigma)
    assert rel_l2_pair(*f32, *f64) <= TOL_FP32


@pytest.mark.parametrize("k", [1, 3])
def test_fast_path_vs_oracle_nonsquare_cells(k):
    nx, ny = 1024, 2048
    dx, dy = 1.0 / 1024, 0.7 / 2048
    rng = np.random.default_rng(k)
    sigma = syn.clumps(nx, ny, seed=k) + 0.1 * rng.random((nx, ny))
    rx, ry = oracle_solver(nx, ny, k, dx, dy).forces(sigma)
    f32 = _forces(nx, ny, k, dx, dy, "fp32", sigma)
    assert rel_l2_pair(*f32, rx, ry) <= TOL_FP32


def test_fast_path_edges_and_ragged_support():
    # density touching every edge of the grid (the truncated spline solve and the zero
    # padding both matter there), order 3, against the oracle
    nx = ny = 1024
    dx = 1.0 / nx
    rng = np.random.default_rng(9)
    sigma = rng.random((nx, ny))
    rx, ry = oracle_solver(nx, ny, 3, dx, dx).forces(sigma)
    f32 = _forces(nx, ny, 3, dx, dx, "fp32", sigma)
    assert rel_l2_pair(*f32, rx, ry) <= TOL_FP32


@pytest.mark.parametrize("shape,k", [((2048, 1024), 3), ((2048, 2048), 2), ((4096, 1024), 1), ((4096, 4096), 3),
                                     ((1536, 768), 3), ((2048, 512), 4), ((2048, 512), 5), ((3072, 2000), 3)])
def test_tc16_form_vs_fp64_gpu(shape, k):
    # the column pass's DFT_16 stages as split TF32 hi/lo tensor-core products (tcgen05.mma),
    # FP32 accumulation; the row passes are the FP32 network kernels
    from paper_1904_07400_gb300.api import Plan
    nx, ny = shape
    dx, dy = 1.0 / nx, 1.0 / ny
    assert Plan(nx, ny, k, dx, dy, precision="fp32_tc16").path() == 3
    sigma = syn.clumps(nx, ny, seed=3 + k)
    tc = _forces(nx, ny, k, dx, dy, "fp32_tc16", sigma)
    f64 = _forces(nx, ny, k, dx, dy, "fp64", sigma)
    assert rel_l2_pair(*tc, *f64) <= TOL_FP32


def test_tc16_form_vs_oracle():
    nx, ny = 2048, 512
    dx, dy = 1.0 / 2048, 0.5 / 512
    sigma = syn.clumps(nx, ny, seed=12)
    rx, ry = oracle_solver(nx, ny, 3, dx, dy).forces(sigma)
    tc = _forces(nx, ny, 3, dx, dy, "fp32_tc16", sigma)
    assert rel_l2_pair(*tc, rx, ry) <= TOL_FP32


def test_tc16_adjoint_matches_fp64_gpu():
    # TC16 plans run the FP32 network adjoint
    import torch
    from paper_1904_07400_gb300.api import Plan
    nx, ny = 2048, 1024
    dx, dy = 1.0 / nx, 1.0 / ny
    gx, gy = syn.adjoint_weights(nx, ny, 6)
    out = {}
    for prec in ("fp32_tc16", "fp64"):
        p = Plan(nx, ny, 3, dx, dy, precision=prec)
        t = lambda a: torch.as_tensor(a, dtype=p.dtype, device=p.device)
        out[prec] = to_np(p.adjoint(t(gx), t(gy)))
        torch.cuda.synchronize()
        assert p.device_error() == 0
    ref = out["fp64"]
    assert np.linalg.norm(out["fp32_tc16"] - ref) / np.linalg.norm(ref) <= TOL_FP32


# sides that are multiples of 16 below the transform length (the plan pads to P = 2L,
# L in {256, 512, 1024, 2048, 4096}; the crop is exact for any P >= 2N - 1)
@pytest.mark.parametrize("shape,k", [((768, 1024), 3), ((1024, 768), 2), ((512, 384), 1), ((384, 512), 3),
                                     ((128, 160), 3), ((1040, 272), 2), ((3072, 4096), 3), ((144, 2000), 1)])
def test_padded_network_sizes_vs_fp64_gpu(shape, k):
    nx, ny = shape
    dx, dy = 1.0 / nx, 1.0 / ny
    sigma = syn.clumps(nx, ny, seed=nx + ny + k)
    f32 = _forces(nx, ny, k, dx, dy, "fp32", sigma)
    f64 = _forces(nx, ny, k, dx, dy, "fp64", sigma)
    assert rel_l2_pair(*f32, *f64) <= TOL_FP32


@pytest.mark.parametrize("shape", [(128, 128), (256, 256), (208, 240), (128, 256), (256, 144)])
@pytest.mark.parametrize("k", [1, 3, 5])
def test_half_warp_lines_vs_oracle(shape, k):
    # sides up to 256 run on the 256-point network, two lines per 32-thread block (an odd
    # number of frequency columns, L + 1: the last block's second half stores nothing)
    from paper_1904_07400_gb300.api import Plan
    nx, ny = shape
    dx, dy = 1.0 / nx, 0.9 / ny
    assert Plan(nx, ny, k, dx, dy, precision="fp32").path() == 2
    rng = np.random.default_rng(nx + ny + k)
    sigma = syn.clumps(nx, ny, seed=nx + 2 * ny) + 0.05 * rng.random((nx, ny))
    rx, ry = oracle_solver(nx, ny, k, dx, dy).forces(sigma)
    f32 = _forces(nx, ny, k, dx, dy, "fp32", sigma)
    assert rel_l2_pair(*f32, rx, ry) <= TOL_FP32


@pytest.mark.parametrize("k", [1, 2, 3])
def test_padded_network_small_grid_vs_oracle(k):
    from paper_1904_07400_gb300.api import Plan
    nx, ny = 176, 144
    dx, dy = 1.0 / nx, 0.8 / ny
    assert Plan(nx, ny, k, dx, dy, precision="fp32").path() == 2
    rng = np.random.default_rng(k)
    sigma = rng.random((nx, ny))  # touches every edge
    rx, ry = oracle_solver(nx, ny, k, dx, dy).forces(sigma)
    f32 = _forces(nx, ny, k, dx, dy, "fp32", sigma)
    assert rel_l2_pair(*f32, rx, ry) <= TOL_FP32


def _adjoint(nx, ny, k, dx, dy, prec, gx, gy):
    import torch
    from paper_1904_07400_gb300.api import Plan
    p = Plan(nx, ny, k, dx, dy, precision=prec)
    tx = torch.as_tensor(gx, dtype=p.dtype, device=p.device)
    ty = torch.as_tensor(gy, dtype=p.dtype, device=p.device)
    gs = p.adjoint(tx, ty)
    torch.cuda.synchronize()
    assert p.device_error() == 0
    return to_np(gs), p.path()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# the adjoint on the network path (same plans as the forward): against the FP64 GPU adjoint
# (generic kernels) and, on a small grid, against the oracle's adjoint
@pytest.mark.parametrize("shape,k", [((4096, 4096), 3), ((2048, 1024), 2), ((1024, 2048), 3), ((768, 1024), 1),
                                     ((384, 512), 3), ((144, 2000), 2)])
def test_network_adjoint_vs_fp64_gpu(shape, k):
    nx, ny = shape
    dx, dy = 1.0 / nx, 1.0 / ny
    gx, gy = syn.adjoint_weights(nx, ny, seed=nx + k)
    a32, path = _adjoint(nx, ny, k, dx, dy, "fp32", gx, gy)
    assert path == 2
    a64, _ = _adjoint(nx, ny, k, dx, dy, "fp64", gx, gy)
    assert _rel(a32, a64) <= TOL_FP32


@pytest.mark.parametrize("k", [1, 2, 3])
def test_network_adjoint_vs_oracle(k):
    nx, ny = 160, 208
    dx, dy = 1.0 / nx, 0.6 / ny
    rng = np.random.default_rng(30 + k)
    gx, gy = rng.standard_normal((nx, ny)), rng.standard_normal((nx, ny))
    ref = oracle_solver(nx, ny, k, dx, dy).adjoint(gx, gy)
    got, path = _adjoint(nx, ny, k, dx, dy, "fp32", gx, gy)
    assert path == 2
    assert _rel(got, ref) <= TOL_FP32
