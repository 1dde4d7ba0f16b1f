"""The slab decomposition of one grid on one GPU: every rank's passes run in the library's
slab kernels (pass A on its rows, pass B on its frequency columns, pass C on its rows), with
the two all-to-all transposes carried out as device copies of the same chunks a multi-GPU
run exchanges.  The assembled forces equal the whole-grid solve bit for bit (the same
kernels on the same data) and the FP64 oracle within the FP32 tolerance."""
import numpy as np
import pytest

from gpu_common import TOL_FP32, library, oracle_solver, rel_l2_pair, to_np
from workloads import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    library()


@pytest.mark.parametrize("nx,ny,k,world", [(256, 512, 3, 2), (512, 384, 2, 4), (1024, 1024, 3, 3),
                                           (2048, 1024, 5, 4), (4096, 4096, 3, 2), (4096, 4096, 3, 8),
                                           (1040, 272, 4, 3), (128, 144, 1, 8)])
def test_simulated_ranks_equal_whole_grid_solve(nx, ny, k, world):
    import torch
    from paper_1904_07400_gb300 import slab
    from paper_1904_07400_gb300.api import Plan
    plan = Plan(nx, ny, k, 1.0 / nx, 1.0 / ny, precision="fp32")
    assert plan.path() == 2
    sigma = torch.as_tensor(syn.clumps(nx, ny, seed=nx + ny + k), dtype=torch.float32, device="cuda:0")
    fx, fy = plan.forces(sigma)
    sx, sy = slab.solve_simulated(plan, sigma, world)
    torch.cuda.synchronize()
    assert plan.device_error() == 0
    assert torch.equal(sx, fx) and torch.equal(sy, fy)


@pytest.mark.parametrize("world", [2, 4])
def test_simulated_ranks_vs_oracle(world):
    import torch
    from paper_1904_07400_gb300 import slab
    from paper_1904_07400_gb300.api import Plan
    nx, ny, k = 256, 192, 3
    dx, dy = 1.0 / nx, 0.8 / ny
    sigma = syn.clumps(nx, ny, seed=31) + 0.05 * np.random.default_rng(31).random((nx, ny))
    rx, ry = oracle_solver(nx, ny, k, dx, dy).forces(sigma)
    plan = Plan(nx, ny, k, dx, dy, precision="fp32")
    sx, sy = slab.solve_simulated(plan, torch.as_tensor(sigma, dtype=torch.float32, device="cuda:0"), world)
    torch.cuda.synchronize()
    assert rel_l2_pair(to_np(sx), to_np(sy), rx, ry) <= TOL_FP32


def test_slab_calls_refuse_bad_arguments():
    import ctypes
    import torch
    from paper_1904_07400_gb300 import native
    from paper_1904_07400_gb300.api import Plan
    lib = native.load()
    p64 = Plan(256, 256, 3, 1.0 / 256, 1.0 / 256, precision="fp64")
    assert lib.tdg_slab_bytes(p64.handle, 2, 0, 0) == 0                       # off the network path
    p = Plan(256, 256, 3, 1.0 / 256, 1.0 / 256, precision="fp32")
    assert lib.tdg_slab_bytes(p.handle, 2, 2, 0) == 0                         # rank outside
    assert lib.tdg_slab_bytes(p.handle, 2, 0, 4) == 0                         # no such buffer
    buf = torch.empty(1 << 20, dtype=torch.float32, device="cuda:0")
    assert lib.tdg_slab_rows_forward(p.handle, 2, 0, None, buf.data_ptr(), None) == 1
    assert lib.tdg_slab_rows_forward(p.handle, 2, 0, buf.data_ptr() + 4, buf.data_ptr(), None) == 1
    assert lib.tdg_slab_rows_forward(p.handle, 2, 5, buf.data_ptr(), buf.data_ptr(), None) == 2
    assert lib.tdg_slab_rows_inverse(p.handle, 2, 0, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), None) == 1
    assert lib.tdg_slab_columns(p64.handle, 2, 0, buf.data_ptr(), buf.data_ptr(), None) == 2
