"""The potential on the GPU (a diagnostic beside the forces) against the FP64 oracle.

Phi = -G sum C w^phi, w^phi the potential integral of the B-spline pair; built on request
(Plan.build_potential) and solved by the generic kernels in every precision form.
Tolerances: FP64 relative L2 <= 1e-12, FP32 <= 1e-5.
"""
import numpy as np
import pytest

from gpu_common import TOL_FP32, TOL_FP64, library, oracle_solver, to_np
from workloads import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    library()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _phi(nx, ny, k, dx, dy, prec, sigma, G=1.0):
    import torch
    from paper_1904_07400_gb300.api import Plan
    p = Plan(nx, ny, k, dx, dy, G=G, precision=prec)
    p.build_potential()
    out = p.potential(torch.as_tensor(sigma, dtype=p.dtype, device=p.device))
    torch.cuda.synchronize()
    return to_np(out)


@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (5, 7), (17, 33), (64, 48)])
@pytest.mark.parametrize("k", [1, 3, 5])
def test_potential_small_and_ragged_vs_oracle(shape, k):
    nx, ny = shape
    d = 1.0 / max(nx, ny)
    sigma = np.random.default_rng(nx + ny + k).standard_normal((nx, ny))
    ref = oracle_solver(nx, ny, k, d, d).potential(sigma, method="direct" if nx * ny <= 4096 else "fft")
    for prec, tol in (("fp64", TOL_FP64), ("fp32", TOL_FP32)):
        assert _rel(_phi(nx, ny, k, d, d, prec, sigma), ref) <= tol, prec


@pytest.mark.parametrize("k", [2, 4])
def test_potential_512_disk_and_G(k):
    N = 512
    _, _, dx, dy = syn.grid(N, N)
    sigma = syn.perturbed_disk(3, N, seed=2)
    ref = oracle_solver(N, N, k, dx, dy, 0.5).potential(sigma)
    assert _rel(_phi(N, N, k, dx, dy, "fp64", sigma, G=0.5), ref) <= TOL_FP64
    assert _rel(_phi(N, N, k, dx, dy, "fp32", sigma, G=0.5), ref) <= TOL_FP32


def test_potential_4096_fp32_vs_fp64_and_network_plan():
    # FP32 plans of network sizes run the potential through the generic kernels on their
    # padded periods
    N = 4096
    _, _, dx, dy = syn.grid(N, N)
    sigma = syn.clumps(N, N, seed=3)
    a = _phi(N, N, 3, dx, dy, "fp64", sigma)
    b = _phi(N, N, 3, dx, dy, "fp32", sigma)
    assert _rel(b, a) <= TOL_FP32


def test_potential_order_of_accuracy_on_gpu():
    # D4 disk on [-1, 1]^2: order 4 for k = 3 (the oracle shows the same)
    from oracle.analytic import disk_potential
    from oracle.norms import orders, paper_norms
    l2 = []
    for N in (32, 64, 128):
        x, y, dx, dy = syn.grid(N, N, -1.0, 1.0)
        phi = _phi(N, N, 3, dx, dy, "fp64", syn.maclaurin_density(4, x, y, 0.5))
        X, Y = np.meshgrid(x, y, indexing="ij")
        Rg = np.round(np.hypot(X, Y), 14)
        ur, inv = np.unique(Rg, return_inverse=True)
        ref = disk_potential(4, ur, 0.5, dps=15)[inv].reshape(Rg.shape)
        l2.append(paper_norms(phi - ref, dx, dy)[1])
    assert abs(orders(l2)[-1] - 4.0) < 0.15, l2


def test_potential_not_built_and_argument_errors():
    import torch
    from paper_1904_07400_gb300 import native
    from paper_1904_07400_gb300.api import Plan
    p = Plan(32, 32, 3, 1 / 32, 1 / 32, precision="fp32")
    s = torch.zeros((32, 32), dtype=torch.float32, device=p.device)
    with pytest.raises(native.TdgError):
        p.potential(s)  # no potential spectrum yet
    p.build_potential()
    with pytest.raises(native.TdgError):
        native.call("tdg_solve_potential", p.handle, s.data_ptr(), s.data_ptr(), None)  # aliased
    assert float(p.potential(s).abs().max()) == 0.0
