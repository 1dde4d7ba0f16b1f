"""Radial-force diagnostics on the GPU (Sec. 3): F_R and the paper's error norms of F^x and
F_R against the analytic D_n forces, computed on the device from the GPU's own forces.

The paper's Tables 4, 6, 7 and 9 (orders 1 and 3 on the D3 and D4 disks) are reproduced to
their printed five digits from GPU FP64 forces with GPU norms, N = 32 ... 256; the norms
equal the oracle's norm definitions applied to the same forces to 1e-12.
"""
import os

import numpy as np
import pytest

from gpu_common import library, to_np
from workloads import synthetic as syn

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    library()


def _rows():
    out = []
    for line in open(os.path.join(GOLDEN, "paper_error_tables.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        out.append((int(f[0]), int(f[1]), int(f[2]), int(f[3]), np.array(list(map(float, f[4:])))))
    return out


def _gpu_norms(k, n, N, prec="fp64"):
    import torch
    from oracle.analytic import cartesian_force
    from paper_1904_07400_gb300.api import Plan
    x, y, dx, dy = syn.grid(N, N, -1.0, 1.0)
    sigma = syn.maclaurin_density(n, x, y, 0.5)
    plan = Plan(N, N, k, dx, dy, precision=prec)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=plan.dtype, device=plan.device)
    fx, fy = plan.forces(t(sigma))
    X, Y = np.meshgrid(x, y, indexing="ij")
    ax, _, ar = cartesian_force(n, X, Y, 0.5)
    fr, norms = plan.radial_diagnostics(fx, fy, -1.0, -1.0, t(ax), t(ar))
    torch.cuda.synchronize()
    assert plan.device_error() == 0
    return np.array(norms), to_np(fx), to_np(fy), to_np(fr), (X, Y, ax, ar, dx, dy)


@pytest.mark.parametrize("row", [r for r in _rows() if r[1] in (1, 3) and r[3] <= 256],
                         ids=lambda r: f"T{r[0]}-N{r[3]}")
def test_gpu_reproduces_printed_error_tables(row):
    from oracle.norms import paper_norms
    tab, k, n, N, printed = row
    ours, fx, fy, fr, (X, Y, ax, ar, dx, dy) = _gpu_norms(k, n, N)
    # the device norms are the oracle's definitions applied to the same forces
    ref = np.array(paper_norms(fx - ax, dx, dy) + paper_norms(fr - ar, dx, dy))
    assert np.all(np.abs(ours - ref) <= 1e-12 * np.abs(ref))
    # F_R itself: (x F^x + y F^y) / R at the cell centres
    np.testing.assert_allclose(fr, (fx * X + fy * Y) / np.hypot(X, Y), rtol=1e-14, atol=1e-15)
    # and the printed five digits
    ulp = 10.0 ** (np.floor(np.log10(np.abs(printed))) - 4)
    assert np.all(np.abs(ours - printed) <= ulp), (ours, printed)


def test_gpu_orders_of_accuracy_up_to_5():
    # order k on D_{k+1}-smooth disks from GPU forces and GPU norms, k = 1 .. 5 (L2 of F^x)
    from oracle.norms import orders
    for k, n in ((1, 4), (2, 4), (3, 4), (4, 5), (5, 6)):
        l2 = [_gpu_norms(k, n, N)[0][1] for N in (64, 128, 256)]
        o = orders(l2)[-1]
        assert k - 0.15 < o < k + 0.6, (k, o)


def test_fp32_radial_force_only_and_zero_radius():
    import torch
    from paper_1904_07400_gb300.api import Plan
    # odd N with dx = 1/64 and the origin at -32.5 dx (all exact in binary): the centre
    # cell sits at R = 0 exactly and gets F_R = 0
    N, dx = 65, 1.0 / 64
    x0 = -32.5 * dx
    x = x0 + (np.arange(N) + 0.5) * dx
    plan = Plan(N, N, 3, dx, dx, precision="fp32")
    s = torch.as_tensor(syn.maclaurin_density(3, x, x, 0.4), dtype=torch.float32, device=plan.device)
    fx, fy = plan.forces(s)
    fr, norms = plan.radial_diagnostics(fx, fy, x0, x0)
    torch.cuda.synchronize()
    assert norms is None
    fr = to_np(fr)
    assert fr[N // 2, N // 2] == 0.0
    X, Y = np.meshgrid(x, x, indexing="ij")
    R = np.hypot(X, Y)
    assert R[N // 2, N // 2] == 0.0
    ok = R > 0
    ref = (to_np(fx) * X + to_np(fy) * Y)[ok] / R[ok]
    np.testing.assert_allclose(fr[ok], ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max())
