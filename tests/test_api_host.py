"""Host-side checks of the Python layer that run before any device work (no GPU needed):
parameter checks of kept kernel tables and of tensors handed to a plan."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def Plan():
    from paper_1904_07400_gb300 import build
    build.build()
    from paper_1904_07400_gb300.api import Plan as P
    return P


def test_build_from_rejects_tables_of_another_plan(Plan, tmp_path):
    p = Plan(16, 12, 3, 0.1, 0.1, precision="fp32", build=False)
    path = str(tmp_path / "t.npz")
    for params in ([16, 12, 2, 0.1, 0.1], [16, 13, 3, 0.1, 0.1], [16, 12, 3, 0.1, 0.2], [16, 12, 3]):
        np.savez(path, wx=np.zeros((16, 12)), wy=np.zeros((16, 12)), params=np.array(params, dtype=float))
        with pytest.raises(ValueError):
            p.build_from(path)
    p.close()


def test_tensor_checks(Plan):
    import torch
    p = Plan(8, 8, 1, 0.1, 0.1, precision="fp64", build=False)
    good_shape_cpu = torch.zeros((8, 8), dtype=torch.float64)
    with pytest.raises(ValueError):
        p.forces(good_shape_cpu)  # not on the plan's device
    with pytest.raises(ValueError):
        p.radial_diagnostics(good_shape_cpu, good_shape_cpu, 0.0, 0.0)
    with pytest.raises(ValueError):
        p.potential(good_shape_cpu)
    p.close()


def test_orders_and_precisions_accepted_at_init(Plan):
    from paper_1904_07400_gb300 import native
    for k in (1, 2, 3, 4, 5):
        for prec in ("fp64", "fp32"):
            Plan(64, 48, k, 0.1, 0.1, precision=prec, build=False).close()
    with pytest.raises(native.TdgError):
        Plan(64, 48, 6, 0.1, 0.1, precision="fp32", build=False)
    # FP32_TC16: columns of 2048 or 4096 transform cells (x sides 1040 .. 4096), any order
    with pytest.raises(native.TdgError):
        Plan(1024, 1024, 3, 0.1, 0.1, precision="fp32_tc16", build=False)
    with pytest.raises(native.TdgError):
        Plan(2000, 1000, 3, 0.1, 0.1, precision="fp32_tc16", build=False)  # y side not a multiple of 16
    for k in (1, 3, 5):
        Plan(2048, 1024, k, 0.1, 0.1, precision="fp32_tc16", build=False).close()
        Plan(1040, 128, k, 0.1, 0.1, precision="fp32_tc16", build=False).close()
