"""The persistent batched kernel on the transform network's item bodies (threads 64): grids on
the network path with sides up to 1024 cells, of every order, in one launch.  Its item
bodies are the ones the single-grid kernels run, so every grid's forces equal its own solve
bit for bit; the oracle checks a few of them (FP32 relative L2 <= 1e-5).  Also: graph
capture and replay, the bounded wait, and the refusal of grids off the network path."""
import pytest

from gpu_common import TOL_FP32, library, oracle_solver, rel_l2_pair, to_np
from workloads import synthetic as syn

pytestmark = pytest.mark.gpu

SPECS = [(256, 192, 3), (1024, 768, 3), (128, 128, 1), (512, 384, 2), (192, 1024, 4), (768, 256, 5),
         (384, 512, 2), (1024, 1024, 3), (144, 528, 3), (640, 128, 1)]


@pytest.fixture(scope="module")
def grids():
    import torch
    from paper_1904_07400_gb300.api import Plan
    library()
    plans, sig, ref = [], [], []
    for (nx, ny, k) in SPECS:
        p = Plan(nx, ny, k, 1.0 / nx, 1.0 / ny, precision="fp32")
        assert p.path() == 2
        s = torch.as_tensor(syn.clumps(nx, ny, seed=5 * nx + ny), dtype=torch.float32, device=p.device)
        plans.append(p)
        sig.append(s)
        ref.append(p.forces(s))
    torch.cuda.synchronize()
    return plans, sig, ref


def _net_batch(plans, sig, units=2):
    from paper_1904_07400_gb300.api import Batch
    b = Batch(plans, sig)
    b.set_config(64, units)
    assert b.info()["threads"] == 64
    return b


@pytest.mark.parametrize("units", [1, 2, 4, 8, 16, 32])
def test_network_batch_equals_single_solves(grids, units):
    import torch
    plans, sig, ref = grids
    b = _net_batch(plans, sig, units)
    for _ in range(2):  # counters are reset by every launch
        for o in b.outs:
            o[0].fill_(float("nan"))
            o[1].fill_(float("nan"))
        b.launch()
        torch.cuda.synchronize()
        assert b.error() == 0
        for (ax, ay), (bx, by) in zip(b.outs, ref):
            assert torch.equal(ax, bx) and torch.equal(ay, by)


def test_network_batch_against_oracle(grids):
    import torch
    plans, sig, _ = grids
    idx = [0, 2, 3, 8]
    b = _net_batch([plans[i] for i in idx], [sig[i] for i in idx])
    b.launch()
    torch.cuda.synchronize()
    for j, i in enumerate(idx):
        nx, ny, k = SPECS[i]
        rx, ry = oracle_solver(nx, ny, k, 1.0 / nx, 1.0 / ny).forces(to_np(sig[i]))
        assert rel_l2_pair(to_np(b.outs[j][0]), to_np(b.outs[j][1]), rx, ry) <= TOL_FP32


def test_network_batch_graph_capture_and_replay(grids):
    import torch
    plans, sig, ref = grids
    b = _net_batch(plans, sig)
    b.launch()
    torch.cuda.synchronize()
    for o in b.outs:
        o[0].zero_()
        o[1].zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            b.launch()
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        for (ax, ay), (bx, by) in zip(b.outs, ref):
            assert torch.equal(ax, bx) and torch.equal(ay, by)
        for o in b.outs:
            o[0].zero_()


def test_network_batch_bounded_wait_times_out_and_device_survives(grids):
    # the row pass of grid 1 is never counted: its column items run out of their bounded
    # wait, the batch reports TIMEOUT, and the next normal launch is exact
    import time
    import torch
    from paper_1904_07400_gb300 import native
    plans, sig, ref = grids
    b = _net_batch(plans[:4], sig[:4])
    b.withhold(1)
    t0 = time.time()
    b.launch()
    torch.cuda.synchronize()
    assert native.STATUS[b.error()] == "TDG_ERR_TIMEOUT"
    assert time.time() - t0 < 30
    b.withhold(-1)
    b.launch()
    torch.cuda.synchronize()
    assert b.error() == 0
    for (ax, ay), (bx, by) in zip(b.outs, ref[:4]):
        assert torch.equal(ax, bx) and torch.equal(ay, by)


def test_network_form_refuses_grids_off_the_network_path(grids):
    import torch
    from paper_1904_07400_gb300 import native
    from paper_1904_07400_gb300.api import Batch, Plan
    plans, sig, _ = grids
    odd = Plan(17, 33, 3, 1.0 / 17, 1.0 / 33, precision="fp32")
    big = Plan(2048, 128, 3, 1.0 / 2048, 1.0 / 128, precision="fp32")
    for extra in (odd, big):
        s = torch.ones((extra.nx, extra.ny), dtype=torch.float32, device=extra.device)
        with pytest.raises(native.TdgError):
            b = Batch([plans[0], extra], [sig[0], s])
            b.set_config(64, 2)


def test_network_batch_beyond_the_shared_tables():
    # more grids than the kernel keeps in shared memory: the item prefix sums and the
    # per-pass grid orders are read from global memory; every grid still equals its own solve
    import torch
    from paper_1904_07400_gb300.api import Batch, Plan
    library()
    specs = [(128 + 16 * (d % 5), 128 + 16 * (d % 7), 1 + d % 3) for d in range(272)]
    plans, sig, ref = [], [], []
    for d, (nx, ny, k) in enumerate(specs):
        p = Plan(nx, ny, k, 1.0 / nx, 1.0 / ny, precision="fp32")
        s = torch.as_tensor(syn.clumps(nx, ny, seed=7000 + d), dtype=torch.float32, device=p.device)
        plans.append(p)
        sig.append(s)
        ref.append(p.forces(s))
    b = Batch(plans, sig)
    b.set_config(64, 4)
    b.launch()
    torch.cuda.synchronize()
    assert b.error() == 0
    for (ax, ay), (bx, by) in zip(b.outs, ref):
        assert torch.equal(ax, bx) and torch.equal(ay, by)
