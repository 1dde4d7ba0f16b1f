"""Persistent batched solves: parity with individual solves and the oracle, reuse, CUDA
graph capture, the bounded-wait timeout path and the autotuner.

Tolerance: FP32 relative L2 <= 1e-5 (per grid)."""
import numpy as np
import pytest

from gpu_common import TOL_FP32, library, oracle_solver, rel_l2_pair, to_np
from workloads import synthetic as syn

pytestmark = pytest.mark.gpu

SPECS = [(128, 192, 1), (192, 128, 2), (256, 256, 3), (384, 128, 3), (96, 40, 2), (768, 192, 1),
         (128, 1024, 3), (17, 33, 3), (512, 384, 2), (64, 64, 1)]


@pytest.fixture(scope="module")
def grids():
    import torch
    from paper_1904_07400_gb300.api import Plan
    library()
    plans, sig, ref = [], [], []
    for (nx, ny, k) in SPECS:
        p = Plan(nx, ny, k, 1.0 / nx, 1.0 / ny, precision="fp32")
        s = torch.as_tensor(syn.clumps(nx, ny, seed=nx * 3 + ny), dtype=torch.float32, device=p.device)
        plans.append(p)
        sig.append(s)
        ref.append(p.forces(s))
    torch.cuda.synchronize()
    return plans, sig, ref


def _check(outs, ref):
    for (ax, ay), (bx, by) in zip(outs, ref):
        assert rel_l2_pair(to_np(ax), to_np(ay), to_np(bx), to_np(by)) <= TOL_FP32


def test_batch_matches_individual_solves_and_reuses(grids):
    import torch
    from paper_1904_07400_gb300.api import Batch
    plans, sig, ref = grids
    b = Batch(plans, sig)
    b.launch()
    torch.cuda.synchronize()
    assert b.error() == 0
    _check(b.outs, ref)
    first = [(x.clone(), y.clone()) for x, y in b.outs]
    b.launch()  # counters are reset by every launch
    torch.cuda.synchronize()
    for (ax, ay), (bx, by) in zip(b.outs, first):
        assert torch.equal(ax, bx) and torch.equal(ay, by)
    info = b.info()
    assert info["items"] > 0 and info["blocks"] > 0


def test_batch_against_oracle_small_grids(grids):
    import torch
    from paper_1904_07400_gb300.api import Batch
    plans, sig, _ = grids
    idx = [4, 7, 9]
    b = Batch([plans[i] for i in idx], [sig[i] for i in idx])
    b.launch()
    torch.cuda.synchronize()
    for j, i in enumerate(idx):
        nx, ny, k = SPECS[i]
        rx, ry = oracle_solver(nx, ny, k, 1.0 / nx, 1.0 / ny).forces(to_np(sig[i]))
        assert rel_l2_pair(to_np(b.outs[j][0]), to_np(b.outs[j][1]), rx, ry) <= TOL_FP32


@pytest.mark.parametrize("threads,radix", [(256, 0), (512, 1), (256, 1)])
def test_batch_configs(grids, threads, radix):
    import torch
    from paper_1904_07400_gb300.api import Batch
    plans, sig, ref = grids
    b = Batch(plans[:6], sig[:6])
    b.set_config(threads, radix)
    b.launch()
    torch.cuda.synchronize()
    _check(b.outs, ref[:6])


def test_batch_graph_capture_and_replay(grids):
    import torch
    from paper_1904_07400_gb300.api import Batch
    plans, sig, ref = grids
    b = Batch(plans, sig)
    b.launch()  # first launch outside the capture
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
    g.replay()
    torch.cuda.synchronize()
    _check(b.outs, ref)
    for o in b.outs:
        o[0].zero_()
    g.replay()
    torch.cuda.synchronize()
    _check(b.outs, ref)


def test_batch_bounded_wait_times_out_and_device_survives(grids):
    # the row pass of grid 2 is never counted: its column items exhaust their bounded
    # wait, the batch reports TIMEOUT, and the next normal launch is correct
    import time
    import torch
    from paper_1904_07400_gb300 import native
    from paper_1904_07400_gb300.api import Batch
    plans, sig, ref = grids
    b = Batch(plans[:4], sig[:4])
    b.withhold(2)
    t0 = time.time()
    b.launch()
    torch.cuda.synchronize()
    assert native.STATUS[b.error()] == "TDG_ERR_TIMEOUT"
    assert time.time() - t0 < 30
    b.withhold(-1)
    b.launch()
    torch.cuda.synchronize()
    assert b.error() == 0
    _check(b.outs, ref[:4])


def test_autotuner_picks_and_caches(grids, tmp_path):
    import torch
    from paper_1904_07400_gb300 import autotune
    from paper_1904_07400_gb300.api import Batch
    plans, sig, ref = grids
    b = Batch(plans, sig)
    path = tmp_path / "tune.json"
    rec = autotune.tune(b, str(path), reps=2)
    assert path.exists() and rec["mode"] in ("persistent", "streams")
    assert set(rec["candidates_ms"]) >= {"512/0", "streams/4"}
    if rec["mode"] == "persistent":
        assert rec["threads"] in (256, 512)
    else:
        assert rec["streams"] in autotune.STREAMS
    rec2 = autotune.tune(b, str(path))
    assert {k: rec2[k] for k in rec2 if k != "candidates_ms"} == {k: rec[k] for k in rec if k != "candidates_ms"}
    b.launch()
    torch.cuda.synchronize()
    _check(b.outs, ref)


def test_solve_forces_batched_convenience(grids):
    import torch
    from paper_1904_07400_gb300.api import forces_batched
    plans, sig, ref = grids
    outs = forces_batched(plans, sig)
    torch.cuda.synchronize()
    _check(outs, ref)


@pytest.mark.parametrize("n", [1, 3, 8])
def test_streams_form_matches_and_switches_back(grids, n):
    import torch
    from paper_1904_07400_gb300.api import Batch
    plans, sig, ref = grids
    b = Batch(plans, sig)
    b.set_streams(n)
    b.launch()
    torch.cuda.synchronize()
    _check(b.outs, ref)
    for o in b.outs:
        o[0].zero_()
        o[1].zero_()
    b.set_config(512, 0)  # back to the persistent kernel
    b.launch()
    torch.cuda.synchronize()
    assert b.error() == 0
    _check(b.outs, ref)


def test_streams_form_graph_capture_and_replay(grids):
    import torch
    from paper_1904_07400_gb300.api import Batch
    plans, sig, ref = grids
    b = Batch(plans, sig)
    b.set_streams(4)
    b.launch()  # first launch outside the capture (kernel attributes, workspaces)
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
    g.replay()
    torch.cuda.synchronize()
    _check(b.outs, ref)
