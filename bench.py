#!/usr/bin/env python
"""Throughput of the thin-disk force solve on GB300 (one JSON line on rank 0).

Workload: 4096 x 4096 cells on [-0.5, 0.5]^2, B-spline order 3, G = 1, sigma = 64 seeded
Gaussian clumps (centres uniform in radius < 0.4, widths U(0.005, 0.05), amplitudes
LogNormal(0, 1)).  One step = one complete force solve (all passes: B-spline solves, padded
forward transform, both spectrum products, both inverse transforms with the crop) through
the library's C ABI.  Kernel tables are built once per plan before timing and excluded.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--gpus N` (N > 1) from a plain `python bench.py` re-launches the script as N ranks with
torch.distributed.run; under a launcher the world size must equal N.

Headline `value`: FP32 form, Mpts/s (nx * ny output points per solve), inputs resident in
HBM.  `e2e`: the same through the public API with the input copied from pinned host memory
and both force components copied back every step.  `forms`: every precision form timed the
same way, each with its relative L2 error against the FP64 CPU oracle (oracle solves of the
same grid, timed on all host cores and on one thread, best of 3: `cpu_baseline`).  With
N > 1 each rank solves its own grid (independent replicas, no collective on the data
path): weak scaling.  A one-GPU run also times, after the headline and outside its timed
region, the method's other workloads (`secondary`: the 256-grid uneven batch as one CUDA
graph, the adjoint at 2048^2, orders 4 and 5 on the headline grid with their table
builds); `--no-secondary` skips them.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mpts/s force solve, order-3 4096^2: FP32/TC vs FP64 GPU at rel err <= 1e-5"
WORKLOAD = "4096x4096 order-3 clumped thin disk (64 Gaussian clumps, seed 3), [-0.5,0.5]^2, G=1"
N_GRID, ORDER, SEED = 4096, 3, 3
PASSES = ("rows_r2c", "cols_conv", "rows_c2r")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--forms", default="fp32,fp32_tc16,fp64")
    ap.add_argument("--size", type=int, default=N_GRID)
    ap.add_argument("--order", type=int, default=ORDER, choices=[1, 2, 3, 4, 5],
                    help="B-spline order of the solve (the headline workload is order 3)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-depth", type=int, default=3,
                    help="end-to-end steps in flight (one stream and workspace each)")
    ap.add_argument("--next2", action="store_true",
                    help="time the in-simulation reuse pieces on the workload grid instead: a table "
                         "build against a rebuild from kept tables, the potential solve and the "
                         "radial diagnostics")
    ap.add_argument("--batched", action="store_true",
                    help="time the uneven batch (256 grids, one persistent launch) instead")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the secondary workloads that a one-GPU run adds to its line (the 256-grid "
                         "batch, the 2048^2 adjoint, orders 4 and 5, the kernel-table build)")
    ap.add_argument("--dry-run", action="store_true",
                    help="check the rank launch only: every rank joins a gloo group on the CPU and rank 0 "
                         "prints the world size it saw (no GPU work)")
    return ap.parse_args()


def launch_ranks(args):
    """`--gpus N` with N > 1 from a plain `python bench.py` re-launches this script as N
    ranks through torch.distributed.run (one process per GPU, 127.0.0.1 rendezvous); under a
    launcher the world size must equal N."""
    world = os.environ.get("WORLD_SIZE")
    if world is not None:
        if int(world) != args.gpus:
            sys.exit(f"bench.py: --gpus {args.gpus} but the launcher started WORLD_SIZE={world} ranks")
        return
    if args.gpus <= 1:
        return
    import socket
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *sys.argv[1:]]
    env = dict(os.environ)
    # NCCL's init log (to stderr, keeping stdout for the JSON line) shows the communicator size
    env.setdefault("NCCL_DEBUG", "INFO")
    env.setdefault("NCCL_DEBUG_SUBSYS", "INIT")
    env.setdefault("NCCL_DEBUG_FILE", "/dev/stderr")
    sys.exit(subprocess.call(cmd, env=env))


# ------------------------------------------------------------------------------------------
# distributed plumbing (one process per GPU, replicas)
# ------------------------------------------------------------------------------------------

def dist_setup(n, cpu=False):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if cpu:
            dist.init_process_group("gloo")
        else:
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    elif not cpu:
        torch.cuda.set_device(0)
    return rank, world, local


def run_dry(args):
    """The multi-rank plumbing without GPU work: ranks, barrier and max over ranks."""
    rank, world, _ = dist_setup(args.gpus, cpu=True)
    barrier(world)
    t = max_over_ranks(float(rank), world)
    if rank == 0:
        print(json.dumps({"dry_run": True, "n_gpus": world, "gpus_requested": args.gpus,
                          "max_over_ranks_of_rank": t}), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def barrier(world):
    from paper_1904_07400_gb300 import dist as pdist
    pdist.barrier(world)


def max_over_ranks(x, world):
    from paper_1904_07400_gb300 import dist as pdist
    return pdist.max_over_ranks(x, world)


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------

class NvmlClocks:
    """SM clock and clock-event reasons read through NVML (read-only queries) by a thread
    polling every 2 ms while the timed region runs, so even a short region gets samples.
    Reason bits are NVML's clocks-event-reason constants."""
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def __init__(self, index):
        import ctypes
        import threading
        self.ct, self.threading = ctypes, threading
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.lib = lib
        self.h = ctypes.c_void_p()
        if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h)) != 0:
            raise RuntimeError("no NVML handle")
        self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint()
        self.max_mhz = float(mx.value) if lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0 else None
        self.rows, self.stop_flag, self.thread = [], None, None

    def _poll(self):
        ct = self.ct
        mhz, mask = ct.c_uint(), ct.c_ulonglong()
        while not self.stop_flag.is_set():
            if self.lib.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(mhz)) == 0 and \
                    self.reasons_fn(self.h, ct.byref(mask)) == 0:
                self.rows.append((float(mhz.value), int(mask.value)))
            self.stop_flag.wait(0.002)

    def start(self):
        self.rows = []
        self.stop_flag = self.threading.Event()
        self.thread = self.threading.Thread(target=self._poll, daemon=True)
        self.thread.start()

    def stop(self):
        self.stop_flag.set()
        self.thread.join(timeout=5)
        if not self.rows:
            return None
        reasons = sorted({n for _, m in self.rows for n, b in self.BITS.items() if m & b})
        return {"sm_mhz": statistics.median(r[0] for r in self.rows),
                "sm_max_mhz": self.max_mhz if self.max_mhz else max(r[0] for r in self.rows),
                "samples": len(self.rows), "reasons": reasons, "source": "nvml"}


def make_clocks(index):
    try:
        return NvmlClocks(index)
    except Exception:
        return Clocks(index)


class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons, "source": "nvidia-smi"}


# ------------------------------------------------------------------------------------------
# algorithmic bytes per pass (FP32: 4-byte reals, 8-byte complex)
# ------------------------------------------------------------------------------------------

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the
# dominant kernel, from one ncu capture of this workload (FP32 network path, 4096x4096,
# order 3).  Valid only for the kernel sources it was taken on: reported when their SHA-256
# still matches, null otherwise.
MEASURED_TRAFFIC = {
    ("cols_conv", 2, 4096): {"bytes": 268_820_736 + 215_590_912,
                             "sha256": "9c3b32e3e86bf85bce6e01d23906a0aefd4b2b0c4725db0bcf5b837c5fa581a5"},
}
TRAFFIC_SOURCES = ("paper_1904_07400_gb300/csrc/net_fp32.cu", "paper_1904_07400_gb300/csrc/fft_net.cuh",
                   "paper_1904_07400_gb300/csrc/fft_reg.cuh")


def measured_traffic(kernel, path, n, form):
    entry = MEASURED_TRAFFIC.get((kernel, path, n))
    if entry is None or form != "fp32" or ORDER != 3:
        return None
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return entry["bytes"] if h.hexdigest() == entry["sha256"] else None


def pass_bytes(nx, ny, px, real, path):
    """Compulsory bytes of each pass: every array it must read or write once, spectra as the
    kernel path stores them (generic: both full spectra, P_x reals per frequency column;
    register path: half spectra, nx + 4 reals per column)."""
    hy = ny + 1
    cplx = 2 * real
    spec = 2 * hy * px * real if path == 0 else hy * (nx + 4) * 2 * real
    a = nx * ny * real + nx * hy * cplx                        # sigma in, Z out
    b = nx * hy * cplx + spec + 2 * nx * hy * cplx             # Z in, spectra, G_x G_y out
    c = 2 * nx * hy * cplx + 2 * nx * ny * real                # G_x G_y in, F^x F^y out
    return {"rows_r2c": a, "cols_conv": b, "rows_c2r": c}


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------

def time_form(form, sigma_host, n, K, W, world, rank, clocks=None):
    import numpy as np
    import torch
    from paper_1904_07400_gb300 import native
    from paper_1904_07400_gb300.api import Plan

    dx = 1.0 / n
    plan = Plan(n, n, ORDER, dx, dx, precision=form, device=torch.cuda.current_device())
    dev = plan.device
    stream = torch.cuda.current_stream(dev)
    sigma = torch.as_tensor(sigma_host, dtype=plan.dtype).to(dev)
    fx = torch.empty_like(sigma)
    fy = torch.empty_like(sigma)
    for _ in range(W):
        plan.forces(sigma, out=(fx, fy))
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        plan.forces(sigma, out=(fx, fy))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    ms = max_over_ranks(e0.elapsed_time(e1) / K, world)

    # per-pass durations: events recorded by the library between its launches
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    for row in evs:
        for e in row:
            e.record(stream)  # materialise the handles
    torch.cuda.synchronize()
    lib = native.load()
    arr = ctypes.c_void_p * 4
    for row in evs:
        handles = arr(*[e.cuda_event for e in row])
        native.check("tdg_set_pass_events", lib.tdg_set_pass_events(plan.handle, handles, 4))
        plan.forces(sigma, out=(fx, fy))
    torch.cuda.synchronize()
    native.check("tdg_set_pass_events", lib.tdg_set_pass_events(plan.handle, None, 0))
    per_pass = {name: statistics.mean(row[i].elapsed_time(row[i + 1]) for row in evs)
                for i, name in enumerate(PASSES)}

    # end to end through the public API: every step copies its input from pinned host
    # memory, solves, and copies both components back to pinned host memory.  Consecutive
    # steps rotate over E2E_DEPTH streams, each with its own device buffers and plan
    # workspace, so one step's copies overlap the next steps' solves (the copy engines
    # and the SMs work at the same time).
    h_sig = torch.as_tensor(sigma_host, dtype=plan.dtype).pin_memory()
    depth = max(1, E2E_DEPTH)
    lanes = []
    for _ in range(depth):
        lanes.append({
            "stream": torch.cuda.Stream(dev),
            "ws": torch.empty(plan.workspace_bytes(), dtype=torch.uint8, device=dev),
            "sig": torch.empty_like(sigma), "fx": torch.empty_like(sigma), "fy": torch.empty_like(sigma),
            "hfx": torch.empty(sigma.shape, dtype=plan.dtype).pin_memory(),
            "hfy": torch.empty(sigma.shape, dtype=plan.dtype).pin_memory(),
        })

    def e2e_step(k):
        ln = lanes[k % depth]
        with torch.cuda.stream(ln["stream"]):
            ln["sig"].copy_(h_sig, non_blocking=True)
            plan.set_workspace(ln["ws"])
            plan.forces(ln["sig"], out=(ln["fx"], ln["fy"]))
            ln["hfx"].copy_(ln["fx"], non_blocking=True)
            ln["hfy"].copy_(ln["fy"], non_blocking=True)

    def run_e2e(nsteps):
        start = torch.cuda.Event()
        start.record(stream)
        for ln in lanes:
            ln["stream"].wait_event(start)
        for k in range(nsteps):
            e2e_step(k)
        for ln in lanes:
            done = torch.cuda.Event()
            done.record(ln["stream"])
            stream.wait_event(done)

    run_e2e(max(depth, W))
    torch.cuda.synchronize()
    barrier(world)
    e0.record(stream)
    run_e2e(K)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / K, world)
    last = lanes[(K - 1) % depth]
    out = (last["hfx"].numpy().astype(np.float64), last["hfy"].numpy().astype(np.float64))
    plan.set_workspace(None)
    info = plan.info()
    res = {"ms": ms, "per_pass_ms": per_pass, "e2e_ms": e2e_ms, "clocks": clk, "px": info["px"],
           "path": plan.path(),
           "real": 8 if form == "fp64" else 4, "h2d": sigma.numel() * sigma.element_size(),
           "d2h": 2 * sigma.numel() * sigma.element_size(), "device_error": plan.device_error()}
    plan.close()
    return res, out


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def oracle_solve(sigma, n, reps=3):
    """FP64 CPU oracle on the same grid, timed on all host cores (scipy's pocketfft with
    workers = os.cpu_count()) and on one thread (numpy's), best of `reps` each; returns
    (forces, seconds all cores, seconds one thread, cores)."""
    from oracle.convolution import Solver
    S = Solver(n, n, ORDER, 1.0 / n, 1.0 / n)
    _ = S.spec  # tables and their transforms: built once, not timed
    cores = os.cpu_count() or 1

    def best(workers):
        out, secs = None, []
        for _ in range(reps):
            t = time.perf_counter()
            out = S.forces(sigma, workers=workers)
            secs.append(time.perf_counter() - t)
        return out, min(secs)
    f, t_all = best(cores)
    _, t_one = best(None)
    return f, t_all, t_one, cores


def rel_l2_pair(ax, ay, bx, by):
    """Relative L2 difference of the pair (ax, ay) from (bx, by) over all cells (FP64)."""
    import numpy as np
    num = np.sum((np.asarray(ax, np.float64) - bx) ** 2) + np.sum((np.asarray(ay, np.float64) - by) ** 2)
    den = np.sum(np.asarray(bx, np.float64) ** 2) + np.sum(np.asarray(by, np.float64) ** 2)
    return float(np.sqrt(num / den))


def run_ours(args):
    import numpy as np
    import torch
    from workloads import synthetic as syn

    rank, world, local = dist_setup(args.gpus)
    n = args.size
    sigma = syn.clumps(n, n, seed=SEED + 1000 * rank)
    forms = [f.strip() for f in args.forms.split(",") if f.strip()]
    results, outputs = {}, {}
    for i, form in enumerate(forms):
        clocks = make_clocks(local) if i == 0 else None
        results[form], outputs[form] = time_form(form, sigma, n, args.steps, args.warmup, world, rank, clocks)

    head = forms[0]
    r = results[head]
    pts = n * n
    value = world * pts / (r["ms"] * 1e-3) / 1e6
    line = {"metric": METRIC, "value": round(value, 1), "unit": "Mpts/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(r["ms"], 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if head != "fp64" else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if n == N_GRID else WORKLOAD.replace("4096x4096", f"{n}x{n}"),
                       "nx": n, "ny": n, "order": ORDER, "form": head, "parallelism": f"replicas{world}",
                       "l2": "no flush: per-step working set ~0.6 GB (sigma, 3 intermediates, spectra, forces) "
                             "exceeds the 126 MB L2"}}
    # roofline of the dominant kernel (largest share of the step)
    pk = peaks()
    dom = max(r["per_pass_ms"], key=r["per_pass_ms"].get)
    algo = pass_bytes(n, n, r["px"], r["real"], r["path"])[dom]
    achieved = algo / (r["per_pass_ms"][dom] * 1e-3) / 1e9
    peak = pk["hbm_gbs"] if pk else 6800.0
    line["roofline"] = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                        "unit": "GB/s", "frac": round(achieved / peak, 4),
                        "traffic": measured_traffic(dom, r["path"], n, head),
                        "peak_source": "measured" if pk else "fallback",
                        "algorithmic_bytes": algo,
                        "pass_ms": {k: round(v, 4) for k, v in r["per_pass_ms"].items()},
                        "step_bytes": sum(pass_bytes(n, n, r["px"], r["real"], r["path"]).values()),
                        # sigma in, F^x and F^y out, one quarter spectrum table: 16 B a point (FP32)
                        "compulsory_bytes": 16 * n * n,
                        "compulsory_frac": round(16 * n * n / (r["ms"] * 1e-3) / 1e9 / peak, 4),
                        "kernel_path": {0: "generic", 2: "network", 3: "network, tensor-core column pass"}.get(r["path"], "generic")}
    line["e2e"] = {"value": round(world * pts / (r["e2e_ms"] * 1e-3) / 1e6, 1), "unit": "Mpts/s",
                   "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"]}
    line["gpu_launches"] = 3 * args.steps  # rows, columns, inverse rows per solve
    if r["clocks"]:
        line["clocks"] = r["clocks"]
    line["forms"] = {f: {"Mpts_s": round(world * pts / (results[f]["ms"] * 1e-3) / 1e6, 1),
                         "ms": round(results[f]["ms"], 4),
                         "pass_ms": {k: round(v, 4) for k, v in results[f]["per_pass_ms"].items()},
                         "e2e_Mpts_s": round(world * pts / (results[f]["e2e_ms"] * 1e-3) / 1e6, 1)}
                     for f in forms}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ref, t_all, t_one, cores = oracle_solve(sigma, n)
        line["cpu_baseline"] = {"value": round(pts / t_all / 1e6, 3), "unit": "Mpts/s", "cores": cores,
                                "kind": "oracle",
                                "single_thread_value": round(pts / t_one / 1e6, 3),
                                "sample": f"FP64 oracle solves of the same {n}x{n} grid, best of 3: value on all "
                                          f"{cores} host cores (scipy pocketfft, workers={cores}), "
                                          "single_thread_value with numpy pocketfft on one thread; kernel tables "
                                          "built beforehand and not timed"}
        for f in forms:
            line["forms"][f]["rel_l2_vs_oracle"] = float(f"{rel_l2_pair(*outputs[f], *ref):.3e}")
        # the 512^2 workload (perturbed D3 disk, seed 2) too, order 3
        s512 = syn.perturbed_disk(3, 512, seed=2)
        _, t5_all, t5_one, _ = oracle_solve(s512, 512)
        line["cpu_baseline"]["config_512"] = {
            "all_cores_ms": round(t5_all * 1e3, 2), "single_thread_ms": round(t5_one * 1e3, 2),
            "all_cores_Mpts_s": round(512 * 512 / t5_all / 1e6, 3),
            "sample": "FP64 oracle solves of the 512x512 perturbed D3 disk (seed 2), order 3, best of 3"}
    if "fp64" in outputs:
        for f in forms:
            if f != "fp64":
                line["forms"][f]["rel_l2_vs_fp64_gpu"] = float(f"{rel_l2_pair(*outputs[f], *outputs['fp64']):.3e}")
    bad = [f for f in forms if results[f]["device_error"]]
    if bad:
        line["device_error"] = bad
    if rank == 0 and world == 1 and not args.no_secondary and n == N_GRID:
        del outputs
        line["secondary"] = secondary_workloads()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle as it stands, on the host cores
# ------------------------------------------------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    from oracle.convolution import Solver
    from workloads import synthetic as syn

    # each step is one oracle solve of the same recipe on all host cores (scipy's pocketfft
    # with workers = os.cpu_count()); the grid is scaled down (by 2 per side at a time, from
    # 4096) only if the whole run would not finish within a few minutes
    cores = os.cpu_count() or 1
    budget = 150.0
    steps = args.steps + args.warmup
    n = min(args.size, 512)
    probe = Solver(n, n, ORDER, 1.0 / n, 1.0 / n)
    _ = probe.spec
    sig = syn.clumps(n, n, seed=SEED)
    probe.forces(sig, workers=cores)
    t = time.perf_counter()
    probe.forces(sig, workers=cores)
    per = time.perf_counter() - t
    while n * 2 <= args.size and per * 4.4 * steps < budget:
        n *= 2
        per *= 4.4
    S = Solver(n, n, ORDER, 1.0 / n, 1.0 / n)
    _ = S.spec
    sigma = syn.clumps(n, n, seed=SEED)
    for _ in range(args.warmup):
        S.forces(sigma, workers=cores)
    t = time.perf_counter()
    for _ in range(args.steps):
        S.forces(sigma, workers=cores)
    secs = (time.perf_counter() - t) / args.steps
    value = n * n / secs / 1e6
    sample = (f"each step one FP64 oracle solve (scipy pocketfft on {cores} host threads) of the {n}x{n} grid "
              f"of the same recipe{'' if n == args.size else ' (scaled down from 4096x4096 to bound the run)'}")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "Mpts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(secs * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if n == N_GRID else WORKLOAD.replace("4096x4096", f"{n}x{n}"),
                       "nx": n, "ny": n, "order": ORDER, "form": "oracle-fp64-cpu"},
            "cpu_baseline": {"value": round(value, 3), "unit": "Mpts/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 3), "unit": "Mpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batched(args):
    """256 independent grids (sides from 128 to 1024, orders 1-3, clumped densities), FP32:
    one persistent launch (captured in a CUDA graph) against 256 separate solves.  On N
    ranks each rank takes its LPT share of the grids (no collective on the data path) and
    the time is the maximum over ranks; the total work is fixed (strong scaling)."""
    import torch
    from paper_1904_07400_gb300 import autotune
    from paper_1904_07400_gb300 import dist as pdist
    from paper_1904_07400_gb300.api import Batch, Plan
    from workloads import synthetic as syn

    rank, world, local = dist_setup(0)
    all_specs = syn.batched_specs(256, seed=4)
    shard = pdist.shard_lpt([pdist.solve_cost(nx, ny) for nx, ny, _, _ in all_specs], world)[rank]
    specs = [all_specs[i] for i in shard]
    plans, sig = [], []
    for nx, ny, k, seed in specs:
        p = Plan(nx, ny, k, 1.0 / nx, 1.0 / ny, precision="fp32")
        plans.append(p)
        sig.append(torch.as_tensor(syn.clumps(nx, ny, seed=seed), dtype=torch.float32, device="cuda"))
    pts = sum(nx * ny for nx, ny, _, _ in all_specs)
    b = Batch(plans, sig)
    tune = autotune.tune(b, None, reps=3)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the persistent kernel at its best setting first, then the tuned form in a graph
    pers = {k: v for k, v in tune["candidates_ms"].items() if not k.startswith("streams")}
    best_p = min(pers, key=pers.get)
    b.set_config(*(int(x) for x in best_p.split("/")))
    for _ in range(args.warmup):
        b.launch()
    torch.cuda.synchronize()
    barrier(world)
    e0.record(stream)
    for _ in range(args.steps):
        b.launch()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms_batch = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
    autotune._apply(b, tune)
    b.launch()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s2 = torch.cuda.Stream()
    s2.wait_stream(stream)
    with torch.cuda.stream(s2):
        with torch.cuda.graph(g, stream=s2):
            b.launch()
    stream.wait_stream(s2)
    g.replay()
    torch.cuda.synchronize()
    barrier(world)
    e0.record(stream)
    for _ in range(args.steps):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms_graph = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
    outs = [(torch.empty_like(x), torch.empty_like(x)) for x in sig]
    for p, x, o in zip(plans, sig, outs):
        p.forces(x, out=o)
    torch.cuda.synchronize()
    barrier(world)
    e0.record(stream)
    for _ in range(args.steps):
        for p, x, o in zip(plans, sig, outs):
            p.forces(x, out=o)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms_sep = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
    err = b.error()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank != 0:
        return
    line = {"metric": "Mpts/s batched force solves, 256 uneven grids (128..1024 per side, orders 1-3)",
            "value": round(pts / (ms_graph * 1e-3) / 1e6, 1), "unit": "Mpts/s", "n_gpus": world,
            "scaling": "strong",
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_graph, 4),
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "256 grids, sides from {128,...,1024}, orders 1-3, clumps, seed 4",
                       "points": pts, "autotuned": tune},
            "form": tune["mode"] if tune["mode"] == "persistent" else f"streams/{tune['streams']}",
            "persistent_ms": round(ms_batch, 4), "persistent_config": best_p, "graph_ms": round(ms_graph, 4),
            "separate_solves_ms": round(ms_sep, 4),
            "separate_Mpts_s": round(pts / (ms_sep * 1e-3) / 1e6, 1), "error": err,
            "grids_on_rank0": len(shard)}
    print(json.dumps(line), flush=True)


E2E_DEPTH = 3


def secondary_workloads(steps=20, warmup=3):
    """The other workloads of the method, timed on the same GPU after the headline (CUDA
    events, device-resident synthetic inputs): the 256-grid uneven batch in the autotuner's
    form replayed as one CUDA graph, the adjoint at 2048^2 (order 3), the 512^2 perturbed
    disk at orders 1-3 (FP32 against FP64), the forward solve at orders 4 and 5 on the
    headline grid, and one kernel-table build of it."""
    import gc
    import torch
    from paper_1904_07400_gb300 import autotune
    from paper_1904_07400_gb300.api import Batch, Plan
    from workloads import synthetic as syn

    gc.collect()
    torch.cuda.empty_cache()
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    out = {}
    # the uneven batch
    specs = syn.batched_specs(256, seed=4)
    plans, sig = [], []
    for nx, ny, k, seed in specs:
        plans.append(Plan(nx, ny, k, 1.0 / nx, 1.0 / ny, precision="fp32"))
        sig.append(torch.as_tensor(syn.clumps(nx, ny, seed=seed), dtype=torch.float32, device="cuda"))
    pts = sum(nx * ny for nx, ny, _, _ in specs)
    b = Batch(plans, sig)
    tune = autotune.tune(b, None, reps=3)
    b.launch()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s2 = torch.cuda.Stream()
    s2.wait_stream(stream)
    with torch.cuda.stream(s2):
        with torch.cuda.graph(g, stream=s2):
            b.launch()
    stream.wait_stream(s2)
    ms = timed(g.replay)
    out["batched_256_grids"] = {
        "ms": round(ms, 4), "Mpts_s": round(pts / (ms * 1e-3) / 1e6, 1), "points": pts,
        "form": "persistent/%d" % tune["radix_pref"] if tune["mode"] == "persistent" else "streams/%d" % tune["streams"],
        "candidates_ms": {k: round(v, 4) for k, v in tune["candidates_ms"].items()}, "error": b.error(),
        "workload": "256 grids, sides from {128,...,1024}, orders 1-3, clumps, seed 4, one CUDA graph"}
    del b, g, plans, sig
    gc.collect()
    torch.cuda.empty_cache()
    # the adjoint (dL/dsigma for L = sum g_x F^x + g_y F^y) at 2048^2
    n2 = 2048
    p = Plan(n2, n2, ORDER, 1.0 / n2, 1.0 / n2, precision="fp32")
    gx, gy = syn.adjoint_weights(n2, n2, seed=6)
    tgx = torch.as_tensor(gx, dtype=torch.float32, device="cuda")
    tgy = torch.as_tensor(gy, dtype=torch.float32, device="cuda")
    res = torch.empty_like(tgx)
    ms = timed(lambda: p.adjoint(tgx, tgy, out=res))
    out["adjoint_2048"] = {"ms": round(ms, 4), "Mpts_s": round(n2 * n2 / (ms * 1e-3) / 1e6, 1),
                           "error": p.device_error(), "workload": "2048x2048 order 3, g_x, g_y ~ N(0, 1) (seed 6)"}
    del p, tgx, tgy, res
    gc.collect()
    torch.cuda.empty_cache()
    # the 512^2 workload: perturbed D3 disk (seed 2), orders 1-3, FP32 against FP64 on the GPU
    n5 = 512
    s5 = torch.as_tensor(syn.perturbed_disk(3, n5, seed=2), dtype=torch.float64, device="cuda")
    s5f = s5.float()
    cfg = {}
    for k in (1, 2, 3):
        p32 = Plan(n5, n5, k, 1.0 / n5, 1.0 / n5, precision="fp32")
        p64 = Plan(n5, n5, k, 1.0 / n5, 1.0 / n5, precision="fp64")
        o32 = (torch.empty_like(s5f), torch.empty_like(s5f))
        o64 = (torch.empty_like(s5), torch.empty_like(s5))
        ms32 = timed(lambda: p32.forces(s5f, out=o32))
        ms64 = timed(lambda: p64.forces(s5, out=o64))
        rel = rel_l2_pair(*(o.cpu().numpy() for o in o32), *(o.cpu().numpy() for o in o64))
        cfg[f"order{k}"] = {"fp32_ms": round(ms32, 4), "fp64_ms": round(ms64, 4),
                            "fp32_Mpts_s": round(n5 * n5 / (ms32 * 1e-3) / 1e6, 1),
                            "fp64_Mpts_s": round(n5 * n5 / (ms64 * 1e-3) / 1e6, 1),
                            "rel_l2_fp32_vs_fp64_gpu": float(f"{rel:.3e}")}
        del p32, p64
    out["disk_512"] = cfg
    gc.collect()
    # orders 4 and 5 on the headline grid, and one table build
    n = N_GRID
    sigma = torch.as_tensor(syn.clumps(n, n, seed=SEED), dtype=torch.float32, device="cuda")
    fx, fy = torch.empty_like(sigma), torch.empty_like(sigma)
    for k in (4, 5):
        t0 = time.perf_counter()
        p = Plan(n, n, k, 1.0 / n, 1.0 / n, precision="fp32")
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t0
        ms = timed(lambda: p.forces(sigma, out=(fx, fy)))
        out[f"order{k}_{n}"] = {"ms": round(ms, 4), "Mpts_s": round(n * n / (ms * 1e-3) / 1e6, 1),
                                "table_build_s": round(build_s, 3), "error": p.device_error()}
        del p
        gc.collect()
    return out


def run_next2(args):
    """One JSON line: the reuse pieces on the workload grid (FP32 plan, device-resident data).
    Builds are timed with host clocks around the synchronising build calls; the potential
    and the diagnostics with CUDA events over K calls after W warm-up calls."""
    import numpy as np
    import torch
    from paper_1904_07400_gb300.api import Plan
    from workloads import synthetic as syn

    n, k = args.size, ORDER
    d = 1.0 / n
    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = time.perf_counter()
    plan = Plan(n, n, k, d, d, precision="fp32", device=dev)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "tables.npz")
        plan.save_tables(path)
        t0 = time.perf_counter()
        again = Plan(n, n, k, d, d, precision="fp32", device=dev, tables=path)
        torch.cuda.synchronize()
        t_from = time.perf_counter() - t0
    again.close()
    t0 = time.perf_counter()
    plan.build_potential()
    torch.cuda.synchronize()
    t_pot_build = time.perf_counter() - t0
    x, y, _, _ = syn.grid(n, n)
    sigma = torch.as_tensor(syn.maclaurin_density(3, x, y, 0.4), dtype=torch.float32, device=dev)
    # reference fields for the norms: the FP64 GPU solve of the same disk (its F^x and F_R)
    p64 = Plan(n, n, k, d, d, precision="fp64", device=dev)
    gx64, gy64 = p64.forces(sigma.double())
    ref_x = gx64.float()
    ref_r = p64.radial_diagnostics(gx64, gy64, -0.5, -0.5)[0].float()
    del p64
    fx, fy = plan.forces(sigma)
    phi = torch.empty_like(sigma)
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    ms_pot = timed(lambda: plan.potential(sigma, out=phi))
    ms_diag = timed(lambda: plan.radial_diagnostics(fx, fy, -0.5, -0.5))  # F_R only: asynchronous
    # with the norms each call copies six values to the host and synchronises
    ms_norms = timed(lambda: plan.radial_diagnostics(fx, fy, -0.5, -0.5, ref_x, ref_r, want_fr=True))
    _, norms = plan.radial_diagnostics(fx, fy, -0.5, -0.5, ref_x, ref_r)
    line = {"metric": "in-simulation reuse pieces, FP32 plan", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "data": "synthetic",
            "config": {"workload": f"{n}x{n} order-{k}, D3 disk (a = 0.4) for the diagnostics", "nx": n, "ny": n,
                       "order": k},
            "table_build_s": round(t_build, 4), "build_from_kept_tables_s": round(t_from, 4),
            "potential_tables_build_s": round(t_pot_build, 4),
            "potential_ms": round(ms_pot, 4), "potential_Mpts_s": round(n * n / (ms_pot * 1e-3) / 1e6, 1),
            "radial_force_ms": round(ms_diag, 4),
            "radial_force_GB_s": round(3 * 4 * n * n / (ms_diag * 1e-3) / 1e9, 1),
            "radial_force_and_norms_ms": round(ms_norms, 4),
            "radial_force_and_norms_GB_s": round(5 * 4 * n * n / (ms_norms * 1e-3) / 1e9, 1),
            "norms_fx_fr_vs_fp64_gpu": [float(f"{v:.4e}") for v in norms],
            "device_error": plan.device_error()}
    print(json.dumps(line), flush=True)


def main():
    global E2E_DEPTH, ORDER, METRIC, WORKLOAD
    args = parse()
    launch_ranks(args)
    if args.dry_run:
        run_dry(args)
        return
    E2E_DEPTH = args.e2e_depth
    if args.order != ORDER:
        METRIC = METRIC.replace("order-3", f"order-{args.order}")
        WORKLOAD = WORKLOAD.replace("order-3", f"order-{args.order}")
        ORDER = args.order
    if args.batched:
        run_batched(args)
        return
    if args.next2:
        run_next2(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
