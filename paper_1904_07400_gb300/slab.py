"""Slab decomposition of one grid over ranks (Sec. 2.3: the spline solves and the transforms
are split over processes in slabs, with transposes between the passes).

Each rank owns a slab of rows of sigma and of the forces, and a slab of frequency columns
for the column pass; the passes run in the library (``tdg_slab_*`` in include/tdgrav.h),
and the two transposes are all-to-all exchanges of contiguous chunks:

* ``solve_distributed``: one rank per process (``torch.distributed``, NCCL on GPUs), each
  with its own plan on its own device;
* ``solve_simulated``: every rank in this process on one device, the all-to-all carried out
  by device copies of the same chunks (the exchange pattern and the kernels are the ones a
  multi-GPU run uses; only the transport differs).

Everything here is argument marshalling and chunk bookkeeping; no step of the method runs in
Python.
"""
from __future__ import annotations

import ctypes

import torch

from . import native
from .api import Plan

CELL = 16  # bytes of one tile cell (two complex floats of adjacent frequency columns)


def partition(nx: int, ny: int, world: int):
    """[(r0, nrows, t0, ntiles)] of every rank (tdg_slab_partition)."""
    lib = native.load()
    out = []
    for r in range(world):
        v = [ctypes.c_int() for _ in range(4)]
        native.check("tdg_slab_partition", lib.tdg_slab_partition(nx, ny, world, r, *[ctypes.byref(x) for x in v]))
        out.append(tuple(x.value for x in v))
    return out


def z_splits(parts, rank):
    """Cells of the Z exchange: (sent to each rank, received from each rank)."""
    _, n_me, _, nt_me = parts[rank]
    return [nt * n_me for _, _, _, nt in parts], [nt_me * n for _, n, _, _ in parts]


def g_splits(parts, rank):
    """Cells of the G exchange, per component: (sent to each rank, received from each rank)."""
    _, n_me, _, nt_me = parts[rank]
    return [nt_me * n for _, n, _, _ in parts], [nt * n_me for _, _, _, nt in parts]


class SlabRank:
    """One rank's share of a slab-decomposed solve: its slab buffers and the library calls."""

    def __init__(self, plan: Plan, world: int, rank: int):
        lib = native.load()
        self.plan, self.world, self.rank = plan, world, rank
        self.parts = partition(plan.nx, plan.ny, world)
        self.r0, self.nrows, self.t0, self.ntiles = self.parts[rank]
        dev = plan.device
        nbytes = [int(lib.tdg_slab_bytes(plan.handle, world, rank, w)) for w in range(4)]
        if not all(nbytes):
            raise native.TdgError("tdg_slab_bytes", native.TDG_OK + 2)
        # float32 views: 4 per cell (all-to-all split sizes count elements)
        self.z_rows = torch.empty(nbytes[0] // 4, dtype=torch.float32, device=dev)
        self.z_recv = torch.empty(nbytes[1] // 4, dtype=torch.float32, device=dev)
        self.z_cols = torch.empty(nbytes[1] // 4, dtype=torch.float32, device=dev)
        self.g_cols = torch.empty(nbytes[2] // 4, dtype=torch.float32, device=dev)
        self.g_send = torch.empty(nbytes[2] // 4, dtype=torch.float32, device=dev)
        self.g_rows = torch.empty(nbytes[3] // 4, dtype=torch.float32, device=dev)

    def _call(self, name, *ptrs, stream):
        native.call(name, self.plan.handle, self.world, self.rank, *ptrs, stream)

    def rows_forward(self, sigma_rows, stream):
        self._call("tdg_slab_rows_forward", sigma_rows.data_ptr(), self.z_rows.data_ptr(), stream=stream)

    def unpack_z(self, stream):
        self._call("tdg_slab_unpack_z", self.z_recv.data_ptr(), self.z_cols.data_ptr(), stream=stream)

    def columns(self, stream):
        self._call("tdg_slab_columns", self.z_cols.data_ptr(), self.g_cols.data_ptr(), stream=stream)

    def pack_g(self, stream):
        self._call("tdg_slab_pack_g", self.g_cols.data_ptr(), self.g_send.data_ptr(), stream=stream)

    def rows_inverse(self, fx_rows, fy_rows, stream):
        self._call("tdg_slab_rows_inverse", self.g_rows.data_ptr(), fx_rows.data_ptr(), fy_rows.data_ptr(),
                   stream=stream)

    # chunk views (float32 elements) of the exchanges
    def z_send_chunks(self):
        sent, _ = z_splits(self.parts, self.rank)
        return list(self.z_rows.split([4 * c for c in sent]))

    def z_recv_chunks(self):
        _, recv = z_splits(self.parts, self.rank)
        return list(self.z_recv.split([4 * c for c in recv]))

    def g_send_chunks(self, comp):
        sent, _ = g_splits(self.parts, self.rank)
        half = self.g_send.numel() // 2
        return list(self.g_send[comp * half:(comp + 1) * half].split([4 * c for c in sent]))

    def g_recv_chunks(self, comp):
        _, recv = g_splits(self.parts, self.rank)
        half = self.g_rows.numel() // 2
        return list(self.g_rows[comp * half:(comp + 1) * half].split([4 * c for c in recv]))


def solve_simulated(plan: Plan, sigma, world: int):
    """The slab-decomposed solve of `sigma` (nx x ny on the plan's device) over `world`
    ranks held in this process; returns (fx, fy) assembled from the ranks' rows."""
    stream = torch.cuda.current_stream(plan.device)
    s = stream.cuda_stream
    ranks = [SlabRank(plan, world, r) for r in range(world)]
    fx = torch.empty_like(sigma)
    fy = torch.empty_like(sigma)
    for rk in ranks:
        rk.rows_forward(sigma[rk.r0:rk.r0 + rk.nrows], s)
    for q, dst in enumerate(ranks):            # chunk q of every source lands at source r of q
        for r, src in enumerate(ranks):
            dst.z_recv_chunks()[r].copy_(src.z_send_chunks()[q])
    for rk in ranks:
        rk.unpack_z(s)
        rk.columns(s)
        rk.pack_g(s)
    for r, dst in enumerate(ranks):
        for q, src in enumerate(ranks):
            for c in range(2):
                dst.g_recv_chunks(c)[q].copy_(src.g_send_chunks(c)[r])
    for rk in ranks:
        rk.rows_inverse(fx[rk.r0:rk.r0 + rk.nrows], fy[rk.r0:rk.r0 + rk.nrows], s)
    return fx, fy


def solve_distributed(plan: Plan, sigma_rows, group=None):
    """This rank's part of the slab-decomposed solve (torch.distributed initialised, one
    rank per device, every rank with the same plan parameters on its own device).
    sigma_rows: this rank's rows (tdg_slab_partition); returns this rank's force rows."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    rk = SlabRank(plan, world, rank)
    s = torch.cuda.current_stream(plan.device).cuda_stream
    fx = torch.empty_like(sigma_rows)
    fy = torch.empty_like(sigma_rows)
    rk.rows_forward(sigma_rows, s)
    sent, recv = z_splits(rk.parts, rank)
    dist.all_to_all_single(rk.z_recv, rk.z_rows, [4 * c for c in recv], [4 * c for c in sent], group=group)
    rk.unpack_z(s)
    rk.columns(s)
    rk.pack_g(s)
    sent, recv = g_splits(rk.parts, rank)
    hs, hr = rk.g_send.numel() // 2, rk.g_rows.numel() // 2
    for c in range(2):
        dist.all_to_all_single(rk.g_rows[c * hr:(c + 1) * hr], rk.g_send[c * hs:(c + 1) * hs],
                               [4 * x for x in recv], [4 * x for x in sent], group=group)
    rk.rows_inverse(fx, fy, s)
    return fx, fy
