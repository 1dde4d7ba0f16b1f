"""The slab decomposition of one grid (Sec. 2.3: the solves and transforms split over
processes in slabs, with transposes between the passes) on CPU gloo ranks.

The GPU kernels do not run here.  Each rank takes its rows and frequency columns from the
library's partition (tdg_slab_partition), does its slab's share of the oracle's solve (the
y solve and row transform on its rows, the x solve, column transforms and spectrum products
on its columns, the row inverse on its rows), and the two transposes go through
all_to_all_single with chunks in rank order, as the library's exchange does.  The gathered
forces equal the single-process oracle.
"""
import json
import socket

import numpy as np
import pytest

NX, NY, K = 128, 144, 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _sigma():
    return np.random.default_rng(21).random((NX, NY))


def _setup():
    from oracle import kernel_tables as kt
    from oracle.convolution import spectra
    from paper_1904_07400_gb300 import build, native, slab
    build.build()
    native.load()
    lx = ly = 256  # the network's transform lengths for 128 and 144 cells
    px, py = 2 * lx, 2 * ly
    wx, wy = kt.kernel_tables(K, NX, NY, 1.0 / NX, 1.0 / NY)
    return slab, px, py, spectra(wx, wy, px, py)


def _a2a(send_blocks, recv_shapes):
    """all_to_all_single of complex blocks (one per rank, in rank order)."""
    import torch
    import torch.distributed as dist
    send = torch.cat([torch.view_as_real(torch.from_numpy(np.ascontiguousarray(b))).reshape(-1)
                      for b in send_blocks])
    sizes_in = [2 * b.size for b in send_blocks]
    sizes_out = [2 * int(np.prod(s)) for s in recv_shapes]
    recv = torch.empty(sum(sizes_out), dtype=torch.float64)
    dist.all_to_all_single(recv, send, sizes_out, sizes_in)
    parts = recv.split(sizes_out)
    return [torch.view_as_complex(p.reshape(-1, 2)).numpy().reshape(s) for p, s in zip(parts, recv_shapes)]


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    from oracle.coefficients import thomas
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        slab, px, py, spec = _setup()
        hy = py // 2 + 1
        parts = slab.partition(NX, NY, world)
        kyr = [(2 * t0, min(2 * (t0 + nt), hy)) for _, _, t0, nt in parts]
        r0, n, _, _ = parts[rank]
        k0, k1 = kyr[rank]
        sigma = _sigma()[r0:r0 + n]
        # pass A on this rank's rows: y solve (Eq. z_system), row transform
        z = thomas(1.0, 6.0, 1.0, sigma.T).T
        zr = np.fft.rfft(z, n=py, axis=1)
        # transpose: rank q gets this rank's rows of q's columns
        zc = np.concatenate(_a2a([zr[:, a:b] for a, b in kyr],
                                 [(pn, k1 - k0) for _, pn, _, _ in parts]), axis=0)
        # pass B on this rank's columns: x solve (Eq. C_system), column transform, products,
        # column inverse, crop
        cx = thomas(1.0, 6.0, 1.0, 64.0 * zc.real) + 1j * thomas(1.0, 6.0, 1.0, 64.0 * zc.imag)
        ch = np.fft.fft(cx, n=px, axis=0)
        gc = [np.fft.ifft(ch * spec[c][:, k0:k1], axis=0)[:NX] for c in range(2)]
        # transpose back, one exchange per component
        gr = [np.concatenate(_a2a([g[pr0:pr0 + pn] for pr0, pn, _, _ in parts],
                                  [(n, b - a) for a, b in kyr]), axis=1) for g in gc]
        f = [np.fft.irfft(g, n=py, axis=1)[:, :NY] for g in gr]
        out = [None] * world
        dist.all_gather_object(out, {"r0": r0, "fx": f[0].tolist(), "fy": f[1].tolist(), "parts": parts})
        if rank == 0:
            with open(out_path, "w") as fh:
                json.dump(out, fh)
    finally:
        dist.destroy_process_group()


def test_partition_covers_rows_and_columns():
    from paper_1904_07400_gb300 import build, native, slab
    build.build()
    native.load()
    for nx, ny, world in ((128, 144, 2), (4096, 4096, 8), (1040, 272, 3), (256, 4096, 16)):
        parts = slab.partition(nx, ny, world)
        ly = {272: 512, 144: 256, 4096: 4096}[ny]
        ntile = (ly + 2) // 2
        assert [p[0] for p in parts] == [sum(q[1] for q in parts[:i]) for i in range(world)]
        assert sum(p[1] for p in parts) == nx and all(p[1] % 16 == 0 and p[1] > 0 for p in parts)
        assert [p[2] for p in parts] == [sum(q[3] for q in parts[:i]) for i in range(world)]
        assert sum(p[3] for p in parts) == ntile and all(p[3] > 0 for p in parts)
        assert max(p[1] for p in parts) - min(p[1] for p in parts) <= 16
    lib = native.load()
    assert lib.tdg_slab_partition(128, 144, 9, 0, None, None, None, None) == 1   # 8 row chunks < 9 ranks
    assert lib.tdg_slab_partition(100, 144, 2, 0, None, None, None, None) == 1   # off the network path
    assert lib.tdg_slab_partition(128, 144, 2, 2, None, None, None, None) == 1   # rank outside


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_slab_solve_equals_oracle(tmp_path, world):
    import torch.multiprocessing as mp
    from oracle.convolution import Solver
    out = tmp_path / "slab.json"
    mp.start_processes(_rank_main, args=(world, _free_port(), str(out)), nprocs=world, join=True,
                       start_method="spawn")
    res = json.loads(out.read_text())
    fx = np.concatenate([np.asarray(r["fx"]) for r in res])
    fy = np.concatenate([np.asarray(r["fy"]) for r in res])
    assert [r["r0"] for r in res] == [p[0] for p in res[0]["parts"]]
    rx, ry = Solver(NX, NY, K, 1.0 / NX, 1.0 / NY).forces(_sigma())
    scale = max(np.abs(rx).max(), np.abs(ry).max())
    assert np.abs(fx - rx).max() < 1e-12 * scale
    assert np.abs(fy - ry).max() < 1e-12 * scale
