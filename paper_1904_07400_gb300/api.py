"""PyTorch-facing API of tdgrav: plans over torch device memory and streams.

    plan = Plan(nx, ny, order, dx, dy, G=1.0, precision="fp32")
    fx, fy = plan.forces(sigma)              # sigma: (nx, ny) CUDA tensor
    gs = plan.adjoint(gx, gy)                # dL/dsigma for L = sum(gx Fx + gy Fy)
    fx, fy = ThinDiskForces.apply(plan, sigma)   # autograd through the hand-written adjoint

Torch provides the device memory and the current stream; every step of the solve runs in
the library's CUDA kernels through the C ABI (paper_1904_07400_gb300.native).
"""
from __future__ import annotations

import ctypes

import torch

from . import native

_DTYPES = {"fp64": torch.float64, "fp32": torch.float32, "fp32_tc16": torch.float32}


def _stream_handle(device: torch.device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


class Plan:
    """One grid (nx x ny cells of dx x dy), B-spline order 1..5, precision form."""

    def __init__(self, nx: int, ny: int, order: int, dx: float, dy: float, G: float = 1.0,
                 precision: str = "fp32", device: int | torch.device = 0, build: bool = True,
                 tables: str | None = None):
        if precision not in native.PRECISION:
            raise ValueError(f"precision must be one of {sorted(native.PRECISION)}")
        dev = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.nx, self.ny, self.order = nx, ny, order
        self.dx, self.dy, self.G = dx, dy, G
        self.precision = precision
        self.dtype = _DTYPES[precision]
        self.device = dev
        h = ctypes.c_void_p()
        native.call("tdg_init", ctypes.byref(h), nx, ny, order, dx, dy, G,
                    native.PRECISION[precision], dev.index)
        self._h = h
        self._built = False
        if tables is not None:
            self.build_from(tables)
        elif build:
            self.build()

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def build(self) -> None:
        with torch.cuda.device(self.device):
            native.call("tdg_build_kernel_tables", self._h, _stream_handle(self.device))
        self._built = True

    def save_tables(self, path: str) -> None:
        """Keep this plan's FP64 kernel tables (w^x, w^y on the quadrant of offsets) and its
        parameters in an .npz file, for plans of later runs (any precision) to start from."""
        import numpy as np
        wx, wy = self.kernel_tables()
        np.savez(path, wx=wx, wy=wy, params=np.array([self.nx, self.ny, self.order, self.dx, self.dy]))

    def build_from(self, path: str) -> None:
        """Build from tables kept by save_tables: their quadrature is skipped, only the
        placement and the spectra are computed."""
        import numpy as np
        d = np.load(path)
        want = np.array([self.nx, self.ny, self.order, self.dx, self.dy])
        if d["params"].shape != want.shape or not np.array_equal(d["params"], want):
            raise ValueError(f"{path} holds tables for (nx, ny, order, dx, dy) = {tuple(d['params'])}")
        wx = np.ascontiguousarray(d["wx"], dtype=np.float64)
        wy = np.ascontiguousarray(d["wy"], dtype=np.float64)
        with torch.cuda.device(self.device):
            native.call("tdg_build_kernel_tables_from", self._h, wx.ctypes.data, wy.ctypes.data,
                        _stream_handle(self.device))
        self._built = True

    def info(self) -> dict:
        px, py, order, prec = (ctypes.c_int() for _ in range(4))
        native.call("tdg_plan_info", self._h, ctypes.byref(px), ctypes.byref(py), ctypes.byref(order),
                    ctypes.byref(prec))
        return {"px": px.value, "py": py.value, "order": order.value, "precision": prec.value}

    def path(self) -> int:
        """0: generic kernels, 2: FP32 transform network, 3: the network with the column pass
        on the tensor cores (FP32_TC16)."""
        return int(native.load().tdg_plan_path(self._h))

    def workspace_bytes(self) -> int:
        return int(native.load().tdg_workspace_bytes(self._h))

    def set_workspace(self, buf: torch.Tensor | None) -> None:
        if buf is None:
            native.call("tdg_set_workspace", self._h, None, 0)
        else:
            native.call("tdg_set_workspace", self._h, _ptr(buf), buf.numel() * buf.element_size())
        self._ws = buf

    def _check(self, t: torch.Tensor, name: str) -> None:
        if t.device != self.device or t.dtype != self.dtype or tuple(t.shape) != (self.nx, self.ny) \
                or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {self.dtype} tensor of shape "
                             f"({self.nx}, {self.ny}) on {self.device}")

    def forces(self, sigma: torch.Tensor, out: tuple | None = None):
        self._check(sigma, "sigma")
        if out is None:
            fx = torch.empty_like(sigma)
            fy = torch.empty_like(sigma)
        else:
            fx, fy = out
            self._check(fx, "fx")
            self._check(fy, "fy")
        native.call("tdg_solve_forces", self._h, _ptr(sigma), _ptr(fx), _ptr(fy), _stream_handle(self.device))
        return fx, fy

    def adjoint(self, gx: torch.Tensor, gy: torch.Tensor, out: torch.Tensor | None = None):
        self._check(gx, "gx")
        self._check(gy, "gy")
        gs = torch.empty_like(gx) if out is None else out
        self._check(gs, "gsigma")
        native.call("tdg_solve_adjoint", self._h, _ptr(gx), _ptr(gy), _ptr(gs), _stream_handle(self.device))
        return gs

    def build_potential(self) -> None:
        """Build the potential kernel's table and spectrum (after the force tables)."""
        with torch.cuda.device(self.device):
            native.call("tdg_build_potential_tables", self._h, _stream_handle(self.device))

    def potential(self, sigma: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """Phi = -G sum C w^phi at the cell centres (build_potential first)."""
        self._check(sigma, "sigma")
        phi = torch.empty_like(sigma) if out is None else out
        self._check(phi, "phi")
        native.call("tdg_solve_potential", self._h, _ptr(sigma), _ptr(phi), _stream_handle(self.device))
        return phi

    def radial_diagnostics(self, fx: torch.Tensor, fy: torch.Tensor, x0: float, y0: float,
                           ref_fx: torch.Tensor | None = None, ref_fr: torch.Tensor | None = None,
                           want_fr: bool = True):
        """F_R = (x F^x + y F^y) / R at the cell centres (x_i = x0 + (i + 1/2) dx, likewise y)
        and, with references, the area-weighted L1, L2, Linf norms of F^x - ref_fx and
        F_R - ref_fr (Sec. 3.1), all on the device.  Returns (F_R or None, six norms or None)."""
        self._check(fx, "fx")
        self._check(fy, "fy")
        for t, name in ((ref_fx, "ref_fx"), (ref_fr, "ref_fr")):
            if t is not None:
                self._check(t, name)
        fr = torch.empty_like(fx) if want_fr else None
        norms = (ctypes.c_double * 6)() if ref_fx is not None else None
        native.call("tdg_radial_diagnostics", self._h, _ptr(fx), _ptr(fy), float(x0), float(y0),
                    _ptr(fr) if fr is not None else None, _ptr(ref_fx) if ref_fx is not None else None,
                    _ptr(ref_fr) if ref_fr is not None else None,
                    ctypes.cast(norms, ctypes.c_void_p) if norms is not None else None,
                    _stream_handle(self.device))
        return fr, (tuple(norms) if norms is not None else None)

    def kernel_tables(self):
        """FP64 quarter tables (w^x, w^y at 0 <= m < nx, 0 <= n < ny) copied to the host."""
        import numpy as np
        wx = np.empty((self.nx, self.ny))
        wy = np.empty((self.nx, self.ny))
        native.call("tdg_copy_kernel_tables", self._h, wx.ctypes.data, wy.ctypes.data)
        return wx, wy

    def device_error(self) -> int:
        return int(native.load().tdg_get_device_error(self._h))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            native.load().tdg_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent FP32 solves in one call (tdg_batch_*).

    The grids' input and output tensors are bound at creation; ``launch()`` solves all of
    them on the current stream with no host synchronisation, so it can be captured in a
    CUDA graph: by default with one persistent kernel, or (``set_streams(n)``) with each
    grid's own kernels on n internal streams forked from and joined to the current one.
    """

    def __init__(self, plans: list[Plan], sigmas: list[torch.Tensor], outs: list[tuple] | None = None):
        if outs is None:
            outs = [(torch.empty_like(s), torch.empty_like(s)) for s in sigmas]
        for p, s, (fx, fy) in zip(plans, sigmas, outs):
            p._check(s, "sigma")
            p._check(fx, "fx")
            p._check(fy, "fy")
        self.plans, self.sigmas, self.outs = list(plans), list(sigmas), list(outs)
        n = len(plans)
        arr = ctypes.c_void_p * n
        h = ctypes.c_void_p()
        native.call("tdg_batch_create", ctypes.byref(h), arr(*[p.handle.value for p in plans]), n,
                    arr(*[_ptr(s) for s in sigmas]), arr(*[_ptr(o[0]) for o in outs]),
                    arr(*[_ptr(o[1]) for o in outs]))
        self._h = h
        self.device = plans[0].device

    def set_config(self, threads: int, radix_pref: int) -> None:
        """Persistent-kernel form: threads per block and radix preference."""
        native.call("tdg_batch_set_streams", self._h, 0)
        native.call("tdg_batch_set_config", self._h, threads, radix_pref)

    def set_streams(self, n: int) -> None:
        """Streams form: each grid's own kernels on n internal streams (0: persistent)."""
        native.call("tdg_batch_set_streams", self._h, n)

    def info(self) -> dict:
        b, t, i, r = (ctypes.c_int() for _ in range(4))
        native.call("tdg_batch_info", self._h, ctypes.byref(b), ctypes.byref(t), ctypes.byref(i), ctypes.byref(r))
        return {"blocks": b.value, "threads": t.value, "items": i.value, "radix_pref": r.value}

    def launch(self) -> None:
        native.call("tdg_batch_launch", self._h, _stream_handle(self.device))

    def error(self) -> int:
        return int(native.load().tdg_batch_get_error(self._h))

    def withhold(self, grid: int) -> None:
        """Test hook: do not count grid `grid`'s row-pass completions (-1 to undo)."""
        native.call("tdg_batch_debug_withhold", self._h, grid)

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            native.load().tdg_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def forces_batched(plans: list[Plan], sigmas: list[torch.Tensor], outs: list[tuple] | None = None):
    """Solve many independent grids in one library call."""
    n = len(plans)
    if outs is None:
        outs = [(torch.empty_like(s), torch.empty_like(s)) for s in sigmas]
    for p, s, (fx, fy) in zip(plans, sigmas, outs):
        p._check(s, "sigma")
        p._check(fx, "fx")
        p._check(fy, "fy")
    arr = ctypes.c_void_p * n
    hs = arr(*[p.handle.value for p in plans])
    ss = arr(*[_ptr(s) for s in sigmas])
    xs = arr(*[_ptr(o[0]) for o in outs])
    ys = arr(*[_ptr(o[1]) for o in outs])
    dev = plans[0].device if plans else torch.device("cuda", 0)
    native.call("tdg_solve_forces_batched", hs, n, ss, xs, ys, _stream_handle(dev))
    return outs


class ThinDiskForces(torch.autograd.Function):
    """(F^x, F^y) = solve(sigma) with the backward given by the library's adjoint."""

    @staticmethod
    def forward(ctx, plan: Plan, sigma: torch.Tensor):
        ctx.plan = plan
        return plan.forces(sigma.contiguous())

    @staticmethod
    def backward(ctx, gx, gy):
        plan = ctx.plan
        gx = torch.zeros((plan.nx, plan.ny), dtype=plan.dtype, device=plan.device) if gx is None else gx.contiguous()
        gy = torch.zeros((plan.nx, plan.ny), dtype=plan.dtype, device=plan.device) if gy is None else gy.contiguous()
        return None, plan.adjoint(gx, gy)
