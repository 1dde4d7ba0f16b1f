"""ctypes binding of libtdgrav (include/tdgrav.h): argument marshalling only.

Every entry point of the C ABI is exposed under the same name.  Pointers are passed as
integers (device addresses from torch tensors, or host arrays from numpy); streams as the
integer handle of a cudaStream_t.  Nothing here computes any part of the method: a
missing library raises, there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libtdgrav.so")

TDG_OK = 0
NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024  # TDG_NOALLOC_SCRATCH_BYTES of include/tdgrav.h
STATUS = {0: "TDG_OK", 1: "TDG_ERR_INVALID_ARG", 2: "TDG_ERR_UNSUPPORTED", 3: "TDG_ERR_NOT_BUILT",
          4: "TDG_ERR_OOM", 5: "TDG_ERR_CUDA", 6: "TDG_ERR_TIMEOUT", 7: "TDG_ERR_DEVICE_BOUNDS"}
PRECISION = {"fp64": 0, "fp32": 1, "fp32_tc16": 2}

_c_int, _c_double, _c_void_p, _c_size_t = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t

# (name, restype, argtypes) for every symbol declared in include/tdgrav.h
SIGNATURES = [
    ("tdg_init", _c_int, [ctypes.POINTER(_c_void_p), _c_int, _c_int, _c_int, _c_double, _c_double,
                          _c_double, _c_int, _c_int]),
    ("tdg_build_kernel_tables", _c_int, [_c_void_p, _c_void_p]),
    ("tdg_build_kernel_tables_from", _c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p]),
    ("tdg_build_potential_tables", _c_int, [_c_void_p, _c_void_p]),
    ("tdg_solve_potential", _c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p]),
    ("tdg_radial_diagnostics", _c_int, [_c_void_p, _c_void_p, _c_void_p, ctypes.c_double, ctypes.c_double,
                                        _c_void_p, _c_void_p, _c_void_p, _c_void_p, _c_void_p]),
    ("tdg_workspace_bytes", _c_size_t, [_c_void_p]),
    ("tdg_set_workspace", _c_int, [_c_void_p, _c_void_p, _c_size_t]),
    ("tdg_solve_forces", _c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _c_void_p]),
    ("tdg_solve_forces_batched", _c_int, [ctypes.POINTER(_c_void_p), _c_int, ctypes.POINTER(_c_void_p),
                                          ctypes.POINTER(_c_void_p), ctypes.POINTER(_c_void_p), _c_void_p]),
    ("tdg_batch_create", _c_int, [ctypes.POINTER(_c_void_p), ctypes.POINTER(_c_void_p), _c_int,
                                  ctypes.POINTER(_c_void_p), ctypes.POINTER(_c_void_p), ctypes.POINTER(_c_void_p)]),
    ("tdg_batch_set_config", _c_int, [_c_void_p, _c_int, _c_int]),
    ("tdg_batch_set_streams", _c_int, [_c_void_p, _c_int]),
    ("tdg_batch_launch", _c_int, [_c_void_p, _c_void_p]),
    ("tdg_batch_get_error", _c_int, [_c_void_p]),
    ("tdg_batch_info", _c_int, [_c_void_p, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                                ctypes.POINTER(_c_int)]),
    ("tdg_batch_debug_withhold", _c_int, [_c_void_p, _c_int]),
    ("tdg_batch_destroy", _c_int, [_c_void_p]),
    ("tdg_solve_adjoint", _c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _c_void_p]),
    ("tdg_get_device_error", _c_int, [_c_void_p]),
    ("tdg_copy_kernel_tables", _c_int, [_c_void_p, _c_void_p, _c_void_p]),
    ("tdg_kernel_entry_host", _c_int, [_c_int, _c_int, _c_int, _c_double, _c_double, _c_int,
                                       ctypes.POINTER(_c_double)]),
    ("tdg_solve_forces_noalloc", _c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _c_void_p]),
    ("tdg_set_pass_events", _c_int, [_c_void_p, ctypes.POINTER(_c_void_p), _c_int]),
    ("tdg_slab_partition", _c_int, [_c_int, _c_int, _c_int, _c_int, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                                    ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)]),
    ("tdg_slab_bytes", _c_size_t, [_c_void_p, _c_int, _c_int, _c_int]),
    ("tdg_slab_rows_forward", _c_int, [_c_void_p, _c_int, _c_int, _c_void_p, _c_void_p, _c_void_p]),
    ("tdg_slab_unpack_z", _c_int, [_c_void_p, _c_int, _c_int, _c_void_p, _c_void_p, _c_void_p]),
    ("tdg_slab_columns", _c_int, [_c_void_p, _c_int, _c_int, _c_void_p, _c_void_p, _c_void_p]),
    ("tdg_slab_pack_g", _c_int, [_c_void_p, _c_int, _c_int, _c_void_p, _c_void_p, _c_void_p]),
    ("tdg_slab_rows_inverse", _c_int, [_c_void_p, _c_int, _c_int, _c_void_p, _c_void_p, _c_void_p, _c_void_p]),
    ("tdg_plan_info", _c_int, [_c_void_p, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                               ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)]),
    ("tdg_plan_path", _c_int, [_c_void_p]),
    ("tdg_destroy", _c_int, [_c_void_p]),
    ("tdg_status_string", ctypes.c_char_p, [_c_int]),
]

_lib = None


class TdgError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        super().__init__(f"{fn} failed: {STATUS.get(status, status)}")


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libtdgrav.so (built in-tree by paper_1904_07400_gb300.build)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"tdgrav library not built: {p} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(p)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def check(fn: str, status: int) -> None:
    if status != TDG_OK:
        raise TdgError(fn, status)


def call(name: str, *args):
    """Call one C entry point; raise TdgError on a non-OK status (status-returning calls)."""
    lib = load()
    res = getattr(lib, name)(*args)
    if name not in ("tdg_workspace_bytes", "tdg_status_string", "tdg_plan_path", "tdg_slab_bytes"):
        check(name, res)
    return res


def kernel_entry_host(order: int, m: int, n: int, dx: float, dy: float, component: int) -> float:
    out = _c_double()
    call("tdg_kernel_entry_host", order, m, n, dx, dy, component, ctypes.byref(out))
    return out.value
