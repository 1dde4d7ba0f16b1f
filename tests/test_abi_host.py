"""The C-ABI library without a GPU: it loads, exports every declared symbol, validates
arguments on the host, and its host-callable table-entry code matches the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1904_07400_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tdgrav.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1904_07400_gb300 import build
    build.build()
    return native.load()


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tdg_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(n for n, _, _ in native.SIGNATURES) == names


def test_status_strings(lib):
    for code in range(8):
        s = lib.tdg_status_string(code)
        assert isinstance(s, bytes) and len(s) > 0
    assert lib.tdg_status_string(0) == b"ok"


def _init(lib, *args):
    h = ctypes.c_void_p()
    st = lib.tdg_init(ctypes.byref(h), *args)
    return st, h


def test_init_validates_arguments(lib):
    ok = (64, 64, 3, 0.1, 0.1, 1.0, 1, 0)
    st, h = _init(lib, *ok)
    assert st == 0 and h.value
    px, py = ctypes.c_int(), ctypes.c_int()
    assert lib.tdg_plan_info(h, ctypes.byref(px), ctypes.byref(py), None, None) == 0
    assert (px.value, py.value) == (128, 128)
    assert lib.tdg_destroy(h) == 0
    bad = [
        (64, 64, 0, 0.1, 0.1, 1.0, 1, 0),      # order
        (64, 64, 6, 0.1, 0.1, 1.0, 1, 0),
        (0, 64, 3, 0.1, 0.1, 1.0, 1, 0),       # size
        (64, 64, 3, 0.0, 0.1, 1.0, 1, 0),      # spacing
        (64, 64, 3, 0.1, -1.0, 1.0, 1, 0),
        (64, 64, 3, float("nan"), 0.1, 1.0, 1, 0),
        (64, 64, 3, 0.1, 0.1, float("inf"), 1, 0),
        (64, 64, 3, 0.1, 0.1, 1.0, 7, 0),      # precision
        (64, 64, 3, 0.1, 0.1, 1.0, 1, -1),     # device
    ]
    for args in bad:
        st, h = _init(lib, *args)
        assert st == 1 and not h.value, args
    st, _ = _init(lib, 4097, 64, 3, 0.1, 0.1, 1.0, 1, 0)
    assert st == 2
    # the tensor-core form needs columns padded to 2048 or 4096 points (nx > 1024)
    st, h = _init(lib, 512, 512, 3, 0.1, 0.1, 1.0, 2, 0)
    assert st == 2 and not h.value
    st, h = _init(lib, 4096, 1024, 3, 0.1, 0.1, 1.0, 2, 0)
    assert st == 0
    lib.tdg_destroy(h)
    # orders 4 and 5 run every form; the tensor-core form still needs nx > 1024
    for k in (4, 5):
        for prec in (0, 1):
            st, h = _init(lib, 64, 48, k, 0.1, 0.1, 1.0, prec, 0)
            assert st == 0 and h.value
            lib.tdg_destroy(h)
        st, h = _init(lib, 1024, 1024, k, 0.1, 0.1, 1.0, 2, 0)
        assert st == 2 and not h.value
    assert lib.tdg_init(None, 64, 64, 3, 0.1, 0.1, 1.0, 1, 0) == 1


@pytest.mark.parametrize("n,period", [(128, 512), (144, 512), (256, 512), (272, 1024), (512, 1024), (528, 2048),
                                      (1024, 2048), (1040, 4096), (2064, 8192), (4096, 8192)])
def test_network_period_choice(lib, n, period):
    # FP32 sides that are multiples of 16 from 128 to 4096 pad to 2L, L the smallest
    # transform-network length (256, 512, 1024, 2048, 4096) not below the side; FP64
    # plans of the same sides keep the smallest even 2^a 3^b >= 2n - 1
    st, h = _init(lib, n, n, 3, 0.1, 0.1, 1.0, 1, 0)
    assert st == 0
    px, py = ctypes.c_int(), ctypes.c_int()
    lib.tdg_plan_info(h, ctypes.byref(px), ctypes.byref(py), None, None)
    assert (px.value, py.value) == (period, period)
    lib.tdg_destroy(h)
    st, h = _init(lib, n, n, 3, 0.1, 0.1, 1.0, 0, 0)
    lib.tdg_plan_info(h, ctypes.byref(px), None, None, None)
    p = px.value
    assert p >= 2 * n - 1 and p % 2 == 0 and p <= period
    lib.tdg_destroy(h)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 17, 33, 64, 100, 192, 4096])
def test_padded_period_choice(lib, n):
    st, h = _init(lib, n, 2, 1, 1.0, 1.0, 1.0, 0, 0)
    assert st == 0
    px = ctypes.c_int()
    lib.tdg_plan_info(h, ctypes.byref(px), None, None, None)
    p = px.value
    q = p // 2
    while q % 2 == 0:
        q //= 2
    while q % 3 == 0:
        q //= 3
    assert p % 2 == 0 and q == 1 and p >= 2 * n - 1 and p >= 2
    lib.tdg_destroy(h)


def test_solve_before_build_and_null_pointers(lib):
    st, h = _init(lib, 16, 16, 2, 0.1, 0.1, 1.0, 1, 0)
    assert lib.tdg_solve_forces(h, 256, 512, 768, None) == 3          # NOT_BUILT
    assert lib.tdg_solve_forces(h, None, 512, 768, None) == 1         # null
    assert lib.tdg_solve_forces(h, 257, 512, 768, None) == 1          # misaligned
    assert lib.tdg_solve_adjoint(h, 256, 512, 768, None) == 3
    wx = np.zeros(256)
    assert lib.tdg_copy_kernel_tables(h, wx.ctypes.data, wx.ctypes.data) == 3
    assert lib.tdg_workspace_bytes(h) > 0
    assert lib.tdg_set_workspace(h, 1024 + 8, 1 << 30) == 1           # not 256-aligned
    assert lib.tdg_set_workspace(h, 4096, 16) == 1                    # too small
    lib.tdg_destroy(h)


def test_kernel_entry_host_matches_oracle_near_field(lib):
    from oracle import kernel_tables as kt
    worst = 0.0
    for k in (1, 2, 3, 4, 5):
        # orders 4, 5: square cells only (their route-I entries cost about a second each;
        # thin cells are covered by the device-against-oracle table tests)
        for ratio in ((1.0, 0.5, 8.0) if k <= 3 else (1.0,)):
            nf = kt.near_field_size(k)
            for m in range(nf):
                for n in range(nf):
                    for comp in (0, 1):
                        got = native.kernel_entry_host(k, m, n, 1.0, ratio, comp)
                        ref = kt._near_entry(k, m, n, ratio, "xy"[comp])
                        if ref == 0.0:
                            assert got == 0.0
                            continue
                        worst = max(worst, abs(got - ref) / abs(ref))
    assert worst < 1e-14


def test_kernel_entry_host_matches_oracle_far_field(lib):
    from oracle import kernel_tables as kt
    rng = np.random.default_rng(0)
    for k in (1, 2, 3, 4, 5):
        for ratio in (1.0, 0.25, 3.0):
            ms = rng.integers(-300, 300, 30)
            ns = rng.integers(-300, 300, 30)
            for comp in ("x", "y"):
                d = kt.band_distance(k, ms, ns, 1.0, ratio)
                for m, n, dd in zip(ms, ns, d):
                    if max(abs(m), abs(n)) < kt.near_field_size(k):
                        continue
                    q = [q for lim, q in kt.FAR_BANDS if lim is None or dd < lim][0]
                    ref = kt.w_far_gl(k, np.array([m]), np.array([n]), 1.0, ratio, q, comp)[0]
                    got = native.kernel_entry_host(k, int(m), int(n), 1.0, ratio, "xy".index(comp))
                    if ref == 0.0:
                        assert got == 0.0
                    else:
                        assert abs(got - ref) < 2e-14 * abs(ref), (k, ratio, m, n, comp)


def test_kernel_entry_host_symmetries(lib):
    e = native.kernel_entry_host
    for k in (1, 2, 3, 4, 5):
        assert e(k, 3, 5, 1.0, 1.0, 0) == -e(k, -3, 5, 1.0, 1.0, 0)
        assert e(k, 3, 5, 1.0, 1.0, 0) == e(k, 3, -5, 1.0, 1.0, 0)
        assert e(k, 3, 5, 1.0, 1.0, 1) == e(k, 5, 3, 1.0, 1.0, 0)
        assert e(k, 0, 7, 1.0, 1.0, 0) == 0.0


def test_build_from_tables_rejects_foreign_tables(lib):
    # the spot check runs before any device work: tables of another order or grid, or
    # missing arrays, are refused with INVALID_ARG
    nx, ny = 12, 10
    st, h = _init(lib, nx, ny, 3, 0.1, 0.1, 1.0, 1, 0)
    assert st == 0
    wx = np.zeros((nx, ny))
    wy = np.zeros((nx, ny))
    assert lib.tdg_build_kernel_tables_from(h, wx.ctypes.data, wy.ctypes.data, None) == 1
    for m in range(nx):  # order-2 entries for an order-3 plan
        for n in range(ny):
            wx[m, n] = native.kernel_entry_host(2, m, n, 0.1, 0.1, 0)
            wy[m, n] = native.kernel_entry_host(2, m, n, 0.1, 0.1, 1)
    assert lib.tdg_build_kernel_tables_from(h, wx.ctypes.data, wy.ctypes.data, None) == 1
    assert lib.tdg_build_kernel_tables_from(h, None, wy.ctypes.data, None) == 1
    lib.tdg_destroy(h)


def test_radial_diagnostics_argument_checks(lib):
    # refused before any device work
    st, h = _init(lib, 16, 16, 3, 0.1, 0.1, 1.0, 0, 0)
    assert st == 0
    buf = (ctypes.c_double * 4)()
    a = ctypes.cast(buf, ctypes.c_void_p)
    norms = (ctypes.c_double * 6)()
    n = ctypes.cast(norms, ctypes.c_void_p)
    f = lib.tdg_radial_diagnostics
    assert f(h, None, a, 0.0, 0.0, a, None, None, None, None) == 1            # no F^x
    assert f(h, a, a, float("nan"), 0.0, a, None, None, None, None) == 1      # origin
    assert f(h, a, a, 0.0, 0.0, None, None, None, None, None) == 1            # nothing asked
    assert f(h, a, a, 0.0, 0.0, a, None, None, n, None) == 1                  # norms, no reference
    assert f(h, a, a, 0.0, 0.0, None, a, None, None, None) == 1               # reference, no norms
    assert f(h, a, a, 0.0, 0.0, None, None, a, n, None) == 1                  # ref_fr without ref_fx
    lib.tdg_destroy(h)


def test_potential_entry_host_matches_oracle(lib):
    from oracle import kernel_tables as kt
    for k in (1, 3, 5):
        nf = kt.near_field_size(k)
        for (m, n) in [(0, 0), (1, 0), (0, 2), (2, 1), (nf - 1, nf - 1)]:
            got = native.kernel_entry_host(k, m, n, 1.0, 1.0, 2)
            ref = kt._near_phi(k, m, n, 1.0)
            assert abs(got - ref) < 5e-15 * ref, (k, m, n)
        rng = np.random.default_rng(k)
        for m, n in zip(rng.integers(0, 300, 20), rng.integers(0, 300, 20)):
            if max(m, n) < nf:
                continue
            d = float(kt.band_distance(k, m, n, 1.0, 0.75))
            q = [q for lim, q in kt.FAR_BANDS if lim is None or d < lim][0]
            ref = kt.w_phi_far_gl(k, np.array([m]), np.array([n]), 1.0, 0.75, q)[0]
            got = native.kernel_entry_host(k, int(m), int(n), 1.0, 0.75, 2)
            assert abs(got - ref) < 5e-15 * ref
        # even in m and n
        assert native.kernel_entry_host(k, -3, 2, 1.0, 1.0, 2) == native.kernel_entry_host(k, 3, -2, 1.0, 1.0, 2)


def test_noalloc_limit_constant_matches_header():
    import re
    from paper_1904_07400_gb300 import native
    hdr = open(os.path.join(ROOT, "include", "tdgrav.h")).read()
    m = re.search(r"#define TDG_NOALLOC_SCRATCH_BYTES \((\d+)u \* (\d+)u \* (\d+)u\)", hdr)
    assert m, "TDG_NOALLOC_SCRATCH_BYTES not found"
    assert int(m.group(1)) * int(m.group(2)) * int(m.group(3)) == native.NOALLOC_SCRATCH_BYTES
