"""Pins of the oracle's potential kernel and potential (a diagnostic beside the forces).

w^phi(m, n) = int int b_k(u/dx + m) b_k(v/dy + n) / r du dv; Phi = -G sum C w^phi.
"""
import numpy as np
import pytest

from oracle import kernel_tables as kt
from oracle.analytic import disk_potential
from oracle.convolution import Solver, potential_direct, potential_fft
from oracle.norms import orders, paper_norms
from workloads.synthetic import grid, maclaurin_density


def test_order1_closed_form_rectangle_potential():
    # route (closed-form inner integral, quadrature outer) = the textbook rectangle formula
    for (m, n, dy) in [(0, 0, 0.5), (1, 0, 1.0), (2, 3, 0.5), (5, 1, 2.0), (0, 7, 1.0)]:
        a = kt.w_phi_k1_closed(m, n, 1.0, dy)
        b = kt.w_phi_route(1, m, n, 1.0, dy, dps=25)
        assert abs(a - b) < 1e-20 * abs(a)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_potential_far_bands_reach_fp64(k):
    nf = kt.near_field_size(k)
    cases = [(nf, 0, 1.0), (1, nf, 1.0), (8, 1, 1.0), (12, 3, 1.0), (33, 0, 1.0), (1, 130, 1.0),
             (1, nf, 0.25), (12, 3, 0.25)]  # thin cells
    for (m, n, dy) in cases:
        d = float(kt.band_distance(k, m, n, 1.0, dy))
        q = [q for lim, q in kt.FAR_BANDS if lim is None or d < lim][0]
        ref = float(kt.w_phi_route(k, m, n, 1.0, dy, dps=25))
        got = kt.w_phi_far_gl(k, np.array([m]), np.array([n]), 1.0, dy, q)[0]
        assert abs(got - ref) < 2e-14 * ref, (k, m, n, dy, q)


@pytest.mark.slow
def test_potential_kernel_order5_scale_and_symmetry():
    """Order 5: w^phi scales with the cell size (4 times for cells four times larger, aspect
    1:2) and the table is even in m and n, as for orders 1 and 3 (about a minute)."""
    a = float(kt.w_phi_route(5, 2, 1, 0.25, 0.5, dps=20))
    b = float(kt.w_phi_route(5, 2, 1, 1.0, 2.0, dps=20))
    assert abs(4 * a - b) < 1e-14 * b
    q = kt.potential_table(5, 6, 5, 0.1, 0.1)
    np.testing.assert_array_equal(q, q[::-1, :])
    np.testing.assert_array_equal(q, q[:, ::-1])


def test_potential_kernel_symmetry_scale_and_moments():
    # proportional to the cell size; even; far away it is the point-mass 1/r with the
    # spline's variance k/12 as the first correction
    for k in (1, 3, 5):
        if k < 5:  # order 5: test_potential_kernel_order5_scale_and_symmetry (slow)
            a = float(kt.w_phi_route(k, 2, 1, 0.25, 0.5, dps=20))
            b = float(kt.w_phi_route(k, 2, 1, 1.0, 2.0, dps=20))
            assert abs(4 * a - b) < 1e-14 * b
            q = kt.potential_table(k, 6, 5, 0.1, 0.1)
            np.testing.assert_array_equal(q, q[::-1, :])
            np.testing.assert_array_equal(q, q[:, ::-1])
        dx, dy = 1.0, 0.75
        for (m, n) in [(400, 150), (-90, 500)]:
            u, v = -m * dx, -n * dy
            r = np.hypot(u, v)
            f, fuu, fvv = 1 / r, (2 * u * u - v * v) / r ** 5, (2 * v * v - u * u) / r ** 5
            ref = dx * dy * (f + k / 24.0 * (dx * dx * fuu + dy * dy * fvv))
            got = kt.w_phi_far_gl(k, np.array([abs(m)]), np.array([abs(n)]), dx, dy, 5)[0]
            assert abs(got - ref) < 1e-10 * ref


def test_disk_potential_quadrature_against_closed_forms():
    # D1 inside: -(pi^2 G sigma0 / (4 a)) (2 a^2 - R^2); any D_n far away: -G M / R
    a = 0.5
    R = np.array([0.05, 0.2, 0.45])
    np.testing.assert_allclose(disk_potential(1, R, a), -(np.pi ** 2 / (4 * a)) * (2 * a * a - R * R), rtol=1e-12)
    for n in (2, 4, 6):
        M = 2 * np.pi * a * a / (2 * n + 1)
        assert abs(disk_potential(n, np.array([60.0]), a)[0] / (-M / 60.0) - 1) < 1e-4


@pytest.mark.parametrize("k", [1, 3, 5])
def test_potential_direct_equals_fft(k):
    rng = np.random.default_rng(k)
    nx, ny = 9, 7
    w = kt.potential_table(k, nx, ny, 0.1, 0.1)
    c = rng.standard_normal((nx, ny))
    a = potential_direct(c, w, 2.0)
    b = potential_fft(c, w, 2.0)
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()
    # a literal scalar loop for one cell
    i, j = 4, 5
    lit = -2.0 * sum(c[p, q] * w[i - p + nx - 1, j - q + ny - 1] for p in range(nx) for q in range(ny))
    assert abs(lit - a[i, j]) < 1e-13 * abs(lit)


def test_potential_order_of_accuracy():
    # against the analytic D4 potential: order 2 for k = 1 and 4 for k = 3 (the potential's
    # kernel is smooth enough that the cell-centre error gains one order for odd k)
    expect = {1: 2.0, 3: 4.0}
    for k, o_exp in expect.items():
        l2 = []
        for N in (32, 64, 128):
            x, y, dx, dy = grid(N, N, -1.0, 1.0)
            phi = Solver(N, N, k, dx, dy).potential(maclaurin_density(4, x, y, 0.5))
            X, Y = np.meshgrid(x, y, indexing="ij")
            Rg = np.round(np.hypot(X, Y), 14)
            ur, inv = np.unique(Rg, return_inverse=True)
            ref = disk_potential(4, ur, 0.5, dps=15)[inv].reshape(Rg.shape)
            l2.append(paper_norms(phi - ref, dx, dy)[1])
        o = orders(l2)[-1]
        assert abs(o - o_exp) < 0.15, (k, l2, o)


@pytest.mark.parametrize("k,m,n", [(2, 3, 2), (3, 4, 2), (4, 3, 3), (5, 4, 3)])
def test_force_kernel_is_the_potential_difference(k, m, n):
    # u r^-3 = -d/du (1/r) and b_k' = b_{k-1}(t + 1/2) - b_{k-1}(t - 1/2), so
    # w^x_k(m, n) = (1/dx) [Phi_{k-1,k}(m + 1/2, n) - Phi_{k-1,k}(m - 1/2, n)] with Phi the
    # potential integral of orders (k-1, k): the potential route against the paper's closed
    # forms (route P) for the force kernel
    import mpmath as mp
    dx = 1.0
    with mp.workdps(25):
        rhs = (kt.w_phi_route(k - 1, m + 0.5, n, dx, 1.0, dps=25, k_v=k)
               - kt.w_phi_route(k - 1, m - 0.5, n, dx, 1.0, dps=25, k_v=k)) / dx
    lhs = kt.w_route_p(k, m, n, dx, 1.0, "x")
    assert abs(lhs - rhs) < mp.mpf(10) ** -15 * abs(lhs)
