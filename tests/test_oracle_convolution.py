"""Pins of the oracle's discrete convolution, its transpose and the invariants (Eq. eqnF)."""
import numpy as np
import pytest

from oracle import kernel_tables as kt
from oracle.coefficients import bspline_coefficients
from oracle.convolution import (Solver, correlate_direct, correlate_fft, forces_direct,
                                forces_fft)


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("k,nx,ny,dy", [(1, 9, 9, 1.0), (2, 12, 20, 1.0), (3, 16, 16, 1.0),
                                        (3, 11, 7, 0.5), (2, 5, 13, 2.0), (4, 10, 13, 1.0), (5, 12, 9, 1.0)])
def test_fft_equals_direct_sum(k, nx, ny, dy):
    wx, wy = kt.kernel_tables(k, nx, ny, 1.0, dy)
    c = _rand((nx, ny), k)
    fx0, fy0 = forces_direct(c, wx, wy)
    fx1, fy1 = forces_fft(c, wx, wy)
    scale = max(np.abs(fx0).max(), np.abs(fy0).max())
    assert np.abs(fx1 - fx0).max() < 1e-13 * scale
    assert np.abs(fy1 - fy0).max() < 1e-13 * scale
    # the transpose, both ways
    gx, gy = _rand((nx, ny), 10 + k), _rand((nx, ny), 20 + k)
    a0 = correlate_direct(gx, gy, wx, wy)
    a1 = correlate_fft(gx, gy, wx, wy)
    assert np.abs(a1 - a0).max() < 1e-13 * np.abs(a0).max()


def test_direct_sum_against_definition_loop():
    # F_ij = sum_{i'j'} C_{i'j'} w(i-i', j-j') with scalar loops, tiny grid
    k, nx, ny = 2, 4, 3
    wx, wy = kt.kernel_tables(k, nx, ny, 1.0, 1.0)
    c = _rand((nx, ny), 3)
    fx, fy = forces_direct(c, wx, wy)
    for i in range(nx):
        for j in range(ny):
            sx = sum(c[a, b] * wx[i - a + nx - 1, j - b + ny - 1] for a in range(nx) for b in range(ny))
            sy = sum(c[a, b] * wy[i - a + nx - 1, j - b + ny - 1] for a in range(nx) for b in range(ny))
            assert abs(sx - fx[i, j]) < 1e-14 and abs(sy - fy[i, j]) < 1e-14


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_invariants(k):
    n = 24
    S = Solver(n, n, k, 1.0 / n, 1.0 / n)
    sig = _rand((n, n), 5)
    fx, fy = S.forces(sig)
    c = bspline_coefficients(sig, k)
    scale = np.abs(c).sum() * np.abs(fx).max()
    # discrete Newton's third law: sum C F = 0 (antisymmetric bilinear form)
    assert abs(np.sum(c * fx)) < 1e-13 * scale and abs(np.sum(c * fy)) < 1e-13 * scale
    # reflection i <-> N-1-i of sigma: F^x odd, F^y even
    sym = sig + sig[::-1, :]
    gx, gy = S.forces(sym)
    np.testing.assert_allclose(gx, -gx[::-1, :], atol=1e-13 * np.abs(gx).max())
    np.testing.assert_allclose(gy, gy[::-1, :], atol=1e-13 * np.abs(gy).max())
    # x <-> y symmetry on a square grid
    sq = sig + sig.T
    hx, hy = S.forces(sq)
    np.testing.assert_allclose(hy, hx.T, atol=1e-13 * np.abs(hx).max())
    # linearity
    s2 = _rand((n, n), 6)
    ax, ay = S.forces(2.0 * sig - 3.0 * s2)
    bx, by = S.forces(s2)
    np.testing.assert_allclose(ax, 2.0 * fx - 3.0 * bx, atol=1e-12 * np.abs(ax).max())


@pytest.mark.parametrize("k", [1, 2, 3])
def test_translation_equivariance(k):
    n = 48
    S = Solver(n, n, k, 1.0, 1.0)
    sig = np.zeros((n, n))
    sig[18:26, 20:27] = _rand((8, 7), 8)
    sh = np.roll(sig, (1, -1), axis=(0, 1))
    fx, fy = S.forces(sig)
    gx, gy = S.forces(sh)
    tol = 1e-10 * np.abs(fx).max()  # order 3: truncated solve leaks r^d, r = 3 - 2 sqrt 2
    np.testing.assert_allclose(gx[10:40, 10:40], np.roll(fx, (1, -1), axis=(0, 1))[10:40, 10:40], atol=tol)
    np.testing.assert_allclose(gy[10:40, 10:40], np.roll(fy, (1, -1), axis=(0, 1))[10:40, 10:40], atol=tol)


@pytest.mark.parametrize("k", [1, 3, 4, 5])
def test_adjoint_identities(k):
    nx, ny = 20, 14
    S = Solver(nx, ny, k, 1.0 / nx, 1.0 / nx)
    sig = _rand((nx, ny), 30)
    gx, gy = _rand((nx, ny), 31), _rand((nx, ny), 32)
    fx, fy = S.forces(sig)
    gs = S.adjoint(gx, gy)
    lhs = np.sum(gx * fx) + np.sum(gy * fy)
    rhs = np.sum(gs * sig)
    assert abs(lhs - rhs) < 1e-13 * (abs(lhs) + np.abs(gs).sum() * np.abs(sig).max())
    np.testing.assert_allclose(S.adjoint(gx, gy, "direct"), gs, atol=1e-13 * np.abs(gs).max())
    # central finite differences: L is linear, so only rounding remains
    for (i, j) in [(0, 0), (3, 5), (nx - 1, ny - 1), (10, 0)]:
        e = np.zeros((nx, ny))
        e[i, j] = 1.0
        px, py = S.forces(sig + e)
        mx, my = S.forces(sig - e)
        fd = 0.5 * (np.sum(gx * (px - mx)) + np.sum(gy * (py - my)))
        assert abs(fd - gs[i, j]) < 1e-11 * np.abs(gs).max()


def test_planted_table3_typo_is_caught(monkeypatch):
    # A mistake planted in the oracle: restore the sign printed in Table 3 for the
    # (y0,y1) x (x1,x2) rectangle's (1,1) term.  Route P then disagrees with route I.
    orig = kt.route_p_terms

    def typo(k, m, n, dx, dy, component="x"):
        rects = orig(k, m, n, dx, dy, component)
        (box, terms) = rects[1 * k + 0]  # x-piece 1, y-piece 0
        rects[1 * k + 0] = (box, [(a, b_, -g if (a, b_) == (1, 1) else g) for a, b_, g in terms])
        return rects

    monkeypatch.setattr(kt, "route_p_terms", typo)
    p = kt.w_route_p(3, 3, 2, 1.0, 1.0)
    i = kt.w_route_i(3, 3, 2, 1.0, 1.0)
    assert abs(p - i) > 1e-6 * abs(i)


def test_planted_transposed_tables_break_invariant():
    # a plausible indexing mistake (the two tables swapped) violates F^x oddness
    n = 16
    S = Solver(n, n, 2, 1.0, 1.0)
    sig = np.random.default_rng(4).standard_normal((n, n))
    sig = sig + sig[::-1, :]
    fx, _ = forces_fft(sig, S.wy, S.wx)
    assert np.abs(fx + fx[::-1, :]).max() > 1e-3 * np.abs(fx).max()


def test_threaded_fft_equals_direct_sum():
    """The multi-threaded FFT primitive (scipy's pocketfft over host threads, used to time
    the oracle on all cores) gives the direct double sum of Eq. (eqnF), like numpy's."""
    import os
    nx, ny, k = 20, 14, 3
    rng = np.random.default_rng(11)
    sigma = rng.standard_normal((nx, ny))
    S = Solver(nx, ny, k, 1.0 / nx, 1.0 / nx)
    rx, ry = S.forces(sigma, method="direct")
    fx, fy = S.forces(sigma, workers=os.cpu_count() or 1)
    scale = max(np.abs(rx).max(), np.abs(ry).max())
    assert np.abs(fx - rx).max() < 1e-13 * scale
    assert np.abs(fy - ry).max() < 1e-13 * scale
