"""Pins of the oracle's B-spline basis and coefficient solve (Sec. 2, Sec. 2.3)."""
import numpy as np
import pytest
import scipy.linalg

from oracle.bspline import b, pieces, pieces_exact, weight_matrix
from oracle.coefficients import apply_interpolation, banded_solve, bspline_coefficients, stencil, thomas


def test_weight_matrix_matches_paper():
    # Eq. (weight_matrix): W = (1/64) [1 6 1; 6 36 6; 1 6 1]
    printed = np.array([[1, 6, 1], [6, 36, 6], [1, 6, 1]]) / 64.0
    np.testing.assert_allclose(weight_matrix(), printed, rtol=0, atol=1e-16)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_partition_of_unity_and_unit_mass(k):
    rng = np.random.default_rng(0)
    for t in rng.uniform(-3, 3, 50):
        s = sum(b(k, t - j) for j in range(-6, 7))
        assert abs(s - 1.0) < 1e-14
    # integral over the support = 1 (exact on polynomial pieces)
    total = sum((p.integ()(hi) - p.integ()(lo)) for lo, hi, p in pieces(k))
    assert abs(total - 1.0) < 1e-15


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_smoothness_at_knots(k):
    # Sec. 2: distinct knots -> the first k-2 derivatives are continuous (C^{k-2})
    ps = pieces(k)
    for (lo0, hi0, p0), (lo1, hi1, p1) in zip(ps[:-1], ps[1:]):
        for d in range(k - 1):
            assert abs(p0.deriv(d)(hi0) - p1.deriv(d)(lo1)) < 1e-13
    # vanishes with its derivatives at the ends of the support (continuity with 0)
    for d in range(k - 1):
        assert abs(ps[0][2].deriv(d)(ps[0][0])) < 1e-13
        assert abs(ps[-1][2].deriv(d)(ps[-1][1])) < 1e-13


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_bspline_is_repeated_box_convolution(k):
    # textbook identity for cardinal splines: b_k(t) = int_{-1/2}^{1/2} b_{k-1}(t - s) ds
    import scipy.integrate
    rng = np.random.default_rng(3)
    knots = [j - (k - 1) / 2.0 for j in range(k)]
    for t in rng.uniform(-k / 2.0, k / 2.0, 25):
        pts = [t - kk for kk in knots if -0.5 < t - kk < 0.5]
        val, _ = scipy.integrate.quad(lambda s: b(k - 1, t - s), -0.5, 0.5, points=pts or None,
                                      epsabs=1e-15, epsrel=1e-14)
        assert abs(val - b(k, t)) < 1e-13


def test_centred_values_at_cell_centres():
    # Fig. 1 / Eq. (weight_matrix): order-3 spline = 1/8, 6/8, 1/8 at centres; order 2 is
    # the hat (1 at its centre, 0 at the neighbours), so C = sigma for k <= 2 (Sec. 2.3)
    assert [b(3, t) for t in (-1, 0, 1)] == [0.125, 0.75, 0.125]
    assert [b(2, t) for t in (-1, 0, 1)] == [0.0, 1.0, 0.0]
    assert [b(1, t) for t in (-1, 0, 1)] == [0.0, 1.0, 0.0]


def test_thomas_matches_lapack_banded():
    rng = np.random.default_rng(1)
    for n in (2, 3, 17, 200):
        rhs = rng.standard_normal((n, 5))
        ab = np.zeros((3, n))
        ab[0, 1:] = 1.0
        ab[1, :] = 6.0
        ab[2, :-1] = 1.0
        ref = scipy.linalg.solve_banded((1, 1), ab, rhs)
        np.testing.assert_allclose(thomas(1.0, 6.0, 1.0, rhs), ref, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("shape", [(2, 3), (5, 7), (17, 33), (64, 48)])
def test_coefficient_solve_reproduces_sigma(shape):
    # residual of Eq. (sigmaW) with the isolated boundary condition C = 0 outside
    rng = np.random.default_rng(2)
    sigma = rng.standard_normal(shape)
    c = bspline_coefficients(sigma, 3)
    np.testing.assert_allclose(apply_interpolation(c, 3), sigma, rtol=0, atol=1e-13)
    for k in (1, 2):
        np.testing.assert_array_equal(bspline_coefficients(sigma, k), sigma)


def test_interpolation_stencil_is_weight_matrix():
    c = np.zeros((7, 7))
    c[3, 3] = 1.0
    s = apply_interpolation(c, 3)
    np.testing.assert_allclose(s[2:5, 2:5], weight_matrix(), atol=1e-17)
    assert np.count_nonzero(s) == 9


# --------------------------------------------------------------------------------------
# Orders 4 and 5: the same interpolation condition with wider stencils
# --------------------------------------------------------------------------------------

def test_stencils_orders_4_5_are_the_cardinal_values():
    # cardinal cubic and quartic B-splines at the integers (Euler-Frobenius numbers):
    # (1, 4, 1)/6 and (1, 76, 230, 76, 1)/384
    np.testing.assert_allclose(stencil(4), np.array([1, 4, 1]) / 6.0, rtol=0, atol=2e-16)
    np.testing.assert_allclose(stencil(5), np.array([1, 76, 230, 76, 1]) / 384.0, rtol=0, atol=2e-16)
    assert stencil(3) == [0.125, 0.75, 0.125]
    # the exact rational pieces: b_5 on its first interval is (t + 5/2)^4 / 24
    from fractions import Fraction as Fr
    lo, hi, cs = pieces_exact(5)[0]
    assert (lo, hi) == (Fr(-5, 2), Fr(-3, 2))
    assert cs == [Fr(625, 384), Fr(125, 48), Fr(25, 16), Fr(5, 12), Fr(1, 24)]


@pytest.mark.parametrize("k", [3, 4, 5])
def test_banded_solve_matches_lapack(k):
    st = stencil(k)
    h = (len(st) - 1) // 2
    rng = np.random.default_rng(k)
    for n in (1, 2, 3, 4, 17, 200):
        rhs = rng.standard_normal((n, 3))
        ab = np.zeros((2 * h + 1, n))
        for d in range(-h, h + 1):
            # LAPACK band storage: ab[h + i - j, j] = A[i, j]; diagonal i - j = -d holds st[d + h]
            row = h - d
            if d >= 0:
                ab[row, d:] = st[d + h]
            else:
                ab[row, :n + d] = st[d + h]
        ref = scipy.linalg.solve_banded((h, h), ab, rhs)
        np.testing.assert_allclose(banded_solve(st, rhs), ref, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("k", [4, 5])
@pytest.mark.parametrize("shape", [(1, 3), (3, 4), (6, 5), (11, 9)])
def test_coefficient_solve_orders_4_5_by_direct_evaluation(k, shape):
    # the interpolation condition itself: sum_{i'j'} C b_k(i - i') b_k(j - j') = sigma at every
    # cell centre, the spline values taken from the recursive definition (C = 0 outside)
    rng = np.random.default_rng(7 + k)
    sigma = rng.standard_normal(shape)
    c = bspline_coefficients(sigma, k)
    nx, ny = shape
    bx = np.array([[b(k, float(i - a)) for a in range(nx)] for i in range(nx)])
    by = np.array([[b(k, float(j - a)) for a in range(ny)] for j in range(ny)])
    np.testing.assert_allclose(bx @ c @ by.T, sigma, rtol=0, atol=1e-13)
    np.testing.assert_allclose(apply_interpolation(c, k), sigma, rtol=0, atol=1e-13)
