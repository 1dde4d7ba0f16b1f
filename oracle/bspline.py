"""B-spline basis of order k, written out from its recursive definition.

TEST INFRASTRUCTURE ONLY: the oracle is imported by tests/, the smoke check and the
CPU-baseline leg of bench.py, never by the product library.

Paper references (arXiv 1904.07400):
  * Eq. (Bspline1) - order-1 B-spline, the indicator of one knot interval.
  * Eq. (eqnBk)    - Cox-de Boor recursion for order k > 1.
  * Eqs. (Bspline2), (Bspline3) - the explicit order-2 and order-3 pieces.
  * Sec. 2.3       - every spline is centred on its cell centre (the symmetric point of
                     B^[k] coincides with (x_i, y_j)), with distinct, uniformly spaced knots.
  * Eq. (weight_matrix) - W = (1/64)[1 6 1; 6 36 6; 1 6 1], the order-3 tensor values at
                     the nine cell centres of its support.

Reading used throughout the oracle: b_k(t) is the centred cardinal B-spline of unit
knot spacing, knots at t = -k/2, -k/2+1, ..., k/2 (faces for odd k, cell centres for
even k).  In a grid with spacing h the coefficient C_i carries b_k((x - x_i)/h).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
from numpy.polynomial import Polynomial


def centred_knots(k: int) -> list[Fraction]:
    """Knots t_0..t_k of the centred order-k spline (unit spacing, symmetric about 0)."""
    half = Fraction(k, 2)
    return [Fraction(j) - half for j in range(k + 1)]


def cox_de_boor(k: int, i: int, knots, x: float) -> float:
    """Value of B^[k]_i(x) by the recursion Eq. (eqnBk), base case Eq. (Bspline1)."""
    if k == 1:
        return 1.0 if float(knots[i]) <= x < float(knots[i + 1]) else 0.0
    ti, tik1 = float(knots[i]), float(knots[i + k - 1])
    ti1, tik = float(knots[i + 1]), float(knots[i + k])
    left = (x - ti) / (tik1 - ti) * cox_de_boor(k - 1, i, knots, x)
    right = (tik - x) / (tik - ti1) * cox_de_boor(k - 1, i + 1, knots, x)
    return left + right


def b(k: int, t: float) -> float:
    """Centred cardinal B-spline b_k(t) = B^[k]_0 on the centred knots."""
    return cox_de_boor(k, 0, centred_knots(k), float(t))


def _poly_on_interval(k: int, i: int, knots, j: int) -> Polynomial:
    """B^[k]_i restricted to the knot interval [t_j, t_{j+1}) as a polynomial.

    Same recursion as Eq. (eqnBk), carried out on polynomial objects instead of values.
    """
    if k == 1:
        return Polynomial([1.0 if i == j else 0.0])
    ti, tik1 = float(knots[i]), float(knots[i + k - 1])
    ti1, tik = float(knots[i + 1]), float(knots[i + k])
    left = Polynomial([-ti, 1.0]) / (tik1 - ti) * _poly_on_interval(k - 1, i, knots, j)
    right = Polynomial([tik, -1.0]) / (tik - ti1) * _poly_on_interval(k - 1, i + 1, knots, j)
    return left + right


def _padd(a: list, b: list) -> list:
    n = max(len(a), len(b))
    return [(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(n)]


def _pmul(a: list, b: list) -> list:
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _exact_on_interval(k: int, i: int, knots, j: int) -> list[Fraction]:
    """Coefficients (by power) of B^[k]_i on [t_j, t_{j+1}), in exact rationals: the same
    recursion Eq. (eqnBk) on polynomials with Fraction coefficients."""
    if k == 1:
        return [Fraction(1 if i == j else 0)]
    ti, tik1 = knots[i], knots[i + k - 1]
    ti1, tik = knots[i + 1], knots[i + k]
    left = _pmul([-ti / (tik1 - ti), 1 / (tik1 - ti)], _exact_on_interval(k - 1, i, knots, j))
    right = _pmul([tik / (tik - ti1), -1 / (tik - ti1)], _exact_on_interval(k - 1, i + 1, knots, j))
    return _padd(left, right)


def pieces_exact(k: int) -> list[tuple[Fraction, Fraction, list[Fraction]]]:
    """The k pieces (lo, hi, coefficients by power of t) of b_k in exact rationals.  Orders
    4 and 5 have coefficients that are not binary fractions, so routes that compose the
    pieces with large offsets start from these, not from their FP64 roundings."""
    knots = centred_knots(k)
    return [(knots[j], knots[j + 1], _exact_on_interval(k, 0, knots, j)) for j in range(k)]


def pieces(k: int) -> list[tuple[float, float, Polynomial]]:
    """The k polynomial pieces (lo, hi, p) of b_k, p valid on [lo, hi) (FP64 coefficients,
    each the rounding of the exact rational)."""
    return [(float(lo), float(hi), Polynomial([float(c) for c in cs])) for lo, hi, cs in pieces_exact(k)]


def eval_exact(k: int, t: float) -> float:
    """b_k(t) for a float t, evaluated in exact rationals and rounded once."""
    ft = Fraction(t)
    for lo, hi, cs in pieces_exact(k):
        if lo <= ft < hi:
            acc = Fraction(0)
            for c in reversed(cs):
                acc = acc * ft + c
            return float(acc)
    return 0.0


def values_at_integers(k: int) -> dict[int, float]:
    """b_k at the integer offsets inside its support (the 1-D interpolation stencil)."""
    half = k // 2 + 1
    return {m: b(k, float(m)) for m in range(-half, half + 1) if b(k, float(m)) != 0.0}


def weight_matrix() -> np.ndarray:
    """Eq. (weight_matrix): order-3 tensor spline evaluated at the 3x3 cell centres."""
    v = np.array([b(3, -1.0), b(3, 0.0), b(3, 1.0)])
    return np.outer(v, v)
