"""Analytic in-plane radial force of generalized Maclaurin disks (Sec. 3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

sigma_{D_n}(R) = sigma_0 (1 - R^2 / a^2)^(n - 1/2) for R < a, 0 outside (Sec. 3), with
eta = a / R.  The paper prints F_R for D_3 and D_4 at z = 0; D_2 (exponent 3/2), needed
for the 64 x 64 and 512 x 512 workloads, is not printed.  Its form below was obtained by
the same pattern (inside: (pi^2 G sigma_0 / 2) eta^(-(2n-1)) P_n(eta); outside: the asin /
sqrt combination whose small-eta expansion has no eta^1 ... eta^(2n-1) terms) and is
pinned in tests against a direct elliptic-integral quadrature of the disk potential.
All forms are attractive (F_R < 0), with F = G x (the convolution), Sec. 1.

D_5 and D_6 (exponents 9/2 and 11/2, the smooth disks that show orders 4 and 5) follow
the same rule, written out in ``rule_coefficients``: inside, F_R is
(pi^2 G sigma_0 / 2) c_n d/ds 2F1(-n, 1/2; 1; s^2) with s = R / a and
c_n = 2 binom(2n, n) / 4^n; outside, Q_n cancels the eta^1 ... eta^(2n-1) Taylor terms of
P_n(eta) asin(eta) / sqrt(1 - eta^2).  The rule reproduces the printed D_3 and D_4
coefficients exactly (tests), and D_5, D_6 are pinned by the same potential quadrature.
"""
from __future__ import annotations

from fractions import Fraction
from math import comb, factorial

import mpmath as mp
import numpy as np

_PI = np.pi

# inside polynomial P_n(eta) and outside sqrt polynomial Q_n(eta), coefficients by power
_INSIDE = {
    1: {0: -1.0},
    2: {0: 9.0 / 8.0, 2: -3.0 / 2.0},
    3: {0: -75.0 / 64.0, 2: 45.0 / 16.0, 4: -15.0 / 8.0},
    4: {0: 1225.0 / 1024.0, 2: -525.0 / 128.0, 4: 315.0 / 64.0, 6: -35.0 / 16.0},
}
_OUTSIDE_SQRT = {
    1: {1: 1.0},
    2: {1: -9.0 / 8.0, 3: 3.0 / 4.0},
    3: {1: 75.0 / 64.0, 3: -65.0 / 32.0, 5: 5.0 / 8.0},
    4: {1: -1225.0 / 1024.0, 3: 5075.0 / 1536.0, 5: -1085.0 / 384.0, 7: 35.0 / 64.0},
}


def rule_coefficients(n: int) -> tuple[dict, dict]:
    """(P_n, Q_n) by power, exact rationals, from the hypergeometric rule above."""
    c_n = Fraction(2 * comb(2 * n, n), 4 ** n)
    inside = {}
    for j in range(1, n + 1):
        # a_j = (-n)_j (1/2)_j / (j!)^2, the coefficient of x^j in 2F1(-n, 1/2; 1; x)
        a = Fraction(1)
        for i in range(j):
            a *= Fraction(-n + i) * (Fraction(1, 2) + i)
        a /= factorial(j) ** 2
        inside[2 * (n - j)] = c_n * 2 * j * a
    # asin(eta) / sqrt(1 - eta^2) = sum_i 4^i (i!)^2 / (2i + 1)! eta^(2i + 1)
    outside = {}
    for p_pow, pc in inside.items():
        for i in range(n):
            deg = p_pow + 2 * i + 1
            if deg <= 2 * n - 1:
                outside[deg] = outside.get(deg, Fraction(0)) - pc * Fraction(4 ** i * factorial(i) ** 2,
                                                                              factorial(2 * i + 1))
    return inside, {q: v for q, v in outside.items() if v != 0}


def _coefs(n: int) -> tuple[dict, dict]:
    if n in _INSIDE:
        return _INSIDE[n], _OUTSIDE_SQRT[n]
    ins, out = rule_coefficients(n)
    return {q: float(v) for q, v in ins.items()}, {q: float(v) for q, v in out.items()}


def _poly(coefs: dict, x):
    return sum(c * x ** p for p, c in coefs.items())


def radial_force(n: int, R, a: float, sigma0: float = 1.0, G: float = 1.0):
    """F_R of the D_n disk at z = 0 (Sec. 3 for n = 3, 4; derived n = 2 and n >= 5; classic
    n = 1).

    D_1 reduces to the classic Maclaurin disk, F_R = -pi^2 G sigma_0 R / (2 a) inside.
    """
    R = np.asarray(R, dtype=np.float64)
    eta = a / R
    p = 2 * n - 1
    out = np.empty_like(R)
    ins, outs = _coefs(n)
    inside = eta >= 1.0
    e = eta[inside]
    out[inside] = (_PI ** 2 * sigma0 * G / 2.0) * e ** (-p) * _poly(ins, e)
    e = eta[~inside]
    out[~inside] = _PI * sigma0 * G * e ** (-p) * (
        _poly(ins, e) * np.arcsin(e) + _poly(outs, e) * np.sqrt(1.0 - e * e))
    # far outside the disk the two outside terms cancel to O(eta^(2n+1)): evaluate there
    # with 50 digits (the loss is about eta^-(2n+1) ulp)
    far = eta < 0.35
    if far.any():
        out[far] = [_outside_mp(n, float(v), sigma0, G) for v in eta[far]]
    return out


def _outside_mp(n: int, eta: float, sigma0: float, G: float) -> float:
    ci, co = (_INSIDE[n], _OUTSIDE_SQRT[n]) if n in _INSIDE else rule_coefficients(n)
    with mp.workdps(50):
        e = mp.mpf(eta)
        ins = sum(mp.mpf(c.numerator) / c.denominator * e ** q if isinstance(c, Fraction) else mp.mpf(c) * e ** q
                  for q, c in ci.items())
        out = sum(mp.mpf(c.numerator) / c.denominator * e ** q if isinstance(c, Fraction) else mp.mpf(c) * e ** q
                  for q, c in co.items())
        return float(mp.pi * sigma0 * G * e ** (-(2 * n - 1)) * (ins * mp.asin(e) + out * mp.sqrt(1 - e * e)))


def cartesian_force(n: int, x, y, a: float, sigma0: float = 1.0, G: float = 1.0):
    """(F^x, F^y) = F_R (x, y) / R."""
    R = np.hypot(x, y)
    fr = radial_force(n, R, a, sigma0, G)
    return fr * x / R, fr * y / R, fr


def disk_potential(n: int, R, a: float, sigma0: float = 1.0, G: float = 1.0, dps: int = 25):
    """Potential of the D_n disk in its plane, Phi(R) = -G int sigma(R') R' dR' dphi / |x - x'|,
    by quadrature: the angular integral is 4 K(k^2) / (R + R'), k^2 = 4 R R' / (R + R')^2,
    with K from the arithmetic-geometric mean, K = pi / (2 agm(1, |R - R'| / (R + R'))).
    D_1 inside the disk has the closed form -(pi^2 G sigma_0 / (4 a)) (2 a^2 - R^2) (tests)."""
    R = np.atleast_1d(np.asarray(R, dtype=np.float64))
    out = np.empty_like(R)
    with mp.workdps(dps):
        for i, Rv in enumerate(R):
            Rm = mp.mpf(Rv)

            def f(Rp):
                return (1 - Rp * Rp / (a * a)) ** (n - mp.mpf(1) / 2) * Rp / (Rm + Rp) \
                    * mp.pi / (2 * mp.agm(1, abs(Rm - Rp) / (Rm + Rp)))
            pts = [0, Rm, a] if Rv < a else [0, a]
            out[i] = float(-4 * G * sigma0 * mp.quad(f, pts))
    return out
