"""Analytic in-plane radial force of generalized Maclaurin disks (Sec. 3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

sigma_{D_n}(R) = sigma_0 (1 - R^2 / a^2)^(n - 1/2) for R < a, 0 outside (Sec. 3), with
eta = a / R.  The paper prints F_R for D_3 and D_4 at z = 0; D_2 (exponent 3/2), needed
for the 64 x 64 and 512 x 512 workloads, is not printed.  Its form below was obtained by
the same pattern (inside: (pi^2 G sigma_0 / 2) eta^(-(2n-1)) P_n(eta); outside: the asin /
sqrt combination whose small-eta expansion has no eta^1 ... eta^(2n-1) terms) and is
pinned in tests against a direct elliptic-integral quadrature of the disk potential.
All forms are attractive (F_R < 0), with F = G x (the convolution), Sec. 1.
"""
from __future__ import annotations

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


def _poly(coefs: dict, x):
    return sum(c * x ** p for p, c in coefs.items())


def radial_force(n: int, R, a: float, sigma0: float = 1.0, G: float = 1.0):
    """F_R of the D_n disk at z = 0 (Sec. 3 for n = 3, 4; derived n = 2; classic n = 1).

    D_1 reduces to the classic Maclaurin disk, F_R = -pi^2 G sigma_0 R / (2 a) inside.
    """
    R = np.asarray(R, dtype=np.float64)
    eta = a / R
    p = 2 * n - 1
    out = np.empty_like(R)
    inside = eta >= 1.0
    e = eta[inside]
    out[inside] = (_PI ** 2 * sigma0 * G / 2.0) * e ** (-p) * _poly(_INSIDE[n], e)
    e = eta[~inside]
    out[~inside] = _PI * sigma0 * G * e ** (-p) * (
        _poly(_INSIDE[n], e) * np.arcsin(e) + _poly(_OUTSIDE_SQRT[n], e) * np.sqrt(1.0 - e * e))
    # far outside the disk the two outside terms cancel to O(eta^(2n+1)): evaluate there
    # with 50 digits (the loss is about eta^-(2n+1) ulp)
    far = eta < 0.35
    if far.any():
        out[far] = [_outside_mp(n, float(v), sigma0, G) for v in eta[far]]
    return out


def _outside_mp(n: int, eta: float, sigma0: float, G: float) -> float:
    with mp.workdps(50):
        e = mp.mpf(eta)
        ins = sum(mp.mpf(c) * e ** q for q, c in _INSIDE[n].items())
        out = sum(mp.mpf(c) * e ** q for q, c in _OUTSIDE_SQRT[n].items())
        return float(mp.pi * sigma0 * G * e ** (-(2 * n - 1)) * (ins * mp.asin(e) + out * mp.sqrt(1 - e * e)))


def cartesian_force(n: int, x, y, a: float, sigma0: float = 1.0, G: float = 1.0):
    """(F^x, F^y) = F_R (x, y) / R."""
    R = np.hypot(x, y)
    fr = radial_force(n, R, a, sigma0, G)
    return fr * x / R, fr * y / R, fr
