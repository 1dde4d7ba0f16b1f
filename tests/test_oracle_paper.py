"""Whole-pipeline pins: the paper's printed error tables and the analytic disk forces.

Sec. 3: D3 and D4 generalized Maclaurin disks (a = 0.5, sigma0 = G = 1) on [-1, 1]^2,
N = 32 ... 512; errors of F^x and F_R against the analytic force (Tables 4-9).
"""
import os

import mpmath as mp
import numpy as np
import pytest

from oracle.analytic import cartesian_force, radial_force
from oracle.convolution import Solver
from oracle.norms import orders, paper_norms
from workloads.synthetic import grid, maclaurin_density

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows():
    out = []
    for line in open(os.path.join(GOLDEN, "paper_error_tables.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        out.append((int(f[0]), int(f[1]), int(f[2]), int(f[3]), np.array(list(map(float, f[4:])))))
    return out


_CACHE = {}


def _norms(k, n, N):
    key = (k, n, N)
    if key not in _CACHE:
        x, y, dx, dy = grid(N, N, -1.0, 1.0)
        sig = maclaurin_density(n, x, y, 0.5)
        fx, fy = Solver(N, N, k, dx, dy).forces(sig)
        X, Y = np.meshgrid(x, y, indexing="ij")
        ax, _, ar = cartesian_force(n, X, Y, 0.5)
        fr = (fx * X + fy * Y) / np.hypot(X, Y)
        _CACHE[key] = np.array(paper_norms(fx - ax, dx, dy) + paper_norms(fr - ar, dx, dy))
    return _CACHE[key]


def _same_5_digits(ours, printed):
    # printed with 5 significant digits: agree to within one unit of the last digit
    ulp = 10.0 ** (np.floor(np.log10(np.abs(printed))) - 4)
    return np.abs(ours - printed) <= 1.0 * ulp


@pytest.mark.parametrize("row", [r for r in _rows() if r[1] in (1, 3)],
                         ids=lambda r: f"T{r[0]}-N{r[3]}")
def test_tables_4_6_7_9_reproduced(row):
    tab, k, n, N, printed = row
    ours = _norms(k, n, N)
    ok = _same_5_digits(ours, printed)
    if N <= 256:
        assert ok.all(), (ours, printed)
    else:
        # N = 512: within 0.5% (L2 of F^x still to the printed digits).  The L1 norms, dominated
        # by the tiny errors far from the disk, differ by ~0.2%, the size of the FP64
        # round-off that closed-form tables carry at offsets ~1000 (Sec. 2.1 forms)
        assert ok[1], (ours, printed)
        assert np.all(np.abs(ours / printed - 1.0) < 5e-3)


@pytest.mark.parametrize("n", [3, 4])
def test_tables_5_8_order_two(n):
    # order 2 reproduces Tables 5 and 8 to leading order only: the difference is O(h^3),
    # so the ratio to the printed norms tends to 1 and the order is 2
    rows = [r for r in _rows() if r[1] == 2 and r[2] == n]
    ratios = []
    for tab, k, nn, N, printed in rows:
        ours = _norms(k, nn, N)
        ratios.append(ours[0] / printed[0])
    assert all(abs(r2 - 1) < 0.6 * abs(r1 - 1) for r1, r2 in zip(ratios[:-1], ratios[1:]))
    assert abs(ratios[-1] - 1) < 0.02
    ours_l1 = [_norms(2, n, N)[0] for N in (64, 128, 256, 512)]
    assert all(abs(o - 2.0) < 0.05 for o in orders(ours_l1))


def test_order_k_on_smooth_disk():
    # Sec. 3.1: order k for B-splines of order k on D_{k+1}-smooth disks (D4 here)
    for k, expect in ((1, 1.0), (2, 2.0), (3, 3.0)):
        l2 = [_norms(k, 4, N)[1] for N in (64, 128, 256)]
        assert abs(orders(l2)[-1] - expect) < 0.15


@pytest.mark.parametrize("k,n", [(4, 5), (5, 6)])
def test_order_k_orders_4_5(k, n):
    # orders 4 and 5 on the next smoother disks (D5, D6): every norm of F^x and F_R falls
    # like h^k (measured 4.13-4.15 and 5.28-5.40 between N = 128 and 256, approaching k
    # from above, the maximum norm from 4.06); a wrong stencil, table or solve leaves a
    # lower order
    N_list = (64, 128, 256)
    norms = np.array([_norms(k, n, N) for N in N_list])
    for col in range(6):
        o = orders(norms[:, col])
        assert k - 0.1 < o[-1] < k + 0.6, (col, o)
        assert min(o) > k - 0.2, (col, o)


# --------------------------------------------------------------------------------------
# Analytic forces (Sec. 3) against a direct quadrature of the disk potential
# --------------------------------------------------------------------------------------

def _potential_force(n, R, a):
    """F_R = -dPhi/dR with Phi(R) = -G int sigma(R') R' int dphi / |x - x'|, the angular
    integral as 4 K(k^2)/(R + R'), k^2 = 4 R R'/(R + R')^2 (complete elliptic integral)."""
    def phi(Rv):
        # K(k^2) = pi / (2 agm(1, k')), k' = |R - R'| / (R + R'), exact near R' = R
        f = lambda Rp: (1 - Rp * Rp / (a * a)) ** (n - mp.mpf(1) / 2) * Rp / (Rv + Rp) \
            * mp.pi / (2 * mp.agm(1, abs(Rv - Rp) / (Rv + Rp)))
        pts = [0, Rv, a] if Rv < a else [0, a]
        return -4 * mp.quad(f, pts)
    with mp.workdps(30):
        return float(-mp.diff(phi, mp.mpf(R)))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_analytic_force_against_potential_quadrature(n):
    a = 0.4
    for R in (0.1, 0.3, 0.45, 0.7, 1.2):
        ref = _potential_force(n, R, a)
        got = float(radial_force(n, np.array([R]), a)[0])
        assert abs(got - ref) < 1e-9 * abs(ref), (n, R, got, ref)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_analytic_force_continuity_and_far_field(n):
    a = 0.5
    eps = 1e-12
    lo, hi = radial_force(n, np.array([a * (1 - eps), a * (1 + eps)]), a)
    # continuous, with a sqrt(1 - eta^2) kink at the edge
    assert abs(lo - hi) < 10 * np.sqrt(eps) * abs(lo)
    # far field -> -G M / R^2 with M = 2 pi sigma0 a^2 / (2n + 1)
    R = 40.0
    M = 2 * np.pi * a * a / (2 * n + 1)
    fr = radial_force(n, np.array([R]), a)[0]
    assert abs(fr / (-M / R ** 2) - 1) < 1e-3


def test_hypergeometric_rule_reproduces_printed_coefficients():
    # the rule behind D5 and D6 gives the printed D3 and D4 forms (Sec. 3) and the classic
    # and derived D1, D2 coefficient for coefficient, in exact rationals
    from oracle.analytic import _INSIDE, _OUTSIDE_SQRT, rule_coefficients
    for n in (1, 2, 3, 4):
        ins, outs = rule_coefficients(n)
        assert {q: float(v) for q, v in ins.items()} == _INSIDE[n]
        assert {q: float(v) for q, v in outs.items()} == _OUTSIDE_SQRT[n]
