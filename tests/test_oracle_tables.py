"""Pins of the oracle's kernel tables w^x, w^y (Sec. 2.1-2.2, Tables 1-3, Appendix A/B)."""
import os

import mpmath as mp
import numpy as np
import pytest
import sympy

from oracle import kernel_tables as kt

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------------------
# Appendix A / B: the antiderivatives
# --------------------------------------------------------------------------------------

def _appendix_a():
    rows = []
    for line in open(os.path.join(GOLDEN, "paper_appendix_a.txt")):
        if line.startswith("#") or not line.strip():
            continue
        left, expr = line.split("|")
        a, b_ = map(int, left.split())
        rows.append((a, b_, expr.strip()))
    return rows


@pytest.mark.parametrize("row", _appendix_a(), ids=lambda r: f"F{r[0]}{r[1]}")
def test_appendix_a_forms_differentiate_to_integrand(row):
    a, b_, expr = row
    x, y = sympy.symbols("x y", positive=True)
    r = sympy.sqrt(x ** 2 + y ** 2)
    F = sympy.sympify(expr, locals={"x": x, "y": y, "r": r})
    integrand = x ** a * y ** b_ / r ** 3
    assert sympy.simplify(sympy.diff(F, x, y) - integrand) == 0


@pytest.mark.parametrize("row", _appendix_a(), ids=lambda r: f"F{r[0]}{r[1]}")
def test_recursion_antiderivative_matches_appendix_a(row):
    # Eq. (intF)/(B10) with Eq. (intMoment)/(B3) gives the same definite integrals
    # (Eq. intFtilde) as the printed closed forms, on rectangles clear of the axes
    a, b_, expr = row
    x, y = sympy.symbols("x y")
    r = sympy.sqrt(x ** 2 + y ** 2)
    F = sympy.lambdify((x, y), sympy.sympify(expr, locals={"x": x, "y": y, "r": r}), "mpmath")
    rng = np.random.default_rng(a * 10 + b_)
    with mp.workdps(40):
        for _ in range(4):
            xl, yl = rng.uniform(0.3, 2.0, 2) * rng.choice([-1, 1], 2)
            xr, yr = xl + rng.uniform(0.1, 0.5), yl + rng.uniform(0.1, 0.5)
            if xl < 0 < xr or yl < 0 < yr:
                continue
            xl, xr, yl, yr = map(mp.mpf, (xl, xr, yl, yr))
            printed = F(xr, yr) - F(xl, yr) - F(xr, yl) + F(xl, yl)
            ours = kt.F_tilde(xl, xr, yl, yr, a, b_)
            assert abs(printed - ours) < mp.mpf(10) ** -30 * max(1, abs(ours))


@pytest.mark.parametrize("a,b_", [(3, 2), (2, 3), (1, 4), (4, 1), (5, 0), (0, 2)])
def test_recursion_beyond_appendix_a(a, b_):
    # alpha + beta = 5 (needed for order 3) is beyond Appendix A: check the recursion's
    # Ftilde against direct 2-D quadrature of the monomial
    with mp.workdps(25):
        xl, xr, yl, yr = mp.mpf("0.7"), mp.mpf("1.3"), mp.mpf("-2.1"), mp.mpf("-1.6")
        direct = mp.quad(lambda u, v: u ** a * v ** b_ / (u * u + v * v) ** 1.5, [xl, xr], [yl, yr])
        assert abs(kt.F_tilde(xl, xr, yl, yr, a, b_) - direct) < mp.mpf(10) ** -18


# --------------------------------------------------------------------------------------
# Tables 1-3: the monomial expansion of each case
# --------------------------------------------------------------------------------------

def _printed_tables():
    rows = []
    for line in open(os.path.join(GOLDEN, "paper_tables_1_3.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, yb, xa, a, b_, g = line.split()
        rows.append((int(k), int(yb), int(xa), int(a), int(b_), g))
    return rows


@pytest.mark.parametrize("k", [1, 2, 3])
def test_expansion_matches_printed_tables(k):
    dx, dy = 0.37, 0.61
    m, n = 5, -3
    rects = kt.route_p_terms(k, m, n, dx, dy, "x")
    xs = [(-m - k / 2.0 + r) * dx for r in range(k + 1)]
    ys = [(-n - k / 2.0 + r) * dy for r in range(k + 1)]
    env = {f"x{r}": xs[r] for r in range(k + 1)}
    env.update({f"y{r}": ys[r] for r in range(k + 1)})
    if k == 3:
        env.update(Ax=sum(xs), Bx=xs[0] * xs[2] + xs[1] * xs[3],
                   Ay=sum(ys), By=ys[0] * ys[2] + ys[1] * ys[3])
    pref = {1: 1.0, 2: 1.0 / (dx * dy), 3: 1.0 / (4 * dx * dx * dy * dy)}[k]
    ours = {}
    for idx, (_, terms) in enumerate(rects):
        xa, yb = idx // k, idx % k
        for a, b_, g in terms:
            ours[(yb, xa, a, b_)] = ours.get((yb, xa, a, b_), 0.0) + g
    printed = {}
    for kk, yb, xa, a, b_, g in _printed_tables():
        if kk == k:
            printed[(yb, xa, a, b_)] = pref * eval(g, {}, env)
    assert set(printed) == {key for key, v in ours.items() if v != 0.0} | set(printed)
    mismatched = [key for key in printed if abs(printed[key] - ours.get(key, 0.0)) > 1e-9 * (1 + abs(printed[key]))]
    if k < 3:
        assert mismatched == []
    else:
        # Table 3, rectangle (y0,y1) x (x1,x2), triplet (1,1,.): expanding
        # x (-2x^2 + Ax x - Bx)(y - y0)^2 gives +2 Bx y0; the printed sign is a typo
        # (its mirror entry for (y2,y3) is printed with the correct sign)
        assert mismatched == [(0, 1, 1, 1)]
        assert abs(printed[(0, 1, 1, 1)] + ours[(0, 1, 1, 1)]) < 1e-9


# --------------------------------------------------------------------------------------
# Routes P / I / brute force / closed form agree
# --------------------------------------------------------------------------------------

ROUTE_CASES = [(k, m, n, comp, dy) for k in (1, 2, 3) for (m, n) in [(2, 2), (3, -2), (-4, 5), (2, 9)]
               for comp in ("x", "y") for dy in (1.0, 0.5)]


@pytest.mark.parametrize("case", ROUTE_CASES[::2] + ROUTE_CASES[1::7])
def test_route_p_equals_route_i(case):
    k, m, n, comp, dy = case
    dx = 1.0
    if not kt.route_p_valid(k, m, n):
        pytest.skip("rectangles touch an axis")
    p = kt.w_route_p(k, m, n, dx, dy, comp)
    i = kt.w_route_i(k, m, n, dx, dy, comp, dps=25)
    assert abs(p - i) < mp.mpf(10) ** -20 * abs(p)


@pytest.mark.parametrize("k,m,n", [(1, 3, 2), (2, 3, -2), (3, -3, 3)])
def test_route_i_equals_brute_force(k, m, n):
    ref = kt.w_brute(k, m, n, 1.0, 1.0, "x", dps=15)
    got = kt.w_route_i(k, m, n, 1.0, 1.0, "x", dps=20)
    assert abs(ref - got) < 1e-12 * abs(ref)


def test_k1_closed_form_rectangle_field():
    for (m, n) in [(1, 0), (1, 1), (2, -3), (7, 2)]:
        a = kt.w_k1_closed(m, n, 1.0, 1.0)
        b_ = kt.w_route_i(1, m, n, 1.0, 1.0, "x", dps=25)
        assert abs(a - b_) < 1e-20


def test_near_origin_principal_value():
    # w^x(0, n) = 0 exactly; w^x(1, 0) is finite and attractive (source at u < 0)
    for k in (1, 2, 3):
        assert abs(kt.w_route_i(k, 0, 1, 1.0, 1.0)) < 1e-25
        assert kt.w_route_i(k, 1, 0, 1.0, 1.0) < 0
    # order 2 near-origin value cross-checked against a thin-disk limit: u/(r^2+h^2)^(3/2)
    with mp.workdps(20):
        h = mp.mpf("1e-4")
        val = 0
        for (ul, uh, pu) in kt._rect_polys(2, 1, 1.0):
            for (vl, vh, pv) in kt._rect_polys(2, 0, 1.0):
                val += mp.quad(lambda u, v: u / (u * u + v * v + h * h) ** 1.5
                               * kt._poly_mp(pu, u) * kt._poly_mp(pv, v), [ul, uh], [vl, 0, vh])
    ref = kt.w_route_i(2, 1, 0, 1.0, 1.0)
    assert abs(val - ref) < 1e-3 * abs(ref)


def test_scale_invariance_and_symmetries():
    for k in (1, 2, 3):
        a = kt.w_route_i(k, 2, 3, 0.25, 0.5)
        b_ = kt.w_route_i(k, 2, 3, 1.0, 2.0)
        assert abs(a - b_) < 1e-20
        # w^y(m, n) = w^x(n, m) for square cells; odd/even reflections
        assert abs(kt.w_route_i(k, 2, 3, 1.0, 1.0, "y") - kt.w_route_i(k, 3, 2, 1.0, 1.0, "x")) < 1e-20
        assert abs(kt.w_route_i(k, -2, 3, 1.0, 1.0) + kt.w_route_i(k, 2, 3, 1.0, 1.0)) < 1e-20
        assert abs(kt.w_route_i(k, 2, -3, 1.0, 1.0) - kt.w_route_i(k, 2, 3, 1.0, 1.0)) < 1e-20


# --------------------------------------------------------------------------------------
# Far field and the assembled table
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("dy", [1.0, 0.5, 0.125])
def test_far_field_bands_reach_fp64(k, dy):
    # each band's Gauss-Legendre order against route I at the band's nearest offsets
    dx = 1.0
    checked = 0
    for (m, n) in [(4, 0), (4, 1), (0, 4), (1, 4), (4, 4), (3, 5), (0, 8), (2, 12), (8, 1),
                   (1, 17), (16, 3), (0, 33), (64, 2), (1, 130)]:
        d = float(kt.effective_distance(m, n, dx, dy))
        q = [q for lim, q in kt.FAR_BANDS if lim is None or d < lim][0]
        for comp in ("x", "y"):
            ref = float(kt.w_route_i(k, m, n, dx, dy, comp, dps=20))
            if ref == 0.0:
                continue
            got = kt.w_far_gl(k, np.array([m]), np.array([n]), dx, dy, q, comp)[0]
            assert abs(got - ref) < 2e-14 * abs(ref), (k, m, n, comp, q)
            checked += 1
    assert checked > 20


def test_far_field_order_converged_on_a_whole_table():
    # raising every band's Gauss-Legendre order by 2 changes nothing beyond rounding
    k, N = 3, 96
    q0 = kt.kernel_table_quarter(k, N, N, 1.0, 1.0)
    saved = kt.FAR_BANDS
    try:
        kt.FAR_BANDS = tuple((lim, q + 2) for lim, q in saved)
        q1 = kt.kernel_table_quarter(k, N, N, 1.0, 1.0)
    finally:
        kt.FAR_BANDS = saved
    nz = q0 != 0.0
    assert np.array_equal(nz, q1 != 0.0)
    assert np.max(np.abs(q1[nz] - q0[nz]) / np.abs(q0[nz])) < 5e-15


def test_assembled_table_symmetries():
    wx, wy = kt.kernel_tables(3, 12, 12, 0.1, 0.1)
    np.testing.assert_allclose(wx, -wx[::-1, :], atol=0)
    np.testing.assert_allclose(wx, wx[:, ::-1], atol=0)
    np.testing.assert_allclose(wy, wx.T, atol=0)
    wx2, wy2 = kt.kernel_tables(2, 6, 9, 0.2, 0.1)
    for (m, n) in [(1, 1), (3, -4), (-5, 8), (2, 0)]:
        ref = float(kt.w_route_i(2, m, n, 0.2, 0.1, "y"))
        assert abs(wy2[m + 5, n + 8] - ref) < 4e-15 * abs(ref) + 1e-18


# --------------------------------------------------------------------------------------
# Orders 4 and 5 (the extension the paper calls straightforward)
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("k,m,n,comp", [(4, 3, 3, "x"), (4, -4, 5, "y"), (5, 3, 4, "x"), (5, 4, -3, "y"),
                                        (5, 9, 4, "x")])
def test_route_p_equals_route_i_orders_4_5(k, m, n, comp):
    # the paper's monomial expansion (now with alpha + beta up to 5, via Eq. intMoment)
    # against integration by parts
    assert kt.route_p_valid(k, m, n)
    p = kt.w_route_p(k, m, n, 1.0, 1.0, comp)
    i = kt.w_route_i(k, m, n, 1.0, 1.0, comp, dps=25)
    assert abs(p - i) < mp.mpf(10) ** -18 * abs(p)


@pytest.mark.parametrize("k,m,n", [(4, 3, 3), (5, 4, 3)])
def test_route_i_equals_brute_force_orders_4_5(k, m, n):
    ref = kt.w_brute(k, m, n, 1.0, 0.5, "x", dps=15)
    got = kt.w_route_i(k, m, n, 1.0, 0.5, "x", dps=20)
    assert abs(ref - got) < 1e-12 * abs(ref)


@pytest.mark.parametrize("k", [4, 5])
def test_near_origin_orders_4_5(k):
    assert abs(kt.w_route_i(k, 0, 1, 1.0, 1.0)) < 1e-25
    assert kt.w_route_i(k, 1, 0, 1.0, 1.0) < 0
    a = kt.w_route_i(k, 2, 1, 0.25, 0.25, dps=20)
    b_ = kt.w_route_i(k, 2, 1, 1.0, 1.0, dps=20)
    assert abs(a - b_) < 1e-17
    # w is dimensionless: scaling both cell sides by 4 (cells of aspect 1:2) leaves it
    # unchanged (u r^-3 du dv is scale invariant), to the 40-digit default of route I
    a = kt.w_route_i(k, 2, 1, 0.25, 0.5)
    b_ = kt.w_route_i(k, 2, 1, 1.0, 2.0)
    assert abs(a - b_) < 1e-20
    assert abs(kt.w_route_i(k, 1, 2, 1.0, 1.0, "y") - kt.w_route_i(k, 2, 1, 1.0, 1.0, "x")) < 1e-20


@pytest.mark.parametrize("k", [4, 5])
@pytest.mark.parametrize("dy", [1.0, 0.125])
def test_far_field_bands_reach_fp64_orders_4_5(k, dy):
    # the nearest offsets of the bands that orders 4, 5 reach (the band distance is shifted
    # by (k - 3)/2 cells and the near field widened by k - 3)
    dx = 1.0
    nf = kt.near_field_size(k)
    checked = 0
    for (m, n) in [(nf, 0), (1, nf), (nf, nf), (0, nf + 2), (12, 3), (33, 0)]:
        d = float(kt.band_distance(k, m, n, dx, dy))
        q = [q for lim, q in kt.FAR_BANDS if lim is None or d < lim][0]
        for comp in ("x", "y"):
            if (comp == "x" and m == 0) or (comp == "y" and n == 0):
                continue
            ref = float(kt.w_route_i(k, m, n, dx, dy, comp, dps=25))
            got = kt.w_far_gl(k, np.array([m]), np.array([n]), dx, dy, q, comp)[0]
            assert abs(got - ref) < 2e-14 * abs(ref), (k, m, n, comp, q)
            checked += 1
    assert checked >= 8


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_far_field_second_moment_expansion(k):
    # far from the origin the spline acts through its moments: mass 1, mean 0, variance
    # k/12 per axis, so w = dx dy [f + (k/24)(dx^2 f_uu + dy^2 f_vv)] + O(d^-7) with
    # f = u r^-3 at the spline's centre (u, v) = (-m dx, -n dy); a dropped or wrong piece
    # of b_k changes the mass or the variance and fails this
    dx, dy = 1.0, 0.75
    for (m, n) in [(400, 150), (-300, 420), (90, -500)]:
        u, v = -m * dx, -n * dy
        r2 = u * u + v * v
        r = np.sqrt(r2)
        f = u / r ** 3
        fuu = -9 * u / r ** 5 + 15 * u ** 3 / r ** 7
        fvv = -3 * u / r ** 5 + 15 * u * v * v / r ** 7
        ref = dx * dy * (f + k / 24.0 * (dx * dx * fuu + dy * dy * fvv))
        got = kt.w_far_gl(k, np.array([m]), np.array([n]), dx, dy, 5, "x")[0]
        assert abs(got - ref) < 1e-9 * abs(ref), (k, m, n, got, ref)
        # the correction term itself is needed (it is ~1e-5 of f here)
        assert abs(got - dx * dy * f) > 1e3 * abs(got - ref)


def test_assembled_table_orders_4_5_against_route_i():
    # near field (route I) and far bands assembled, square cells, against route I
    for k in (4, 5):
        wx, wy = kt.kernel_tables(k, 9, 11, 0.1, 0.1)
        for (m, n) in [(1, 1), (3, -4), (-7, 8), (8, 10)]:
            refx = float(kt.w_route_i(k, m, n, 0.1, 0.1, "x", dps=20))
            refy = float(kt.w_route_i(k, m, n, 0.1, 0.1, "y", dps=20))
            assert abs(wx[m + 8, n + 10] - refx) < 2e-14 * abs(refx) + 1e-18
            assert abs(wy[m + 8, n + 10] - refy) < 2e-14 * abs(refy) + 1e-18
