"""Force-kernel tables w^x(m, n), w^y(m, n) (Sec. 2.1-2.2, Eqs. eqnw, eqnwB).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Definition (Eq. eqnwB with the change of variables of Eq. wk1, u = x' - x, v = y' - y,
m = i - i', n = j - j'):

    w^x(m, n) = PV int int  u (u^2 + v^2)^(-3/2)  b_k(u/dx + m) b_k(v/dy + n)  du dv
    w^y(m, n) = PV int int  v (u^2 + v^2)^(-3/2)  b_k(u/dx + m) b_k(v/dy + n)  du dv

so that F^x_ij = G sum_{i'j'} C_{i'j'} w^x(i-i', j-j') (Eq. eqnF).  The integrand is
only conditionally integrable at u = v = 0 (Sec. 1 calls the singularity removable); the
value taken is the symmetric principal value, which equals the thin-disk limit.

Three independent evaluations are provided:

* route P (the paper's): the integrand on each of the k x k polynomial rectangles is
  expanded in monomials u^alpha v^beta / r^3 (Tables 1-3 list exactly these triplets),
  and each monomial is integrated with the closed-form antiderivative F of Eq. (intF),
  built from G of Eq. (G_function) via the recursion Eq. (intMoment) and the base
  integrals Eqs. (B11)-(B13), evaluated at the four corners (Eq. intFtilde).  Done in
  mpmath at high precision, because the corner terms cancel catastrophically at large
  offsets.  Valid only where no rectangle touches an axis (the antiderivatives carry
  log singularities on the axes).
* route I (integration by parts): u/r^3 = -d/du (1/r), so
      w^x(m, n) = int dv b_k(v/dy + n) int dt b_k'(t) / sqrt(((t - m) dx)^2 + v^2),
  absolutely convergent everywhere; the inner integral is closed form (asinh, r), the
  outer one is an mpmath quadrature split at v = 0 and at the knots.
* far field: tensor Gauss-Legendre quadrature on each polynomial piece in plain FP64
  numpy, used where the rectangles are far enough from the origin for the smooth
  integrand to converge geometrically; the node count falls with distance.

``kernel_table`` assembles a whole table from route I (near field) and the far-field
quadrature.  Both are pinned against route P and against each other in tests/.
"""
from __future__ import annotations

import functools

import mpmath as mp
import numpy as np
from numpy.polynomial import Polynomial

from .bspline import eval_exact, pieces, pieces_exact

# ----------------------------------------------------------------------------------
# Route P: the paper's closed forms (Eqs. intF, G_function, intMoment, B11-B13)
# ----------------------------------------------------------------------------------


def G_anti(x, a, alpha: int):
    """Antiderivative in x of x^alpha / (x^2 + a^2)^(3/2)  (Eq. G_function).

    alpha = 0, 1, 2 from Eqs. (B11)-(B13); larger alpha by the recursion Eq. (intMoment).
    """
    r = mp.sqrt(x * x + a * a)
    if alpha == 0:
        return x / (a * a * r)
    if alpha == 1:
        return -1 / r
    if alpha == 2:
        return -x / r + mp.log(abs(x + r))
    return x ** (alpha - 1) / ((alpha - 2) * r) - mp.mpf(alpha - 1) / (alpha - 2) * a * a * G_anti(x, a, alpha - 2)


def F_anti(x, y, alpha: int, beta: int):
    """Antiderivative F(x, y, alpha, beta) of x^alpha y^beta / r^3 (Eq. intF / B10).

    alpha + beta = 1 is the one case Eq. (intF) excludes; Appendix A gives those forms.
    """
    r = mp.sqrt(x * x + y * y)
    if (alpha, beta) == (1, 0):
        return -mp.log(y + r)
    if (alpha, beta) == (0, 1):
        return -mp.log(x + r)
    s = alpha + beta - 1
    return (y ** (beta + 1) * G_anti(x, y, alpha) + x ** (alpha + 1) * G_anti(y, x, beta)) / s


def F_tilde(xl, xr, yl, yr, alpha: int, beta: int):
    """Definite integral over [xl, xr] x [yl, yr] (Eq. intFtilde), four-corner form."""
    return (F_anti(xr, yr, alpha, beta) - F_anti(xl, yr, alpha, beta)
            - F_anti(xr, yl, alpha, beta) + F_anti(xl, yl, alpha, beta))


class _MPoly:
    """Polynomial with mpmath coefficients, by power."""

    def __init__(self, coef):
        self.coef = list(coef)


def _mpf(fr) -> mp.mpf:
    return mp.mpf(fr.numerator) / fr.denominator


def _compose(cs, m: int, h: float) -> list:
    """Coefficients (by power of u) of p(u/h + m) for p given by exact rationals cs, in
    mpmath at the working precision (Horner on polynomials)."""
    a, s = mp.mpf(m), 1 / mp.mpf(h)
    acc = [mp.mpf(0)]
    for c in reversed(cs):
        nxt = [mp.mpf(0)] * (len(acc) + 1)
        for i, x in enumerate(acc):
            nxt[i] += x * a
            nxt[i + 1] += x * s
        nxt[0] += _mpf(c)
        acc = nxt
    return acc[:len(cs)]


def _rect_polys(k: int, m: int, h: float):
    """Pieces of b_k(u/h + m) as (u_lo, u_hi, polynomial in u), composed in mpmath from the
    exact rational pieces.

    Composition t = u/h + m of the unit-spacing pieces (Sec. 2.2: the rectangles of
    Cases 1-3 are the knot intervals of the shifted splines).
    """
    out = []
    for lo, hi, cs in pieces_exact(k):
        out.append(((_mpf(lo) - m) * mp.mpf(h), (_mpf(hi) - m) * mp.mpf(h), _MPoly(_compose(cs, m, h))))
    return out


def route_p_terms(k: int, m: int, n: int, dx: float, dy: float, component: str = "x"):
    """Monomial triplets (alpha, beta, gamma) per rectangle, i.e. the content of
    Tables 1-3 for this offset: the integrand u^a v^b / r^3 with coefficient gamma on
    [xl, xr] x [yl, yr].  The 1/(dx dy) and 1/(4 dx^2 dy^2) prefactors of Cases 2 and 3
    are folded into gamma."""
    rects = []
    for (ul, uh, pu) in _rect_polys(k, m, dx):
        for (vl, vh, pv) in _rect_polys(k, n, dy):
            terms = []
            cu = list(pu.coef) + [0.0] * (k + 1)
            cv = list(pv.coef) + [0.0] * (k + 1)
            for ia in range(k):
                for ib in range(k):
                    g = cu[ia] * cv[ib]
                    if g == 0.0:
                        continue
                    if component == "x":
                        terms.append((ia + 1, ib, g))
                    else:
                        terms.append((ia, ib + 1, g))
            rects.append(((ul, uh, vl, vh), terms))
    return rects


def route_p_valid(k: int, m: int, n: int) -> bool:
    """True when no rectangle of the offset touches the u or v axis (closed sets)."""
    half = k / 2.0
    for c in (m, n):
        lo, hi = -c - half, -c + half
        if lo <= 0.0 <= hi:
            return False
    return True


def w_route_p(k: int, m: int, n: int, dx: float, dy: float, component: str = "x", dps: int = 60):
    """w at one offset by the paper's route (Tables 1-3 expansion + Eq. intFtilde)."""
    if not route_p_valid(k, m, n):
        raise ValueError("route P needs rectangles clear of both axes")
    with mp.workdps(dps):
        total = mp.mpf(0)
        for (ul, uh, vl, vh), terms in route_p_terms(k, m, n, dx, dy, component):
            for a, b_, g in terms:
                total += mp.mpf(g) * F_tilde(mp.mpf(ul), mp.mpf(uh), mp.mpf(vl), mp.mpf(vh), a, b_)
        return total


# ----------------------------------------------------------------------------------
# Route I: integration by parts, absolutely convergent
# ----------------------------------------------------------------------------------


def _J(j: int, u, v):
    """Antiderivative in u of u^j / sqrt(u^2 + v^2), v != 0."""
    r = mp.sqrt(u * u + v * v)
    if j == 0:
        return mp.asinh(u / abs(v))
    if j == 1:
        return r
    return u ** (j - 1) * r / j - mp.mpf(j - 1) / j * v * v * _J(j - 2, u, v)


def _inner_ibp(k: int, m: int, h: float, v):
    """int dt b_k'(t) / sqrt(((t - m) h)^2 + v^2)  (the u-integral after parts)."""
    if k == 1:
        # b_1 jumps +1 at t = -1/2 and -1 at t = +1/2
        a0 = (-0.5 - m) * h
        a1 = (0.5 - m) * h
        return 1 / mp.sqrt(a0 * a0 + v * v) - 1 / mp.sqrt(a1 * a1 + v * v)
    total = mp.mpf(0)
    for lo, hi, cs in pieces_exact(k):
        dcs = [i * c for i, c in enumerate(cs)][1:]
        q = _compose(dcs, m, h)  # b'(u/h + m) as a polynomial in u
        ul, uh = (_mpf(lo) - m) * mp.mpf(h), (_mpf(hi) - m) * mp.mpf(h)
        for j, c in enumerate(q):
            if c != 0:
                total += c / h * (_J(j, uh, v) - _J(j, ul, v))
    return total


def w_route_i(k: int, m: int, n: int, dx: float, dy: float, component: str = "x", dps: int = 30):
    """w at one offset by integration by parts in the force direction."""
    if component == "y":
        # same integral with the roles of (u, m, dx) and (v, n, dy) exchanged
        return w_route_i(k, n, m, dy, dx, "x", dps)
    with mp.workdps(dps):
        total = mp.mpf(0)
        for lo, hi, cs in pieces_exact(k):
            vl, vh = (_mpf(lo) - n) * mp.mpf(dy), (_mpf(hi) - n) * mp.mpf(dy)
            pts = [vl, vh]
            if vl < 0 < vh:
                pts = [vl, mp.mpf(0), vh]
            pv = _MPoly(_compose(cs, n, dy))  # b(v/dy + n) as a polynomial in v

            def f(v, pv=pv):
                return _poly_mp(pv, v) * _inner_ibp(k, m, dx, v)

            total += mp.quad(f, pts)
        return total


def _poly_mp(p, t):
    acc = mp.mpf(0)
    for c in reversed(p.coef):
        acc = acc * t + mp.mpf(c)
    return acc


def w_k1_closed(m: int, n: int, dx: float, dy: float):
    """Order 1 in closed form: the x-field of a uniform rectangle (textbook result),
    obtained from route I with the v-integral done analytically."""
    with mp.workdps(40):
        vl, vh = mp.mpf((-0.5 - n) * dy), mp.mpf((0.5 - n) * dy)

        def edge(a):
            a = abs(mp.mpf(a))
            return mp.asinh(vh / a) - mp.asinh(vl / a)

        return edge((-0.5 - m) * dx) - edge((0.5 - m) * dx)


def w_brute(k: int, m: int, n: int, dx: float, dy: float, component: str = "x", dps: int = 20):
    """Direct 2-D quadrature of the definition, per polynomial rectangle.  Only for
    offsets whose support is clear of the origin (no principal value needed)."""
    if not route_p_valid(k, m, n):
        raise ValueError("brute force needs the support clear of both axes")
    with mp.workdps(dps):
        total = mp.mpf(0)
        for (ul, uh, pu) in _rect_polys(k, m, dx):
            for (vl, vh, pv) in _rect_polys(k, n, dy):
                def f(u, v, pu=pu, pv=pv):
                    r3 = (u * u + v * v) ** mp.mpf(1.5)
                    num = u if component == "x" else v
                    return num / r3 * _poly_mp(pu, u) * _poly_mp(pv, v)
                total += mp.quad(f, [ul, uh], [vl, vh])
        return total


# ----------------------------------------------------------------------------------
# Far field: tensor Gauss-Legendre per polynomial piece (plain FP64)
# ----------------------------------------------------------------------------------


@functools.lru_cache(maxsize=None)
def _gl_nodes(k: int, q: int):
    """Nodes t_a and weights b_k(t_a) * gl_a over the k pieces of b_k."""
    x, wgl = np.polynomial.legendre.leggauss(q)
    ts, ws = [], []
    for lo, hi, p in pieces(k):
        t = 0.5 * (hi - lo) * x + 0.5 * (hi + lo)
        ts.append(t)
        ws.append(0.5 * (hi - lo) * wgl * np.array([eval_exact(k, ti) for ti in t]))
    return np.concatenate(ts), np.concatenate(ws)


def w_far_gl(k: int, ms: np.ndarray, ns: np.ndarray, dx: float, dy: float, q: int,
             component: str = "x") -> np.ndarray:
    """sum_a sum_b W_a W_b f((t_a - m) dx, (t_b - n) dy) dx dy for arrays of offsets."""
    ms = np.asarray(ms, dtype=np.float64)
    ns = np.asarray(ns, dtype=np.float64)
    t, wt = _gl_nodes(k, q)
    out = np.zeros(np.broadcast(ms, ns).shape)
    for ta, wa in zip(t, wt):
        u = (ta - ms) * dx
        for tb, wb in zip(t, wt):
            v = (tb - ns) * dy
            r2 = u * u + v * v
            num = u if component == "x" else v
            out += (wa * wb) * num / (r2 * np.sqrt(r2))
    return out * dx * dy


# distance bands (Chebyshev distance max(|m|, |n|) in cells) -> Gauss-Legendre order
NEAR_FIELD = 4  # index distance max(|m|, |n|) below which route I is used
# (upper limit of the effective distance, Gauss-Legendre nodes per piece); measured
# against route I to reach FP64 round-off, including cells with dy/dx down to 1/8
FAR_BANDS = ((1, 32), (2, 24), (4, 16), (8, 10), (16, 7), (64, 5), (None, 4))


def near_field_size(k: int) -> int:
    """Index distance below which route I is used.  Orders above 3 have wider supports,
    so their nearest polynomial piece sits (k - 3)/2 cells closer to the origin."""
    return NEAR_FIELD + max(0, k - 3)


def band_distance(k: int, m, n, dx: float, dy: float):
    """Distance that selects the Gauss-Legendre band: the effective distance less the
    (k - 3)/2 cells by which the support of orders above 3 reaches closer to the origin
    (orders 4, 5 measured against route I like orders 1-3)."""
    return effective_distance(m, n, dx, dy) - max(0, k - 3) / 2.0


def effective_distance(m, n, dx: float, dy: float):
    """Distance of offset (m, n) in units of the longer cell side.  Gauss-Legendre
    convergence on a piece depends on its distance from the origin over its width, so
    the band of an offset is chosen by this, not by the index distance."""
    return np.maximum(np.abs(m) * dx, np.abs(n) * dy) / max(dx, dy)


@functools.lru_cache(maxsize=None)
def _near_entry(k: int, m: int, n: int, ratio: float, component: str) -> float:
    if (component == "x" and m == 0) or (component == "y" and n == 0):
        return 0.0  # odd in the force direction
    if component == "y":
        # w^y(m, n; 1, ratio) = w^x(n, m; ratio, 1) = w^x(n, m; 1, 1/ratio) (scale
        # invariance), so square cells share one set of entries
        return _near_entry(k, n, m, 1.0 / ratio, "x")
    return float(w_route_i(k, m, n, 1.0, ratio, "x", dps=20))


def kernel_table_quarter(k: int, nx: int, ny: int, dx: float, dy: float, component: str = "x",
                         chunk: int = 256) -> np.ndarray:
    """w at offsets 0 <= m < nx, 0 <= n < ny (the other quadrants follow by symmetry:
    w^x is odd in m and even in n, w^y even in m and odd in n)."""
    out = np.zeros((nx, ny))
    # near field by route I; w depends on the cells only through dy/dx (scale invariance
    # of u r^-3 du dv), so those entries are cached per (k, m, n, dy/dx)
    nf = near_field_size(k)
    for m in range(min(nx, nf)):
        for n in range(min(ny, nf)):
            out[m, n] = _near_entry(k, m, n, dy / dx, component)
    mm_all = np.arange(nx)
    nn_all = np.arange(ny)
    for m0 in range(0, nx, chunk):
        mm = mm_all[m0:m0 + chunk, None]
        nn = nn_all[None, :]
        d = band_distance(k, mm, nn, dx, dy)
        near = np.maximum(mm, nn) < nf
        block = np.zeros(d.shape)
        lower = 0.0
        for limit, q in FAR_BANDS:
            upper = np.inf if limit is None else limit
            sel = (d >= lower) & (d < upper) & ~near
            if sel.any():
                mi, ni = np.nonzero(sel)
                block[mi, ni] = w_far_gl(k, mm[mi, 0], nn[0, ni], dx, dy, q, component)
            if limit is None:
                break
            lower = limit
        block[near] = out[m0:m0 + chunk][near]
        out[m0:m0 + chunk] = block
    # odd in the force direction: the m = 0 row of w^x (n = 0 column of w^y) is 0
    if component == "x":
        out[0, :] = 0.0
    else:
        out[:, 0] = 0.0
    return out


def kernel_tables(k: int, nx: int, ny: int, dx: float, dy: float):
    """Full tables wx, wy of shape (2nx-1, 2ny-1), index [m + nx - 1, n + ny - 1]."""
    qx = kernel_table_quarter(k, nx, ny, dx, dy, "x")
    if nx == ny and dx == dy:
        qy = qx.T.copy()  # w^y(m, n) = w^x(n, m) for square cells
    else:
        qy = kernel_table_quarter(k, nx, ny, dx, dy, "y")
    return _unfold(qx, odd_axis=0), _unfold(qy, odd_axis=1)


def _unfold(q: np.ndarray, odd_axis: int) -> np.ndarray:
    nx, ny = q.shape
    full = np.zeros((2 * nx - 1, 2 * ny - 1))
    sm = -1.0 if odd_axis == 0 else 1.0
    sn = -1.0 if odd_axis == 1 else 1.0
    full[nx - 1:, ny - 1:] = q
    full[:nx - 1, ny - 1:] = sm * q[:0:-1, :]
    full[nx - 1:, :ny - 1] = sn * q[:, :0:-1]
    full[:nx - 1, :ny - 1] = sm * sn * q[:0:-1, :0:-1]
    # w^x(0, n) = 0 and w^y(m, 0) = 0 exactly (oddness)
    if odd_axis == 0:
        full[nx - 1, :] = 0.0
    else:
        full[:, ny - 1] = 0.0
    return full


# ----------------------------------------------------------------------------------
# Potential kernel (a diagnostic beside the forces; the paper itself never forms the
# potential, Sec. 1): Phi_ij = -G sum C_{i'j'} w^phi(i - i', j - j') with
#     w^phi(m, n) = int int b_k(u/dx + m) b_k(v/dy + n) (u^2 + v^2)^(-1/2) du dv,
# even in m and n, absolutely convergent (1/r is integrable in 2-D), and proportional to
# the cell size (w^phi(m, n; s dx, s dy) = s w^phi(m, n; dx, dy)).
# ----------------------------------------------------------------------------------


def _inner_phi(k: int, m: int, h: float, v):
    """int b_k(u/h + m) / sqrt(u^2 + v^2) du, v != 0: closed form on each piece."""
    total = mp.mpf(0)
    for lo, hi, cs in pieces_exact(k):
        q = _compose(cs, m, h)  # b(u/h + m) as a polynomial in u
        ul, uh = (_mpf(lo) - m) * mp.mpf(h), (_mpf(hi) - m) * mp.mpf(h)
        for j, c in enumerate(q):
            if c != 0:
                total += c * (_J(j, uh, v) - _J(j, ul, v))
    return total


def w_phi_route(k: int, m, n: int, dx: float, dy: float, dps: int = 30, k_v: int | None = None):
    """w^phi at one offset: the u-integral in closed form, then an mpmath quadrature in v
    split at v = 0 (a logarithmic endpoint singularity) and at the knots.  With k_v the
    spline along v has that order instead (the mixed integrals of the force-potential
    identity, where m may also be a half-integer)."""
    kv = k if k_v is None else k_v
    with mp.workdps(dps):
        total = mp.mpf(0)
        for lo, hi, cs in pieces_exact(kv):
            vl, vh = (_mpf(lo) - n) * mp.mpf(dy), (_mpf(hi) - n) * mp.mpf(dy)
            pts = [vl, vh]
            if vl < 0 < vh:
                pts = [vl, mp.mpf(0), vh]
            pv = _MPoly(_compose(cs, n, dy))

            def f(v, pv=pv):
                return _poly_mp(pv, v) * _inner_phi(k, m, dx, v)

            total += mp.quad(f, pts)
        return total


def w_phi_k1_closed(m: int, n: int, dx: float, dy: float):
    """Order 1 in closed form: the potential integral of a uniform rectangle, with the
    textbook antiderivative of 1/r, u ln(v + r) + v ln(u + r), written as
    A(u, v) = u asinh(v/|u|) + v asinh(u/|v|) (the two differ by functions of u alone and
    of v alone, which cancel at the four corners; A's terms vanish on the axes)."""
    with mp.workdps(40):
        def A(u, v):
            u, v = mp.mpf(u), mp.mpf(v)
            a = u * mp.asinh(v / abs(u)) if u != 0 else mp.mpf(0)
            b = v * mp.asinh(u / abs(v)) if v != 0 else mp.mpf(0)
            return a + b
        ul, uh = (-0.5 - m) * dx, (0.5 - m) * dx
        vl, vh = (-0.5 - n) * dy, (0.5 - n) * dy
        return A(uh, vh) - A(ul, vh) - A(uh, vl) + A(ul, vl)


def w_phi_far_gl(k: int, ms: np.ndarray, ns: np.ndarray, dx: float, dy: float, q: int) -> np.ndarray:
    """sum_a sum_b W_a W_b / r((t_a - m) dx, (t_b - n) dy) dx dy for arrays of offsets."""
    ms = np.asarray(ms, dtype=np.float64)
    ns = np.asarray(ns, dtype=np.float64)
    t, wt = _gl_nodes(k, q)
    out = np.zeros(np.broadcast(ms, ns).shape)
    for ta, wa in zip(t, wt):
        u = (ta - ms) * dx
        for tb, wb in zip(t, wt):
            v = (tb - ns) * dy
            out += (wa * wb) / np.sqrt(u * u + v * v)
    return out * dx * dy


@functools.lru_cache(maxsize=None)
def _near_phi(k: int, m: int, n: int, ratio: float) -> float:
    # unit dx; scaled by dx by the caller.  Square cells: symmetric in (m, n)
    if ratio == 1.0 and n < m:
        return _near_phi(k, n, m, ratio)
    return float(w_phi_route(k, m, n, 1.0, ratio, dps=20))


def potential_table_quarter(k: int, nx: int, ny: int, dx: float, dy: float, chunk: int = 256) -> np.ndarray:
    """w^phi at offsets 0 <= m < nx, 0 <= n < ny (even in both), assembled like the force
    tables: near field by the closed-form inner integral and quadrature, far field by the
    Gauss-Legendre bands."""
    out = np.zeros((nx, ny))
    nf = near_field_size(k)
    for m in range(min(nx, nf)):
        for n in range(min(ny, nf)):
            out[m, n] = dx * _near_phi(k, m, n, dy / dx)
    for m0 in range(0, nx, chunk):
        mm = np.arange(m0, min(nx, m0 + chunk))[:, None]
        nn = np.arange(ny)[None, :]
        d = band_distance(k, mm, nn, dx, dy)
        near = np.maximum(mm, nn) < nf
        block = np.zeros(d.shape)
        lower = 0.0
        for limit, q in FAR_BANDS:
            upper = np.inf if limit is None else limit
            sel = (d >= lower) & (d < upper) & ~near
            if sel.any():
                mi, ni = np.nonzero(sel)
                block[mi, ni] = w_phi_far_gl(k, mm[mi, 0], nn[0, ni], dx, dy, q)
            if limit is None:
                break
            lower = limit
        block[near] = out[m0:m0 + chunk][near]
        out[m0:m0 + chunk] = block
    return out


def potential_table(k: int, nx: int, ny: int, dx: float, dy: float) -> np.ndarray:
    """Full table of shape (2nx-1, 2ny-1), index [m + nx - 1, n + ny - 1]."""
    q = potential_table_quarter(k, nx, ny, dx, dy)
    full = np.zeros((2 * nx - 1, 2 * ny - 1))
    full[nx - 1:, ny - 1:] = q
    full[:nx - 1, ny - 1:] = q[:0:-1, :]
    full[nx - 1:, :ny - 1] = q[:, :0:-1]
    full[:nx - 1, :ny - 1] = q[:0:-1, :0:-1]
    return full
