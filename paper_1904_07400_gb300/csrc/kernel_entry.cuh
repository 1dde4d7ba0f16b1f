// One entry of the force-kernel tables, in FP64, callable on host and device.
//
//   w^x(m, n) = PV int int u (u^2+v^2)^(-3/2) b_k(u/dx + m) b_k(v/dy + n) du dv
//
// (Eq. eqnwB after the change of variables of Eq. wk1; m = i - i', n = j - j').
// w^y(m, n; dx, dy) = w^x(n, m; dy, dx), so only the x form is coded.
//
// The closed forms of Eqs. (intF)-(intMoment) cancel catastrophically at large offsets
// (every corner term is O(d^(alpha+beta-1)) while w is O(d^-2)), so two FP64-stable
// evaluations are used instead:
//
//  * far field: tensor Gauss-Legendre on each of the k x k polynomial rectangles of the
//    integrand, which is analytic there; the node count follows from a Bernstein-ellipse
//    bound on each rectangle (entry_rho below), chosen to reach 1e-18.
//  * near field (offsets where no order up to 32 meets that bound, i.e. rectangles that
//    touch the singular point): integrate by parts in u (u r^-3 = -d/du r^-1), which
//    makes the integral absolutely convergent:
//       w = int dv b_k(v/dy + n) g(v),  g(v) = int dt b_k'(t) / sqrt(((t - m) dx)^2 + v^2)
//    The u-integral is closed form (asinh, r).  g has at most a logarithmic singularity
//    at v = 0, g = A(v) + L ln|v| with A analytic on each side of 0; the ln|v| part is
//    integrated in closed form against the polynomial b_k piece, the rest by composite
//    Gauss-Legendre on sub-intervals no wider than dx/2.
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define TDG_HD __host__ __device__ __forceinline__
#else
#define TDG_HD inline
#endif

namespace tdg {

// Polynomial pieces of the centred cardinal B-spline b_k, unit knot spacing, support
// [-k/2, k/2]; piece p covers [lo + p, lo + p + 1) and is sum_i c[p][i] t^i.
struct SplinePieces {
    int k;
    double lo;
    double c[3][3];
};

TDG_HD SplinePieces spline_pieces(int k) {
    SplinePieces s;
    for (int p = 0; p < 3; ++p)
        for (int i = 0; i < 3; ++i) s.c[p][i] = 0.0;
    s.k = k;
    if (k == 1) {
        s.lo = -0.5;
        s.c[0][0] = 1.0;
    } else if (k == 2) {
        s.lo = -1.0;
        s.c[0][0] = 1.0;  s.c[0][1] = 1.0;   // 1 + t on [-1, 0)
        s.c[1][0] = 1.0;  s.c[1][1] = -1.0;  // 1 - t on [0, 1)
    } else {
        s.lo = -1.5;
        s.c[0][0] = 1.125; s.c[0][1] = 1.5;  s.c[0][2] = 0.5;   // (t + 3/2)^2 / 2
        s.c[1][0] = 0.75;  s.c[1][1] = 0.0;  s.c[1][2] = -1.0;  // 3/4 - t^2
        s.c[2][0] = 1.125; s.c[2][1] = -1.5; s.c[2][2] = 0.5;   // (3/2 - t)^2 / 2
    }
    return s;
}

TDG_HD double piece_eval(const SplinePieces& s, int p, double t) {
    return s.c[p][0] + t * (s.c[p][1] + t * s.c[p][2]);
}

// Gauss-Legendre rule on [-1, 1]: nodes x[i], weights w[i], i < q.
struct GLRule {
    const double* x;
    const double* w;
    int q;
};

TDG_HD double kernel_f(double u, double v) {
    double r2 = u * u + v * v;
    double inv = 1.0 / sqrt(r2);
    return u * inv * inv * inv;
}

// Far field: sum over the k x k rectangles of the tensor Gauss-Legendre rule.
TDG_HD double entry_far(int k, int m, int n, double dx, double dy, const GLRule& g) {
    SplinePieces s = spline_pieces(k);
    double acc = 0.0;
    for (int pu = 0; pu < k; ++pu) {
        double cu = s.lo + pu + 0.5;
        for (int a = 0; a < g.q; ++a) {
            double tu = cu + 0.5 * g.x[a];
            double wu = 0.5 * g.w[a] * piece_eval(s, pu, tu);
            double u = (tu - m) * dx;
            double inner = 0.0;
            for (int pv = 0; pv < k; ++pv) {
                double cv = s.lo + pv + 0.5;
                for (int b = 0; b < g.q; ++b) {
                    double tv = cv + 0.5 * g.x[b];
                    double wv = 0.5 * g.w[b] * piece_eval(s, pv, tv);
                    inner += wv * kernel_f(u, (tv - n) * dy);
                }
            }
            acc += wu * inner;
        }
    }
    return acc * dx * dy;
}

TDG_HD double sgn(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }

// Bernstein-ellipse parameter guaranteeing analyticity of u r^-3 on every polynomial
// rectangle of offset (m, n).  The integrand is singular only where u = +-i v.  For a
// rectangle with centre (cu, cv) and half-widths (hu, hv), the product of the ellipses
// E_rho (foci at the rectangle's edges) stays clear of that set if the smallest |Re u| on
// E_rho(u) exceeds the largest |Im v| on E_rho(v), or the same with u and v exchanged; the
// largest such rho solves a quadratic.  Tensor Gauss-Legendre with q nodes then converges
// like rho^(-2q).  Returns the smallest rho over the k x k rectangles (1 = no bound).
TDG_HD double entry_rho(int k, int m, int n, double dx, double dy) {
    SplinePieces s = spline_pieces(k);
    const double hu = 0.5 * dx, hv = 0.5 * dy;
    double rmin = 1e300;
    for (int pu = 0; pu < k; ++pu) {
        double cu = fabs((s.lo + pu + 0.5 - m) * dx);
        double r1 = cu > hu ? (cu + sqrt(cu * cu - hu * hu + hv * hv)) / (hu + hv) : 1.0;
        for (int pv = 0; pv < k; ++pv) {
            double cv = fabs((s.lo + pv + 0.5 - n) * dy);
            double r2 = cv > hv ? (cv + sqrt(cv * cv - hv * hv + hu * hu)) / (hu + hv) : 1.0;
            double r = r1 > r2 ? r1 : r2;
            if (r < rmin) rmin = r;
        }
    }
    return rmin;
}

// Gauss-Legendre orders available to the far field; the near field uses rule 4 (16 nodes)
constexpr int kNumOrders = 7;
constexpr int kNearRule = 4;
TDG_HD int rule_order(int i) {
    const int q[kNumOrders] = {4, 5, 7, 10, 16, 24, 32};
    return q[i];
}

// smallest order with rho^(-2q) <= 1e-18, or 0 if even 32 nodes do not reach it
TDG_HD int choose_order(double rho) {
    if (rho <= 1.0) return 0;
    double need = 18.0 * 2.302585092994046 / (2.0 * log(rho));
    for (int i = 0; i < kNumOrders; ++i)
        if (rule_order(i) >= need) return rule_order(i);
    return 0;
}

// g(v) = int u r^-3 b_k(u/dx + m) du for v != 0, by parts (u r^-3 = -d/du r^-1):
// g = int dt b_k'(t) / sqrt(((t - m) dx)^2 + v^2) = A(v) + L ln|v|, A analytic on either
// side of v = 0.  Returns A and sets L.
TDG_HD double near_inner(int k, int m, double dx, double v, double* L) {
    if (k == 1) {
        // b_1' = delta(t + 1/2) - delta(t - 1/2): two point evaluations, no log part
        double a0 = (-0.5 - m) * dx, a1 = (0.5 - m) * dx;
        *L = 0.0;
        return 1.0 / sqrt(a0 * a0 + v * v) - 1.0 / sqrt(a1 * a1 + v * v);
    }
    SplinePieces s = spline_pieces(k);
    double A = 0.0, Lsum = 0.0;
    for (int p = 0; p < k; ++p) {
        // derivative piece b'(t) = d0 + d1 t; as a polynomial in u: c0 + c1 u
        double d0 = s.c[p][1], d1 = 2.0 * s.c[p][2];
        double c0 = d0 + d1 * m, c1 = d1 / dx;
        double ul = (s.lo + p - m) * dx, uh = (s.lo + p + 1 - m) * dx;
        double rl = sqrt(ul * ul + v * v), rh = sqrt(uh * uh + v * v);
        // int du / r = asinh(u/|v|) = sgn(u) [ln(|u| + r) - ln|v|]  (u != 0); 0 at u = 0
        double jl = (ul != 0.0) ? sgn(ul) * log(fabs(ul) + rl) : 0.0;
        double jh = (uh != 0.0) ? sgn(uh) * log(fabs(uh) + rh) : 0.0;
        A += c0 * (jh - jl) + c1 * (rh - rl);
        Lsum -= c0 * (sgn(uh) - sgn(ul));
    }
    *L = Lsum / dx;
    return A / dx;
}

// g(v) directly, Gauss-Legendre in u on each piece (for |v| >= 2 dx, where the
// integrand is smooth in u and the by-parts form would cancel)
TDG_HD double direct_inner(int k, int m, double dx, double v, const GLRule& g) {
    SplinePieces s = spline_pieces(k);
    double acc = 0.0;
    for (int p = 0; p < k; ++p) {
        double c = s.lo + p + 0.5;
        for (int a = 0; a < g.q; ++a) {
            double t = c + 0.5 * g.x[a];
            acc += 0.5 * g.w[a] * piece_eval(s, p, t) * kernel_f((t - m) * dx, v);
        }
    }
    return acc * dx;
}

// int_a^b v^i ln|v| dv for a, b on the same side of 0 (either may be 0)
TDG_HD double int_vlog(int i, double a, double b) {
    double e = i + 1.0;
    double pa = a, pb = b;
    for (int j = 0; j < i; ++j) {
        pa *= a;
        pb *= b;
    }
    double fb = (b != 0.0) ? pb / e * (log(fabs(b)) - 1.0 / e) : 0.0;
    double fa = (a != 0.0) ? pa / e * (log(fabs(a)) - 1.0 / e) : 0.0;
    return fb - fa;
}

// Near field: w = int dv b_k(v/dy + n) g(v) over the k pieces in v, each split at v = 0
// and cut into sub-intervals no wider than dx/2.  On the sub-interval touching v = 0
// the ln|v| part of g is integrated in closed form and A by Gauss-Legendre; elsewhere g
// is smooth and integrated by Gauss-Legendre (by-parts form for |v| < 2 dx, direct form
// beyond).
TDG_HD double entry_near(int k, int m, int n, double dx, double dy, const GLRule& g) {
    SplinePieces s = spline_pieces(k);
    double total = 0.0;
    for (int pv = 0; pv < k; ++pv) {
        double tl = s.lo + pv, th = tl + 1.0;
        double vl = (tl - n) * dy, vh = (th - n) * dy;
        // the piece as a polynomial in v: b(v/dy + n) = e0 + e1 v + e2 v^2
        double p0 = s.c[pv][0], p1 = s.c[pv][1], p2 = s.c[pv][2];
        double e0 = p0 + p1 * n + p2 * n * n;
        double e1 = (p1 + 2.0 * p2 * n) / dy;
        double e2 = p2 / (dy * dy);
        double cuts[3] = {vl, vh, vh};
        int ncut = 2;
        if (vl < 0.0 && vh > 0.0) {
            cuts[1] = 0.0;
            ncut = 3;
        }
        for (int h = 0; h + 1 < ncut; ++h) {
            double a = cuts[h], b = cuts[h + 1];
            int nsub = (int)ceil(2.0 * (b - a) / dx);
            if (nsub < 1) nsub = 1;
            double width = (b - a) / nsub;
            for (int si = 0; si < nsub; ++si) {
                double sa = a + si * width, sb = (si == nsub - 1) ? b : sa + width;
                bool at_zero = (sa == 0.0) || (sb == 0.0);
                double vmax = fmax(fabs(sa), fabs(sb));
                double c = 0.5 * (sa + sb), hw = 0.5 * (sb - sa);
                double acc = 0.0, L = 0.0;
                for (int q = 0; q < g.q; ++q) {
                    double v = c + hw * g.x[q];
                    double poly = e0 + v * (e1 + v * e2);
                    double gv;
                    if (at_zero) {
                        gv = near_inner(k, m, dx, v, &L);             // A(v) only
                    } else if (vmax < 2.0 * dx) {
                        gv = near_inner(k, m, dx, v, &L);
                        gv += L * log(fabs(v));                      // full g(v)
                    } else {
                        gv = direct_inner(k, m, dx, v, g);
                    }
                    acc += g.w[q] * poly * gv;
                }
                total += hw * acc;
                if (at_zero) {
                    near_inner(k, m, dx, c, &L);  // L does not depend on v
                    if (L != 0.0)
                        total += L * (e0 * int_vlog(0, sa, sb) + e1 * int_vlog(1, sa, sb) + e2 * int_vlog(2, sa, sb));
                }
            }
        }
    }
    return total;
}

// One table entry w^x(m, n), m, n >= 0, on host or device; rules[i] is the order
// rule_order(i) Gauss-Legendre rule.
TDG_HD double entry_x(int k, int m, int n, double dx, double dy, const GLRule* rules) {
    if (m == 0) return 0.0;  // odd in m
    int q = choose_order(entry_rho(k, m, n, dx, dy));
    if (q == 0) return entry_near(k, m, n, dx, dy, rules[kNearRule]);
    int i = 0;
    while (rule_order(i) != q) ++i;
    return entry_far(k, m, n, dx, dy, rules[i]);
}

}  // namespace tdg
