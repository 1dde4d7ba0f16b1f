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

// Polynomial pieces of the centred cardinal B-spline b_k (k <= 5), unit knot spacing,
// support [-k/2, k/2].  Piece p covers t in [lo + p, lo + p + 1) and is held in the local
// variable s = t - (lo + p) in [0, 1): sum_i c[p][i] s^i (the uniform B-spline basis,
// whose coefficients are those of (k-1)! b_k; well conditioned for every order).
struct SplinePieces {
    int k;
    double lo;
    double c[5][5];
};

TDG_HD SplinePieces spline_pieces(int k) {
    SplinePieces sp;
    for (int p = 0; p < 5; ++p)
        for (int i = 0; i < 5; ++i) sp.c[p][i] = 0.0;
    sp.k = k;
    sp.lo = -0.5 * k;
    // (k-1)! times the pieces, by power of s (zero entries omitted)
    if (k == 1) {
        sp.c[0][0] = 1.0;
    } else if (k == 2) {
        sp.c[0][1] = 1.0; sp.c[1][0] = 1.0; sp.c[1][1] = -1.0;
    } else if (k == 3) {
        sp.c[0][2] = 1.0; sp.c[1][0] = 1.0; sp.c[1][1] = 2.0; sp.c[1][2] = -2.0; sp.c[2][0] = 1.0;
        sp.c[2][1] = -2.0; sp.c[2][2] = 1.0;
    } else if (k == 4) {
        sp.c[0][3] = 1.0; sp.c[1][0] = 1.0; sp.c[1][1] = 3.0; sp.c[1][2] = 3.0; sp.c[1][3] = -3.0;
        sp.c[2][0] = 4.0; sp.c[2][2] = -6.0; sp.c[2][3] = 3.0; sp.c[3][0] = 1.0; sp.c[3][1] = -3.0;
        sp.c[3][2] = 3.0; sp.c[3][3] = -1.0;
    } else if (k == 5) {
        sp.c[0][4] = 1.0; sp.c[1][0] = 1.0; sp.c[1][1] = 4.0; sp.c[1][2] = 6.0; sp.c[1][3] = 4.0;
        sp.c[1][4] = -4.0; sp.c[2][0] = 11.0; sp.c[2][1] = 12.0; sp.c[2][2] = -6.0; sp.c[2][3] = -12.0;
        sp.c[2][4] = 6.0; sp.c[3][0] = 11.0; sp.c[3][1] = -12.0; sp.c[3][2] = -6.0; sp.c[3][3] = 12.0;
        sp.c[3][4] = -4.0; sp.c[4][0] = 1.0; sp.c[4][1] = -4.0; sp.c[4][2] = 6.0; sp.c[4][3] = -4.0;
        sp.c[4][4] = 1.0;
    }
    double f = 1.0;
    for (int q = 2; q < k; ++q) f *= q;
    for (int p = 0; p < k; ++p)
        for (int i = 0; i < k; ++i) sp.c[p][i] /= f;
    return sp;
}

// piece p at local coordinate s
TDG_HD double piece_eval(const SplinePieces& sp, int p, double s) {
    double acc = 0.0;
    for (int i = sp.k - 1; i >= 0; --i) acc = acc * s + sp.c[p][i];
    return acc;
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
    SplinePieces sp = spline_pieces(k);
    double acc = 0.0;
    for (int pu = 0; pu < k; ++pu) {
        double cu = sp.lo + pu + 0.5;
        for (int a = 0; a < g.q; ++a) {
            double su = 0.5 + 0.5 * g.x[a];
            double wu = 0.5 * g.w[a] * piece_eval(sp, pu, su);
            double u = (cu + 0.5 * g.x[a] - m) * dx;
            double inner = 0.0;
            for (int pv = 0; pv < k; ++pv) {
                double cv = sp.lo + pv + 0.5;
                for (int b = 0; b < g.q; ++b) {
                    double sv = 0.5 + 0.5 * g.x[b];
                    double wv = 0.5 * g.w[b] * piece_eval(sp, pv, sv);
                    inner += wv * kernel_f(u, (cv + 0.5 * g.x[b] - n) * dy);
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
    const double lo = -0.5 * k;
    const double hu = 0.5 * dx, hv = 0.5 * dy;
    double rmin = 1e300;
    for (int pu = 0; pu < k; ++pu) {
        double cu = fabs((lo + pu + 0.5 - m) * dx);
        double r1 = cu > hu ? (cu + sqrt(cu * cu - hu * hu + hv * hv)) / (hu + hv) : 1.0;
        for (int pv = 0; pv < k; ++pv) {
            double cv = fabs((lo + pv + 0.5 - n) * dy);
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

// the piece's polynomial in u (by power of u) from its local form, s = (u - ul) / h;
// used only for pieces with |ul| <= k h / 2 + 1 (near the origin), where expanding the
// powers of (u - ul) loses little
TDG_HD void piece_in_u(const SplinePieces& sp, int p, double ul, double h, double* e) {
    for (int i = 0; i < 5; ++i) e[i] = 0.0;
    // Horner on polynomials: acc = acc * (u - ul)/h + c_i
    for (int i = sp.k - 1; i >= 0; --i) {
        for (int q = 4; q >= 1; --q) e[q] = (e[q - 1] - ul * e[q]) / h;
        e[0] = -ul * e[0] / h + sp.c[p][i];
    }
}

// g(v) = int u r^-3 b_k(u/dx + m) du for v != 0, by parts (u r^-3 = -d/du r^-1):
// g = int dt b_k'(t) / sqrt(((t - m) dx)^2 + v^2) = A(v) + (L0 + L2 v^2) ln|v|, A analytic
// on either side of v = 0.  Pieces whose u-range contains 0 are integrated in closed form
// (int u^j / r du for j <= 3: asinh, r, (u r - v^2 asinh)/2, r (u^2 - 2 v^2)/3, whose
// asinh terms carry the ln|v|); the others are smooth in u and taken by the rule g.
// Returns A and sets L0, L2.
TDG_HD double near_inner(int k, int m, double dx, double v, double* L0, double* L2, const GLRule& g) {
    *L0 = 0.0;
    *L2 = 0.0;
    if (k == 1) {
        // b_1' = delta(t + 1/2) - delta(t - 1/2): two point evaluations, no log part
        double a0 = (-0.5 - m) * dx, a1 = (0.5 - m) * dx;
        return 1.0 / sqrt(a0 * a0 + v * v) - 1.0 / sqrt(a1 * a1 + v * v);
    }
    SplinePieces sp = spline_pieces(k);
    const double v2 = v * v;
    double A = 0.0;
    for (int p = 0; p < k; ++p) {
        const double ul = (sp.lo + p - m) * dx, uh = ul + dx;
        if (ul <= 0.0 && uh >= 0.0) {
            // b as a polynomial in u, then b'(t) = dx sum_j q_j u^j; with dt = du / dx the
            // piece contributes sum_j q_j int u^j / r du
            double e[5];
            piece_in_u(sp, p, ul, dx, e);
            double q[4];
            for (int j = 0; j < 4; ++j) q[j] = (j + 1) * e[j + 1];
            double J[2][4];
            const double us[2] = {ul, uh};
            for (int z = 0; z < 2; ++z) {
                const double u = us[z];
                const double r = sqrt(u * u + v2);
                const double j0 = (u != 0.0) ? sgn(u) * log(fabs(u) + r) : 0.0;  // asinh minus its log part
                J[z][0] = j0;
                J[z][1] = r;
                J[z][2] = 0.5 * (u * r - v2 * j0);
                J[z][3] = r * (u * u - 2.0 * v2) / 3.0;
            }
            for (int j = 0; j < 4; ++j) A += q[j] * (J[1][j] - J[0][j]);
            const double ds = sgn(uh) - sgn(ul);
            *L0 -= q[0] * ds;
            *L2 += 0.5 * q[2] * ds;
        } else {
            // smooth: int b'(t) / r dt over the piece by Gauss-Legendre in s = t - (lo + p)
            double acc = 0.0;
            for (int a = 0; a < g.q; ++a) {
                const double s = 0.5 + 0.5 * g.x[a];
                double d = 0.0;
                for (int i = sp.k - 1; i >= 1; --i) d = d * s + i * sp.c[p][i];
                const double u = ul + s * dx;
                acc += 0.5 * g.w[a] * d / sqrt(u * u + v2);
            }
            A += acc;
        }
    }
    return A;
}

// g(v) directly, Gauss-Legendre in u on each piece (for |v| >= 2 dx, where the
// integrand is smooth in u and the by-parts form would cancel)
TDG_HD double direct_inner(int k, int m, double dx, double v, const GLRule& g) {
    SplinePieces sp = spline_pieces(k);
    double acc = 0.0;
    for (int p = 0; p < k; ++p) {
        double c = sp.lo + p + 0.5;
        for (int a = 0; a < g.q; ++a) {
            double t = c + 0.5 * g.x[a];
            acc += 0.5 * g.w[a] * piece_eval(sp, p, 0.5 + 0.5 * g.x[a]) * kernel_f((t - m) * dx, v);
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
    SplinePieces sp = spline_pieces(k);
    double total = 0.0;
    for (int pv = 0; pv < k; ++pv) {
        double vl = (sp.lo + pv - n) * dy, vh = vl + dy;
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
                double acc = 0.0, L0 = 0.0, L2 = 0.0;
                for (int q = 0; q < g.q; ++q) {
                    double v = c + hw * g.x[q];
                    double poly = piece_eval(sp, pv, (v - vl) / dy);
                    double gv;
                    if (at_zero) {
                        gv = near_inner(k, m, dx, v, &L0, &L2, g);   // A(v) only
                    } else if (vmax < 2.0 * dx) {
                        gv = near_inner(k, m, dx, v, &L0, &L2, g);
                        gv += (L0 + L2 * v * v) * log(fabs(v));     // full g(v)
                    } else {
                        gv = direct_inner(k, m, dx, v, g);
                    }
                    acc += g.w[q] * poly * gv;
                }
                total += hw * acc;
                if (at_zero) {
                    near_inner(k, m, dx, c, &L0, &L2, g);  // L0, L2 do not depend on v
                    if (L0 != 0.0 || L2 != 0.0) {
                        // the piece as a polynomial in v (it contains v = 0, so |vl| <= k dy / 2)
                        double e[5];
                        piece_in_u(sp, pv, vl, dy, e);
                        double lp = 0.0;
                        for (int i = 0; i < sp.k; ++i)
                            lp += e[i] * (L0 * int_vlog(i, sa, sb) + L2 * int_vlog(i + 2, sa, sb));
                        total += lp;
                    }
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

// ---------------------------------------------------------------------------------------
// Potential kernel (a diagnostic beside the forces; Sec. 1 notes that the method never
// forms the potential): w^phi(m, n) = int int b_k(u/dx + m) b_k(v/dy + n) / r du dv, even in
// m and n and absolutely convergent.  Same structure as the force entries:
//  * far field: tensor Gauss-Legendre with 1/r (same rectangles and node counts);
//  * near field: w = int dv b_k(v/dy + n) h(v), h(v) = int b_k(u/dx + m) / r du =
//    A(v) + (L0 + L2 v^2 + L4 v^4) ln|v|; the piece whose u-range contains 0 in closed form
//    (int u^j / r du, j <= 4: asinh, r, (u r - v^2 asinh)/2, r (u^2 - 2 v^2)/3,
//    u^3 r / 4 - (3/4) v^2 J_2), the others by Gauss-Legendre.
// ---------------------------------------------------------------------------------------
TDG_HD double phi_far(int k, int m, int n, double dx, double dy, const GLRule& g) {
    SplinePieces sp = spline_pieces(k);
    double acc = 0.0;
    for (int pu = 0; pu < k; ++pu) {
        double cu = sp.lo + pu + 0.5;
        for (int a = 0; a < g.q; ++a) {
            double wu = 0.5 * g.w[a] * piece_eval(sp, pu, 0.5 + 0.5 * g.x[a]);
            double u = (cu + 0.5 * g.x[a] - m) * dx;
            double inner = 0.0;
            for (int pv = 0; pv < k; ++pv) {
                double cv = sp.lo + pv + 0.5;
                for (int b = 0; b < g.q; ++b) {
                    double wv = 0.5 * g.w[b] * piece_eval(sp, pv, 0.5 + 0.5 * g.x[b]);
                    double v = (cv + 0.5 * g.x[b] - n) * dy;
                    inner += wv / sqrt(u * u + v * v);
                }
            }
            acc += wu * inner;
        }
    }
    return acc * dx * dy;
}

// h(v) for |v| < 2 dx: returns A(v), sets L0, L2, L4
TDG_HD double phi_inner_near(int k, int m, double dx, double v, double* L0, double* L2, double* L4, const GLRule& g) {
    SplinePieces sp = spline_pieces(k);
    const double v2 = v * v;
    double A = 0.0;
    *L0 = *L2 = *L4 = 0.0;
    for (int p = 0; p < k; ++p) {
        const double ul = (sp.lo + p - m) * dx, uh = ul + dx;
        if (ul <= 0.0 && uh >= 0.0) {
            double e[5];
            piece_in_u(sp, p, ul, dx, e);  // b(u/dx + m) = sum_j e_j u^j on the piece
            double J[2][5];
            const double us[2] = {ul, uh};
            for (int z = 0; z < 2; ++z) {
                const double u = us[z];
                const double r = sqrt(u * u + v2);
                const double j0 = (u != 0.0) ? sgn(u) * log(fabs(u) + r) : 0.0;
                J[z][0] = j0;
                J[z][1] = r;
                J[z][2] = 0.5 * (u * r - v2 * j0);
                J[z][3] = r * (u * u - 2.0 * v2) / 3.0;
                J[z][4] = 0.25 * u * u * u * r - 0.75 * v2 * J[z][2];
            }
            for (int j = 0; j < 5; ++j) A += e[j] * (J[1][j] - J[0][j]);
            const double ds = sgn(uh) - sgn(ul);
            *L0 -= e[0] * ds;
            *L2 += 0.5 * e[2] * ds;
            *L4 -= 0.375 * e[4] * ds;
        } else {
            double acc = 0.0;
            for (int a = 0; a < g.q; ++a) {
                const double s = 0.5 + 0.5 * g.x[a];
                const double u = ul + s * dx;
                acc += 0.5 * g.w[a] * piece_eval(sp, p, s) / sqrt(u * u + v2);
            }
            A += acc * dx;
        }
    }
    return A;
}

TDG_HD double phi_inner_direct(int k, int m, double dx, double v, const GLRule& g) {
    SplinePieces sp = spline_pieces(k);
    double acc = 0.0;
    for (int p = 0; p < k; ++p) {
        for (int a = 0; a < g.q; ++a) {
            const double s = 0.5 + 0.5 * g.x[a];
            const double u = (sp.lo + p + s - m) * dx;
            acc += 0.5 * g.w[a] * piece_eval(sp, p, s) / sqrt(u * u + v * v);
        }
    }
    return acc * dx;
}

TDG_HD double phi_near(int k, int m, int n, double dx, double dy, const GLRule& g) {
    SplinePieces sp = spline_pieces(k);
    double total = 0.0;
    for (int pv = 0; pv < k; ++pv) {
        double vl = (sp.lo + pv - n) * dy, vh = vl + dy;
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
                double acc = 0.0, L0 = 0.0, L2 = 0.0, L4 = 0.0;
                for (int q = 0; q < g.q; ++q) {
                    double v = c + hw * g.x[q];
                    double poly = piece_eval(sp, pv, (v - vl) / dy);
                    double hv;
                    if (at_zero) {
                        hv = phi_inner_near(k, m, dx, v, &L0, &L2, &L4, g);
                    } else if (vmax < 2.0 * dx) {
                        hv = phi_inner_near(k, m, dx, v, &L0, &L2, &L4, g);
                        const double v2 = v * v;
                        hv += (L0 + v2 * (L2 + v2 * L4)) * log(fabs(v));
                    } else {
                        hv = phi_inner_direct(k, m, dx, v, g);
                    }
                    acc += g.w[q] * poly * hv;
                }
                total += hw * acc;
                if (at_zero) {
                    phi_inner_near(k, m, dx, c, &L0, &L2, &L4, g);  // L0, L2, L4 do not depend on v
                    if (L0 != 0.0 || L2 != 0.0 || L4 != 0.0) {
                        double e[5];
                        piece_in_u(sp, pv, vl, dy, e);
                        double lp = 0.0;
                        for (int i = 0; i < sp.k; ++i)
                            lp += e[i] * (L0 * int_vlog(i, sa, sb) + L2 * int_vlog(i + 2, sa, sb) +
                                          L4 * int_vlog(i + 4, sa, sb));
                        total += lp;
                    }
                }
            }
        }
    }
    return total;
}

// One potential-table entry w^phi(m, n), m, n >= 0
TDG_HD double entry_phi(int k, int m, int n, double dx, double dy, const GLRule* rules) {
    int q = choose_order(entry_rho(k, m, n, dx, dy));
    if (q == 0) return phi_near(k, m, n, dx, dy, rules[kNearRule]);
    int i = 0;
    while (rule_order(i) != q) ++i;
    return phi_far(k, m, n, dx, dy, rules[i]);
}

}  // namespace tdg
