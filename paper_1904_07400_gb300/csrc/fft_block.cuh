// Block-cooperative building blocks operating on lines held in shared memory:
//   * Stockham autosort FFT (radix 2, 3, 4, 8), in place, several interleaved lines;
//   * the real <-> half-length complex packing of real transforms;
//   * the truncated tridiagonal solve of the order-3 B-spline coefficients.
//
// Layout: `nl` lines of length L interleaved, element e of line c at s[e * nl + c], so
// that consecutive threads touch consecutive words.
#pragma once

#include "tdg_internal.cuh"

namespace tdg {

template <typename T> struct Consts;
template <> struct Consts<float> {
    static constexpr float kS3 = 0.866025403784438646763723f;   // sin(pi/3)
    static constexpr float kR2 = 0.707106781186547524400844f;   // 1/sqrt(2)
};
template <> struct Consts<double> {
    static constexpr double kS3 = 0.866025403784438646763723;
    static constexpr double kR2 = 0.707106781186547524400844;
};

__device__ __forceinline__ cpx<float> ldg_c(const cpx<float>* p) {
    float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return mk(v.x, v.y);
}
__device__ __forceinline__ cpx<double> ldg_c(const cpx<double>* p) {
    double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return mk(v.x, v.y);
}

// multiply by -i (forward) or +i (inverse)
template <typename T>
__device__ __forceinline__ cpx<T> rot90(cpx<T> a, bool inv) {
    return inv ? mk(-a.y, a.x) : mk(a.y, -a.x);
}

template <typename T, int R>
__device__ __forceinline__ void butterfly(cpx<T>* v, bool inv) {
    if constexpr (R == 2) {
        cpx<T> a = v[0], b = v[1];
        v[0] = a + b;
        v[1] = a - b;
    } else if constexpr (R == 3) {
        // DFT_3 with w = exp(-+ 2 pi i / 3) = -1/2 -+ i sqrt(3)/2
        cpx<T> a = v[0], b = v[1], c = v[2];
        cpx<T> s = b + c, d = b - c;
        cpx<T> m = a - scl(s, T(0.5));
        cpx<T> r = rot90(scl(d, Consts<T>::kS3), inv);
        v[0] = a + s;
        v[1] = m + r;
        v[2] = m - r;
    } else if constexpr (R == 4) {
        cpx<T> t0 = v[0] + v[2], t1 = v[0] - v[2];
        cpx<T> t2 = v[1] + v[3], t3 = rot90(v[1] - v[3], inv);
        v[0] = t0 + t2;
        v[2] = t0 - t2;
        v[1] = t1 + t3;
        v[3] = t1 - t3;
    } else if constexpr (R == 8) {
        // two radix-4 halves on even/odd inputs, then twiddles exp(-+ 2 pi i q / 8)
        cpx<T> e[4] = {v[0], v[2], v[4], v[6]};
        cpx<T> o[4] = {v[1], v[3], v[5], v[7]};
        butterfly<T, 4>(e, inv);
        butterfly<T, 4>(o, inv);
        const T h = Consts<T>::kR2;
        // o1 *= w^1, o2 *= w^2, o3 *= w^3 with w = exp(-+ i pi / 4)
        cpx<T> o1 = inv ? mk(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
                        : mk(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
        cpx<T> o2 = rot90(o[2], inv);
        cpx<T> o3 = inv ? mk(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
                        : mk(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
        v[0] = e[0] + o[0];
        v[4] = e[0] - o[0];
        v[1] = e[1] + o1;
        v[5] = e[1] - o1;
        v[2] = e[2] + o2;
        v[6] = e[2] - o2;
        v[3] = e[3] + o3;
        v[7] = e[3] - o3;
    }
}

// One Stockham stage of radix R over nl interleaved lines of length L.  Ns = product of
// the radices already applied.  tw is the table exp(-2 pi i t / P) with P = L * tstride.
template <typename T, int R, int EPT>
__device__ __forceinline__ void fft_stage(cpx<T>* s, int L, int nl, int Ns, const cpx<T>* __restrict__ tw,
                                          int tstride, bool inv) {
    constexpr int MB = (EPT + R - 1) / R;
    cpx<T> v[MB][R];
    const int LR = L / R;
    const int nb = nl * LR;
#pragma unroll
    for (int q = 0; q < MB; ++q) {
        int b = threadIdx.x + q * blockDim.x;
        if (b < nb) {
            int c = b % nl, j = b / nl;
#pragma unroll
            for (int r = 0; r < R; ++r) v[q][r] = s[(j + r * LR) * nl + c];
        }
    }
    __syncthreads();
    const int step = (LR / Ns) * tstride;
#pragma unroll
    for (int q = 0; q < MB; ++q) {
        int b = threadIdx.x + q * blockDim.x;
        if (b < nb) {
            int c = b % nl, j = b / nl;
            int k = j % Ns;
            if (k != 0) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    cpx<T> w = ldg_c(tw + r * k * step);
                    v[q][r] = inv ? cmulc(v[q][r], w) : cmul(v[q][r], w);
                }
            }
            butterfly<T, R>(v[q], inv);
            int base = (j / Ns) * Ns * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) s[(base + r * Ns) * nl + c] = v[q][r];
        }
    }
    __syncthreads();
}

// Full transform (forward: exp(-2 pi i ...), inverse: exp(+2 pi i ...), unnormalised).
template <typename T, int EPT>
__device__ void fft_lines(cpx<T>* s, const FftPlan& fp, int nl, const cpx<T>* tw, int tstride, bool inv) {
    int Ns = 1;
    for (int st = 0; st < fp.nst; ++st) {
        int R = fp.radix[st];
        switch (R) {
            case 8: fft_stage<T, 8, EPT>(s, fp.L, nl, Ns, tw, tstride, inv); break;
            case 4: fft_stage<T, 4, EPT>(s, fp.L, nl, Ns, tw, tstride, inv); break;
            case 3: fft_stage<T, 3, EPT>(s, fp.L, nl, Ns, tw, tstride, inv); break;
            default: fft_stage<T, 2, EPT>(s, fp.L, nl, Ns, tw, tstride, inv); break;
        }
        Ns *= R;
    }
}

// ---------------------------------------------------------------------------------------
// Truncated interpolation solves along one axis, c = 0 outside [0, n) (Sec. 2.3, Eqs.
// z_system / C_system with the isolated boundary condition; orders 4 and 5 the same
// condition with wider stencils): sum_d st_d c_{i+d} = s_i with st = b_k at the integers.
// Scaled to integer matrices A c = S s:
//   order 3: tridiag(1, 6, 1), S = 8        order 4: tridiag(1, 4, 1), S = 6
//   order 5: pentadiag(1, 76, 230, 76, 1), S = 384
// Tridiagonal (exact LU): d_0 = D, d_i = D - 1/d_{i-1}, lam_i = 1/d_i; forward
// y_i = S s_i - lam_{i-1} y_{i-1}, backward c_i = lam_i (y_i - c_{i+1}).
// Pentadiagonal (exact L D L^T, two subdiagonals l1_i, l2_i): forward
// y_i = S s_i - l1_i y_{i-1} - l2_i y_{i-2}, backward c_i = y_i / D_i - l1_{i+1} c_{i+1}
// - l2_{i+2} c_{i+2}.  The factors reach their limits to double precision within 32 rows.
// Each thread takes a contiguous chunk of a line and starts each sweep W rows early from
// a zero state, or exactly at the line's end when that is near.  The error of the early
// start decays as rho^W with rho the recurrence's slowest root: 0.172 (order 3), 0.268
// (order 4), 0.361 (order 5); W is chosen to put rho^W below the working precision.
// ---------------------------------------------------------------------------------------

constexpr int kLamTable = 32;
constexpr int kSolveTab = 3 * kLamTable;  // values of T in a solve's table

template <typename T>
__host__ __device__ __forceinline__ int solve_warm(int order) {
    const bool dbl = sizeof(T) == 8;
    return order == 5 ? (dbl ? 40 : 18) : order == 4 ? (dbl ? 30 : 14) : (dbl ? 24 : 12);
}

__host__ __device__ __forceinline__ float solve_scale(int order) {
    return order == 5 ? 384.f : order == 4 ? 6.f : 8.f;
}

// fills the per-row factors (thread 0); caller syncs.  order 3, 4: tab[i] = lam_i;
// order 5: tab[i] = l1_i, tab[K + i] = l2_i, tab[2K + i] = 1 / D_i (K = kLamTable)
template <typename T>
__device__ __forceinline__ void init_solve_tables(T* tab, int order) {
    if (threadIdx.x != 0) return;
    if (order == 5) {
        double Dm2 = 0.0, Dm1 = 0.0, l1m1 = 0.0;
        for (int i = 0; i < kLamTable; ++i) {
            const double l2 = i >= 2 ? 1.0 / Dm2 : 0.0;
            const double l1 = i >= 1 ? (76.0 - l2 * l1m1 * Dm2) / Dm1 : 0.0;
            const double D = 230.0 - l1 * l1 * Dm1 - l2 * l2 * Dm2;
            tab[i] = T(l1);
            tab[kLamTable + i] = T(l2);
            tab[2 * kLamTable + i] = T(1.0 / D);
            Dm2 = Dm1;
            Dm1 = D;
            l1m1 = l1;
        }
    } else {
        const double Dg = order == 4 ? 4.0 : 6.0;
        double d = Dg;
        for (int i = 0; i < kLamTable; ++i) {
            tab[i] = T(1.0 / d);
            d = Dg - 1.0 / d;
        }
    }
}

template <typename T> __device__ __forceinline__ T vscale(T a, T s) { return a * s; }
template <typename T> __device__ __forceinline__ cpx<T> vscale(cpx<T> a, T s) { return scl(a, s); }
template <typename T> __device__ __forceinline__ T vzero(T*) { return T(0); }
template <typename T> __device__ __forceinline__ cpx<T> vzero(cpx<T>*) { return mk(T(0), T(0)); }

__device__ __forceinline__ int tab_row(int i) { return i < kLamTable ? i : kLamTable - 1; }

template <typename T, typename V>
__device__ void tridiag_lines(const V* src, V* tmp, V* dst, int n, int nl, const T* lam, int W, T S) {
    const T lamInf = lam[kLamTable - 1];
    const int tpl = blockDim.x / nl;           // threads per line
    const int line = threadIdx.x / tpl;
    const int t = threadIdx.x % tpl;
    const int chunk = (n + tpl - 1) / tpl;
    const int a = t * chunk;
    const int b = min(n, a + chunk);
    const bool active = line < nl && a < n;
    // forward sweep -> tmp
    if (active) {
        int s0 = a - W;
        V y;
        if (s0 < kLamTable) {
            s0 = 0;
            y = vscale(src[line], S);
        } else {
            y = vzero((V*)nullptr);
        }
        int start = (s0 == 0) ? 1 : s0;
        if (s0 == 0 && a == 0) tmp[line] = y;
        for (int i = start; i < b; ++i) {
            T l = (i - 1 < kLamTable) ? lam[i - 1] : lamInf;
            V si = vscale(src[i * nl + line], S);
            y = si - vscale(y, l);
            if (i >= a) tmp[i * nl + line] = y;
        }
    }
    __syncthreads();
    // backward sweep tmp -> dst
    if (active) {
        int e0 = b - 1 + W;
        V c;
        int i0;
        if (e0 >= n - 1) {
            i0 = n - 1;
            T l = (i0 < kLamTable) ? lam[i0] : lamInf;
            c = vscale(tmp[i0 * nl + line], l);
            if (i0 < b) dst[i0 * nl + line] = c;
            --i0;
        } else {
            i0 = e0;
            c = vzero((V*)nullptr);
        }
        for (int i = i0; i >= a; --i) {
            T l = (i < kLamTable) ? lam[i] : lamInf;
            c = vscale(tmp[i * nl + line] - c, l);
            if (i < b) dst[i * nl + line] = c;
        }
    }
    __syncthreads();
}

template <typename T, typename V>
__device__ void pentadiag_lines(const V* src, V* tmp, V* dst, int n, int nl, const T* tab, int W, T S) {
    const T* l1 = tab;
    const T* l2 = tab + kLamTable;
    const T* rD = tab + 2 * kLamTable;
    const int tpl = blockDim.x / nl;
    const int line = threadIdx.x / tpl;
    const int t = threadIdx.x % tpl;
    const int chunk = (n + tpl - 1) / tpl;
    const int a = t * chunk;
    const int b = min(n, a + chunk);
    const bool active = line < nl && a < n;
    if (active) {
        // rows before max(s0, 0) count as zero: exact from row 0, else an early start
        int s0 = a - W;
        if (s0 < kLamTable) s0 = 0;
        V y1 = vzero((V*)nullptr), y2 = y1;  // y_{i-1}, y_{i-2}
        for (int i = s0; i < b; ++i) {
            const int r = tab_row(i);
            V y = vscale(src[i * nl + line], S) - vscale(y1, l1[r]) - vscale(y2, l2[r]);
            if (i >= a) tmp[i * nl + line] = y;
            y2 = y1;
            y1 = y;
        }
    }
    __syncthreads();
    if (active) {
        int e0 = b - 1 + W;
        if (e0 >= n - 1) e0 = n - 1;  // exact: c_n = c_{n+1} = 0
        V c1 = vzero((V*)nullptr), c2 = c1;  // c_{i+1}, c_{i+2}
        for (int i = e0; i >= a; --i) {
            V c = vscale(tmp[i * nl + line], rD[tab_row(i)]) - vscale(c1, l1[tab_row(i + 1)]) -
                  vscale(c2, l2[tab_row(i + 2)]);
            if (i < b) dst[i * nl + line] = c;
            c2 = c1;
            c1 = c;
        }
    }
    __syncthreads();
}

// src, dst: nl interleaved lines of n values (V = T or cpx<T>); tmp: same size scratch.
// Result (c) in dst; src and dst may be the same array, tmp must differ from both.  tab:
// filled by init_solve_tables for the same order.
template <typename T, typename V>
__device__ void spline_solve_lines(const V* src, V* tmp, V* dst, int n, int nl, const T* tab, int order) {
    const int W = solve_warm<T>(order);
    const T S = T(solve_scale(order));
    if (order == 5)
        pentadiag_lines<T, V>(src, tmp, dst, n, nl, tab, W, S);
    else
        tridiag_lines<T, V>(src, tmp, dst, n, nl, tab, W, S);
}

}  // namespace tdg
