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
// Truncated tridiagonal solve (1/8) (c_{i-1} + 6 c_i + c_{i+1}) = s_i, c = 0 outside
// [0, n) (Sec. 2.3, Eqs. z_system / C_system with the isolated boundary condition).
//
// Exact LU of tridiag(1, 6, 1): d_0 = 6, d_i = 6 - 1/d_{i-1}, lam_i = 1/d_i; forward
// y_i = 8 s_i - lam_{i-1} y_{i-1}, backward c_i = lam_i (y_i - c_{i+1}).  lam_i reaches its
// limit 3 - 2 sqrt(2) to double precision within 32 steps.  Each thread takes a contiguous
// chunk of a line; it starts its recurrence W steps early from a zero state (the error
// decays as lam^W, below the working precision for W = 12 (float) / 24 (double)), or
// exactly from the end of the line when that is near.
// ---------------------------------------------------------------------------------------

template <typename T> struct SolveWarm;
template <> struct SolveWarm<float> { static constexpr int W = 12; };
template <> struct SolveWarm<double> { static constexpr int W = 24; };

constexpr int kLamTable = 32;

// fills lam[0..31] (thread 0); caller syncs
template <typename T>
__device__ __forceinline__ void init_lambda(T* lam) {
    if (threadIdx.x == 0) {
        double d = 6.0;
        for (int i = 0; i < kLamTable; ++i) {
            lam[i] = T(1.0 / d);
            d = 6.0 - 1.0 / d;
        }
    }
}

template <typename T> __device__ __forceinline__ T vscale(T a, T s) { return a * s; }
template <typename T> __device__ __forceinline__ cpx<T> vscale(cpx<T> a, T s) { return scl(a, s); }
template <typename T> __device__ __forceinline__ T vzero(T*) { return T(0); }
template <typename T> __device__ __forceinline__ cpx<T> vzero(cpx<T>*) { return mk(T(0), T(0)); }

// src, dst: nl interleaved lines of n values (V = T or cpx<T>); tmp: same size scratch.
// Result (c) in dst; src and dst may be the same array, tmp must differ from both.
template <typename T, typename V>
__device__ void tridiag_solve_lines(const V* src, V* tmp, V* dst, int n, int nl, const T* lam) {
    constexpr int W = SolveWarm<T>::W;
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
            y = vscale(src[line], T(8));
        } else {
            y = vzero((V*)nullptr);
        }
        int start = (s0 == 0) ? 1 : s0;
        if (s0 == 0 && a == 0) tmp[line] = y;
        for (int i = start; i < b; ++i) {
            T l = (i - 1 < kLamTable) ? lam[i - 1] : lamInf;
            V si = vscale(src[i * nl + line], T(8));
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

}  // namespace tdg
