// Device bodies of the generic passes (any grid size with padded periods 2^a 3^b), shared
// by the one-kernel-per-pass launches and by the persistent batched kernel.
#pragma once

#include "fft_block.cuh"
#include "tdg_internal.cuh"

namespace tdg {

template <typename T> struct RowCfg;
template <> struct RowCfg<float> { static constexpr int TR = 4; static constexpr int TW = 4; };
template <> struct RowCfg<double> { static constexpr int TR = 2; static constexpr int TW = 2; };

constexpr int kEPT = 16;  // elements per thread held in registers by one FFT stage

struct Tiled {
    int tw;           // tile width
    size_t slab;      // elements per tile slab = rows * tw
};

__device__ __forceinline__ size_t tidx(const Tiled& t, int row, int ky) {
    return (size_t)(ky / t.tw) * t.slab + (size_t)row * t.tw + (ky % t.tw);
}

template <typename T>
__device__ __forceinline__ cpx<T> r2c_unpack(cpx<T> za, cpx<T> zb, cpx<T> w) {
    // X = (Za + conj Zb)/2 - i w (Za - conj Zb)/2
    cpx<T> e = mk(T(0.5) * (za.x + zb.x), T(0.5) * (za.y - zb.y));
    cpx<T> d = mk(T(0.5) * (za.x - zb.x), T(0.5) * (za.y + zb.y));
    cpx<T> wd = cmul(w, d);
    return mk(e.x + wd.y, e.y - wd.x);
}

template <typename T>
__device__ __forceinline__ cpx<T> c2r_pack(cpx<T> xa, cpx<T> xb, cpx<T> w) {
    // Z = (Xa + conj Xb) + i conj(w) (Xa - conj Xb)
    cpx<T> e = mk(xa.x + xb.x, xa.y - xb.y);
    cpx<T> d = mk(xa.x - xb.x, xa.y + xb.y);
    cpx<T> wd = cmulc(d, w);
    return mk(e.x - wd.y, e.y + wd.x);
}

// ---------------------------------------------------------------------------------------
// Pass A: real rows -> hy complex frequencies (tiled output).
// in: rows of `ld` reals, the first `ncols` valid (the rest of the period is zero).
// ---------------------------------------------------------------------------------------
template <typename T> struct Bounds;
template <> struct Bounds<float> { static constexpr int ROWS = 1024; };
template <> struct Bounds<double> { static constexpr int ROWS = 512; };
constexpr int kColThreads = 512;

template <typename T, int EPT = kEPT>
__device__ void row_r2c_body(const T* __restrict__ in, int nrows, int ld, int ncols, int solve, const FftPlan& fp,
                             const cpx<T>* __restrict__ tw, cpx<T>* __restrict__ out, const Tiled& ot, int hy, int bx,
                             unsigned char* smem_raw) {
    constexpr int TR = RowCfg<T>::TR;
    const int M = fp.L;
    cpx<T>* cbuf = reinterpret_cast<cpx<T>*>(smem_raw);                 // (M + 1) * TR
    T* rbuf = reinterpret_cast<T*>(cbuf + (size_t)(M + 1) * TR);        // ncols * TR
    T* lam = rbuf + (size_t)ncols * TR;                                 // kSolveTab
    const int r0 = bx * TR;
    const int nr = min(TR, nrows - r0);

    if (solve) {
        for (int idx = threadIdx.x; idx < TR * ncols; idx += blockDim.x) {
            int c = idx / ncols, j = idx % ncols;
            rbuf[j * TR + c] = (c < nr) ? in[(size_t)(r0 + c) * ld + j] : T(0);
        }
        init_solve_tables(lam, solve);
        __syncthreads();
        spline_solve_lines<T, T>(rbuf, reinterpret_cast<T*>(cbuf), rbuf, ncols, TR, lam, solve);
        // pack z[n] = x[2n] + i x[2n+1], x zero beyond ncols
        for (int idx = threadIdx.x; idx < TR * M; idx += blockDim.x) {
            int c = idx % TR, n = idx / TR;
            int j0 = 2 * n, j1 = 2 * n + 1;
            T a = (j0 < ncols) ? rbuf[j0 * TR + c] : T(0);
            T b = (j1 < ncols) ? rbuf[j1 * TR + c] : T(0);
            cbuf[n * TR + c] = mk(a, b);
        }
    } else {
        // pack straight from the rows
        for (int idx = threadIdx.x; idx < TR * M; idx += blockDim.x) {
            int c = idx / M, n = idx % M;
            int j0 = 2 * n, j1 = 2 * n + 1;
            const T* row = in + (size_t)(r0 + c) * ld;
            T a = (c < nr && j0 < ncols) ? row[j0] : T(0);
            T b = (c < nr && j1 < ncols) ? row[j1] : T(0);
            cbuf[n * TR + c] = mk(a, b);
        }
    }
    __syncthreads();
    fft_lines<T, EPT>(cbuf, fp, TR, tw, 2, false);

    // unpack to X[k], k = 0..M; thread owns the pair (k, M - k)
    const int half = M / 2;
    for (int idx = threadIdx.x; idx < TR * (half + 1); idx += blockDim.x) {
        int c = idx % TR, k = idx / TR;
        if (k == 0) {
            cpx<T> z0 = cbuf[c];
            cbuf[c] = mk(z0.x + z0.y, T(0));
            cbuf[M * TR + c] = mk(z0.x - z0.y, T(0));
        } else if (2 * k == M) {
            cpx<T> z = cbuf[k * TR + c];
            cbuf[k * TR + c] = r2c_unpack(z, z, ldg_c(tw + k));
        } else {
            cpx<T> za = cbuf[k * TR + c], zb = cbuf[(M - k) * TR + c];
            cbuf[k * TR + c] = r2c_unpack(za, zb, ldg_c(tw + k));
            cbuf[(M - k) * TR + c] = r2c_unpack(zb, za, ldg_c(tw + (M - k)));
        }
    }
    __syncthreads();

    // tiled write: for each slab, TR rows x TW frequencies are contiguous
    const int TW = ot.tw;
    const int ntile = (hy + TW - 1) / TW;
    for (int idx = threadIdx.x; idx < ntile * TR * TW; idx += blockDim.x) {
        int w = idx % TW, c = (idx / TW) % TR, t = idx / (TW * TR);
        int ky = t * TW + w;
        if (c < nr && ky < hy) out[tidx(ot, r0 + c, ky)] = cbuf[ky * TR + c];
    }
}

// ---------------------------------------------------------------------------------------
// Pass C: hy complex frequencies -> real rows (first ncols of the period), optional
// tridiagonal solve along the row after the crop (adjoint).
// ---------------------------------------------------------------------------------------
template <typename T, int EPT = kEPT>
__device__ void row_c2r_body(const cpx<T>* __restrict__ in0, const cpx<T>* __restrict__ in1, const Tiled& it,
                             int nrows, int hy, int solve, const FftPlan& fp, const cpx<T>* __restrict__ tw,
                             T* __restrict__ out0, T* __restrict__ out1, int ncols, int bx, int by,
                             unsigned char* smem_raw) {
    constexpr int TR = RowCfg<T>::TR;
    const int M = fp.L;
    cpx<T>* cbuf = reinterpret_cast<cpx<T>*>(smem_raw);
    T* rbuf = reinterpret_cast<T*>(cbuf + (size_t)(M + 1) * TR);
    T* lam = rbuf + (size_t)ncols * TR;
    const cpx<T>* in = by ? in1 : in0;
    T* out = by ? out1 : out0;
    const int r0 = bx * TR;
    const int nr = min(TR, nrows - r0);
    const int TW = it.tw;
    const int ntile = (hy + TW - 1) / TW;

    for (int idx = threadIdx.x; idx < ntile * TR * TW; idx += blockDim.x) {
        int w = idx % TW, c = (idx / TW) % TR, t = idx / (TW * TR);
        int ky = t * TW + w;
        if (ky < hy) cbuf[ky * TR + c] = (c < nr) ? in[tidx(it, r0 + c, ky)] : mk(T(0), T(0));
    }
    if (solve) init_solve_tables(lam, solve);
    __syncthreads();

    // Hermitian repack into Z[k], k < M; thread owns the pair (k, M - k)
    const int half = M / 2;
    for (int idx = threadIdx.x; idx < TR * (half + 1); idx += blockDim.x) {
        int c = idx % TR, k = idx / TR;
        if (k == 0) {
            cpx<T> x0 = cbuf[c], xm = cbuf[M * TR + c];
            cbuf[c] = c2r_pack(x0, xm, mk(T(1), T(0)));
        } else if (2 * k == M) {
            cpx<T> x = cbuf[k * TR + c];
            cbuf[k * TR + c] = c2r_pack(x, x, ldg_c(tw + k));
        } else {
            cpx<T> xa = cbuf[k * TR + c], xb = cbuf[(M - k) * TR + c];
            cbuf[k * TR + c] = c2r_pack(xa, xb, ldg_c(tw + k));
            cbuf[(M - k) * TR + c] = c2r_pack(xb, xa, ldg_c(tw + (M - k)));
        }
    }
    __syncthreads();
    fft_lines<T, EPT>(cbuf, fp, TR, tw, 2, true);

    if (!solve) {
        for (int idx = threadIdx.x; idx < TR * ncols; idx += blockDim.x) {
            int c = idx / ncols, j = idx % ncols;
            if (c < nr) {
                cpx<T> z = cbuf[(j >> 1) * TR + c];
                out[(size_t)(r0 + c) * ncols + j] = (j & 1) ? z.y : z.x;
            }
        }
        return;
    }
    for (int idx = threadIdx.x; idx < TR * ncols; idx += blockDim.x) {
        int c = idx % TR, j = idx / TR;
        cpx<T> z = cbuf[(j >> 1) * TR + c];
        rbuf[j * TR + c] = (j & 1) ? z.y : z.x;
    }
    __syncthreads();
    spline_solve_lines<T, T>(rbuf, reinterpret_cast<T*>(cbuf), rbuf, ncols, TR, lam, solve);
    for (int idx = threadIdx.x; idx < TR * ncols; idx += blockDim.x) {
        int c = idx / ncols, j = idx % ncols;
        if (c < nr) out[(size_t)(r0 + c) * ncols + j] = rbuf[j * TR + c];
    }
}

// ---------------------------------------------------------------------------------------
// Pass B (forward): one column ky per block.
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void load_column(cpx<T>* s, const cpx<T>* __restrict__ z, const Tiled& t, int ky,
                                            int nx, int P) {
    for (int i = threadIdx.x; i < P; i += blockDim.x) s[i] = (i < nx) ? z[tidx(t, i, ky)] : mk(T(0), T(0));
}

// s holds the column in [0, nx) and zeros beyond; solves along x in place, restores zeros
template <typename T>
__device__ __forceinline__ void column_solve(cpx<T>* s, int nx, int P, const T* lam, int order) {
    spline_solve_lines<T, cpx<T>>(s, s + nx, s, nx, 1, lam, order);
    for (int i = nx + threadIdx.x; i < P; i += blockDim.x) s[i] = mk(T(0), T(0));
    __syncthreads();
}

template <typename T, bool KEEP, int EPT = kEPT>
__device__ void col_conv_body(const cpx<T>* __restrict__ z, const Tiled& t, int nx, int hy, int solve,
                              const FftPlan& fp, const cpx<T>* __restrict__ tw, const T* __restrict__ spec,
                              cpx<T>* __restrict__ gx, cpx<T>* __restrict__ gy, int bx, unsigned char* smem_raw) {
    const int P = fp.L;
    cpx<T>* s = reinterpret_cast<cpx<T>*>(smem_raw);
    T* lam = reinterpret_cast<T*>(s + P);
    const int ky = bx;
    const size_t sstride = (size_t)hy * P;
    cpx<T> keep[KEEP ? EPT : 1];

    for (int comp = 0; comp < 2; ++comp) {
        if (comp == 0 || !KEEP) {
            load_column(s, z, t, ky, nx, P);
            if (solve) init_solve_tables(lam, solve);
            __syncthreads();
            if (solve) column_solve(s, nx, P, lam, solve);
            fft_lines<T, EPT>(s, fp, 1, tw, 1, false);
            if (KEEP) {
#pragma unroll
                for (int q = 0; q < EPT; ++q) {
                    int e = threadIdx.x + q * blockDim.x;
                    if (e < P) keep[q] = s[e];
                }
                __syncthreads();
            }
        }
        const T* sc = spec + comp * sstride + (size_t)ky * P;
        cpx<T>* g = comp ? gy : gx;
        // times i s_c
        if (KEEP) {
#pragma unroll
            for (int q = 0; q < EPT; ++q) {
                int e = threadIdx.x + q * blockDim.x;
                if (e < P) {
                    T sv = __ldg(sc + e);
                    s[e] = mk(-sv * keep[q].y, sv * keep[q].x);
                }
            }
        } else {
            for (int e = threadIdx.x; e < P; e += blockDim.x) {
                T sv = __ldg(sc + e);
                cpx<T> v = s[e];
                s[e] = mk(-sv * v.y, sv * v.x);
            }
        }
        __syncthreads();
        fft_lines<T, EPT>(s, fp, 1, tw, 1, true);
        for (int i = threadIdx.x; i < nx; i += blockDim.x) g[tidx(t, i, ky)] = s[i];
        __syncthreads();
    }
}


}  // namespace tdg
