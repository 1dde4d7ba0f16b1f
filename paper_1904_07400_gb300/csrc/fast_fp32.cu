// FP32 force solve for grids whose sides are 1024, 2048 or 4096 cells: the same three
// passes as solve_kernels.cu, with register-resident transforms (fft_reg.cuh) and two
// structural savings:
//
//  * Zero padding used exactly.  The column transform of length 2N of a column whose upper
//    half is zero splits into two transforms of length N: even frequencies
//    X_e = FFT_N(x), odd frequencies X_o = FFT_N(x_n W_2N^n).  The inverse, cropped to the
//    first N rows, splits the same way: y = IFFT_N(Y_e) + W_2N^-n IFFT_N(Y_o).  Nothing of
//    length 2N is ever formed.
//  * Half spectra.  For fixed ky, s_x is odd and s_y even in kx, so each of the even and odd
//    half-tables is (anti)symmetric about its middle; only the first half of each is stored
//    (8 bytes per output point for both spectra together).
//
// Intermediates use two-column tiles: element (row i, frequency ky) of an nx x hy complex
// array lives at [ky / 2][i][ky % 2], so a column-pass block reads and writes contiguous
// nx x 16-byte slabs.
#include <cuda_runtime.h>

#include "fft_reg.cuh"
#include "tdg_internal.cuh"

namespace tdg {
namespace {

using reg::cf;
using reg::pad;

constexpr int kTW = 2;  // tile width of the intermediates


// ---------------------------------------------------------------------------------------
// truncated tridiagonal solve (1/8)(c_{i-1} + 6 c_i + c_{i+1}) = s_i on one line held in
// shared memory (element i at idx(i)); tpl threads per line, thread t owns a contiguous
// chunk and starts its recurrences W steps early from zero (error lam^W, lam = 3 - 2 sqrt 2)
// ---------------------------------------------------------------------------------------
constexpr int kLam = 32;
constexpr int kWarm = 12;

__device__ __forceinline__ void fill_lambda(float* lam) {
    if (threadIdx.x == 0) {
        double d = 6.0;
        for (int i = 0; i < kLam; ++i) {
            lam[i] = (float)(1.0 / d);
            d = 6.0 - 1.0 / d;
        }
    }
}

__device__ __forceinline__ float vs(float a, float s) { return a * s; }
__device__ __forceinline__ cf vs(cf a, float s) { return scl(a, s); }

template <typename V, bool PAD>
__device__ __forceinline__ int ix(int i) { return PAD ? pad(i) : i; }

// all threads of the block call this (it synchronises); each line handled by tpl threads
template <typename V, bool PAD>
__device__ void solve_line(const V* src, V* tmp, V* dst, int n, int t, int tpl, const float* lam) {
    const float linf = lam[kLam - 1];
    const int chunk = (n + tpl - 1) / tpl;
    const int a = t * chunk;
    const int b = min(n, a + chunk);
    if (a < n) {
        int s0 = a - kWarm;
        V y;
        int start;
        if (s0 < kLam) {
            y = vs(src[ix<V, PAD>(0)], 8.0f);
            if (a == 0) tmp[ix<V, PAD>(0)] = y;
            start = 1;
        } else {
            y = vs(src[ix<V, PAD>(0)], 0.0f);
            start = s0;
        }
        for (int i = start; i < b; ++i) {
            float l = (i - 1 < kLam) ? lam[i - 1] : linf;
            y = vs(src[ix<V, PAD>(i)], 8.0f) - vs(y, l);
            if (i >= a) tmp[ix<V, PAD>(i)] = y;
        }
    }
    __syncthreads();
    if (a < n) {
        int e0 = b - 1 + kWarm;
        V c;
        int i0;
        if (e0 >= n - 1) {
            i0 = n - 1;
            float l = (i0 < kLam) ? lam[i0] : linf;
            c = vs(tmp[ix<V, PAD>(i0)], l);
            if (i0 < b) dst[ix<V, PAD>(i0)] = c;
            --i0;
        } else {
            i0 = e0;
            c = vs(tmp[ix<V, PAD>(0)], 0.0f);
        }
        for (int i = i0; i >= a; --i) {
            float l = (i < kLam) ? lam[i] : linf;
            c = vs(tmp[ix<V, PAD>(i)] - c, l);
            if (i < b) dst[ix<V, PAD>(i)] = c;
        }
    }
    __syncthreads();
}

// Same solve for a line of exactly CH * T elements with thread t owning [t CH, t CH + CH):
// fully unrolled, and branch-free for every thread but the first, because
// lam_i = 1/d_i equals its limit 3 - 2 sqrt 2 to float precision for i >= 6 (|d_i - d_inf|
// shrinks by lam^2 ~ 0.03 per step).  Warm-up of W = 10 steps: lam^10 = 2e-8.
constexpr int kWarmFast = 10;
constexpr int kExactRows = 6;

template <typename V, int CH>
__device__ __forceinline__ void solve_line_fast(const V* src, V* tmp, V* dst, int n, int t, const float* lam) {
    constexpr int W = kWarmFast;
    const float li = lam[kLam - 1];
    const int a = t * CH;
    V x[CH + W];
    // forward sweep y_i = 8 s_i - lam_{i-1} y_{i-1}: all loads first, then the recurrence
    // in registers
    if (t == 0) {
#pragma unroll
        for (int i = 0; i < CH; ++i) x[i] = src[pad(i)];
        V y = vs(x[0], 8.0f);
        tmp[pad(0)] = y;
#pragma unroll
        for (int i = 1; i < CH; ++i) {
            float l = i - 1 < kExactRows ? lam[i - 1] : li;
            y = vs(x[i], 8.0f) - vs(y, l);
            tmp[pad(i)] = y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < CH + W; ++i) x[i] = src[pad(a - W + i)];
        V y = vs(x[0], 8.0f);
#pragma unroll
        for (int i = 1; i < W; ++i) y = vs(x[i], 8.0f) - vs(y, li);
#pragma unroll
        for (int i = 0; i < CH; ++i) {
            y = vs(x[W + i], 8.0f) - vs(y, li);
            tmp[pad(a + i)] = y;
        }
    }
    __syncthreads();
    // backward sweep c_i = lam_i (y_i - c_{i+1}), exact at the end of the line
    const int b = a + CH;
    if (b == n) {
#pragma unroll
        for (int i = 0; i < CH; ++i) x[i] = tmp[pad(a + i)];
        V c = vs(x[CH - 1], li);
        dst[pad(n - 1)] = c;
#pragma unroll
        for (int i = CH - 2; i >= 0; --i) {
            float l = a + i < kExactRows ? lam[a + i] : li;
            c = vs(x[i] - c, l);
            dst[pad(a + i)] = c;
        }
    } else {
#pragma unroll
        for (int i = 0; i < CH + W; ++i) x[i] = tmp[pad(a + i)];
        V c = vs(x[CH + W - 1], li);
#pragma unroll
        for (int i = CH + W - 2; i >= CH; --i) c = vs(x[i] - c, li);
#pragma unroll
        for (int i = CH - 1; i >= 0; --i) {
            float l = a + i < kExactRows ? lam[a + i] : li;
            c = vs(x[i] - c, l);
            dst[pad(a + i)] = c;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ cf ld2(const cf* p) {
    float2 v = *reinterpret_cast<const float2*>(p);
    return mk(v.x, v.y);
}

// X = (Za + conj Zb)/2 - i w (Za - conj Zb)/2
__device__ __forceinline__ cf unpack_r2c(cf za, cf zb, cf w) {
    cf e = mk(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y));
    cf d = mk(0.5f * (za.x - zb.x), 0.5f * (za.y + zb.y));
    cf wd = cmul(w, d);
    return mk(e.x + wd.y, e.y - wd.x);
}

// Z = (Xa + conj Xb) + i conj(w) (Xa - conj Xb)
__device__ __forceinline__ cf pack_c2r(cf xa, cf xb, cf w) {
    cf e = mk(xa.x + xb.x, xa.y - xb.y);
    cf d = mk(xa.x - xb.x, xa.y + xb.y);
    cf wd = cmulc(d, w);
    return mk(e.x - wd.y, e.y + wd.x);
}

// ---------------------------------------------------------------------------------------
// pass A: one row per block (T = L / 16 threads), row length L = ny (packed complex length
// L, period 2L).  Several blocks share an SM, so one block's barrier waits overlap with
// another's work.
// ---------------------------------------------------------------------------------------
template <int L, bool TC>
__global__ void __launch_bounds__(L / 16, TC ? 2 : 3) k_fast_rows(const float* __restrict__ sigma, int nx, int solve,
                                                         const cf* __restrict__ tw, cf* __restrict__ z) {
    constexpr int T = L / 16;
    constexpr int R1 = reg::Mid<L>::R1;
    constexpr int LP = L + L / 16 + 16;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cf* eb = reinterpret_cast<cf*>(smem_raw);                 // LP
    float* rbuf = reinterpret_cast<float*>(eb + LP);          // LP floats (order 3 only)
    float* lam = rbuf + LP;
    const int t = threadIdx.x;
    const int i = blockIdx.x;
    const reg::TwBase<L, R1> tb = reg::load_tw_base<L, R1, 2>(tw, t);
    cf* ws = TC ? reinterpret_cast<cf*>(lam + kLam) + (t >> 5) * reg::kTcWarpScratch : nullptr;
    reg::TcConst K;
    if constexpr (TC) K = reg::make_tc_const(t & 31);
    cf v[16];
    if (solve) {
        // row into shared memory with one pad word per 16 (the solve's per-thread chunks
        // of 16 then fall in distinct banks)
        const float4* src = reinterpret_cast<const float4*>(sigma + (size_t)i * L);
        float4 x[4];  // all loads in flight before the first shared store
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = src[t + q * T];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float* d = rbuf + pad(4 * (t + q * T));
            d[0] = x[q].x;
            d[1] = x[q].y;
            d[2] = x[q].z;
            d[3] = x[q].w;
        }
        fill_lambda(lam);
        __syncthreads();
        solve_line_fast<float, 16>(rbuf, reinterpret_cast<float*>(eb), rbuf, L, t, lam);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            int n = t + r * T;
            v[r] = mk(rbuf[pad(2 * n)], rbuf[pad(2 * n + 1)]);
        }
    } else {
        const float2* row = reinterpret_cast<const float2*>(sigma + (size_t)i * L);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            float2 x = row[t + r * T];
            v[r] = mk(x.x, x.y);
        }
    }
#pragma unroll
    for (int r = 8; r < 16; ++r) v[r] = mk(0.f, 0.f);
    reg::fft<L, R1, TC>(v, eb, tb, t, ws, &K);
    // unpack the real transform: X[k] from Z[k] and Z[L - k]
#pragma unroll
    for (int r = 0; r < 16; ++r) eb[pad(t + r * T)] = v[r];
    __syncthreads();
    const size_t slab = (size_t)nx * kTW;
    const cf wt = reg::ld_tw(tw, t);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        int k = t + r * T;
        cf zb = eb[pad((L - k) & (L - 1))];
        z[(size_t)(k >> 1) * slab + (size_t)i * kTW + (k & 1)] = unpack_r2c(v[r], zb, reg::twist(wt, r));
    }
    if (t == 0) z[(size_t)(L >> 1) * slab + (size_t)i * kTW] = mk(v[0].x - v[0].y, 0.f);
}

// ---------------------------------------------------------------------------------------
// pass B: one column ky per block, column length L = nx
// spec: per ky, the even half (L/2 + 1 values, padded to HS) then the odd half (L/2), each
// value (s_x, s_y) already scaled by G / (P_x P_y)
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float2 ld_spec(const float2* p) { return __ldg(p); }

// (i s_x X, i s_y X) for the even (H = 0) or odd (H = 1) half at k = t + r T: wx gets the
// x product, v is overwritten with the y product (one load of each spectrum value)
template <int L, int H>
__device__ __forceinline__ void spec_products(cf* wx, cf* v, const float2* sh, int t) {
    constexpr int T = L / 16;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        int k = t + r * T;
        bool direct = H == 0 ? (r < 8 || (r == 8 && t == 0)) : (r < 8);
        float2 q = ld_spec(sh + (direct ? k : (H == 0 ? L - k : L - 1 - k)));
        float sx = direct ? q.x : -q.x;  // s_x odd, s_y even about the middle of the half
        float sy = q.y;
        cf x = v[r];
        wx[r] = mk(-sx * x.y, sx * x.x);
        v[r] = mk(-sy * x.y, sy * x.x);
    }
}

// blocks per SM the column kernel is compiled for (register budget 65536 / (blocks * L/16))
#ifndef TDG_COLS_BLOCKS
#define TDG_COLS_BLOCKS 2
#endif
// 1: one force component per column block (see k_fast_cols_split)
#ifndef TDG_COLS_SPLIT
#define TDG_COLS_SPLIT 0
#endif

template <int L, bool TC>
__global__ void __launch_bounds__(L / 16, TC ? 1 : TDG_COLS_BLOCKS) k_fast_cols(const cf* __restrict__ z, int hy, int solve,
                                                         const cf* __restrict__ tw,
                                                         const float2* __restrict__ spec, cf* __restrict__ gx,
                                                         cf* __restrict__ gy) {
    constexpr int T = L / 16;
    constexpr int R1 = reg::Mid<L>::R1;
    constexpr int LP = L + L / 16 + 16;
    constexpr int HS = L / 2 + 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cf* xb = reinterpret_cast<cf*>(smem_raw);   // LP: the column, later the even-half y result
    cf* eb = xb + LP;                            // LP: transform exchanges, solve scratch
    cf* sb = eb + LP;                            // LP: the even-half x result
    float* lam = reinterpret_cast<float*>(sb + LP);
    const int t = threadIdx.x;
    cf* ws = TC ? reinterpret_cast<cf*>(lam + kLam) + (t >> 5) * reg::kTcWarpScratch : nullptr;
    reg::TcConst K;
    if constexpr (TC) K = reg::make_tc_const(t & 31);
    const int ky = blockIdx.x;
    const int tile = ky >> 1, c = ky & 1;
    const size_t slab = (size_t)L * kTW;
    const cf* zc = z + (size_t)tile * slab + c;
    // the column's half spectra are read only after the solve and the first transform:
    // start moving them into L2 now (one bulk prefetch per half)
    if (t == 0) {
        const float2* sp = spec + (size_t)ky * 2 * HS;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(sp), "r"((unsigned)(HS * sizeof(float2)))
                     : "memory");
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(sp + HS),
                     "r"((unsigned)(HS * sizeof(float2)))
                     : "memory");
    }
    const reg::TwBase<L, R1> tb = reg::load_tw_base<L, R1, 2>(tw, t);
    {
        cf x[16];  // all loads in flight before the first shared store
#pragma unroll
        for (int r = 0; r < 16; ++r) x[r] = ld2(zc + (size_t)(t + r * T) * kTW);
#pragma unroll
        for (int r = 0; r < 16; ++r) xb[pad(t + r * T)] = x[r];
    }
    if (solve) fill_lambda(lam);
    __syncthreads();
    if (solve) solve_line_fast<cf, 16>(xb, eb, xb, L, t, lam);

    const float2* se = spec + (size_t)ky * 2 * HS;
    const float2* so = se + HS;
    const cf wt = reg::ld_tw(tw, t);
    cf v[16], w[16];
    // even frequencies: X_e = FFT_N(x); both products; both inverse transforms
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = xb[pad(t + r * T)];
    reg::fft<L, R1, TC>(v, eb, tb, t, ws, &K);
    spec_products<L, 0>(w, v, se, t);
    reg::ifft<L, R1, TC>(w, eb, tb, t, ws, &K);
#pragma unroll
    for (int r = 0; r < 16; ++r) sb[pad(t + r * T)] = w[r];  // own positions only
    reg::ifft<L, R1, TC>(v, eb, tb, t, ws, &K);
    // odd frequencies: read the twisted column, then park the even y result in its place
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        int n = t + r * T;
        w[r] = cmul(xb[pad(n)], reg::twist(wt, r));  // x_n W_2L^n
        xb[pad(n)] = v[r];
    }
    reg::fft<L, R1, TC>(w, eb, tb, t, ws, &K);
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = w[r];
    spec_products<L, 1>(w, v, so, t);
    reg::ifft<L, R1, TC>(w, eb, tb, t, ws, &K);
    cf* gxc = gx + (size_t)tile * slab + c;
    cf* gyc = gy + (size_t)tile * slab + c;
    const cf wtc = reg::ld_tw(tw, (2 * L - t) & (2 * L - 1));
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        int n = t + r * T;
        gxc[(size_t)n * kTW] = sb[pad(n)] + cmul(w[r], reg::untwist(wtc, r));
    }
    reg::ifft<L, R1, TC>(v, eb, tb, t, ws, &K);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        int n = t + r * T;
        gyc[(size_t)n * kTW] = xb[pad(n)] + cmul(v[r], reg::untwist(wtc, r));
    }
}

// Variant with one force component per block (grid 2 hy, blockIdx.x = 2 ky + comp): four
// transforms per block instead of six per column-pair of components, but a single
// 16-element array live at a time (no register spills at two blocks per SM).
template <int L, int H>
__device__ __forceinline__ void spec_product_one(cf* v, const float2* sh, int comp, int t) {
    constexpr int T = L / 16;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        int k = t + r * T;
        bool direct = H == 0 ? (r < 8 || (r == 8 && t == 0)) : (r < 8);
        float2 q = ld_spec(sh + (direct ? k : (H == 0 ? L - k : L - 1 - k)));
        float s = comp ? q.y : (direct ? q.x : -q.x);
        cf x = v[r];
        v[r] = mk(-s * x.y, s * x.x);
    }
}

template <int L, bool TC = false>
__global__ void __launch_bounds__(L / 16, TDG_COLS_BLOCKS) k_fast_cols_split(const cf* __restrict__ z, int hy, int solve,
                                                               const cf* __restrict__ tw,
                                                               const float2* __restrict__ spec,
                                                               cf* __restrict__ gx, cf* __restrict__ gy) {
    constexpr int T = L / 16;
    constexpr int R1 = reg::Mid<L>::R1;
    constexpr int LP = L + L / 16 + 16;
    constexpr int HS = L / 2 + 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cf* xb = reinterpret_cast<cf*>(smem_raw);   // LP: the column
    cf* eb = xb + LP;                            // LP: exchanges, solve scratch
    cf* sb = eb + LP;                            // LP: the even-half result
    float* lam = reinterpret_cast<float*>(sb + LP);
    const int t = threadIdx.x;
    const int ky = blockIdx.x >> 1, comp = blockIdx.x & 1;
    const int tile = ky >> 1, c = ky & 1;
    const size_t slab = (size_t)L * kTW;
    const cf* zc = z + (size_t)tile * slab + c;
    const reg::TwBase<L, R1> tb = reg::load_tw_base<L, R1, 2>(tw, t);
    cf* ws = nullptr;  // no tensor-core stages in this variant
    reg::TcConst K;
    {
        cf x[16];  // all loads in flight before the first shared store
#pragma unroll
        for (int r = 0; r < 16; ++r) x[r] = ld2(zc + (size_t)(t + r * T) * kTW);
#pragma unroll
        for (int r = 0; r < 16; ++r) xb[pad(t + r * T)] = x[r];
    }
    if (solve) fill_lambda(lam);
    __syncthreads();
    if (solve) solve_line_fast<cf, 16>(xb, eb, xb, L, t, lam);
    const float2* se = spec + (size_t)ky * 2 * HS;
    const cf wt = reg::ld_tw(tw, t);
    cf v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = xb[pad(t + r * T)];
    reg::fft<L, R1, TC>(v, eb, tb, t, ws, &K);
    spec_product_one<L, 0>(v, se, comp, t);
    reg::ifft<L, R1, TC>(v, eb, tb, t, ws, &K);
#pragma unroll
    for (int r = 0; r < 16; ++r) sb[pad(t + r * T)] = v[r];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = cmul(xb[pad(t + r * T)], reg::twist(wt, r));
    reg::fft<L, R1, TC>(v, eb, tb, t, ws, &K);
    spec_product_one<L, 1>(v, se + HS, comp, t);
    reg::ifft<L, R1, TC>(v, eb, tb, t, ws, &K);
    cf* gc = (comp ? gy : gx) + (size_t)tile * slab + c;
    const cf wtc = reg::ld_tw(tw, (2 * L - t) & (2 * L - 1));
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        int n = t + r * T;
        gc[(size_t)n * kTW] = sb[pad(n)] + cmul(v[r], reg::untwist(wtc, r));
    }
}

// ---------------------------------------------------------------------------------------
// pass C: one row of one component per block (blockIdx.y = component)
// ---------------------------------------------------------------------------------------
template <int L, bool TC>
__global__ void __launch_bounds__(L / 16, TC ? 2 : 3) k_fast_rows_inv(const cf* __restrict__ g0,
                                                             const cf* __restrict__ g1, int nx,
                                                             const cf* __restrict__ tw, float* __restrict__ f0,
                                                             float* __restrict__ f1) {
    constexpr int T = L / 16;
    constexpr int R1 = reg::Mid<L>::R1;
    constexpr int LP = L + L / 16 + 16;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cf* xb = reinterpret_cast<cf*>(smem_raw);  // LP
    const cf* g = blockIdx.y ? g1 : g0;
    float* f = blockIdx.y ? f1 : f0;
    const int t = threadIdx.x;
    cf* ws = TC ? xb + LP + (t >> 5) * reg::kTcWarpScratch : nullptr;
    reg::TcConst K;
    if constexpr (TC) K = reg::make_tc_const(t & 31);
    const int i = blockIdx.x;
    const size_t slab = (size_t)nx * kTW;
    const reg::TwBase<L, R1> tb = reg::load_tw_base<L, R1, 2>(tw, t);
    // X[k], k = 0..L (the tile pair (2p, 2p + 1) of row i is one 16-byte word)
    {
        float4 d[8];  // all loads in flight before the first shared store
#pragma unroll
        for (int q = 0; q < 8; ++q) d[q] = *reinterpret_cast<const float4*>(g + (size_t)(t + q * T) * slab + (size_t)i * kTW);
        float4 dl = make_float4(0.f, 0.f, 0.f, 0.f);
        if (t == 0) dl = *reinterpret_cast<const float4*>(g + (size_t)(L / 2) * slab + (size_t)i * kTW);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            int p = t + q * T;
            xb[pad(2 * p)] = mk(d[q].x, d[q].y);
            xb[pad(2 * p + 1)] = mk(d[q].z, d[q].w);
        }
        if (t == 0) xb[pad(L)] = mk(dl.x, dl.y);
    }
    __syncthreads();
    cf v[16];
    const cf wt = reg::ld_tw(tw, t);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        int k = t + r * T;
        v[r] = pack_c2r(xb[pad(k)], xb[pad(L - k)], reg::twist(wt, r));
    }
    __syncthreads();
    reg::ifft<L, R1, TC>(v, xb, tb, t, ws, &K);
    float2* out = reinterpret_cast<float2*>(f + (size_t)i * L);
#pragma unroll
    for (int r = 0; r < 8; ++r) out[t + r * T] = make_float2(v[r].x, v[r].y);
}

// spectra in the half layout from the full FP32 spectra [c][ky][kx]
__global__ void k_half_spectra(const float* __restrict__ full, int hy, int Px, float2* __restrict__ half) {
    const int L = Px / 2;
    const int HS = L / 2 + 2;
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long total = (long)hy * 2 * HS;
    if (idx >= total) return;
    int ky = (int)(idx / (2 * HS));
    int rem = (int)(idx % (2 * HS));
    int h = rem / HS, k = rem % HS;
    int kx = 2 * k + h;
    float2 v = make_float2(0.f, 0.f);
    bool ok = (h == 0) ? (k <= L / 2) : (k < L / 2);
    if (ok) {
        v.x = full[(size_t)ky * Px + kx];
        v.y = full[(size_t)hy * Px + (size_t)ky * Px + kx];
    }
    half[idx] = v;
}

template <int L>
size_t tc_scratch(bool tc) {
    return tc ? (size_t)(L / 16 / 32) * reg::kTcWarpScratch * sizeof(cf) : 0;
}

template <int L>
size_t rows_smem(int solve, bool tc) {
    constexpr int LP = L + L / 16 + 16;
    // the order-3 row buffer is always reserved so the TC scratch has a fixed offset
    (void)solve;
    return LP * sizeof(cf) + LP * sizeof(float) + kLam * sizeof(float) + tc_scratch<L>(tc);
}

template <int L>
size_t cols_smem(bool tc) {
    constexpr int LP = L + L / 16 + 16;
    return 3 * LP * sizeof(cf) + kLam * sizeof(float) + tc_scratch<L>(tc);
}

template <int L>
size_t inv_smem(bool tc) {
    constexpr int LP = L + L / 16 + 16;
    return LP * sizeof(cf) + tc_scratch<L>(tc);
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int LX, int LY, bool TC>
cudaError_t run_fast(const Plan& p, const float* sigma, float* fx, float* fy, void* work, cudaStream_t s) {
    const int hy = p.hy;
    const int ntile = (hy + kTW - 1) / kTW;
    const size_t n_el = (size_t)ntile * p.nx * kTW;
    cf* z = reinterpret_cast<cf*>(work);
    cf* gx = z + n_el;
    cf* gy = gx + n_el;
    const cf* twx = reinterpret_cast<const cf*>(p.tw_x);
    const cf* twy = reinterpret_cast<const cf*>(p.tw_y);
    const int solve = p.order == 3;
    cudaError_t e;
    size_t sm = rows_smem<LY>(solve, TC);
    if ((e = set_smem(k_fast_rows<LY, TC>, sm)))
        return e;
    mark(p, 0, s);
    k_fast_rows<LY, TC><<<p.nx, LY / 16, sm, s>>>(sigma, p.nx, solve, twy, z);
    if ((e = cudaGetLastError())) return e;
    mark(p, 1, s);
    sm = cols_smem<LX>(TC);
#if TDG_COLS_SPLIT
    if ((e = set_smem(k_fast_cols_split<LX>, sm)))
        return e;
    k_fast_cols_split<LX><<<2 * hy, LX / 16, sm, s>>>(z, hy, solve, twx,
                                                       reinterpret_cast<const float2*>(p.spec_half), gx, gy);
#else
    if ((e = set_smem(k_fast_cols<LX, TC>, sm)))
        return e;
    k_fast_cols<LX, TC><<<hy, LX / 16, sm, s>>>(z, hy, solve, twx, reinterpret_cast<const float2*>(p.spec_half), gx,
                                                 gy);
#endif
    if ((e = cudaGetLastError())) return e;
    mark(p, 2, s);
    sm = inv_smem<LY>(TC);
    if ((e = set_smem(k_fast_rows_inv<LY, TC>, sm)))
        return e;
    dim3 grid(p.nx, 2);
    k_fast_rows_inv<LY, TC><<<grid, LY / 16, sm, s>>>(gx, gy, p.nx, twy, fx, fy);
    e = cudaGetLastError();
    mark(p, 3, s);
    return e;
}

template <int LX, bool TC>
cudaError_t run_fast_x(const Plan& p, const float* sigma, float* fx, float* fy, void* work, cudaStream_t s) {
    switch (p.ny) {
        case 1024: return run_fast<LX, 1024, TC>(p, sigma, fx, fy, work, s);
        case 2048: return run_fast<LX, 2048, TC>(p, sigma, fx, fy, work, s);
        default: return run_fast<LX, 4096, TC>(p, sigma, fx, fy, work, s);
    }
}

template <bool TC>
cudaError_t run_fast_xy(const Plan& p, const float* sigma, float* fx, float* fy, void* work, cudaStream_t s) {
    switch (p.nx) {
        case 1024: return run_fast_x<1024, TC>(p, sigma, fx, fy, work, s);
        case 2048: return run_fast_x<2048, TC>(p, sigma, fx, fy, work, s);
        default: return run_fast_x<4096, TC>(p, sigma, fx, fy, work, s);
    }
}

bool fast_side(int n) { return n == 1024 || n == 2048 || n == 4096; }

}  // namespace

bool fast_fp32_eligible(const Plan& p) {
    return p.prec != TDG_FP64 && p.order <= 3 && fast_side(p.nx) && fast_side(p.ny) && p.ax.P == 2 * p.nx &&
           p.ay.P == 2 * p.ny;
}

size_t fast_fp32_spec_bytes(const Plan& p) {
    const int HS = p.nx / 2 + 2;
    return (size_t)p.hy * 2 * HS * sizeof(float2);
}

cudaError_t launch_half_spectra(const Plan& p, cudaStream_t s) {
    const int HS = p.nx / 2 + 2;
    long total = (long)p.hy * 2 * HS;
    k_half_spectra<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(reinterpret_cast<const float*>(p.spec), p.hy,
                                                                    p.ax.P, reinterpret_cast<float2*>(p.spec_half));
    return cudaGetLastError();
}

cudaError_t launch_forward_fast(const Plan& p, const float* sigma, float* fx, float* fy, void* work,
                                cudaStream_t s) {
    if (p.prec == TDG_FP32_TC16) return run_fast_xy<true>(p, sigma, fx, fy, work, s);
    return run_fast_xy<false>(p, sigma, fx, fy, work, s);
}

}  // namespace tdg
