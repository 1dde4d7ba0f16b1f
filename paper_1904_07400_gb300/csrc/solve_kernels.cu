// The three passes of the force solve and of its adjoint (Sec. 4.1: one forward transform
// of C, two inverse transforms), plus the forward transform of the kernel tables.
//
// Data flow of a forward solve (P_x, P_y the padded periods, M = P_y / 2, hy = M + 1):
//   pass A (rows, y):    sigma row -> [order 3: tridiagonal solve along y] -> zero-pad to
//                        P_y -> real transform (complex length-M FFT + unpacking) ->
//                        hy frequencies written to the tiled buffer Z
//   pass B (columns, x): Z column ky -> [order 3: tridiagonal solve along x on the complex
//                        column, which commutes with the y transform] -> zero-pad to P_x
//                        -> FFT -> times i s_x and i s_y -> two inverse FFTs -> first nx
//                        rows written to the tiled buffers G_x, G_y
//   pass C (rows, y):    G row -> Hermitian repacking -> inverse complex FFT of length M ->
//                        first ny reals = F^x (resp. F^y)
// The adjoint runs the transposed chain: A on g_x and g_y, B with the conjugate spectra
// (correlation) summed into one column and the x solve after the crop, C with the y solve
// after the crop.
//
// Tiled intermediates: element (row i, frequency ky) of an nx x hy complex array lives at
// [ky / TW][i][ky % TW]; a pass-B column is a strided walk through one contiguous slab and
// the row passes move whole TW-wide slices of TR rows.
#include <cuda_runtime.h>

#include "fft_block.cuh"
#include "generic_passes.cuh"
#include "tdg_internal.cuh"

namespace tdg {

// one block per row group / column: thin wrappers around the device bodies
template <typename T>
__global__ void __launch_bounds__(Bounds<T>::ROWS) k_rows_r2c(const T* __restrict__ in, int nrows, int ld, int ncols,
                                                   int solve, FftPlan fp, const cpx<T>* __restrict__ tw,
                                                   cpx<T>* __restrict__ out, Tiled ot, int hy) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    row_r2c_body<T>(in, nrows, ld, ncols, solve, fp, tw, out, ot, hy, blockIdx.x, smem_raw);
}

template <typename T>
__global__ void __launch_bounds__(Bounds<T>::ROWS) k_rows_c2r(const cpx<T>* __restrict__ in0, const cpx<T>* __restrict__ in1,
                                                   Tiled it, int nrows, int hy, int solve, FftPlan fp,
                                                   const cpx<T>* __restrict__ tw, T* __restrict__ out0,
                                                   T* __restrict__ out1, int ncols) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    row_c2r_body<T>(in0, in1, it, nrows, hy, solve, fp, tw, out0, out1, ncols, blockIdx.x, blockIdx.y, smem_raw);
}

template <typename T, bool KEEP>
__global__ void __launch_bounds__(kColThreads) k_cols_conv(const cpx<T>* __restrict__ z, Tiled t, int nx, int hy,
                                                    int solve, FftPlan fp, const cpx<T>* __restrict__ tw,
                                                    const T* __restrict__ spec, cpx<T>* __restrict__ gx,
                                                    cpx<T>* __restrict__ gy) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    col_conv_body<T, KEEP>(z, t, nx, hy, solve, fp, tw, spec, gx, gy, blockIdx.x, smem_raw);
}

// Pass B (adjoint): dL/dC-hat = -i (s_x Gx-hat + s_y Gy-hat), one inverse FFT, crop,
// x solve after the crop.
template <typename T>
__global__ void __launch_bounds__(kColThreads) k_cols_adj(const cpx<T>* __restrict__ zx, const cpx<T>* __restrict__ zy,
                                                   Tiled t, int nx, int hy, int solve, FftPlan fp,
                                                   const cpx<T>* __restrict__ tw, const T* __restrict__ spec,
                                                   cpx<T>* __restrict__ gout) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = fp.L;
    cpx<T>* s = reinterpret_cast<cpx<T>*>(smem_raw);
    T* lam = reinterpret_cast<T*>(s + P);
    const int ky = blockIdx.x;
    const size_t sstride = (size_t)hy * P;
    cpx<T> acc[kEPT];

    for (int comp = 0; comp < 2; ++comp) {
        load_column(s, comp ? zy : zx, t, ky, nx, P);
        __syncthreads();
        fft_lines<T, kEPT>(s, fp, 1, tw, 1, false);
        const T* sc = spec + comp * sstride + (size_t)ky * P;
#pragma unroll
        for (int q = 0; q < kEPT; ++q) {
            int e = threadIdx.x + q * blockDim.x;
            if (e < P) {
                T sv = __ldg(sc + e);
                cpx<T> v = s[e];
                // -i s v
                cpx<T> r = mk(sv * v.y, -sv * v.x);
                acc[q] = comp ? acc[q] + r : r;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < kEPT; ++q) {
        int e = threadIdx.x + q * blockDim.x;
        if (e < P) s[e] = acc[q];
    }
    if (solve) init_solve_tables(lam, solve);
    __syncthreads();
    fft_lines<T, kEPT>(s, fp, 1, tw, 1, true);
    if (solve) column_solve(s, nx, P, lam, solve);
    for (int i = threadIdx.x; i < nx; i += blockDim.x) gout[tidx(t, i, ky)] = s[i];
}

// Spectrum of the placed tables: column FFT of the row-transformed tables, keep the
// imaginary part (force tables: odd along the force axis) or the real part (potential
// table: even in both), times the scale (G or -G over P_x P_y).
template <typename T>
__global__ void __launch_bounds__(kColThreads) k_cols_spectrum(const cpx<double>* __restrict__ z, Tiled t, int hy,
                                                        FftPlan fp, const cpx<double>* __restrict__ tw,
                                                        double scale, int real_part, T* __restrict__ spec) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = fp.L;
    cpx<double>* s = reinterpret_cast<cpx<double>*>(smem_raw);
    const int ky = blockIdx.x;
    for (int i = threadIdx.x; i < P; i += blockDim.x) s[i] = z[tidx(t, i, ky)];
    __syncthreads();
    fft_lines<double, kEPT>(s, fp, 1, tw, 1, false);
    for (int e = threadIdx.x; e < P; e += blockDim.x)
        spec[(size_t)ky * P + e] = T(scale * (real_part ? s[e].x : s[e].y));
}

// Pass B of the potential: column ky of Z, x solve, transform, times the real potential
// spectrum, inverse transform, crop
template <typename T>
__global__ void __launch_bounds__(kColThreads) k_cols_pot(const cpx<T>* __restrict__ z, Tiled t, int nx, int hy,
                                                   int solve, FftPlan fp, const cpx<T>* __restrict__ tw,
                                                   const T* __restrict__ spec, cpx<T>* __restrict__ g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = fp.L;
    cpx<T>* s = reinterpret_cast<cpx<T>*>(smem_raw);
    T* lam = reinterpret_cast<T*>(s + P);
    const int ky = blockIdx.x;
    load_column(s, z, t, ky, nx, P);
    if (solve) init_solve_tables(lam, solve);
    __syncthreads();
    if (solve) column_solve(s, nx, P, lam, solve);
    fft_lines<T, kEPT>(s, fp, 1, tw, 1, false);
    const T* sc = spec + (size_t)ky * P;
    for (int e = threadIdx.x; e < P; e += blockDim.x) s[e] = scl(s[e], __ldg(sc + e));
    __syncthreads();
    fft_lines<T, kEPT>(s, fp, 1, tw, 1, true);
    for (int i = threadIdx.x; i < nx; i += blockDim.x) g[tidx(t, i, ky)] = s[i];
}

template <typename T>
__global__ void k_twiddles(cpx<T>* tw, int P) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P) {
        double sn, cs;
        sincospi(2.0 * (double)k / (double)P, &sn, &cs);
        tw[k] = mk(T(cs), T(-sn));
    }
}

// ---------------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------------

static int round_threads(long work, int cap) {
    long nt = (work + kEPT - 1) / kEPT;
    nt = ((nt + 31) / 32) * 32;
    if (nt < 64) nt = 64;
    if (nt > cap) nt = cap;
    return (int)nt;
}

template <typename T>
static size_t row_smem(int M, int ncols, int solve) {
    if (!solve) ncols = 0;
    constexpr int TR = RowCfg<T>::TR;
    return (size_t)(M + 1) * TR * sizeof(cpx<T>) + (size_t)ncols * TR * sizeof(T) + kSolveTab * sizeof(T);
}

template <typename T>
static size_t col_smem(int P) {
    return (size_t)P * sizeof(cpx<T>) + kSolveTab * sizeof(T);
}

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T>
static cudaError_t rows_r2c(const T* in, int nrows, int ld, int ncols, int solve, const FftPlan& fp,
                            const cpx<T>* tw, cpx<T>* out, Tiled ot, int hy, cudaStream_t s) {
    constexpr int TR = RowCfg<T>::TR;
    size_t sm = row_smem<T>(fp.L, ncols, solve);
    cudaError_t e = set_smem(k_rows_r2c<T>, sm);
    if (e != cudaSuccess) return e;
    int nt = round_threads((long)TR * fp.L, Bounds<T>::ROWS);
    k_rows_r2c<T><<<(nrows + TR - 1) / TR, nt, sm, s>>>(in, nrows, ld, ncols, solve, fp, tw, out, ot, hy);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t rows_c2r(const cpx<T>* in0, const cpx<T>* in1, Tiled it, int nrows, int hy, int solve,
                            const FftPlan& fp, const cpx<T>* tw, T* out0, T* out1, int ncols, cudaStream_t s) {
    constexpr int TR = RowCfg<T>::TR;
    size_t sm = row_smem<T>(fp.L, ncols, solve);
    cudaError_t e = set_smem(k_rows_c2r<T>, sm);
    if (e != cudaSuccess) return e;
    int nt = round_threads((long)TR * fp.L, Bounds<T>::ROWS);
    dim3 grid((nrows + TR - 1) / TR, in1 ? 2 : 1);
    k_rows_c2r<T><<<grid, nt, sm, s>>>(in0, in1, it, nrows, hy, solve, fp, tw, out0, out1, ncols);
    return cudaGetLastError();
}

template <typename T>
static Tiled tiled_of(const Plan& p, int rows) {
    Tiled t;
    t.tw = RowCfg<T>::TW;
    t.slab = (size_t)rows * t.tw;
    return t;
}

template <typename T>
cudaError_t launch_twiddles(cpx<T>* tw, int P, cudaStream_t s) {
    k_twiddles<T><<<(P + 255) / 256, 256, 0, s>>>(tw, P);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_forward(const Plan& p, const T* sigma, T* fx, T* fy, void* work, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        // the transform network for sides that are multiples of 16 from 128 to 4096 cells
        if (p.spec_half && p.net_tw) return launch_forward_net(p, sigma, fx, fy, work, s);
    }
    const Tiled t = tiled_of<T>(p, p.nx);
    const size_t n_el = (size_t)p.ntile * t.slab;
    cpx<T>* z = reinterpret_cast<cpx<T>*>(work);
    cpx<T>* gx = z + n_el;
    cpx<T>* gy = gx + n_el;
    const cpx<T>* twx = reinterpret_cast<const cpx<T>*>(p.tw_x);
    const cpx<T>* twy = reinterpret_cast<const cpx<T>*>(p.tw_y);
    const int solve = solve_order(p);
    mark(p, 0, s);
    cudaError_t e = rows_r2c<T>(sigma, p.nx, p.ny, p.ny, solve, p.ay.half, twy, z, t, p.hy, s);
    if (e != cudaSuccess) return e;
    mark(p, 1, s);
    // one column per block; FP32 keeps the transformed column in registers, FP64 redoes
    // the forward transform for the second component (register budget)
    constexpr bool KEEP = sizeof(T) == 4;
    size_t sm = col_smem<T>(p.ax.full.L);
    e = set_smem(k_cols_conv<T, KEEP>, sm);
    if (e != cudaSuccess) return e;
    int nt = round_threads(p.ax.full.L, kColThreads);
    k_cols_conv<T, KEEP><<<p.hy, nt, sm, s>>>(z, t, p.nx, p.hy, solve, p.ax.full, twx,
                                              reinterpret_cast<const T*>(p.spec), gx, gy);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    mark(p, 2, s);
    e = rows_c2r<T>(gx, gy, t, p.nx, p.hy, 0, p.ay.half, twy, fx, fy, p.ny, s);
    mark(p, 3, s);
    return e;
}

template <typename T>
cudaError_t launch_adjoint(const Plan& p, const T* gxin, const T* gyin, T* gsig, void* work, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (p.spec_half && p.net_tw) return launch_adjoint_net(p, gxin, gyin, gsig, work, s);
    }
    const Tiled t = tiled_of<T>(p, p.nx);
    const size_t n_el = (size_t)p.ntile * t.slab;
    cpx<T>* zx = reinterpret_cast<cpx<T>*>(work);
    cpx<T>* zy = zx + n_el;
    cpx<T>* gc = zy + n_el;
    const cpx<T>* twx = reinterpret_cast<const cpx<T>*>(p.tw_x);
    const cpx<T>* twy = reinterpret_cast<const cpx<T>*>(p.tw_y);
    const int solve = solve_order(p);
    mark(p, 0, s);
    cudaError_t e = rows_r2c<T>(gxin, p.nx, p.ny, p.ny, 0, p.ay.half, twy, zx, t, p.hy, s);
    if (e != cudaSuccess) return e;
    e = rows_r2c<T>(gyin, p.nx, p.ny, p.ny, 0, p.ay.half, twy, zy, t, p.hy, s);
    if (e != cudaSuccess) return e;
    mark(p, 1, s);
    size_t sm = col_smem<T>(p.ax.full.L);
    e = set_smem(k_cols_adj<T>, sm);
    if (e != cudaSuccess) return e;
    int nt = round_threads(p.ax.full.L, kColThreads);
    k_cols_adj<T><<<p.hy, nt, sm, s>>>(zx, zy, t, p.nx, p.hy, solve, p.ax.full, twx,
                                       reinterpret_cast<const T*>(p.spec), gc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    mark(p, 2, s);
    e = rows_c2r<T>(gc, nullptr, t, p.nx, p.hy, solve, p.ay.half, twy, gsig, nullptr, p.ny, s);
    mark(p, 3, s);
    return e;
}

template <typename T>
cudaError_t launch_spectra(const Plan& p, const double* placed_x, const double* placed_y, void* scratch,
                           T* spec, cudaStream_t s) {
    // FP64 transforms of the two placed P_x x P_y tables (twiddles in FP64)
    const int Px = p.ax.P, Py = p.ay.P;
    Tiled t;
    t.tw = RowCfg<double>::TW;
    t.slab = (size_t)Px * t.tw;
    cpx<double>* z = reinterpret_cast<cpx<double>*>(scratch);
    cudaError_t e;
    // twiddle tables in FP64 for this build (the plan's own may be FP32)
    cpx<double>* tw64x = z + (size_t)((p.hy + t.tw - 1) / t.tw) * t.slab;
    cpx<double>* tw64y = tw64x + Px;
    if ((e = launch_twiddles<double>(tw64x, Px, s)) != cudaSuccess) return e;
    if ((e = launch_twiddles<double>(tw64y, Py, s)) != cudaSuccess) return e;
    const double scale = p.G / ((double)Px * (double)Py);
    size_t sm = col_smem<double>(Px);
    if ((e = set_smem(k_cols_spectrum<T>, sm)) != cudaSuccess) return e;
    int nt = round_threads(Px, kColThreads);
    for (int comp = 0; comp < 2; ++comp) {
        const double* placed = comp ? placed_y : placed_x;
        e = rows_r2c<double>(placed, Px, Py, Py, 0, p.ay.half, tw64y, z, t, p.hy, s);
        if (e != cudaSuccess) return e;
        k_cols_spectrum<T><<<p.hy, nt, sm, s>>>(z, t, p.hy, p.ax.full, tw64x, scale, 0,
                                                spec + (size_t)comp * p.hy * Px);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_potential_spectrum(const Plan& p, const double* placed, void* scratch, T* spec, cudaStream_t s) {
    const int Px = p.ax.P, Py = p.ay.P;
    Tiled t;
    t.tw = RowCfg<double>::TW;
    t.slab = (size_t)Px * t.tw;
    cpx<double>* z = reinterpret_cast<cpx<double>*>(scratch);
    cudaError_t e;
    cpx<double>* tw64x = z + (size_t)((p.hy + t.tw - 1) / t.tw) * t.slab;
    cpx<double>* tw64y = tw64x + Px;
    if ((e = launch_twiddles<double>(tw64x, Px, s)) != cudaSuccess) return e;
    if ((e = launch_twiddles<double>(tw64y, Py, s)) != cudaSuccess) return e;
    const double scale = -p.G / ((double)Px * (double)Py);  // Phi = -G (C * w^phi)
    size_t sm = col_smem<double>(Px);
    if ((e = set_smem(k_cols_spectrum<T>, sm)) != cudaSuccess) return e;
    int nt = round_threads(Px, kColThreads);
    if ((e = rows_r2c<double>(placed, Px, Py, Py, 0, p.ay.half, tw64y, z, t, p.hy, s)) != cudaSuccess) return e;
    k_cols_spectrum<T><<<p.hy, nt, sm, s>>>(z, t, p.hy, p.ax.full, tw64x, scale, 1, spec);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_potential(const Plan& p, const T* sigma, T* phi, void* work, cudaStream_t s) {
    const Tiled t = tiled_of<T>(p, p.nx);
    const size_t n_el = (size_t)p.ntile * t.slab;
    cpx<T>* z = reinterpret_cast<cpx<T>*>(work);
    cpx<T>* g = z + n_el;
    const cpx<T>* twx = reinterpret_cast<const cpx<T>*>(p.tw_x);
    const cpx<T>* twy = reinterpret_cast<const cpx<T>*>(p.tw_y);
    const int solve = solve_order(p);
    cudaError_t e = rows_r2c<T>(sigma, p.nx, p.ny, p.ny, solve, p.ay.half, twy, z, t, p.hy, s);
    if (e != cudaSuccess) return e;
    size_t sm = col_smem<T>(p.ax.full.L);
    if ((e = set_smem(k_cols_pot<T>, sm)) != cudaSuccess) return e;
    int nt = round_threads(p.ax.full.L, kColThreads);
    k_cols_pot<T><<<p.hy, nt, sm, s>>>(z, t, p.nx, p.hy, solve, p.ax.full, twx,
                                       reinterpret_cast<const T*>(p.spec_phi), g);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return rows_c2r<T>(g, nullptr, t, p.nx, p.hy, 0, p.ay.half, twy, phi, nullptr, p.ny, s);
}

template cudaError_t launch_potential_spectrum<float>(const Plan&, const double*, void*, float*, cudaStream_t);
template cudaError_t launch_potential_spectrum<double>(const Plan&, const double*, void*, double*, cudaStream_t);
template cudaError_t launch_potential<float>(const Plan&, const float*, float*, void*, cudaStream_t);
template cudaError_t launch_potential<double>(const Plan&, const double*, double*, void*, cudaStream_t);
template cudaError_t launch_twiddles<float>(cpx<float>*, int, cudaStream_t);
template cudaError_t launch_twiddles<double>(cpx<double>*, int, cudaStream_t);
template cudaError_t launch_forward<float>(const Plan&, const float*, float*, float*, void*, cudaStream_t);
template cudaError_t launch_forward<double>(const Plan&, const double*, double*, double*, void*, cudaStream_t);
template cudaError_t launch_adjoint<float>(const Plan&, const float*, const float*, float*, void*, cudaStream_t);
template cudaError_t launch_adjoint<double>(const Plan&, const double*, const double*, double*, void*,
                                            cudaStream_t);
template cudaError_t launch_spectra<float>(const Plan&, const double*, const double*, void*, float*,
                                           cudaStream_t);
template cudaError_t launch_spectra<double>(const Plan&, const double*, const double*, void*, double*,
                                            cudaStream_t);

}  // namespace tdg
