// Radial force and error norms at the cell centres (Sec. 3: the validation of the paper
// measures F^x and F_R = (x F^x + y F^y) / R against the analytic forces of the
// generalized Maclaurin disks, with one-, two- and infinity-norms, Sec. 3.1).
//
// One grid-stride pass over the cells writes F_R (if asked) and accumulates sum |e|,
// sum e^2 and max |e| of e_x = F^x - ref_x and e_R = F_R - ref_R, per thread in the data's
// precision (compensated for FP32), per block in FP64; a second one-block pass reduces the
// block partials in a fixed order (the result does not depend on timing).  The norms are area-weighted: L1 = dx dy sum |e|, L2 = (dx dy sum e^2)^(1/2),
// Linf = max |e|.
#include <cuda_runtime.h>

#include "tdg_internal.cuh"

namespace tdg {
namespace {

constexpr int kDiagThreads = 256;

struct Acc6 {
    double v[6];  // sum|ex|, sum ex^2, max|ex|, sum|er|, sum er^2, max|er|
};

// block-wide reduction of six values into red[0..5] (thread 0 holds the result)
__device__ void block_reduce(Acc6 a, double* red) {
    __shared__ double sh[6][kDiagThreads];
    for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] = a.v[q];
    __syncthreads();
    for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < 6; ++q) {
                const double o = sh[q][threadIdx.x + w];
                sh[q][threadIdx.x] = (q == 2 || q == 5) ? fmax(sh[q][threadIdx.x], o) : sh[q][threadIdx.x] + o;
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 6; ++q) red[q] = sh[q][0];
}

// per-thread sums: FP64 for FP64 data; for FP32 data, FP32 with compensated (Kahan)
// additions, so that the per-cell work stays on the FP32 pipes (FP64 arithmetic is slow on
// this part) while each thread's sums keep about FP32 precision; blocks reduce in FP64
template <typename T>
struct ThreadSums {
    T s[4], comp[4], mx[2];  // sum|ex|, sum ex^2, sum|er|, sum er^2; compensations; maxima
    __device__ __forceinline__ ThreadSums() {
        for (int q = 0; q < 4; ++q) s[q] = comp[q] = T(0);
        mx[0] = mx[1] = T(0);
    }
    __device__ __forceinline__ void add(int q, T v) {
        if constexpr (sizeof(T) == 8) {
            s[q] += v;
        } else {
            const T y = v - comp[q];
            const T t = s[q] + y;
            comp[q] = (t - s[q]) - y;
            s[q] = t;
        }
    }
    __device__ __forceinline__ void push(T ex, T er) {
        const T ax = fabs(ex), ar = fabs(er);
        add(0, ax);
        add(1, ex * ex);
        add(2, ar);
        add(3, er * er);
        mx[0] = fmax(mx[0], ax);
        mx[1] = fmax(mx[1], ar);
    }
    __device__ __forceinline__ Acc6 to_acc() const {
        Acc6 a;
        a.v[0] = (double)s[0] - (double)comp[0];
        a.v[1] = (double)s[1] - (double)comp[1];
        a.v[2] = (double)mx[0];
        a.v[3] = (double)s[2] - (double)comp[2];
        a.v[4] = (double)s[3] - (double)comp[3];
        a.v[5] = (double)mx[1];
        return a;
    }
};

template <typename T>
__global__ void __launch_bounds__(kDiagThreads) k_radial(int nx, int ny, double dx, double dy, double x0, double y0,
                                                         const T* __restrict__ fx, const T* __restrict__ fy,
                                                         T* __restrict__ fr, const T* __restrict__ rx,
                                                         const T* __restrict__ rr, double* __restrict__ part) {
    ThreadSums<T> acc;
    const long n = (long)nx * ny;
    const T tx0 = (T)x0, ty0 = (T)y0, tdx = (T)dx, tdy = (T)dy;
    // (i, j) of cell c, advanced by the grid stride without a division per cell
    const long stride = (long)gridDim.x * blockDim.x;
    const int di = (int)(stride / ny), dj = (int)(stride % ny);
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    int i = (int)(c / ny), j = (int)(c % ny);
    for (; c < n; c += stride) {
        const T x = tx0 + (T)(i + 0.5) * tdx, y = ty0 + (T)(j + 0.5) * tdy;
        const T R = sqrt(x * x + y * y);
        const T gx = fx[c];
        const T g = R > T(0) ? (x * gx + y * fy[c]) / R : T(0);
        if (fr) fr[c] = g;
        if (rx) acc.push(gx - rx[c], rr ? g - rr[c] : T(0));
        i += di;
        j += dj;
        if (j >= ny) {
            j -= ny;
            ++i;
        }
    }
    if (part) block_reduce(acc.to_acc(), part + 6 * blockIdx.x);
}

__global__ void __launch_bounds__(kDiagThreads) k_reduce6(int nblocks, double area, const double* __restrict__ part,
                                                          double* __restrict__ out) {
    Acc6 a;
    for (int q = 0; q < 6; ++q) a.v[q] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        const double* p = part + 6 * b;
        a.v[0] += p[0];
        a.v[1] += p[1];
        a.v[2] = fmax(a.v[2], p[2]);
        a.v[3] += p[3];
        a.v[4] += p[4];
        a.v[5] = fmax(a.v[5], p[5]);
    }
    __shared__ double red[6];
    block_reduce(a, red);
    if (threadIdx.x == 0) {
        out[0] = area * red[0];
        out[1] = sqrt(area * red[1]);
        out[2] = red[2];
        out[3] = area * red[3];
        out[4] = sqrt(area * red[4]);
        out[5] = red[5];
    }
}

}  // namespace

int diag_blocks(const Plan& p) {
    const long n = (long)p.nx * p.ny;
    const long b = (n + kDiagThreads - 1) / kDiagThreads;
    return (int)(b < kDiagMaxBlocks ? b : kDiagMaxBlocks);
}

template <typename T>
cudaError_t launch_radial(const Plan& p, const T* fx, const T* fy, double x0, double y0, T* fr, const T* rx,
                          const T* rr, double* part, double* out, cudaStream_t s) {
    const int nb = diag_blocks(p);
    k_radial<T><<<nb, kDiagThreads, 0, s>>>(p.nx, p.ny, p.dx, p.dy, x0, y0, fx, fy, fr, rx, rr, rx ? part : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !rx) return e;
    k_reduce6<<<1, kDiagThreads, 0, s>>>(nb, p.dx * p.dy, part, out);
    return cudaGetLastError();
}

template cudaError_t launch_radial<float>(const Plan&, const float*, const float*, double, double, float*,
                                          const float*, const float*, double*, double*, cudaStream_t);
template cudaError_t launch_radial<double>(const Plan&, const double*, const double*, double, double, double*,
                                           const double*, const double*, double*, double*, cudaStream_t);

}  // namespace tdg
