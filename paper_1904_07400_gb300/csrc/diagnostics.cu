// Radial force and error norms at the cell centres (Sec. 3: the validation of the paper
// measures F^x and F_R = (x F^x + y F^y) / R against the analytic forces of the
// generalized Maclaurin disks, with one-, two- and infinity-norms, Sec. 3.1).
//
// One grid-stride pass over the cells writes F_R (if asked) and accumulates, per block in
// FP64, sum |e|, sum e^2 and max |e| of e_x = F^x - ref_x and e_R = F_R - ref_R; a second
// one-block pass reduces the block partials in a fixed order (the result does not depend
// on timing).  The norms are area-weighted: L1 = dx dy sum |e|, L2 = (dx dy sum e^2)^(1/2),
// Linf = max |e|.
#include <cuda_runtime.h>

#include "tdg_internal.cuh"

namespace tdg {
namespace {

constexpr int kDiagThreads = 256;

struct Acc6 {
    double v[6];  // sum|ex|, sum ex^2, max|ex|, sum|er|, sum er^2, max|er|
};

__device__ __forceinline__ void acc_add(Acc6& a, double ex, double er) {
    const double ax = fabs(ex), ar = fabs(er);
    a.v[0] += ax;
    a.v[1] += ex * ex;
    a.v[2] = fmax(a.v[2], ax);
    a.v[3] += ar;
    a.v[4] += er * er;
    a.v[5] = fmax(a.v[5], ar);
}

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

template <typename T>
__global__ void __launch_bounds__(kDiagThreads) k_radial(int nx, int ny, double dx, double dy, double x0, double y0,
                                                         const T* __restrict__ fx, const T* __restrict__ fy,
                                                         T* __restrict__ fr, const T* __restrict__ rx,
                                                         const T* __restrict__ rr, double* __restrict__ part) {
    Acc6 a;
    for (int q = 0; q < 6; ++q) a.v[q] = 0.0;
    const long n = (long)nx * ny;
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
        const int i = (int)(c / ny), j = (int)(c % ny);
        const double x = x0 + (i + 0.5) * dx, y = y0 + (j + 0.5) * dy;
        const double R = sqrt(x * x + y * y);
        const double gx = (double)fx[c];
        const double g = R > 0.0 ? (x * gx + y * (double)fy[c]) / R : 0.0;
        if (fr) fr[c] = (T)g;
        if (rx) acc_add(a, gx - (double)rx[c], rr ? g - (double)rr[c] : 0.0);
    }
    if (part) block_reduce(a, part + 6 * blockIdx.x);
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
