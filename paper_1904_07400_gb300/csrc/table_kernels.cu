// Kernel-table construction on the device, FP64 (Sec. 2.1-2.2; the paper computes the
// tables once at the start, Sec. 4.2).  One thread per offset (m, n) of the quadrant
// 0 <= m < nx, 0 <= n < ny computes w^x and w^y and writes them into the quarter arrays and
// into the four mirrored positions of the zero-padded periodic tables (offset m at index
// m mod P_x); index P/2 and everything beyond |m| < nx stay zero.
#include <cuda_runtime.h>

#include "kernel_entry.cuh"
#include "tdg_internal.cuh"

namespace tdg {

struct GLSet {
    const double* x;  // the kNumOrders rules, concatenated in order
    const double* w;
};

__global__ void k_build_tables(int k, int nx, int ny, double dx, double dy, GLSet g, double* __restrict__ wq,
                               double* __restrict__ px_tab, double* __restrict__ py_tab, int Px, int Py) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)nx * ny) return;
    int m = (int)(idx / ny), n = (int)(idx % ny);
    GLRule rules[kNumOrders];
    int off = 0;
    for (int i = 0; i < kNumOrders; ++i) {
        rules[i].x = g.x + off;
        rules[i].w = g.w + off;
        rules[i].q = rule_order(i);
        off += rule_order(i);
    }
    double wx = entry_x(k, m, n, dx, dy, rules);
    double wy = entry_x(k, n, m, dy, dx, rules);  // w^y(m, n; dx, dy) = w^x(n, m; dy, dx)
    wq[idx] = wx;
    wq[(long)nx * ny + idx] = wy;
    for (int sm = 0; sm < 2; ++sm) {
        if (sm && m == 0) continue;
        int im = sm ? Px - m : m;
        for (int sn = 0; sn < 2; ++sn) {
            if (sn && n == 0) continue;
            int in = sn ? Py - n : n;
            size_t o = (size_t)im * Py + in;
            px_tab[o] = sm ? -wx : wx;  // odd in m, even in n
            py_tab[o] = sn ? -wy : wy;  // even in m, odd in n
        }
    }
}

// the placement alone, from quarter tables already in wq (tables built earlier and kept by
// the caller): the same four mirrored positions as k_build_tables
__global__ void k_place_tables(int nx, int ny, const double* __restrict__ wq, double* __restrict__ px_tab,
                               double* __restrict__ py_tab, int Px, int Py) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)nx * ny) return;
    int m = (int)(idx / ny), n = (int)(idx % ny);
    const double wx = wq[idx];
    const double wy = wq[(long)nx * ny + idx];
    for (int sm = 0; sm < 2; ++sm) {
        if (sm && m == 0) continue;
        int im = sm ? Px - m : m;
        for (int sn = 0; sn < 2; ++sn) {
            if (sn && n == 0) continue;
            int in = sn ? Py - n : n;
            size_t o = (size_t)im * Py + in;
            px_tab[o] = sm ? -wx : wx;
            py_tab[o] = sn ? -wy : wy;
        }
    }
}

cudaError_t launch_place_tables(const Plan& p, const double* wq, double* placed_x, double* placed_y,
                                cudaStream_t s) {
    long n = (long)p.nx * p.ny;
    int nt = 256;
    k_place_tables<<<(unsigned)((n + nt - 1) / nt), nt, 0, s>>>(p.nx, p.ny, wq, placed_x, placed_y, p.ax.P, p.ay.P);
    return cudaGetLastError();
}

// the potential kernel's quadrant, placed even-even on the periodic grid
__global__ void k_build_phi_table(int k, int nx, int ny, double dx, double dy, GLSet g, double* __restrict__ placed,
                                  int Px, int Py) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)nx * ny) return;
    int m = (int)(idx / ny), n = (int)(idx % ny);
    GLRule rules[kNumOrders];
    int off = 0;
    for (int i = 0; i < kNumOrders; ++i) {
        rules[i].x = g.x + off;
        rules[i].w = g.w + off;
        rules[i].q = rule_order(i);
        off += rule_order(i);
    }
    const double w = entry_phi(k, m, n, dx, dy, rules);
    for (int sm = 0; sm < 2; ++sm) {
        if (sm && m == 0) continue;
        int im = sm ? Px - m : m;
        for (int sn = 0; sn < 2; ++sn) {
            if (sn && n == 0) continue;
            int in = sn ? Py - n : n;
            placed[(size_t)im * Py + in] = w;
        }
    }
}

cudaError_t launch_build_phi_table(const Plan& p, double* placed, const double* glx, const double* glw,
                                   cudaStream_t s) {
    GLSet g;
    g.x = glx;
    g.w = glw;
    long n = (long)p.nx * p.ny;
    int nt = 128;
    k_build_phi_table<<<(unsigned)((n + nt - 1) / nt), nt, 0, s>>>(p.order, p.nx, p.ny, p.dx, p.dy, g, placed,
                                                                   p.ax.P, p.ay.P);
    return cudaGetLastError();
}

cudaError_t launch_build_tables(const Plan& p, double* wq, double* placed_x, double* placed_y, const double* glx,
                                const double* glw, cudaStream_t s) {
    GLSet g;
    g.x = glx;
    g.w = glw;
    long n = (long)p.nx * p.ny;
    int nt = 128;
    k_build_tables<<<(unsigned)((n + nt - 1) / nt), nt, 0, s>>>(p.order, p.nx, p.ny, p.dx, p.dy, g, wq, placed_x,
                                                                placed_y, p.ax.P, p.ay.P);
    return cudaGetLastError();
}

}  // namespace tdg
