// Internal declarations shared by the tdgrav translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tdgrav.h"

namespace tdg {

template <typename T>
struct cpx {
    T x, y;
};

template <typename T>
__host__ __device__ __forceinline__ cpx<T> mk(T a, T b) {
    cpx<T> r;
    r.x = a;
    r.y = b;
    return r;
}
template <typename T>
__host__ __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T>
__host__ __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T>
__host__ __device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T>
__host__ __device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> b) {
    return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T>
__host__ __device__ __forceinline__ cpx<T> conjg(cpx<T> a) { return mk(a.x, -a.y); }
template <typename T>
__host__ __device__ __forceinline__ cpx<T> scl(cpx<T> a, T s) { return mk(a.x * s, a.y * s); }

// Maximum number of radix stages of one transform.
constexpr int kMaxStages = 16;

// Radix schedule of one transform length L = prod radix[s] (radices 2, 3, 4, 8).
struct FftPlan {
    int L;
    int nst;
    int radix[kMaxStages];
};

// Per-axis description used by the kernels.
struct AxisInfo {
    int n;        // cells along the axis
    int P;        // padded period (even, 2^a 3^b, >= 2n - 1)
    FftPlan half; // complex transform of length P/2 (rows: real transform of length P)
    FftPlan full; // complex transform of length P (columns)
};

struct Plan {
    int nx, ny, order, device;
    double dx, dy, G;
    tdg_precision prec;
    AxisInfo ax, ay;       // x: columns (axis 0), y: rows (axis 1, contiguous)
    int hy;                // number of y frequencies kept: P_y/2 + 1
    int tw;                // tile width (complex elements) of the tiled intermediates
    int ntile;             // ceil(hy / tw)
    size_t ld_tile;        // elements per tile slab: nx * tw
    size_t elem;           // sizeof(real)
    bool built;
    // device allocations
    void* tw_x;            // twiddles exp(-2 pi i k / P_x), k < P_x, complex<real>
    void* tw_y;            // twiddles exp(-2 pi i k / P_y), k < P_y
    void* spec;            // spectra s_x, s_y: 2 x hy x P_x reals, layout [c][ky][kx]
    void* spec_half;       // FP32 fast path: half spectra [ky][even|odd][k] of (s_x, s_y)
    void* net_tw;          // FP32 network path: per-thread twiddle bases, x axis then y
    double* wq;            // FP64 quarter tables w^x, w^y: 2 x nx x ny (kept for tests)
    void* work;            // workspace (plan-owned or caller-owned)
    size_t work_bytes;
    bool work_owned;
    int* err;              // device error word
    double* diag;          // diagnostics: block partials and the six norms (on first use)
    void* spec_phi;        // potential spectrum (-G s_phi / (P_x P_y)), hy x P_x reals, on request
    void* noalloc;         // device address of the allocation-free solve's scratch array
    int n_ev;              // 0 or 4: events recorded around the passes (instrumentation)
    cudaEvent_t ev[4];
};

// record the plan's instrumentation event i on stream s (no-op when none are set)
// the potential (a diagnostic): table, spectrum, solve
cudaError_t launch_build_phi_table(const Plan& p, double* placed, const double* glx, const double* glw,
                                   cudaStream_t s);
template <typename T>
cudaError_t launch_potential_spectrum(const Plan& p, const double* placed, void* scratch, T* spec, cudaStream_t s);
template <typename T>
cudaError_t launch_potential(const Plan& p, const T* sigma, T* phi, void* work, cudaStream_t s);

// radial-force diagnostics (diagnostics.cu): at most kDiagMaxBlocks partial sums
constexpr int kDiagMaxBlocks = 1024;
int diag_blocks(const Plan& p);
template <typename T>
cudaError_t launch_radial(const Plan& p, const T* fx, const T* fy, double x0, double y0, T* fr, const T* rx,
                          const T* rr, double* part, double* out, cudaStream_t s);

// order of the interpolation solve a plan's passes run (0: none, C = sigma for k <= 2)
inline int solve_order(const Plan& p) { return p.order >= 3 ? p.order : 0; }

inline void mark(const Plan& p, int i, cudaStream_t s) {
    if (p.n_ev > i) cudaEventRecord(p.ev[i], s);
}

size_t workspace_bytes(const Plan& p);
cudaError_t noalloc_scratch(void** out);  // noalloc.cu: the scratch array on the current device

}  // namespace tdg

// the plan behind a C handle
const tdg::Plan& tdg_plan_internal(const tdg_plan_s* h);

namespace tdg {

// launchers (return cudaError_t of the launch)
cudaError_t launch_build_tables(const Plan& p, double* wq, double* placed_x, double* placed_y,
                                const double* glx, const double* glw, cudaStream_t s);
cudaError_t launch_place_tables(const Plan& p, const double* wq, double* placed_x, double* placed_y,
                                cudaStream_t s);
template <typename T>
cudaError_t launch_twiddles(cpx<T>* tw, int P, cudaStream_t s);
template <typename T>
cudaError_t launch_spectra(const Plan& p, const double* placed_x, const double* placed_y,
                           void* scratch, T* spec, cudaStream_t s);
template <typename T>
cudaError_t launch_forward(const Plan& p, const T* sigma, T* fx, T* fy, void* work,
                           cudaStream_t s);
int net_fp32_length(int n);  // FP32 network transform length for a side of n cells, 0: none
bool net_fp32_eligible(const Plan& p);
size_t net_fp32_table_bytes(const Plan& p);
size_t net_fp32_spec_bytes(const Plan& p);
cudaError_t launch_net_tables(const Plan& p, cudaStream_t s);
cudaError_t launch_forward_net(const Plan& p, const float* sigma, float* fx, float* fy, void* work,
                               cudaStream_t s);
cudaError_t launch_adjoint_net(const Plan& p, const float* gx, const float* gy, float* gsig, void* work,
                               cudaStream_t s);
// slab decomposition of one grid (network path): pass A on `nrows` rows into a Z row slab,
// pass B on columns ky0 .. ky0 + nky - 1 (a column slab of `ntiles` two-column tiles, G_y
// after G_x), pass C on `nrows` rows of a G row slab (G_y after G_x)
cudaError_t launch_slab_rows(const Plan& p, const float* sigma_rows, int nrows, void* zr, cudaStream_t s);
cudaError_t launch_slab_cols(const Plan& p, const void* zc, int ky0, int nky, int ntiles, void* gc, cudaStream_t s);
cudaError_t launch_slab_rows_inv(const Plan& p, const void* gr, int nrows, float* fx, float* fy, cudaStream_t s);
constexpr int kSlabCell = 16;  // bytes of one tile cell of the intermediates (two complex floats)

// One grid of a batch run by the persistent kernel on the transform network's item bodies
// (sides that are multiples of 16 up to 1024 cells: transform lengths lx, ly of 512 or
// 1024).  Units per pass: rows (pass A), frequency columns (pass B), rows of one force
// component (pass C); a 512-length unit holds two of them, one per warp.  An item is a run
// of consecutive units of one grid and pass.
struct NetDisk {
    const float* sigma;
    float* fx;
    float* fy;
    void* z;               // Z, then G_x, G_y in the plan's network workspace layout
    void* gx;
    void* gy;
    const void* nbx;       // network twiddle bases, x axis and y axis
    const void* nby;
    const void* twx;       // W_2L tables
    const void* twy;
    const void* spec;      // half spectra in network order
    int nx, ny, hy, ord, lx, ly;
    int uA, uB, uC;        // units per pass (a unit: one 1024-length transform, two 512-length)
    int nA, nB, nC;        // items per pass (units grouped by the batch's units per item)
};
struct NetBatchDev {
    const NetDisk* disks;
    const int* start;      // [3][count + 1] prefix sums of items per pass, then [3][count] grid orders
    int* done;             // [3][count] finished items per pass and grid
    int* ticket;
    int* err;
    int count;
    int total;
    int withhold;          // grid whose row-pass completions are not counted (test hook), or -1
    int units;             // units per item
};
int net_batch_units(const Plan& p, int pass);  // units of pass 0, 1, 2 for one grid; 0: not eligible
size_t net_batch_smem();                        // dynamic shared memory of the kernel
cudaError_t net_batch_blocks(int device, int* blocks);  // one persistent wave
cudaError_t launch_batched_net(const NetBatchDev& d, int blocks, cudaStream_t s);
template <typename T>
cudaError_t launch_adjoint(const Plan& p, const T* gx, const T* gy, T* gsig, void* work,
                           cudaStream_t s);

}  // namespace tdg
