// C ABI of tdgrav: plan lifecycle, transform-length choice and dispatch to the kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "kernel_entry.cuh"
#include "tdg_internal.cuh"

using namespace tdg;

struct tdg_plan_s {
    Plan p;
};

const Plan& tdg_plan_internal(const tdg_plan_s* h) { return h->p; }

namespace {

constexpr int kMaxN = 4096;            // longest grid side: P = 2M <= 8192 fits one block

bool smooth23(int n) {
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

// smallest 2^a 3^b >= n
int next_smooth(int n) {
    int m = n < 1 ? 1 : n;
    while (!smooth23(m)) ++m;
    return m;
}

FftPlan make_fft_plan(int L) {
    FftPlan fp;
    fp.L = L;
    fp.nst = 0;
    int e2 = 0, e3 = 0, t = L;
    while (t % 2 == 0) { t /= 2; ++e2; }
    while (t % 3 == 0) { t /= 3; ++e3; }
    for (int i = 0; i < e3; ++i) fp.radix[fp.nst++] = 3;
    while (e2 >= 3) { fp.radix[fp.nst++] = 8; e2 -= 3; }
    if (e2 == 2) fp.radix[fp.nst++] = 4;
    if (e2 == 1) fp.radix[fp.nst++] = 2;
    return fp;
}

// padded period 2M; M = the smallest 2^a 3^b >= n unless a longer M is given
AxisInfo make_axis(int n, int M = 0) {
    AxisInfo a;
    a.n = n;
    if (M < n) M = next_smooth(n);
    a.P = 2 * M;
    a.half = make_fft_plan(M);
    a.full = make_fft_plan(2 * M);
    return a;
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_q
void gauss_legendre(int q, double* x, double* w) {
    const double pi = 3.14159265358979323846264338327950288;
    for (int i = 0; i < (q + 1) / 2; ++i) {
        double z = cos(pi * (i + 0.75) / (q + 0.5));
        double pp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= q; ++j) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = q * (z * p1 - p2) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (fabs(dz) < 1e-17) break;
        }
        x[i] = -z;
        x[q - 1 - i] = z;
        w[i] = w[q - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

// the kNumOrders Gauss-Legendre rules, concatenated in order
struct HostRules {
    std::vector<double> x, w;
    GLRule rules[kNumOrders];
    HostRules() {
        int off[kNumOrders];
        for (int i = 0; i < kNumOrders; ++i) {
            off[i] = (int)x.size();
            x.resize(x.size() + rule_order(i));
            w.resize(w.size() + rule_order(i));
        }
        for (int i = 0; i < kNumOrders; ++i) {
            gauss_legendre(rule_order(i), x.data() + off[i], w.data() + off[i]);
            rules[i].x = x.data() + off[i];
            rules[i].w = w.data() + off[i];
            rules[i].q = rule_order(i);
        }
    }
};

const HostRules& host_rules() {
    static HostRules r;
    return r;
}

tdg_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return TDG_OK;
    if (e == cudaErrorMemoryAllocation) return TDG_ERR_OOM;
    return TDG_ERR_CUDA;
}

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool aligned16(const void* ptr) { return ((uintptr_t)ptr & 15u) == 0; }

size_t real_size(tdg_precision prec) { return prec == TDG_FP64 ? sizeof(double) : sizeof(float); }

int tile_width(tdg_precision prec) { return prec == TDG_FP64 ? 2 : 4; }

void free_plan_memory(Plan& p) {
    cudaFree(p.tw_x);
    cudaFree(p.tw_y);
    cudaFree(p.spec);
    cudaFree(p.spec_half);
    cudaFree(p.net_tw);
    cudaFree(p.wq);
    cudaFree(p.err);
    cudaFree(p.diag);
    p.diag = nullptr;
    cudaFree(p.spec_phi);
    p.spec_phi = nullptr;
    if (p.work_owned) cudaFree(p.work);
    p.tw_x = p.tw_y = p.spec = p.spec_half = p.net_tw = nullptr;
    p.wq = nullptr;
    p.err = nullptr;
    p.work = nullptr;
    p.work_bytes = 0;
    p.work_owned = false;
    p.built = false;
}

tdg_status ensure_workspace(Plan& p) {
    size_t need = workspace_bytes(p);
    if (p.work && p.work_bytes >= need) return TDG_OK;
    if (p.work && !p.work_owned) return TDG_ERR_INVALID_ARG;
    if (p.work) cudaFree(p.work);
    p.work = nullptr;
    cudaError_t e = cudaMalloc(&p.work, need);
    if (e != cudaSuccess) {
        p.work = nullptr;
        return from_cuda(e);
    }
    p.work_bytes = need;
    p.work_owned = true;
    return TDG_OK;
}

// the tensor-core form runs on the register-transform kernels: sides of 1024, 2048, 4096
// FP32_TC16 runs the network path with its column pass on the tensor cores: sides that the
// network takes, columns (x) of a transform length of 2048 or 4096 (two warp groups of 128
// rows, or one, per product)
bool tc16_available(int nx, int ny) { return net_fp32_length(nx) >= 2048 && net_fp32_length(ny) != 0; }

}  // namespace

namespace tdg {
size_t workspace_bytes(const Plan& p) {
    // three tiled nx x hy complex arrays (Z, G_x, G_y; adjoint: Z_x, Z_y, G)
    return 3 * (size_t)p.ntile * p.nx * p.tw * 2 * p.elem;
}
}  // namespace tdg

extern "C" {

const char* tdg_status_string(tdg_status s) {
    switch (s) {
        case TDG_OK: return "ok";
        case TDG_ERR_INVALID_ARG: return "invalid argument";
        case TDG_ERR_UNSUPPORTED: return "unsupported size";
        case TDG_ERR_NOT_BUILT: return "kernel tables not built";
        case TDG_ERR_OOM: return "device allocation failed";
        case TDG_ERR_CUDA: return "CUDA error";
        case TDG_ERR_TIMEOUT: return "device-side wait timed out";
        case TDG_ERR_DEVICE_BOUNDS: return "device-side bounds check failed";
    }
    return "unknown status";
}

tdg_status tdg_init(tdg_plan* out, int nx, int ny, int order, double dx, double dy, double G,
                    tdg_precision prec, int device) {
    if (!out) return TDG_ERR_INVALID_ARG;
    *out = nullptr;
    if (order < 1 || order > 5 || nx < 1 || ny < 1) return TDG_ERR_INVALID_ARG;
    if (!(dx > 0.0) || !(dy > 0.0) || !isfinite(dx) || !isfinite(dy) || !isfinite(G)) return TDG_ERR_INVALID_ARG;
    if (prec != TDG_FP64 && prec != TDG_FP32 && prec != TDG_FP32_TC16) return TDG_ERR_INVALID_ARG;
    if (prec == TDG_FP32_TC16 && !tc16_available(nx, ny)) return TDG_ERR_UNSUPPORTED;
    if (device < 0) return TDG_ERR_INVALID_ARG;
    if (nx > kMaxN || ny > kMaxN) return TDG_ERR_UNSUPPORTED;
    tdg_plan_s* h = new (std::nothrow) tdg_plan_s();
    if (!h) return TDG_ERR_OOM;
    Plan& p = h->p;
    memset(&p, 0, sizeof(Plan));
    p.nx = nx;
    p.ny = ny;
    p.order = order;
    p.device = device;
    p.dx = dx;
    p.dy = dy;
    p.G = G;
    p.prec = prec;
    // FP32 grids whose sides are multiples of 16 from 128 to 4096 cells run the transform
    // network, whose lengths are 512 .. 4096: pad to twice that length (any padded period
    // of at least 2n - 1 gives the same cropped result)
    const bool net = (prec == TDG_FP32 || prec == TDG_FP32_TC16) && net_fp32_length(nx) && net_fp32_length(ny);
    p.ax = make_axis(nx, net ? net_fp32_length(nx) : 0);
    p.ay = make_axis(ny, net ? net_fp32_length(ny) : 0);
    p.hy = p.ay.P / 2 + 1;
    p.tw = tile_width(prec);
    p.ntile = (p.hy + p.tw - 1) / p.tw;
    p.ld_tile = (size_t)nx * p.tw;
    p.elem = real_size(prec);
    *out = h;
    return TDG_OK;
}

size_t tdg_workspace_bytes(const tdg_plan h) {
    if (!h) return 0;
    return workspace_bytes(h->p);
}

tdg_status tdg_set_workspace(tdg_plan h, void* ptr, size_t bytes) {
    if (!h) return TDG_ERR_INVALID_ARG;
    Plan& p = h->p;
    if (ptr && (((uintptr_t)ptr & 255u) != 0 || bytes < workspace_bytes(p))) return TDG_ERR_INVALID_ARG;
    DeviceGuard g(p.device);
    if (p.work_owned && p.work) cudaFree(p.work);
    p.work = ptr;
    p.work_bytes = ptr ? bytes : 0;
    p.work_owned = false;
    return TDG_OK;
}

// the build; with wx_host / wy_host (quarter tables the caller kept) the quadrature is
// skipped and the tables are copied in and placed
static tdg_status build_plan(tdg_plan h, const double* wx_host, const double* wy_host, tdg_stream stream) {
    Plan& p = h->p;
    DeviceGuard g(p.device);
    if (!g.ok) return TDG_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int Px = p.ax.P, Py = p.ay.P;
    const size_t cx = p.prec == TDG_FP64 ? sizeof(cpx<double>) : sizeof(cpx<float>);
    // drop an earlier build, keep a caller workspace
    void* keep_work = p.work;
    bool keep_owned = p.work_owned;
    size_t keep_bytes = p.work_bytes;
    p.work = nullptr;
    p.work_owned = false;
    free_plan_memory(p);
    p.work = keep_work;
    p.work_owned = keep_owned;
    p.work_bytes = keep_bytes;

    cudaError_t e;
    double *placed_x = nullptr, *placed_y = nullptr, *glx = nullptr, *glw = nullptr;
    void* scratch = nullptr;
    const HostRules& R = host_rules();
    const size_t ntile64 = (size_t)(p.hy + 1) / 2;
    const size_t scratch_bytes = (ntile64 * Px * 2 + Px + Py) * sizeof(cpx<double>);
#define TDG_TRY(call)              \
    do {                           \
        e = (call);                \
        if (e != cudaSuccess) goto fail; \
    } while (0)
    TDG_TRY(cudaMalloc(&p.err, sizeof(int)));
    TDG_TRY(cudaMemsetAsync(p.err, 0, sizeof(int), s));
    TDG_TRY(cudaMalloc(&p.tw_x, Px * cx));
    TDG_TRY(cudaMalloc(&p.tw_y, Py * cx));
    TDG_TRY(cudaMalloc(&p.wq, 2 * (size_t)p.nx * p.ny * sizeof(double)));
    TDG_TRY(cudaMalloc(&p.spec, 2 * (size_t)p.hy * Px * p.elem));
    TDG_TRY(cudaMalloc(&placed_x, (size_t)Px * Py * sizeof(double)));
    TDG_TRY(cudaMalloc(&placed_y, (size_t)Px * Py * sizeof(double)));
    TDG_TRY(cudaMalloc(&scratch, scratch_bytes));
    if (!wx_host) {
        TDG_TRY(cudaMalloc(&glx, R.x.size() * sizeof(double)));
        TDG_TRY(cudaMalloc(&glw, R.w.size() * sizeof(double)));
        TDG_TRY(cudaMemcpyAsync(glx, R.x.data(), R.x.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        TDG_TRY(cudaMemcpyAsync(glw, R.w.data(), R.w.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    TDG_TRY(cudaMemsetAsync(placed_x, 0, (size_t)Px * Py * sizeof(double), s));
    TDG_TRY(cudaMemsetAsync(placed_y, 0, (size_t)Px * Py * sizeof(double), s));
    if (p.prec == TDG_FP64) {
        TDG_TRY(launch_twiddles<double>(reinterpret_cast<cpx<double>*>(p.tw_x), Px, s));
        TDG_TRY(launch_twiddles<double>(reinterpret_cast<cpx<double>*>(p.tw_y), Py, s));
    } else {
        TDG_TRY(launch_twiddles<float>(reinterpret_cast<cpx<float>*>(p.tw_x), Px, s));
        TDG_TRY(launch_twiddles<float>(reinterpret_cast<cpx<float>*>(p.tw_y), Py, s));
    }
    if (wx_host) {
        const size_t n = (size_t)p.nx * p.ny;
        TDG_TRY(cudaMemcpyAsync(p.wq, wx_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
        TDG_TRY(cudaMemcpyAsync(p.wq + n, wy_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
        TDG_TRY(launch_place_tables(p, p.wq, placed_x, placed_y, s));
    } else {
        TDG_TRY(launch_build_tables(p, p.wq, placed_x, placed_y, glx, glw, s));
    }
    if (p.prec == TDG_FP64)
        TDG_TRY(launch_spectra<double>(p, placed_x, placed_y, scratch, reinterpret_cast<double*>(p.spec), s));
    else
        TDG_TRY(launch_spectra<float>(p, placed_x, placed_y, scratch, reinterpret_cast<float*>(p.spec), s));
    if (net_fp32_eligible(p)) {
        // FP32 and FP32_TC16: one-barrier network kernels, spectra in the network's order
        TDG_TRY(cudaMalloc(&p.spec_half, net_fp32_spec_bytes(p)));
        TDG_TRY(cudaMalloc(&p.net_tw, net_fp32_table_bytes(p)));
        TDG_TRY(launch_net_tables(p, s));
    }
    TDG_TRY(cudaStreamSynchronize(s));
    if (noalloc_scratch(&p.noalloc) != cudaSuccess) p.noalloc = nullptr;  // set-up of tdg_solve_forces_noalloc
    cudaFree(placed_x);
    cudaFree(placed_y);
    cudaFree(glx);
    cudaFree(glw);
    cudaFree(scratch);
    p.built = true;
    return TDG_OK;
fail:
    cudaStreamSynchronize(s);
    cudaFree(placed_x);
    cudaFree(placed_y);
    cudaFree(glx);
    cudaFree(glw);
    cudaFree(scratch);
    keep_work = p.work;
    keep_owned = p.work_owned;
    keep_bytes = p.work_bytes;
    p.work = nullptr;
    p.work_owned = false;
    free_plan_memory(p);
    p.work = keep_work;
    p.work_owned = keep_owned;
    p.work_bytes = keep_bytes;
    return from_cuda(e);
#undef TDG_TRY
}

tdg_status tdg_build_kernel_tables(tdg_plan h, tdg_stream stream) {
    if (!h) return TDG_ERR_INVALID_ARG;
    return build_plan(h, nullptr, nullptr, stream);
}

tdg_status tdg_build_kernel_tables_from(tdg_plan h, const double* wx, const double* wy, tdg_stream stream) {
    if (!h || !wx || !wy) return TDG_ERR_INVALID_ARG;
    const Plan& p = h->p;
    // spot check against the table code: the corners, the near field and a far entry of
    // both components must agree (tables of another order, cell shape or size fail here);
    // entries that vanish by symmetry are held to 1e-15 of the largest one checked
    const int ms[5] = {0, 1, 2, p.nx - 1, p.nx / 2};
    const int ns[5] = {1, 0, 3, p.ny - 1, p.ny / 3};
    double ref[5][2], amax = 0.0;
    for (int q = 0; q < 5; ++q)
        for (int c = 0; c < 2; ++c) {
            const int m = ms[q] < p.nx ? ms[q] : p.nx - 1, n = ns[q] < p.ny ? ns[q] : p.ny - 1;
            if (tdg_kernel_entry_host(p.order, m, n, p.dx, p.dy, c, &ref[q][c]) != TDG_OK) return TDG_ERR_INVALID_ARG;
            amax = fmax(amax, fabs(ref[q][c]));
        }
    for (int q = 0; q < 5; ++q)
        for (int c = 0; c < 2; ++c) {
            const int m = ms[q] < p.nx ? ms[q] : p.nx - 1, n = ns[q] < p.ny ? ns[q] : p.ny - 1;
            const double got = (c ? wy : wx)[(size_t)m * p.ny + n];
            if (!(fabs(got - ref[q][c]) <= 1e-12 * fabs(ref[q][c]) + 1e-15 * amax)) return TDG_ERR_INVALID_ARG;
        }
    return build_plan(h, wx, wy, stream);
}

static tdg_status check_solve_args(const Plan& p, const void* a, const void* b, const void* c) {
    if (!a || !b || !c || !aligned16(a) || !aligned16(b) || !aligned16(c)) return TDG_ERR_INVALID_ARG;
    if (!p.built) return TDG_ERR_NOT_BUILT;
    return TDG_OK;
}

tdg_status tdg_solve_forces(tdg_plan h, const void* sigma, void* fx, void* fy, tdg_stream stream) {
    if (!h) return TDG_ERR_INVALID_ARG;
    Plan& p = h->p;
    tdg_status st = check_solve_args(p, sigma, fx, fy);
    if (st != TDG_OK) return st;
    if (fx == fy || fx == sigma || fy == sigma) return TDG_ERR_INVALID_ARG;
    DeviceGuard g(p.device);
    if (!g.ok) return TDG_ERR_CUDA;
    if ((st = ensure_workspace(p)) != TDG_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (p.prec == TDG_FP64)
        e = launch_forward<double>(p, (const double*)sigma, (double*)fx, (double*)fy, p.work, s);
    else
        e = launch_forward<float>(p, (const float*)sigma, (float*)fx, (float*)fy, p.work, s);
    return from_cuda(e);
}

tdg_status tdg_build_potential_tables(tdg_plan h, tdg_stream stream) {
    if (!h) return TDG_ERR_INVALID_ARG;
    Plan& p = h->p;
    if (!p.built) return TDG_ERR_NOT_BUILT;
    DeviceGuard g(p.device);
    if (!g.ok) return TDG_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int Px = p.ax.P, Py = p.ay.P;
    const HostRules& R = host_rules();
    const size_t ntile64 = (size_t)(p.hy + 1) / 2;
    const size_t scratch_bytes = (ntile64 * Px * 2 + Px + Py) * sizeof(cpx<double>);
    double *placed = nullptr, *glx = nullptr, *glw = nullptr;
    void* scratch = nullptr;
    cudaFree(p.spec_phi);
    p.spec_phi = nullptr;
    cudaError_t e;
#define TDG_TRY(call)              \
    do {                           \
        e = (call);                \
        if (e != cudaSuccess) goto fail; \
    } while (0)
    TDG_TRY(cudaMalloc(&p.spec_phi, (size_t)p.hy * Px * p.elem));
    TDG_TRY(cudaMalloc(&placed, (size_t)Px * Py * sizeof(double)));
    TDG_TRY(cudaMalloc(&scratch, scratch_bytes));
    TDG_TRY(cudaMalloc(&glx, R.x.size() * sizeof(double)));
    TDG_TRY(cudaMalloc(&glw, R.w.size() * sizeof(double)));
    TDG_TRY(cudaMemcpyAsync(glx, R.x.data(), R.x.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    TDG_TRY(cudaMemcpyAsync(glw, R.w.data(), R.w.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    TDG_TRY(cudaMemsetAsync(placed, 0, (size_t)Px * Py * sizeof(double), s));
    TDG_TRY(launch_build_phi_table(p, placed, glx, glw, s));
    if (p.prec == TDG_FP64)
        TDG_TRY(launch_potential_spectrum<double>(p, placed, scratch, reinterpret_cast<double*>(p.spec_phi), s));
    else
        TDG_TRY(launch_potential_spectrum<float>(p, placed, scratch, reinterpret_cast<float*>(p.spec_phi), s));
    TDG_TRY(cudaStreamSynchronize(s));
    cudaFree(placed);
    cudaFree(scratch);
    cudaFree(glx);
    cudaFree(glw);
    return TDG_OK;
fail:
    cudaStreamSynchronize(s);
    cudaFree(placed);
    cudaFree(scratch);
    cudaFree(glx);
    cudaFree(glw);
    cudaFree(p.spec_phi);
    p.spec_phi = nullptr;
    return from_cuda(e);
#undef TDG_TRY
}

tdg_status tdg_solve_potential(tdg_plan h, const void* sigma, void* phi, tdg_stream stream) {
    if (!h || !sigma || !phi || !aligned16(sigma) || !aligned16(phi) || sigma == phi) return TDG_ERR_INVALID_ARG;
    Plan& p = h->p;
    if (!p.built || !p.spec_phi) return TDG_ERR_NOT_BUILT;
    DeviceGuard g(p.device);
    if (!g.ok) return TDG_ERR_CUDA;
    tdg_status st = ensure_workspace(p);
    if (st != TDG_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (p.prec == TDG_FP64)
        e = launch_potential<double>(p, (const double*)sigma, (double*)phi, p.work, s);
    else
        e = launch_potential<float>(p, (const float*)sigma, (float*)phi, p.work, s);
    return from_cuda(e);
}

tdg_status tdg_radial_diagnostics(tdg_plan h, const void* fx, const void* fy, double x0, double y0, void* fr,
                                  const void* ref_fx, const void* ref_fr, double* norms, tdg_stream stream) {
    if (!h || !fx || !fy || !aligned16(fx) || !aligned16(fy)) return TDG_ERR_INVALID_ARG;
    if (!isfinite(x0) || !isfinite(y0)) return TDG_ERR_INVALID_ARG;
    if ((norms != nullptr) != (ref_fx != nullptr) || (ref_fr && !ref_fx)) return TDG_ERR_INVALID_ARG;
    if (!fr && !norms) return TDG_ERR_INVALID_ARG;
    Plan& p = h->p;
    DeviceGuard g(p.device);
    if (!g.ok) return TDG_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (norms && !p.diag) {
        e = cudaMalloc(&p.diag, (6 * (size_t)kDiagMaxBlocks + 6) * sizeof(double));
        if (e != cudaSuccess) return from_cuda(e);
    }
    double* part = p.diag;
    double* out = p.diag ? p.diag + 6 * (size_t)kDiagMaxBlocks : nullptr;
    if (p.prec == TDG_FP64)
        e = launch_radial<double>(p, (const double*)fx, (const double*)fy, x0, y0, (double*)fr, (const double*)ref_fx,
                                  (const double*)ref_fr, part, out, s);
    else
        e = launch_radial<float>(p, (const float*)fx, (const float*)fy, x0, y0, (float*)fr, (const float*)ref_fx,
                                 (const float*)ref_fr, part, out, s);
    if (e != cudaSuccess) return from_cuda(e);
    if (norms) {
        double tmp[6];
        if ((e = cudaMemcpyAsync(tmp, out, sizeof(tmp), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return from_cuda(e);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return from_cuda(e);
        for (int q = 0; q < 6; ++q) norms[q] = tmp[q];
        if (!ref_fr) norms[3] = norms[4] = norms[5] = 0.0;
    }
    return TDG_OK;
}

tdg_status tdg_solve_adjoint(tdg_plan h, const void* gfx, const void* gfy, void* gsigma, tdg_stream stream) {
    if (!h) return TDG_ERR_INVALID_ARG;
    Plan& p = h->p;
    tdg_status st = check_solve_args(p, gfx, gfy, gsigma);
    if (st != TDG_OK) return st;
    if (gsigma == gfx || gsigma == gfy) return TDG_ERR_INVALID_ARG;
    DeviceGuard g(p.device);
    if (!g.ok) return TDG_ERR_CUDA;
    if ((st = ensure_workspace(p)) != TDG_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (p.prec == TDG_FP64)
        e = launch_adjoint<double>(p, (const double*)gfx, (const double*)gfy, (double*)gsigma, p.work, s);
    else
        e = launch_adjoint<float>(p, (const float*)gfx, (const float*)gfy, (float*)gsigma, p.work, s);
    return from_cuda(e);
}

tdg_status tdg_solve_forces_batched(const tdg_plan* plans, int count, const void* const* sigma, void* const* fx,
                                    void* const* fy, tdg_stream stream) {
    if (count == 0 && plans) return TDG_OK;
    tdg_batch b = nullptr;
    tdg_status st = tdg_batch_create(&b, plans, count, sigma, fx, fy);
    if (st != TDG_OK) return st;
    st = tdg_batch_launch(b, stream);
    tdg_status st2 = tdg_batch_destroy(b);
    return st != TDG_OK ? st : st2;
}

tdg_status tdg_get_device_error(tdg_plan h) {
    if (!h) return TDG_ERR_INVALID_ARG;
    Plan& p = h->p;
    if (!p.err) return TDG_OK;
    DeviceGuard g(p.device);
    int v = 0;
    cudaError_t e = cudaMemcpy(&v, p.err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return from_cuda(e);
    if (v != 0) cudaMemset(p.err, 0, sizeof(int));
    return (tdg_status)v;
}

tdg_status tdg_copy_kernel_tables(const tdg_plan h, double* wx, double* wy) {
    if (!h || !wx || !wy) return TDG_ERR_INVALID_ARG;
    const Plan& p = h->p;
    if (!p.built) return TDG_ERR_NOT_BUILT;
    DeviceGuard g(p.device);
    size_t n = (size_t)p.nx * p.ny;
    cudaError_t e = cudaMemcpy(wx, p.wq, n * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(wy, p.wq + n, n * sizeof(double), cudaMemcpyDeviceToHost);
    return from_cuda(e);
}

tdg_status tdg_kernel_entry_host(int order, int m, int n, double dx, double dy, int component, double* out) {
    if (!out || order < 1 || order > 5 || component < 0 || component > 2) return TDG_ERR_INVALID_ARG;
    if (!(dx > 0.0) || !(dy > 0.0) || !isfinite(dx) || !isfinite(dy)) return TDG_ERR_INVALID_ARG;
    if (component == 2) {  // the potential kernel, even in m and n
        *out = entry_phi(order, m < 0 ? -m : m, n < 0 ? -n : n, dx, dy, host_rules().rules);
        return TDG_OK;
    }
    if (component == 1) {  // w^y(m, n; dx, dy) = w^x(n, m; dy, dx)
        int t = m;
        m = n;
        n = t;
        double d = dx;
        dx = dy;
        dy = d;
    }
    // the quadrant m, n >= 0 by symmetry: odd in the force direction, even across it
    double sign = m < 0 ? -1.0 : 1.0;
    int am = m < 0 ? -m : m, an = n < 0 ? -n : n;
    *out = sign * entry_x(order, am, an, dx, dy, host_rules().rules);
    return TDG_OK;
}

tdg_status tdg_set_pass_events(tdg_plan h, void* const* events, int count) {
    if (!h || (count != 0 && count != 4) || (count == 4 && !events)) return TDG_ERR_INVALID_ARG;
    Plan& p = h->p;
    for (int i = 0; i < count; ++i)
        if (!events[i]) return TDG_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i) p.ev[i] = reinterpret_cast<cudaEvent_t>(events[i]);
    p.n_ev = count;
    return TDG_OK;
}

tdg_status tdg_plan_info(const tdg_plan h, int* px, int* py, int* order, int* precision) {
    if (!h) return TDG_ERR_INVALID_ARG;
    if (px) *px = h->p.ax.P;
    if (py) *py = h->p.ay.P;
    if (order) *order = h->p.order;
    if (precision) *precision = (int)h->p.prec;
    return TDG_OK;
}

int tdg_plan_path(const tdg_plan h) {
    if (!h) return -1;
    if (h->p.spec_half && h->p.net_tw) return h->p.prec == TDG_FP32_TC16 ? 3 : 2;
    return 0;
}

tdg_status tdg_destroy(tdg_plan h) {
    if (!h) return TDG_ERR_INVALID_ARG;
    Plan& p = h->p;
    {
        DeviceGuard g(p.device);
        if (p.built || p.work_owned) cudaDeviceSynchronize();
        free_plan_memory(p);
    }
    delete h;
    return TDG_OK;
}

}  // extern "C"
