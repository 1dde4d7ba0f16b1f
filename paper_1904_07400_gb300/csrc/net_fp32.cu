// FP32 force solve (and its adjoint) for grids whose sides are multiples of 16 from 128 to
// 4096 cells, padded to transform lengths L in {256, 512, 1024, 2048, 4096}, built around
// the one-barrier register FFT network of fft_net.cuh and the data movement of sm_103a
// (lines of 256 points are half a warp: their kernels run two lines per 32-thread block):
//
//  * pass A (rows): chunked register spline solve, packed real transform, unpack, and
//    16-byte stores of the row's cells into the tiled intermediate Z (rows of 2048 and
//    4096 points in pairs: the rows at adjacent positions of Z, sigma by TMA, each tile's
//    two cells with one 32-byte store);
//  * pass B (columns): chunked register spline solve, the zero-padded column transform as
//    two half-length transforms (even and odd frequencies), both spectrum products and
//    four inverse half-length transforms, with the spectra stored in the network's
//    output order;
//  * pass C (rows): TMA bulk-tensor load of one row of G (of a pair of rows, as 32-byte
//    pieces, for 2048 and 4096 points), Hermitian repack, transform, crop and store.
//
// The padded transforms use the zero padding exactly (no length-2N transform is formed)
// and the spectra use their parity in kx (half of each half table is stored).
//
// Intermediates Z, G_x, G_y: nx x hy complex values in two-column tiles, element
// (row, ky) at [ky / 2][row][ky % 2].  For order 3, Z stores row i at position
// (i % 16) * (nx / 16) + i / 16, so a column block's thread t reads its rows 16 t .. 16 t + 15
// (the chunk its spline solve owns) with coalesced loads.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "fft_net.cuh"
#include "tdg_internal.cuh"

namespace tdg {
namespace {

using net::cf;
using reg::pad;

// Tile widths (complex values per row of a tile) of the intermediates.  Row passes move
// one tile cell per tile, so wider tiles mean fewer, larger cells for them, while the column
// pass's stores then touch more cache lines per warp; measured at 4096^2, widening G to
// four columns saved pass C 10 us and cost pass B 52 us, so both stay at two.
constexpr int kTW = 2;  // Z (pass A -> pass B) and the adjoint's intermediates
constexpr int kGW = 2;  // G_x, G_y (pass B -> pass C)


// ---------------------------------------------------------------------------------------
// Spline coefficients by the truncated interpolation solve along a line of length 16 T,
// thread t owning the chunk [16 t, 16 t + 16) in registers (c = 0 outside the line).
// Scaled matrices A c = S s (Sec. 2.3; orders 4 and 5 the same condition with the wider
// stencils): order 3 tridiag(1, 6, 1), S = 8; order 4 tridiag(1, 4, 1), S = 6; order 5
// pentadiag(1, 76, 230, 76, 1), S = 384.
//
// Tridiagonal, exact LU: y_0 = S s_0, y_i = S s_i - lam_{i-1} y_{i-1}; c_{n-1} =
// lam_{n-1} y_{n-1}, c_i = lam_i (y_i - c_{i+1}), lam_i = 1 / d_i, d_0 = D, d_i = D -
// 1 / d_{i-1}.  Pentadiagonal, exact L D L^T with subdiagonals l1_i, l2_i: y_i = S s_i -
// l1_i y_{i-1} - l2_i y_{i-2}; c_i = y_i / D_i - l1_{i+1} c_{i+1} - l2_{i+2} c_{i+2}.  The
// factors reach their limits to float precision within the first chunk (exact there).
//
// Each thread sweeps its chunk from zero in both directions (first chunk: exact factors).
// The true values differ from the local ones by the homogeneous solutions driven by the
// chunk edges: tridiagonal c = c_local + Y h + C g (Y = y at the end of the previous chunk,
// C = c at the start of the next one); pentadiagonal the same with two values per edge,
// c = c_local + Y1 h1 + Y2 h2 + C1 g1 + C2 g2.  Y and C are the neighbours' local values
// (their own corrections are rho^16 relative, rho the slowest root: 6e-13, 7e-10, 9e-8 for
// orders 3, 4, 5), exchanged by shuffles and, across warps, through shared memory with one
// barrier.
// ---------------------------------------------------------------------------------------
template <int ORD>
struct TriSpec;
template <>
struct TriSpec<3> {
    static constexpr double D = 6.0, S = 8.0;
};
template <>
struct TriSpec<4> {
    static constexpr double D = 4.0, S = 6.0;
};
constexpr int kTriExact = 8;   // rows of the first chunk with their exact LU factor
constexpr int kPentaExact = 10;

__host__ __device__ constexpr double tri_lam(double D, int i) {
    double d = D;
    for (int k = 0; k < i; ++k) d = D - 1.0 / d;
    return 1.0 / d;
}

// the tridiagonal solve's constants, folded at compile time
struct TriTabs {
    float h[16], g[16], lam[kTriExact], lamInf, S;
};
template <int ORD>
__host__ __device__ constexpr TriTabs make_tri_tabs() {
    TriTabs s{};
    constexpr double D = TriSpec<ORD>::D;
    const double li = tri_lam(D, 80);
    double pw[18] = {};  // (-lam)^k
    pw[0] = 1.0;
    for (int k = 1; k < 18; ++k) pw[k] = -li * pw[k - 1];
    // h_r: backward local sweep of e_r = (-lam)^(r+1)
    double c = li * pw[16];
    s.h[15] = (float)c;
    for (int q = 14; q >= 0; --q) {
        c = li * (pw[q + 1] - c);
        s.h[q] = (float)c;
    }
    for (int r = 0; r < 16; ++r) s.g[r] = (float)pw[16 - r];
    for (int i = 0; i < kTriExact; ++i) s.lam[i] = (float)tri_lam(D, i);
    s.lamInf = (float)li;
    s.S = (float)TriSpec<ORD>::S;
    return s;
}

// exact L D L^T factors of pentadiag(1, 76, 230, 76, 1), row i
struct PentaRow {
    double l1, l2, D;
};
__host__ __device__ constexpr PentaRow penta_row(int i) {
    double Dm2 = 0.0, Dm1 = 0.0, l1m1 = 0.0;
    PentaRow r{0.0, 0.0, 230.0};
    for (int k = 0; k <= i; ++k) {
        const double l2 = k >= 2 ? 1.0 / Dm2 : 0.0;
        const double l1 = k >= 1 ? (76.0 - l2 * l1m1 * Dm2) / Dm1 : 0.0;
        const double D = 230.0 - l1 * l1 * Dm1 - l2 * l2 * Dm2;
        r = PentaRow{l1, l2, D};
        Dm2 = Dm1;
        Dm1 = D;
        l1m1 = l1;
    }
    return r;
}

struct PentaTabs {
    float h1[16], h2[16], g1[16], g2[16];
    float l1[kPentaExact], l2[kPentaExact], rD[kPentaExact];
    float l1i, l2i, rDi;
};
__host__ __device__ constexpr PentaTabs make_penta_tabs() {
    PentaTabs s{};
    const PentaRow inf = penta_row(120);
    const double l1 = inf.l1, l2 = inf.l2, rD = 1.0 / inf.D;
    // forward responses to the incoming y_{-1} (phi) and y_{-2} (psi)
    double phi[16] = {}, psi[16] = {};
    {
        double a1 = 1.0, a2 = 0.0, b1 = 0.0, b2 = 1.0;  // (y_{r-1}, y_{r-2}) of phi and psi
        for (int r = 0; r < 16; ++r) {
            phi[r] = -l1 * a1 - l2 * a2;
            psi[r] = -l1 * b1 - l2 * b2;
            a2 = a1;
            a1 = phi[r];
            b2 = b1;
            b1 = psi[r];
        }
    }
    // backward sweeps from a zero future (h1, h2) and of a unit c_16 or c_17 (g1, g2)
    double c1a = 0.0, c2a = 0.0, c1b = 0.0, c2b = 0.0;  // c_{r+1}, c_{r+2} of h1 / h2
    double d1a = 1.0, d2a = 0.0, d1b = 0.0, d2b = 1.0;  // c_{r+1}, c_{r+2} of g1 / g2
    for (int r = 15; r >= 0; --r) {
        const double ha = phi[r] * rD - l1 * c1a - l2 * c2a;
        const double hb = psi[r] * rD - l1 * c1b - l2 * c2b;
        const double ga = -l1 * d1a - l2 * d2a;
        const double gb = -l1 * d1b - l2 * d2b;
        s.h1[r] = (float)ha;
        s.h2[r] = (float)hb;
        s.g1[r] = (float)ga;
        s.g2[r] = (float)gb;
        c2a = c1a;
        c1a = ha;
        c2b = c1b;
        c1b = hb;
        d2a = d1a;
        d1a = ga;
        d2b = d1b;
        d1b = gb;
    }
    for (int i = 0; i < kPentaExact; ++i) {
        const PentaRow r = penta_row(i);
        s.l1[i] = (float)r.l1;
        s.l2[i] = (float)r.l2;
        s.rD[i] = (float)(1.0 / r.D);
    }
    s.l1i = (float)l1;
    s.l2i = (float)l2;
    s.rDi = (float)rD;
    return s;
}

__device__ __forceinline__ float vs(float a, float s) { return a * s; }
__device__ __forceinline__ cf vs(cf a, float s) { return scl(a, s); }
__device__ __forceinline__ float vfma(float a, float s, float b) { return fmaf(a, s, b); }
__device__ __forceinline__ cf vfma(cf a, float s, cf b) { return mk(fmaf(a.x, s, b.x), fmaf(a.y, s, b.y)); }
__device__ __forceinline__ float vzero(float) { return 0.f; }
__device__ __forceinline__ cf vzero(cf) { return mk(0.f, 0.f); }
__device__ __forceinline__ float shfl_up1(float a) { return __shfl_up_sync(0xffffffffu, a, 1); }
__device__ __forceinline__ cf shfl_up1(cf a) {
    return mk(__shfl_up_sync(0xffffffffu, a.x, 1), __shfl_up_sync(0xffffffffu, a.y, 1));
}
__device__ __forceinline__ float shfl_down1(float a) { return __shfl_down_sync(0xffffffffu, a, 1); }
__device__ __forceinline__ cf shfl_down1(cf a) {
    return mk(__shfl_down_sync(0xffffffffu, a.x, 1), __shfl_down_sync(0xffffffffu, a.y, 1));
}

// x: the thread's chunk (in: s, out: c).  The line has 16 nact values (threads t < nact
// own them; the others hold zeros and get zeros back).  edge: 4 * (nthreads / 32) values
// of shared memory.  Called by all nthreads threads of the block (one __syncthreads).
template <int ORD, typename V>
__device__ __forceinline__ void solve_chunk_tri(V* x, int t, int nact, int nthreads, V* edge) {
    constexpr TriTabs K = make_tri_tabs<ORD>();
    const float li = K.lamInf;
    // forward sweep from zero (exact start on the first chunk)
    x[0] = vs(x[0], K.S);
#pragma unroll
    for (int r = 1; r < 16; ++r) {
        const float l = (t == 0 && r - 1 < kTriExact) ? K.lam[r - 1] : li;
        x[r] = vs(x[r], K.S) - vs(x[r - 1], l);
    }
    const V ylast = x[15];
    // backward sweep from zero (lam_{n-1} = lam: exact on the last chunk)
    x[15] = vs(x[15], li);
#pragma unroll
    for (int r = 14; r >= 0; --r) {
        const float l = (t == 0 && r < kTriExact) ? K.lam[r] : li;
        x[r] = vs(x[r] - x[r + 1], l);
    }
    const V cfirst = x[0];
    // neighbours' edge values
    const int lane = t & 31, w = t >> 5, nw = nthreads >> 5;
    V yprev = shfl_up1(ylast);
    V cnext = shfl_down1(cfirst);
    if (lane == 31) edge[w] = ylast;
    if (lane == 0) edge[nw + w] = cfirst;
    __syncthreads();
    if (lane == 0) yprev = w > 0 ? edge[w - 1] : vzero(ylast);
    if (lane == 31) cnext = w + 1 < nw ? edge[nw + w + 1] : vzero(ylast);
    const V Y = t > 0 ? yprev : vzero(ylast);
    const V C = t + 1 < nact ? vfma(ylast, K.h[0], cnext) : vzero(ylast);
    const float keep = t < nact ? 1.0f : 0.0f;
#pragma unroll
    for (int r = 0; r < 16; ++r) x[r] = vs(vfma(C, K.g[r], vfma(Y, K.h[r], x[r])), keep);
}

template <typename V>
__device__ __forceinline__ void solve_chunk_penta(V* x, int t, int nact, int nthreads, V* edge) {
    constexpr PentaTabs K = make_penta_tabs();
    const bool first = t == 0;
    // forward sweep from zero (exact factors on the first chunk)
    x[0] = vs(x[0], 384.f);
    x[1] = vs(x[1], 384.f) - vs(x[0], first ? K.l1[1] : K.l1i);
#pragma unroll
    for (int r = 2; r < 16; ++r) {
        const bool ex = first && r < kPentaExact;
        x[r] = vs(x[r], 384.f) - vs(x[r - 1], ex ? K.l1[r] : K.l1i) - vs(x[r - 2], ex ? K.l2[r] : K.l2i);
    }
    const V y1 = x[15], y2 = x[14];
    // backward sweep from a zero future (exact on the last chunk: c_n = c_{n+1} = 0)
    x[15] = vs(x[15], K.rDi);
    x[14] = vs(x[14], K.rDi) - vs(x[15], K.l1i);
#pragma unroll
    for (int r = 13; r >= 0; --r) {
        const bool ex = first && r + 2 < kPentaExact;
        const float rd = (first && r < kPentaExact) ? K.rD[r] : K.rDi;
        const float a1 = (first && r + 1 < kPentaExact) ? K.l1[r + 1] : K.l1i;
        const float a2 = ex ? K.l2[r + 2] : K.l2i;
        x[r] = vs(x[r], rd) - vs(x[r + 1], a1) - vs(x[r + 2], a2);
    }
    const V c0 = x[0], c1 = x[1];
    // neighbours' edge values: y_15, y_14 of the previous chunk, c_0, c_1 of the next
    const int lane = t & 31, w = t >> 5, nw = nthreads >> 5;
    V Y1 = shfl_up1(y1), Y2 = shfl_up1(y2);
    V N0 = shfl_down1(c0), N1 = shfl_down1(c1);
    if (lane == 31) {
        edge[w] = y1;
        edge[nw + w] = y2;
    }
    if (lane == 0) {
        edge[2 * nw + w] = c0;
        edge[3 * nw + w] = c1;
    }
    __syncthreads();
    if (lane == 0) {
        Y1 = w > 0 ? edge[w - 1] : vzero(y1);
        Y2 = w > 0 ? edge[nw + w - 1] : vzero(y1);
    }
    if (lane == 31) {
        N0 = w + 1 < nw ? edge[2 * nw + w + 1] : vzero(y1);
        N1 = w + 1 < nw ? edge[3 * nw + w + 1] : vzero(y1);
    }
    if (t == 0) {
        Y1 = vzero(y1);
        Y2 = vzero(y1);
    }
    const bool more = t + 1 < nact;
    const V C1 = more ? vfma(y2, K.h2[0], vfma(y1, K.h1[0], N0)) : vzero(y1);
    const V C2 = more ? vfma(y2, K.h2[1], vfma(y1, K.h1[1], N1)) : vzero(y1);
    const float keep = t < nact ? 1.0f : 0.0f;
#pragma unroll
    for (int r = 0; r < 16; ++r)
        x[r] = vs(vfma(C2, K.g2[r], vfma(C1, K.g1[r], vfma(Y2, K.h2[r], vfma(Y1, K.h1[r], x[r])))), keep);
}

// order known at compile time (the forward kernels are instantiated per order)
template <int ORD, typename V>
__device__ __forceinline__ void solve_chunk_o(V* x, int t, int nact, int nthreads, V* edge) {
    if constexpr (ORD == 5)
        solve_chunk_penta<V>(x, t, nact, nthreads, edge);
    else
        solve_chunk_tri<ORD, V>(x, t, nact, nthreads, edge);
}

// order 3, 4 or 5 (uniform across the block)
template <typename V>
__device__ __forceinline__ void solve_chunk(V* x, int t, int nact, int nthreads, V* edge, int order) {
    if (order == 5)
        solve_chunk_penta<V>(x, t, nact, nthreads, edge);
    else if (order == 4)
        solve_chunk_tri<4, V>(x, t, nact, nthreads, edge);
    else
        solve_chunk_tri<3, V>(x, t, nact, nthreads, edge);
}

// ---------------------------------------------------------------------------------------
// TMA (cp.async.bulk.tensor) and mbarrier helpers
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// bounded wait for phase `parity` of the barrier: false after about a second of naps
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    const unsigned a = smem_u32(bar);
    for (int it = 0; it < (1 << 20); ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (it > 64) __nanosleep(1000);
    }
    return false;
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// generic-proxy shared-memory writes become visible to the async proxy (TMA, tensor core)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void flag_error(int* err, int code) {
    if (err) atomicCAS(err, 0, code);
}

constexpr int kBox = 256;  // tile cells per TMA box (the box-dimension limit)

// shared values of the chunked spline solve's edge exchange (solve_chunk_*): four per warp
// of the line's threads, and four for a line of half a warp (T = 16)
template <int T>
__host__ __device__ constexpr int edge_slots() {
    return 4 * (T / 32 > 0 ? T / 32 : 1);
}

// ---------------------------------------------------------------------------------------
// Tensor memory (tcgen05) as a per-thread stash of 16 complex values: warp w uses TMEM
// lanes 32 (w % 4) .. + 31 (one per thread) and 32 columns starting at 32 (w / 4).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(unsigned* slot, unsigned ncols) {  // one whole warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {  // one whole warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_store16(unsigned a, const cf* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(a),
        "f"(v[0].x), "f"(v[0].y), "f"(v[1].x), "f"(v[1].y), "f"(v[2].x), "f"(v[2].y), "f"(v[3].x), "f"(v[3].y),
        "f"(v[4].x), "f"(v[4].y), "f"(v[5].x), "f"(v[5].y), "f"(v[6].x), "f"(v[6].y), "f"(v[7].x), "f"(v[7].y),
        "f"(v[8].x), "f"(v[8].y), "f"(v[9].x), "f"(v[9].y), "f"(v[10].x), "f"(v[10].y), "f"(v[11].x), "f"(v[11].y),
        "f"(v[12].x), "f"(v[12].y), "f"(v[13].x), "f"(v[13].y), "f"(v[14].x), "f"(v[14].y), "f"(v[15].x),
        "f"(v[15].y)
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// four complex values (8 columns) at column offset of a; no wait
__device__ __forceinline__ void tmem_store4_nowait(unsigned a, const cf* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(a),
                 "f"(v[0].x), "f"(v[0].y), "f"(v[1].x), "f"(v[1].y), "f"(v[2].x), "f"(v[2].y), "f"(v[3].x),
                 "f"(v[3].y)
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_load4(unsigned a, cf* v) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(v[0].x), "=f"(v[0].y), "=f"(v[1].x), "=f"(v[1].y), "=f"(v[2].x), "=f"(v[2].y),
                   "=f"(v[3].x), "=f"(v[3].y)
                 : "r"(a)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_load16(unsigned a, cf* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=f"(v[0].x), "=f"(v[0].y), "=f"(v[1].x), "=f"(v[1].y), "=f"(v[2].x), "=f"(v[2].y), "=f"(v[3].x),
          "=f"(v[3].y), "=f"(v[4].x), "=f"(v[4].y), "=f"(v[5].x), "=f"(v[5].y), "=f"(v[6].x), "=f"(v[6].y),
          "=f"(v[7].x), "=f"(v[7].y), "=f"(v[8].x), "=f"(v[8].y), "=f"(v[9].x), "=f"(v[9].y), "=f"(v[10].x),
          "=f"(v[10].y), "=f"(v[11].x), "=f"(v[11].y), "=f"(v[12].x), "=f"(v[12].y), "=f"(v[13].x), "=f"(v[13].y),
          "=f"(v[14].x), "=f"(v[14].y), "=f"(v[15].x), "=f"(v[15].y)
        : "r"(a)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 16 values (16 columns) at a; no wait
__device__ __forceinline__ void tmem_store16f_nowait(unsigned a, const float* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(a),
        "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]),
        "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15])
        : "memory");
}

// ---------------------------------------------------------------------------------------
// DFT_16 as tensor-core products (the FP32_TC16 form's column pass).  The 16 complex values
// of each thread form one row of A (32 reals: Re x_r, Im x_r at 2 r, 2 r + 1); the forward
// DFT_16 in real form is B (K = 32 inputs x N = 32 outputs); D = A B lands in tensor memory.
// Operands are TF32 (tcgen05.mma kind::tf32, FP32 accumulation), each split into hi + lo:
// hi keeps the top 10 mantissa bits (exact in TF32), lo = x - hi, and three products
// A_hi B_hi + A_lo B_hi + A_hi B_lo keep the error near FP32's (the dropped lo lo term is
// below 2^-20 of the product).  A warp group (128 threads, lanes 0..127) shares one product:
// its threads store their rows, meet at a named barrier, one thread issues the twelve MMAs
// (K = 8 each) and commits them to the group's mbarrier, and every thread reads its row of
// D back.  Tensor memory of a group (column c0): A_hi [c0, +32), A_lo [+32, +64),
// D [+64, +96).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// instruction descriptor: D F32, A and B TF32, both K-major, M = 128, N = 32
constexpr unsigned kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

// shared-memory descriptor of a K-major operand without swizzle: core matrices of 8 rows x
// 16 bytes, LBO = byte step between core matrices along K, SBO = along N
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (unsigned long long)((addr >> 4) & 0x3FFF) | ((unsigned long long)((lbo >> 4) & 0x3FFF) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma_tf32_ts(unsigned d, unsigned a, unsigned long long bdesc, int acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %3, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %4, p;\n}" ::"r"(d),
        "r"(a), "l"(bdesc), "r"(acc), "r"(kTcIdesc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// B of the forward DFT_16 in real form, as the kernels stage it in shared memory: element
// (k, n) (input real k = 2 r + part, output real n = 2 q + part) at float offset
// (n / 8) 256 + (k / 4) 32 + (n % 8) 4 + k % 4 (K-major core matrices: LBO 128 B, SBO 1024 B);
// hi at [0, 1024), lo at [1024, 2048)
constexpr int kTcBFloats = 2048;
__global__ void k_tc_bmat(float* __restrict__ b) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 1024) return;
    const int k = e >> 5, n = e & 31;
    const int r = k >> 1, kp = k & 1, q = n >> 1, np = n & 1;
    double sn, cs;
    sincospi(-2.0 * (double)((r * q) & 15) / 16.0, &sn, &cs);  // W_16^(r q) = cs + i sn
    // y_q = sum_r W_16^(r q) x_r: Re y = cs Re x - sn Im x, Im y = sn Re x + cs Im x
    const double w = np == 0 ? (kp == 0 ? cs : -sn) : (kp == 0 ? sn : cs);
    const float hi = tf32_hi((float)w);
    const int off = (n >> 3) * 256 + (k >> 2) * 32 + (n & 7) * 4 + (k & 3);
    b[off] = hi;
    b[1024 + off] = (float)(w - (double)hi);
}

struct TcDft {
    unsigned arow;  // this thread's lane at the group's A_hi column (A_lo + 32, D + 64)
    unsigned a0;    // lane 0 of the group at its A_hi column (the MMA operands)
    unsigned bhi;   // shared address of B hi (B lo at + 4096)
    unsigned long long* bar;  // the group's mbarrier
    int* err;
    int g;          // warp group (named barrier 1 + g)
    bool leader;    // the group's thread that issues the MMAs
    unsigned ph;    // phase of the group's next mbarrier completion

    template <int R>
    __device__ __forceinline__ void stage(cf* v) {
        if constexpr (R != 16) {
            reg::butterflies<R>(v);
        } else {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float hi[16], lo[16];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const cf x = v[8 * h + i];
                    hi[2 * i] = tf32_hi(x.x);
                    hi[2 * i + 1] = tf32_hi(x.y);
                    lo[2 * i] = x.x - hi[2 * i];
                    lo[2 * i + 1] = x.y - hi[2 * i + 1];
                }
                tmem_store16f_nowait(arow + 16 * h, hi);
                tmem_store16f_nowait(arow + 32 + 16 * h, lo);
            }
            tmem_wait_st();
            tmem_fence_before();
            asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory");
            if (leader) {
                tmem_fence_after();
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) mma_tf32_ts(a0 + 64, a0 + 8 * ks, smem_desc(bhi + 256 * ks, 128, 1024), ks);
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)
                    mma_tf32_ts(a0 + 64, a0 + 32 + 8 * ks, smem_desc(bhi + 256 * ks, 128, 1024), 1);
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)
                    mma_tf32_ts(a0 + 64, a0 + 8 * ks, smem_desc(bhi + 4096 + 256 * ks, 128, 1024), 1);
                mma_commit(bar);
            }
            if (!mbar_wait(bar, ph)) flag_error(err, TDG_ERR_TIMEOUT);
            ph ^= 1u;
            tmem_fence_after();
            tmem_load16(arow + 64, v);
        }
    }
};

// ---------------------------------------------------------------------------------------
// Tables
// ---------------------------------------------------------------------------------------
// per-thread twiddle bases of the network: [0, T) W_L^perm(t), [T, 2T) W_{16R}^(t / 16)
template <int L>
__global__ void k_net_bases(cf* tab) {
    constexpr int T = L / 16, R = L / 256;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    double s, c;
    sincospi(-2.0 * (double)net::perm<L>(t) / (double)L, &s, &c);
    tab[t] = mk((float)c, (float)s);
    sincospi(-2.0 * (double)(t >> 4) / (double)(16 * R), &s, &c);
    tab[T + t] = mk((float)c, (float)s);
}

// half spectra in the network's output order, per ky: the even half (X_e, kx = 2k) as
// rows k_a < 8 of T entries (entry k_a T + t holds k = perm(t) + T k_a) then k = L/2 and a
// pad entry; the odd half (X_o, kx = 2k + 1) as rows k_a < 8.  Values (s_x, s_y).
template <int L>
__global__ void k_net_spectra(const float* __restrict__ full, int hy, float2* __restrict__ half) {
    constexpr int T = L / 16, HS = L / 2 + 2, Px = 2 * L;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)hy * 2 * HS) return;
    const int ky = (int)(idx / (2 * HS));
    const int rem = (int)(idx % (2 * HS));
    const int h = rem / HS, q = rem % HS;
    int kx = -1;
    if (q < L / 2) kx = 2 * (net::perm<L>(q % T) + T * (q / T)) + h;
    else if (q == L / 2 && h == 0) kx = L;
    float2 v = make_float2(0.f, 0.f);
    if (kx >= 0) {
        v.x = full[(size_t)ky * Px + kx];
        v.y = full[(size_t)hy * Px + (size_t)ky * Px + kx];
    }
    half[idx] = v;
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
// pass A: one row i per block (T = L / 16 threads); row length L = ny, transformed as the
// packed complex sequence z_n = s_2n + i s_2n+1 of length L (period 2L, upper half zero).
// Shared memory: E = network buffer; U = the float row for the solve's transposition, later
// Z in padded natural order for the unpack; edge.  Each thread unpacks its cells
// (X[2p], X[2p+1]), p = t + T q, and stores them from registers with 16-byte stores: per
// row there are L/2 cells, one per two-column tile, so every store touches its own tile
// whichever unit issues it, and storing from registers needs neither a staging buffer nor
// the block to wait for a bulk copy before it exits.
// ---------------------------------------------------------------------------------------
// ORD: the order of the row solve (0: none), or -1: the order `ord` given at run time.
// The body of one row (thread t of the row's T threads, shared memory `smem`): row i of
// sigma to its unpacked cells, each handed to sink(q, cell) for p = t + T q; returns
// X[L] (valid in thread 0).  A row that is solved comes as the thread's chunk
// s[16 t .. 16 t + 15] (zeros past the row) from load(x); hook() runs once the row's
// transform is done with the network buffer E (after a block barrier), before the unpack.
__device__ __forceinline__ void load_chunk(const float* __restrict__ sigma, int i, int ny, int t, float (&x)[16]) {
    const float4* src = reinterpret_cast<const float4*>(sigma + (size_t)i * ny) + 4 * t;
    const bool in = t < (ny >> 4);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 f = in ? src[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        x[4 * q] = f.x;
        x[4 * q + 1] = f.y;
        x[4 * q + 2] = f.z;
        x[4 * q + 3] = f.w;
    }
}

template <int L, int ORD, class Load, class Hook, class Sink>
__device__ __forceinline__ float rows_body(unsigned char* smem, int t, int ny, int ord, const cf* __restrict__ nb,
                                           const cf* __restrict__ tw, const float* __restrict__ row_plain,
                                           Load&& load, Hook&& hook, Sink&& sink) {
    constexpr int T = L / 16;
    constexpr int BUF = net::Cfg<L>::BUF;
    cf* E = reinterpret_cast<cf*>(smem);
    cf* U = E + BUF;
    float* edge = reinterpret_cast<float*>(U + BUF);
    const net::Bases bs = net::load_bases<L>(nb, t);
    cf v[16];
    const int nact = ny >> 4;  // threads owning a 16-value chunk of the row
    const bool solve = ORD < 0 ? ord != 0 : ORD != 0;
    if (solve) {
        float x[16];
        load(x);
        if constexpr (ORD < 0)
            solve_chunk<float>(x, t, nact, T, edge, ord);
        else if constexpr (ORD != 0)
            solve_chunk_o<ORD, float>(x, t, nact, T, edge);
        // chunk -> natural-strided pairs through U (float index f at f + 4 (f / 32))
        float* uf = reinterpret_cast<float*>(U);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<float4*>(uf + 16 * t + 4 * q + 4 * (t >> 1)) =
                make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
        __syncthreads();
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int n = t + T * c;
            const float2 p = *reinterpret_cast<const float2*>(uf + 2 * n + 4 * (n >> 4));
            v[c] = mk(p.x, p.y);
        }
    } else {
        const float2* row = reinterpret_cast<const float2*>(row_plain);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float2 p = 2 * (t + T * c) < ny ? row[t + T * c] : make_float2(0.f, 0.f);
            v[c] = mk(p.x, p.y);
        }
    }
#pragma unroll
    for (int c = 8; c < 16; ++c) v[c] = mk(0.f, 0.f);
    net::fwd<L>(v, E, bs, t);
    // Z (network order) -> U, natural padded (every thread read its pairs from U before the
    // barrier inside fwd)
    const int pt = net::perm<L>(t);
#pragma unroll
    for (int ka = 0; ka < 16; ++ka) U[pad(pt + T * ka)] = v[ka];
    const float znyq = v[0].x - v[0].y;  // X[L] (thread 0: v[0] = Z[0])
    __syncthreads();
    hook();
    // cells p = t + T q: (X[2p], X[2p+1]) with X[k] = unpack(Z[k], Z[L-k], W_2L^k)
    const cf w2t = reg::ld_tw(tw, 2 * t);  // W_2L^(2t)
    const cf w1 = reg::ld_tw(tw, 1);       // W_2L
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int p = t + T * q;
        const int k0 = 2 * p;
        const cf wk0 = reg::mul_w16(w2t, q);  // W_2L^(2t + 2Tq), 2T = L / 8
        const cf wk1 = cmul(wk0, w1);
        const cf x0 = unpack_r2c(U[pad(k0)], U[pad((L - k0) & (L - 1))], wk0);
        const cf x1 = unpack_r2c(U[pad(k0 + 1)], U[pad(L - k0 - 1)], wk1);
        sink(q, make_float4(x0.x, x0.y, x1.x, x1.y));
    }
    return znyq;
}

// Z row position of sigma row i: for solves of order >= 3 row i sits at (i % 16) (nx / 16) +
// i / 16, so that the column pass's thread t reads its 16-row solve chunk from consecutive
// positions; otherwise at i
__device__ __forceinline__ int row_pos(int i, int rowmap, int nx) { return rowmap ? (i & 15) * (nx >> 4) + (i >> 4) : i; }
__device__ __forceinline__ int pos_row(int rp, int rowmap, int nx) {
    return rowmap ? 16 * (rp % (nx >> 4)) + rp / (nx >> 4) : rp;
}

// One row: row i of sigma, its cells stored to tile p of row position row_pos(i) with one
// 16-byte store each.  Used by k_net_rows and by the batched persistent kernel.
template <int L, int ORD>
__device__ __forceinline__ void rows_item(unsigned char* smem, int t, int i, const float* __restrict__ sigma, int ny,
                                          int ord, int rowmap, int nx, const cf* __restrict__ nb,
                                          const cf* __restrict__ tw, cf* __restrict__ z) {
    constexpr int T = L / 16;
    cf* zr = z + (size_t)row_pos(i, rowmap, nx) * kTW;
    const float* row = sigma + (size_t)i * ny;
    const float znyq = rows_body<L, ORD>(
        smem, t, ny, ord, nb, tw, row, [&](float(&x)[16]) { load_chunk(sigma, i, ny, t, x); }, [] {},
        [&](int q, float4 c) { *reinterpret_cast<float4*>(zr + (size_t)(t + T * q) * nx * kTW) = c; });
    if (t == 0) zr[(size_t)(L / 2) * nx * kTW] = mk(znyq, 0.f);
}

template <int L, int ORD>
__global__ void __launch_bounds__(L / 16, 3)
    k_net_rows(const float* __restrict__ sigma, int ny, int ord, int rowmap, int nx, const cf* __restrict__ nb,
               const cf* __restrict__ tw, cf* __restrict__ z) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    rows_item<L, ORD>(smem_raw, threadIdx.x, blockIdx.x, sigma, ny, ord, rowmap, nx, nb, tw, z);
}

__device__ __forceinline__ void st_global_v8(void* p, float4 a, float4 b) {
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(a.x), "f"(a.y), "f"(a.z),
                 "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
                 : "memory");
}

// Pass A on pairs of row positions (2b, 2b + 1), one pair per block: the rows that sit at
// adjacent positions of Z share every 32-byte sector of Z, so the block transforms both and
// writes each tile's two cells with one 32-byte store.  The first row's cells wait in tensor
// memory (32 columns per thread: warp w at lanes 32 (w % 4), columns 32 (w / 4)) while the
// second row is transformed.  nx even (every side on the network path is a multiple of 16).
//
// Rows that are solved (order >= 3) and span whole 128-byte pieces (ny % 32 == 0, smap
// valid: sma != 0) arrive by TMA, one box per row, into the network buffer E under the
// 128-byte swizzle (the box's inner extent is the swizzle span, so its footprint is the
// dense row): thread t's chunk is the two halves of piece t / 2, 16-byte unit u of a piece
// at u ^ (piece % 8), so that the eight threads of a quarter-warp read eight different
// bank groups.  The first row's load is issued at the start, the second row's as soon as
// the first row's transform is done with E.  Shared memory: rows_bytes, then the mbarrier
// and the tensor-memory address.
template <int L>
constexpr size_t rows2_bytes() {
    return (size_t)2 * net::Cfg<L>::BUF * sizeof(cf) + edge_slots<L / 16>() * sizeof(float) + 16;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

template <int L, int ORD>
__global__ void __launch_bounds__(L / 16, 3)
    k_net_rows2(const __grid_constant__ CUtensorMap smap, int sma, const float* __restrict__ sigma, int ny, int ord,
                int rowmap, int nx, const cf* __restrict__ nb, const cf* __restrict__ tw, cf* __restrict__ z,
                int* __restrict__ err) {
    constexpr int T = L / 16;
    constexpr int BUF = net::Cfg<L>::BUF;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned long long* bar =
        reinterpret_cast<unsigned long long*>(smem_raw + 2 * BUF * sizeof(cf) + edge_slots<T>() * sizeof(float));
    unsigned* tslot = reinterpret_cast<unsigned*>(bar + 1);
    const int t = threadIdx.x;
    const bool solve = ORD < 0 ? ord != 0 : ORD != 0;
    const bool tma = solve && sma != 0;
    const int rp = 2 * blockIdx.x;
    const int i0 = pos_row(rp, rowmap, nx), i1 = pos_row(rp + 1, rowmap, nx);
    if (t < 32) tmem_alloc(tslot, 64);
    if (t == 0 && tma) {
        mbar_init(bar, 1);
        mbar_expect_tx(bar, (unsigned)(ny * sizeof(float)));
        tma_load_3d(smem_raw, &smap, 0, 0, i0, bar);
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const unsigned ta = *tslot + ((unsigned)(32 * ((t >> 5) & 3)) << 16) + 32u * (unsigned)(t >> 7);
    cf* zr = z + (size_t)rp * kTW;
    unsigned ph = 0;
    auto load = [&](int i, float(&x)[16]) {
        if (!tma) {
            load_chunk(sigma, i, ny, t, x);
            return;
        }
        if (!mbar_wait(bar, ph)) {
            flag_error(err, TDG_ERR_TIMEOUT);
            mbar_wait(bar, ph);  // a late copy lands before E is reused
        }
        ph ^= 1u;
        const float4* e = reinterpret_cast<const float4*>(smem_raw) + 8 * (t >> 1);
        const int sw = (t >> 1) & 7, h = 4 * (t & 1);
        const bool in = t < (ny >> 4);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 f = in ? e[(h + q) ^ sw] : make_float4(0.f, 0.f, 0.f, 0.f);
            x[4 * q] = f.x;
            x[4 * q + 1] = f.y;
            x[4 * q + 2] = f.z;
            x[4 * q + 3] = f.w;
        }
    };
    // row at position rp: its cells to tensor memory
    {
        float4 c0[8];
        const float znyq = rows_body<L, ORD>(
            smem_raw, t, ny, ord, nb, tw, sigma + (size_t)i0 * ny, [&](float(&x)[16]) { load(i0, x); },
            [&] {
                if (t == 0 && tma) {  // E is free: the second row's load
                    fence_async_smem();
                    mbar_expect_tx(bar, (unsigned)(ny * sizeof(float)));
                    tma_load_3d(smem_raw, &smap, 0, 0, i1, bar);
                }
            },
            [&](int q, float4 c) { c0[q] = c; });
        tmem_store16(ta, reinterpret_cast<const cf*>(c0));
        if (t == 0) zr[(size_t)(L / 2) * nx * kTW] = mk(znyq, 0.f);
    }
    // row at position rp + 1: each tile's two cells with one store.  No barrier between the
    // rows: the first row last read the edge values before its transposition barrier and E
    // before its unpack barrier, which every thread has passed, and this row writes U only
    // after a barrier of its own (its solve's or its transform's), which no thread reaches
    // before finishing the first row's unpack
    cf c0[16];
    const float znyq = rows_body<L, ORD>(
        smem_raw, t, ny, ord, nb, tw, sigma + (size_t)i1 * ny, [&](float(&x)[16]) { load(i1, x); }, [] {},
        [&](int q, float4 c) {
            if (q == 0) tmem_load16(ta, c0);
            st_global_v8(zr + (size_t)(t + T * q) * nx * kTW,
                         make_float4(c0[2 * q].x, c0[2 * q].y, c0[2 * q + 1].x, c0[2 * q + 1].y), c);
        });
    if (t == 0) zr[(size_t)(L / 2) * nx * kTW + kTW] = mk(znyq, 0.f);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (t < 32) tmem_dealloc(*tslot, 64);
}

// ---------------------------------------------------------------------------------------
// pass C: rows i of one component at a time.  A row's L/kGW tile cells arrive by TMA, its
// Nyquist value by a plain load.  Shared memory: S = the row (L + 2 complex values),
// E = network buffer, bar = the row's mbarrier.
// ---------------------------------------------------------------------------------------
template <int L>
constexpr int inv_e_offset() {
    constexpr int a = L >= 512 ? 1024 : 128;  // 256-length rows: four of them share a batch block
    return (((L + 2) * 8 + a - 1) / a) * a;   // bytes
}


// Persistent: each block walks the (row, component) items b, b + G, ..., issuing the next
// item's TMA load as soon as every thread has repacked the current one, so that the load
// overlaps the transform and the stores.  The cropped output goes back through E (the
// network buffer), since S by then receives the next row.
template <int L>
__global__ void __launch_bounds__(L / 16, 3)
    k_net_rows_inv(const __grid_constant__ CUtensorMap gmap, const cf* __restrict__ g0,
                     const cf* __restrict__ g1, int nx, int ny, const cf* __restrict__ nb, const cf* __restrict__ tw,
                     float* __restrict__ f0, float* __restrict__ f1, int* __restrict__ err) {
    constexpr int T = L / 16;
    constexpr int BUF = net::Cfg<L>::BUF;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    cf* S = reinterpret_cast<cf*>(smem_raw);
    cf* E = reinterpret_cast<cf*>(smem_raw + inv_e_offset<L>());
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(E + BUF);
    const int t = threadIdx.x;
    const int nitems = 2 * nx;
    int w = blockIdx.x;
    if (w >= nitems) return;
    // thread 0: start moving item `it` into S (cells by TMA, the Nyquist cell by hand)
    auto issue = [&](int it) {
        const int i = it % nx, comp = it / nx;
        constexpr int kB = L / kGW < kBox ? L / kGW : kBox;  // cells per box
        mbar_expect_tx(bar, (unsigned)(L * sizeof(cf)));
#pragma unroll 1
        for (int b = 0; b < L / kGW / kB; ++b) tma_load_4d(S + kGW * b * kB, &gmap, 0, i, b * kB, comp, bar);
        const cf* g = comp ? g1 : g0;
        S[L] = ld2(g + (size_t)(L / kGW) * nx * kGW + (size_t)i * kGW);  // read back by thread 0 only
    };
    if (t == 0) mbar_init(bar, 1);
    __syncthreads();
    if (t == 0) issue(w);
    const net::Bases bs = net::load_bases<L>(nb, t);
    const cf wt = reg::ld_tw(tw, t);
    const int pt = net::perm<L>(t);
    unsigned ph = 0;
    for (; w < nitems; w += gridDim.x, ph ^= 1u) {
        const int i = w % nx, comp = w / nx;
        const int ok = __syncthreads_and(mbar_wait(bar, ph) ? 1 : 0);
        if (!ok) {
            if (t == 0) flag_error(err, TDG_ERR_TIMEOUT);
            mbar_wait(bar, ph);
            return;
        }
        cf v[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int k = t + T * r;
            v[r] = conjg(pack_c2r(S[k], S[L - k], reg::twist(wt, r)));
        }
        net::fwd<L>(v, E, bs, t);  // its barrier: every thread is done with S
        if (t == 0 && w + (int)gridDim.x < nitems) issue(w + gridDim.x);
        __syncthreads();  // every half-warp is done with its slab of E
#pragma unroll
        for (int ka = 0; ka < 8; ++ka) E[pad(pt + T * ka)] = conjg(v[ka]);
        __syncthreads();
        float2* out = reinterpret_cast<float2*>((comp ? f1 : f0) + (size_t)i * ny);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int n = t + T * c;
            const cf o = E[pad(n)];
            if (2 * n < ny) out[n] = make_float2(o.x, o.y);  // crop to the grid
        }
    }
}

// Pass C on pairs of rows (2j, 2j + 1) of one component, for the long rows (L >= 2048).
// Rows 2j and 2j + 1 are adjacent in every tile of G, so one TMA box over the pair view of G
// (32-byte pieces: both rows' cells of a tile) brings both, with half as many pieces as
// two single-row loads.  S holds the pair as [tile][row][column] (4 complex per tile) under
// the TMA's 32-byte swizzle, which exchanges the two 16-byte halves of a tile (the rows)
// when bit 2 of the tile index is set, and the two Nyquist values at 2L and 2L + 2: value
// k of row r sits at 4 p + 2 (r ^ (p / 4 % 2)) + k % 2, p = k / 2, for every k <= L.  Without
// the swizzle, tiles p and p + 4 read by one half-warp would fall in the same banks.  The
// second row, repacked, waits in tensor memory
// (32 columns per thread, as in pass A's pairs) while the first is transformed and stored.
// Persistent over the items w = (component, pair), the next item's load issued as soon as
// both rows are repacked.
template <int L>
constexpr int inv2_e_offset() {
    return (((2 * L + 4) * 8 + 1023) / 1024) * 1024;  // bytes
}

template <int L>
__global__ void __launch_bounds__(L / 16, 2)
    k_net_rows_inv2(const __grid_constant__ CUtensorMap gmap2, const cf* __restrict__ g0, const cf* __restrict__ g1,
                    int nx, int ny, const cf* __restrict__ nb, const cf* __restrict__ tw, float* __restrict__ f0,
                    float* __restrict__ f1, int* __restrict__ err) {
    constexpr int T = L / 16;
    constexpr int BUF = net::Cfg<L>::BUF;
    constexpr int kB = L / 2 < kBox ? L / 2 : kBox;  // tiles per box
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    cf* S = reinterpret_cast<cf*>(smem_raw);
    cf* E = reinterpret_cast<cf*>(smem_raw + inv2_e_offset<L>());
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(E + BUF);
    unsigned* tslot = reinterpret_cast<unsigned*>(bar + 1);
    const int t = threadIdx.x;
    const int npair = nx >> 1;
    const int nitems = 2 * npair;
    if ((int)blockIdx.x >= nitems) return;
    if (t < 32) tmem_alloc(tslot, 64);
    // thread 0: start moving item `it` into S (both rows' cells by TMA, the Nyquist values by hand)
    auto issue = [&](int it) {
        const int j = it % npair, comp = it / npair;
        mbar_expect_tx(bar, (unsigned)(2 * L * sizeof(cf)));
#pragma unroll 1
        for (int b = 0; b < L / 2 / kB; ++b) tma_load_4d(S + 4 * b * kB, &gmap2, 0, j, b * kB, comp, bar);
        const cf* g = (comp ? g1 : g0) + (size_t)(L / 2) * nx * kGW + (size_t)(2 * j) * kGW;
        S[2 * L] = ld2(g);  // read back after the next item's barrier
        S[2 * L + 2] = ld2(g + kGW);
    };
    if (t == 0) mbar_init(bar, 1);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const unsigned ta = *tslot + ((unsigned)(32 * ((t >> 5) & 3)) << 16) + 32u * (unsigned)(t >> 7);
    if (t == 0) issue(blockIdx.x);
    const net::Bases bs = net::load_bases<L>(nb, t);
    const cf wt = reg::ld_tw(tw, t);
    const int pt = net::perm<L>(t);
    // k = t + T r and its mirror L - k: as T r is a multiple of 16, the tile index moves by
    // T r / 2 and the swizzle bit and column parity are the thread's own
    const int sk = (t >> 3) & 1, sm = ((L - t) >> 3) & 1;
    const cf* Sk = S + 4 * (t >> 1) + (t & 1);
    const cf* Sm = S + 4 * ((L - t) >> 1) + (t & 1);
    unsigned ph = 0;
    for (int w = blockIdx.x; w < nitems; w += gridDim.x, ph ^= 1u) {
        const int j = w % npair, comp = w / npair;
        const int ok = __syncthreads_and(mbar_wait(bar, ph) ? 1 : 0);
        if (!ok) {
            if (t == 0) flag_error(err, TDG_ERR_TIMEOUT);
            mbar_wait(bar, ph);  // the load in flight lands before the block leaves
            break;
        }
        cf v[16];
        // both rows, four values at a time: the first row's to registers, the second row's
        // to tensor memory
#pragma unroll
        for (int r0 = 0; r0 < 16; r0 += 4) {
            cf u[4];
#pragma unroll
            for (int r = r0; r < r0 + 4; ++r) {
                const cf wr = reg::twist(wt, r);
                v[r] = conjg(pack_c2r(Sk[2 * T * r + 2 * sk], Sm[-2 * T * r + 2 * sm], wr));
                u[r - r0] = conjg(pack_c2r(Sk[2 * T * r + 2 * (sk ^ 1)], Sm[-2 * T * r + 2 * (sm ^ 1)], wr));
            }
            tmem_store4_nowait(ta + 2 * r0, u);
        }
        tmem_wait_st();
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            if (h == 1) tmem_load16(ta, v);
            net::fwd<L>(v, E, bs, t);  // its barrier: every thread is done with S (h = 0)
            if (h == 0 && t == 0 && w + (int)gridDim.x < nitems) issue(w + gridDim.x);
            __syncthreads();  // every half-warp is done with its slab of E
#pragma unroll
            for (int ka = 0; ka < 8; ++ka) E[pad(pt + T * ka)] = conjg(v[ka]);
            __syncthreads();
            float2* out = reinterpret_cast<float2*>((comp ? f1 : f0) + (size_t)(2 * j + h) * ny);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int n = t + T * c;
                const cf o = E[pad(n)];
                if (2 * n < ny) out[n] = make_float2(o.x, o.y);  // crop to the grid
            }
            // E is read before the next transform writes it: the second row's reads are
            // separated from the next item's transform by the barrier at the top of the loop
            if (h == 0) __syncthreads();
        }
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (t < 32) tmem_dealloc(*tslot, 64);
}

// Pass C body for the batched persistent kernel: row i of one component of G (cells of two
// columns, 16-byte loads into S), then the repack, transform, crop and store of
// k_net_rows_inv.  Shared memory as k_net_rows_inv (S, then E at inv_e_offset).
template <int L>
__device__ __forceinline__ void inv_item(unsigned char* smem, int t, int i, const cf* __restrict__ g, int nx, int ny,
                                         const cf* __restrict__ nb, const cf* __restrict__ tw, float* __restrict__ f) {
    constexpr int T = L / 16;
    cf* S = reinterpret_cast<cf*>(smem);
    cf* E = reinterpret_cast<cf*>(smem + inv_e_offset<L>());
    const cf* gr = g + (size_t)i * kGW;
#pragma unroll
    for (int q = 0; q < L / 2 / T; ++q) {
        const int p = t + T * q;
        *reinterpret_cast<float4*>(S + 2 * p) = __ldg(reinterpret_cast<const float4*>(gr + (size_t)p * nx * kGW));
    }
    if (t == 0) S[L] = ld2(gr + (size_t)(L / 2) * nx * kGW);
    __syncthreads();
    const net::Bases bs = net::load_bases<L>(nb, t);
    const cf wt = reg::ld_tw(tw, t);
    const int pt = net::perm<L>(t);
    cf v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int k = t + T * r;
        v[r] = conjg(pack_c2r(S[k], S[L - k], reg::twist(wt, r)));
    }
    net::fwd<L>(v, E, bs, t);
    __syncthreads();  // every half-warp is done with its slab of E
#pragma unroll
    for (int ka = 0; ka < 8; ++ka) E[pad(pt + T * ka)] = conjg(v[ka]);
    __syncthreads();
    float2* out = reinterpret_cast<float2*>(f + (size_t)i * ny);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int n = t + T * c;
        const cf o = E[pad(n)];
        if (2 * n < ny) out[n] = make_float2(o.x, o.y);
    }
}

// twiddle factors kept in tensor memory: 32 columns of stage-2 factors at a2, 32 of
// stage-3 factors at a3 (16 complex values each, in the order the network applies them)
template <int L>
struct TmemTw {
    unsigned a2, a3;
    // v[i] *= f[i] where the factor is not 1 (i % G != 0)
    template <int G>
    __device__ __forceinline__ static void mul16(cf* v, unsigned a) {
        cf f[16];
        tmem_load16(a, f);
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (i % G) v[i] = cmul(v[i], f[i]);
    }
    __device__ __forceinline__ void apply2(cf* v) const { mul16<net::Cfg<L>::R>(v, a2); }
    __device__ __forceinline__ void apply3(cf* v) const { mul16<16>(v, a3); }
};

// ---------------------------------------------------------------------------------------
// pass B: one frequency column ky per block, column length L = nx.
//
// Spectra (k_net_spectra): per ky the even half then the odd half, HS = L/2 + 2 entries
// each, in network order.  The products are conj(i s X) (the inverse transforms run as
// conj(inv_t(conj(.)))).  For fixed ky, s_x is odd and s_y even in kx, so entries past
// the middle of a half come from the mirrored entry, with s_x negated.
//
// Only the 16 values of the transform in flight live in registers; the rest waits in
// tensor memory (tcgen05.st / tcgen05.ld, 32 columns a slot, warps w and w + 4 sharing
// the lane quarter w % 4) or in shared memory:
//   slot A: the even half's y product, then the even y result;
//   slot B: the twisted column x_n W_2L^n, then the odd half's y product;
//   xb (shared): the column (and the solve's transposition), then the even x result;
//   4096-cell columns: the stage-2 and stage-3 twiddle factors, formed once per block, in
//   two more slots (256 columns a block, two blocks an SM: the whole tensor memory).
// ---------------------------------------------------------------------------------------
// Per-thread stash of 16 complex values: tensor memory (32 columns of the thread's lane)
// for columns of 1024 cells and more; shared memory ([r][t], the thread's own slots) for
// 512, whose one-warp blocks would need more tensor memory per SM than there is.
template <int L, bool TM = (L >= 1024)>
struct Stash {
    static constexpr bool kTmem = TM;
    unsigned ta;  // tensor memory address of the slot (kTmem)
    cf* sa;       // shared slot base (!kTmem): element r of thread t at sa[r T + t]
    int t;
    __device__ __forceinline__ void store16(const cf* v) const {
        if constexpr (kTmem) {
            tmem_store16(ta, v);
        } else {
#pragma unroll
            for (int r = 0; r < 16; ++r) sa[r * (L / 16) + t] = v[r];
        }
    }
    __device__ __forceinline__ void load16(cf* v) const {
        if constexpr (kTmem) {
            tmem_load16(ta, v);
        } else {
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = sa[r * (L / 16) + t];
        }
    }
    // group g of four values (r = 4 g .. 4 g + 3); stores complete at store_done()
    __device__ __forceinline__ void store4(int g, const cf* v) const {
        if constexpr (kTmem) {
            tmem_store4_nowait(ta + 8 * g, v);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) sa[(4 * g + e) * (L / 16) + t] = v[e];
        }
    }
    __device__ __forceinline__ void store_done() const {
        if constexpr (kTmem) tmem_wait_st();
    }
    __device__ __forceinline__ void load4(int g, cf* v) const {
        if constexpr (kTmem) {
            tmem_load4(ta + 8 * g, v);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = sa[(4 * g + e) * (L / 16) + t];
        }
    }
};

template <int L, int H, typename ST>
__device__ __forceinline__ void spec_products(cf* v, const float2* __restrict__ sh, int t, int pt, int tm,
                                              const ST& ys) {
    constexpr int T = L / 16;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        cf y[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int ka = 4 * g + e;
            int idx;
            bool direct;
            if (ka < 8) {
                idx = ka * T + t;
                direct = true;
            } else if (H == 0 && pt == 0) {
                idx = (16 - ka) * T;  // k = T ka, mirror T (16 - ka); ka = 8 is the middle itself
                direct = ka == 8;
            } else {
                idx = (15 - ka) * T + tm;
                direct = false;
            }
            const float2 q = __ldg(sh + idx);
            const float sx = direct ? q.x : -q.x;
            const float sy = q.y;
            const cf x = v[ka];
            v[ka] = mk(-sx * x.y, -sx * x.x);  // x product, stays in v
            y[e] = mk(-sy * x.y, -sy * x.x);   // y product, to the stash
        }
        ys.store4(g, y);
    }
    ys.store_done();
}

template <int L>
constexpr bool cols_twiddles_in_tmem() {
    return L == 4096;
}

template <int L>
constexpr size_t cols_smem_bytes() {
    constexpr int T = L / 16, BUF = net::Cfg<L>::BUF;
    return (size_t)(2 * BUF) * sizeof(cf) + edge_slots<T>() * sizeof(cf) + 16 +
           (Stash<L>::kTmem ? 0 : (size_t)2 * 16 * T * sizeof(cf));
}

// column length nx <= L (a multiple of 16); Z, G_x, G_y hold nx rows
// ORD: the order of the column solve (0: none), or -1: the order `ord` given at run time.
// 1024-cell columns keep five blocks an
// SM (registers capped at 204), as they had before the solve order was compiled in: the
// batched streams form relies on blocks of many small grids sharing the SMs
template <int L>
constexpr int cols_min_blocks() {
    return L == 1024 ? 5 : 2;
}
// The body of one column (thread t of the column's T threads, shared memory `smem`), used by
// k_net_cols and by the batched persistent kernel: column kl of Z, G_x, G_y (as stored) and
// ky of the spectra; rows at or past nstore are not stored.  TM: the stashes in tensor
// memory (its address at *tslot, published to every thread by the body's first barrier).
template <int L, int ORD, bool TM = (L >= 1024)>
__device__ __forceinline__ void cols_item(unsigned char* smem, int t, int kl, int ky, const cf* __restrict__ z,
                                          int nx, int nstore, int ord, const cf* __restrict__ nb,
                                          const cf* __restrict__ tw, const float2* __restrict__ spec,
                                          cf* __restrict__ gx, cf* __restrict__ gy, const unsigned* tslot) {
    constexpr int T = L / 16;
    constexpr int BUF = net::Cfg<L>::BUF;
    constexpr int HS = L / 2 + 2;
    constexpr bool kTm = TM;
    constexpr bool kTwt = cols_twiddles_in_tmem<L>();
    constexpr unsigned kWarpCols = kTwt ? 128 : 64;
    cf* E = reinterpret_cast<cf*>(smem);  // network buffer
    cf* xb = E + BUF;                     // the column (padded natural), later the even x result
    cf* edge = xb + BUF;
    cf* sslots = reinterpret_cast<cf*>(reinterpret_cast<unsigned*>(edge + edge_slots<T>()) + 4);  // shared stash slots A, B
    const int tile = kl >> 1, c = kl & 1;
    const size_t slab = (size_t)nx * kTW;
    const cf* zc = z + (size_t)tile * slab + c;
    const float2* se = spec + (size_t)ky * 2 * HS;
    const float2* so = se + HS;
    if (t == 0) {
        // the column's spectra are read after the solve and the first transform
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(se), "r"((unsigned)(2 * HS * sizeof(float2)))
                     : "memory");
    }
    const net::Bases bs = net::load_bases<L>(nb, t);
    const int nact = nx >> 4;
    cf v[16];
    const bool solve = ORD < 0 ? ord != 0 : ORD != 0;
    if (solve) {
#pragma unroll
        for (int r = 0; r < 16; ++r)  // row 16 t + r sits at r (nx / 16) + t
            v[r] = t < nact ? ld2(zc + (size_t)(r * nact + t) * kTW) : mk(0.f, 0.f);
        if constexpr (ORD < 0)
            solve_chunk<cf>(v, t, nact, T, edge, ord);
        else if constexpr (ORD != 0)
            solve_chunk_o<ORD, cf>(v, t, nact, T, edge);
#pragma unroll
        for (int r = 0; r < 16; ++r) xb[pad(16 * t + r)] = v[r];
        tmem_fence_before();
        __syncthreads();  // also publishes the tensor-memory address
        tmem_fence_after();
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = xb[pad(t + r * T)];
    } else {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int n = t + r * T;
            v[r] = n < nx ? ld2(zc + (size_t)n * kTW) : mk(0.f, 0.f);
        }
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
    }
    // tensor-memory lanes of this hardware warp (a block may run one column per warp)
    const unsigned tA = kTm ? *tslot + ((unsigned)(32 * ((threadIdx.x >> 5) & 3)) << 16) +
                                  kWarpCols * (unsigned)(threadIdx.x >> 7)
                            : 0u;
    const Stash<L, kTm> sA{tA, sslots, t};
    const Stash<L, kTm> sB{tA + 32, sslots + 16 * T, t};
    const TmemTw<L> tt{tA + 64, tA + 96};
    if constexpr (kTwt) {
        cf f[16], g[16];
        net::stage_factors<L>(bs, f, g);
        tmem_store16(tt.a2, f);
        tmem_store16(tt.a3, g);
    }
    auto FWD = [&](cf* vv) {
        if constexpr (kTwt) net::fwd_p<L>(vv, E, tt, t);
        else net::fwd<L>(vv, E, bs, t);
    };
    auto INV = [&](cf* vv) {
        if constexpr (kTwt) net::inv_t_p<L>(vv, E, tt, t);
        else net::inv_t<L>(vv, E, bs, t);
    };
    const int pt = net::perm<L>(t);
    const int te = pt == 0 ? 0 : net::perm_inv<L>(T - pt);  // even half: mirror of k is L - k
    const int to = net::perm_inv<L>(T - 1 - pt);             // odd half: mirror of k is L - 1 - k
    // the odd half's input x_n W_2L^n waits in slot B
    {
        const cf wt = reg::ld_tw(tw, t);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            cf y[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) y[e] = cmul(v[4 * g + e], reg::twist(wt, 4 * g + e));
            sB.store4(g, y);
        }
        sB.store_done();
    }
    // even frequencies X_e = FFT_L(x)
    FWD(v);
    spec_products<L, 0>(v, se, t, pt, te, sA);
    INV(v);
    // every thread read its column values from xb before the first barrier of FWD
#pragma unroll
    for (int r = 0; r < 16; ++r) xb[pad(t + r * T)] = v[r];  // even x result, own slots
    sA.load16(v);
    __syncthreads();
    INV(v);
    sA.store16(v);  // even y result
    sB.load16(v);   // x W_2L^n
    __syncthreads();
    // odd frequencies X_o = FFT_L(x_n W_2L^n)
    FWD(v);
    spec_products<L, 1>(v, so, t, pt, to, sB);
    INV(v);
    // G = conj(u_even + W_2L^n u_odd); W_2L^n as conj of W_2L^-n (table entry 2L - t);
    // rows past the grid are not stored
    const cf wtc = reg::ld_tw(tw, (2 * L - t) & (2 * L - 1));
    cf* gxc = gx + (size_t)(kl / kGW) * nx * kGW + kl % kGW;
    cf* gyc = gy + (size_t)(kl / kGW) * nx * kGW + kl % kGW;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int n = t + r * T;
        if (n < nstore) gxc[(size_t)n * kGW] = conjg(xb[pad(n)] + cmulc(v[r], reg::untwist(wtc, r)));
    }
    sB.load16(v);
    __syncthreads();
    INV(v);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        cf ey[4];
        sA.load4(g, ey);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int r = 4 * g + e;
            const int n = t + r * T;
            if (n < nstore) gyc[(size_t)n * kGW] = conjg(ey[e] + cmulc(v[r], reg::untwist(wtc, r)));
        }
    }
}

template <int L, int ORD>
__global__ void __launch_bounds__(L / 16, cols_min_blocks<L>())
    k_net_cols(const cf* __restrict__ z, int nx, int ord, const cf* __restrict__ nb, const cf* __restrict__ tw,
               const float2* __restrict__ spec, cf* __restrict__ gx, cf* __restrict__ gy, int ky0) {
    constexpr int T = L / 16;
    constexpr bool kTm = Stash<L>::kTmem;
    constexpr unsigned kCols = cols_twiddles_in_tmem<L>() ? 256 : (T > 128 ? 128 : 64);
    constexpr int BUF = net::Cfg<L>::BUF;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned* tslot = reinterpret_cast<unsigned*>(reinterpret_cast<cf*>(smem_raw) + 2 * BUF + edge_slots<T>());
    const int t = threadIdx.x;
    if constexpr (kTm) {
        if (t < 32) tmem_alloc(tslot, kCols);
    }
    // column ky0 + b of the spectra; Z, G_x, G_y hold the columns from ky0 on (ky0 even)
    cols_item<L, ORD>(smem_raw, t, blockIdx.x, ky0 + blockIdx.x, z, nx, nx, ord, nb, tw, spec, gx, gy, tslot);
    if constexpr (kTm) {
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
        if (t < 32) tmem_dealloc(*tslot, kCols);
    }
}

// ---------------------------------------------------------------------------------------
// pass B of the FP32_TC16 form (columns of 2048 or 4096 cells): k_net_cols with every
// DFT_16 of the network as tensor-core products (TcDft).  Tensor memory per warp group:
// A_hi, A_lo, D and stash slot B (32 columns each, 128 a group); stash slot A lives in shared
// memory, and the twiddle powers are formed at every stage (tensor memory is full).
// ---------------------------------------------------------------------------------------
template <int L>
constexpr size_t tc_cols_bmat_offset() {  // bytes: E, xb, edge, tensor slot and mbarriers, aligned
    constexpr int T = L / 16, BUF = net::Cfg<L>::BUF;
    return (((size_t)(2 * BUF) * sizeof(cf) + edge_slots<T>() * sizeof(cf) + 32 + 1023) / 1024) * 1024;
}
template <int L>
constexpr size_t tc_cols_smem_bytes() {
    return tc_cols_bmat_offset<L>() + kTcBFloats * sizeof(float) + (size_t)16 * (L / 16) * sizeof(cf);
}

template <int L, int ORD>
__global__ void __launch_bounds__(L / 16, 2)
    k_net_cols_tc(const cf* __restrict__ z, int nx, int ord, const cf* __restrict__ nb, const cf* __restrict__ tw,
                  const float2* __restrict__ spec, const float* __restrict__ bmat, cf* __restrict__ gx,
                  cf* __restrict__ gy, int* __restrict__ err) {
    constexpr int T = L / 16;
    constexpr int BUF = net::Cfg<L>::BUF;
    constexpr int HS = L / 2 + 2;
    constexpr unsigned kCols = T;  // 128 columns per warp group
    static_assert(T == 128 || T == 256, "columns of 2048 or 4096 cells");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    cf* E = reinterpret_cast<cf*>(smem_raw);  // network buffer
    cf* xb = E + BUF;                         // the column (padded natural), later the even x result
    cf* edge = xb + BUF;
    unsigned* tslot = reinterpret_cast<unsigned*>(edge + edge_slots<T>());
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(tslot + 4);  // one per warp group
    float* bsm = reinterpret_cast<float*>(smem_raw + tc_cols_bmat_offset<L>());
    cf* sslot = reinterpret_cast<cf*>(bsm + kTcBFloats);  // stash slot A, [r][t]
    const int t = threadIdx.x;
    if (t < 32) tmem_alloc(tslot, kCols);
    if (t == 0) {
        mbar_init(bars, 1);
        mbar_init(bars + 1, 1);
    }
    // B (hi, lo) into shared memory, seen by the tensor core's proxy after the barrier below
    for (int i = t; i < kTcBFloats / 4; i += T)
        reinterpret_cast<float4*>(bsm)[i] = __ldg(reinterpret_cast<const float4*>(bmat) + i);
    fence_async_smem();
    const int ky = blockIdx.x;
    const int tile = ky >> 1, c = ky & 1;
    const size_t slab = (size_t)nx * kTW;
    const cf* zc = z + (size_t)tile * slab + c;
    const float2* se = spec + (size_t)ky * 2 * HS;
    const float2* so = se + HS;
    if (t == 0) {
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(se), "r"((unsigned)(2 * HS * sizeof(float2)))
                     : "memory");
    }
    const net::Bases bs = net::load_bases<L>(nb, t);
    const int nact = nx >> 4;
    cf v[16];
    const bool solve = ORD < 0 ? ord != 0 : ORD != 0;
    if (solve) {
#pragma unroll
        for (int r = 0; r < 16; ++r)  // row 16 t + r sits at r (nx / 16) + t
            v[r] = t < nact ? ld2(zc + (size_t)(r * nact + t) * kTW) : mk(0.f, 0.f);
        if constexpr (ORD < 0)
            solve_chunk<cf>(v, t, nact, T, edge, ord);
        else if constexpr (ORD != 0)
            solve_chunk_o<ORD, cf>(v, t, nact, T, edge);
#pragma unroll
        for (int r = 0; r < 16; ++r) xb[pad(16 * t + r)] = v[r];
        tmem_fence_before();
        __syncthreads();  // also publishes the tensor-memory address, the mbarriers and B
        tmem_fence_after();
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = xb[pad(t + r * T)];
    } else {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int n = t + r * T;
            v[r] = n < nx ? ld2(zc + (size_t)n * kTW) : mk(0.f, 0.f);
        }
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
    }
    const int g = t >> 7;
    const unsigned gcol = *tslot + 128u * (unsigned)g;
    const unsigned arow = gcol + ((unsigned)(32 * ((t >> 5) & 3)) << 16);
    TcDft df{arow, gcol, smem_u32(bsm), bars + g, err, g, (t & 127) == 0, 0u};
    const Stash<L, false> sA{0u, sslot, t};
    const Stash<L, true> sB{arow + 96, nullptr, t};
    const net::GenTw<L> gt{bs};
    auto FWD = [&](cf* vv) { net::fwd_p<L>(vv, E, gt, t, df); };
    auto INV = [&](cf* vv) { net::inv_t_p<L>(vv, E, gt, t, df); };
    const int pt = net::perm<L>(t);
    const int te = pt == 0 ? 0 : net::perm_inv<L>(T - pt);  // even half: mirror of k is L - k
    const int to = net::perm_inv<L>(T - 1 - pt);             // odd half: mirror of k is L - 1 - k
    {
        const cf wt = reg::ld_tw(tw, t);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            cf y[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) y[e] = cmul(v[4 * q + e], reg::twist(wt, 4 * q + e));
            sB.store4(q, y);
        }
        sB.store_done();
    }
    FWD(v);
    spec_products<L, 0>(v, se, t, pt, te, sA);
    INV(v);
#pragma unroll
    for (int r = 0; r < 16; ++r) xb[pad(t + r * T)] = v[r];  // even x result, own slots
    sA.load16(v);
    __syncthreads();
    INV(v);
    sA.store16(v);  // even y result
    sB.load16(v);   // x W_2L^n
    __syncthreads();
    FWD(v);
    spec_products<L, 1>(v, so, t, pt, to, sB);
    INV(v);
    const cf wtc = reg::ld_tw(tw, (2 * L - t) & (2 * L - 1));
    cf* gxc = gx + (size_t)(ky / kGW) * nx * kGW + ky % kGW;
    cf* gyc = gy + (size_t)(ky / kGW) * nx * kGW + ky % kGW;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int n = t + r * T;
        if (n < nx) gxc[(size_t)n * kGW] = conjg(xb[pad(n)] + cmulc(v[r], reg::untwist(wtc, r)));
    }
    sB.load16(v);
    __syncthreads();
    INV(v);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        cf ey[4];
        sA.load4(q, ey);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int r = 4 * q + e;
            const int n = t + r * T;
            if (n < nx) gyc[(size_t)n * kGW] = conjg(ey[e] + cmulc(v[r], reg::untwist(wtc, r)));
        }
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (t < 32) tmem_dealloc(*tslot, kCols);
}

// ---------------------------------------------------------------------------------------
// The adjoint (dL/dsigma for L = sum g_x F^x + g_y F^y): the same passes transposed.
// w^x and w^y are odd in their force direction, so the transpose of each convolution is
// its negation: dL/dC = -(K_x g_x + K_y g_y) on the grid, then the spline solves (T is
// symmetric).  Pass A runs k_net_rows on g_x and g_y (no solve, natural row order).
// ---------------------------------------------------------------------------------------
// conj(-i s X) = i s conj(X) = (s X.y, s X.x) for one component, in place on v; with a
// stash, the stashed partial sum (groups of four) is added
template <int L, int H, typename ST>
__device__ __forceinline__ void adj_products(cf* v, const float2* __restrict__ sh, int t, int pt, int tm, int comp,
                                             const ST* add) {
    constexpr int T = L / 16;
#pragma unroll
    for (int g4 = 0; g4 < 4; ++g4) {
        cf prev[4];
        if (add) add->load4(g4, prev);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int ka = 4 * g4 + e;
            int idx;
            bool direct;
            if (ka < 8) {
                idx = ka * T + t;
                direct = true;
            } else if (H == 0 && pt == 0) {
                idx = (16 - ka) * T;
                direct = ka == 8;
            } else {
                idx = (15 - ka) * T + tm;
                direct = false;
            }
            const float2 q = __ldg(sh + idx);
            const float sv = comp ? q.y : (direct ? q.x : -q.x);
            const cf r = mk(sv * v[ka].y, sv * v[ka].x);
            v[ka] = add ? prev[e] + r : r;
        }
    }
}

// pass B of the adjoint: column ky of Z_x and Z_y (natural rows) -> G column, x solve
// applied, rows stored at the chunk-permuted positions (i % 16) (nx / 16) + i / 16.
// Stashes: A, B in tensor memory (shared slots for 512), C in xb (shared, own slots).
// The body of one column (thread t of the column's T threads, shared memory `smem`, column
// ky); `store` false: the column is computed but nothing is stored (a half-warp that has no
// column of its own in a block of two columns).  TMEM address at *tslot (L >= 1024).
template <int L>
__device__ __forceinline__ void cols_adj_item(unsigned char* smem, int t, int ky, bool store,
                                              const cf* __restrict__ zx, const cf* __restrict__ zy, int nx, int solve,
                                              const cf* __restrict__ nb, const cf* __restrict__ tw,
                                              const float2* __restrict__ spec, cf* __restrict__ g,
                                              const unsigned* tslot) {
    constexpr int T = L / 16;
    constexpr int BUF = net::Cfg<L>::BUF;
    constexpr int HS = L / 2 + 2;
    constexpr bool kTm = Stash<L>::kTmem;
    constexpr bool kTwt = cols_twiddles_in_tmem<L>();
    constexpr unsigned kWarpCols = kTwt ? 128 : 64;
    cf* E = reinterpret_cast<cf*>(smem);  // network buffer
    cf* xb = E + BUF;                     // stash C ([r][t]), then the solve's transposition
    cf* edge = xb + BUF;
    cf* sslots = reinterpret_cast<cf*>(reinterpret_cast<unsigned*>(edge + edge_slots<T>()) + 4);
    const int tile = ky >> 1, c = ky & 1;
    const size_t slab = (size_t)nx * kTW;
    const float2* se = spec + (size_t)ky * 2 * HS;
    const float2* so = se + HS;
    if (t == 0) {
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(se), "r"((unsigned)(2 * HS * sizeof(float2)))
                     : "memory");
    }
    const net::Bases bs = net::load_bases<L>(nb, t);
    tmem_fence_before();
    __syncthreads();  // publishes the tensor-memory address
    tmem_fence_after();
    const unsigned tA = kTm ? *tslot + ((unsigned)(32 * ((t >> 5) & 3)) << 16) + kWarpCols * (unsigned)(t >> 7) : 0u;
    const Stash<L> sA{tA, sslots, t};
    const Stash<L> sB{tA + 32, sslots + 16 * T, t};
    const Stash<L, false> sC{0u, xb, t};  // shared ([r][t], own slots)
    const TmemTw<L> tt{tA + 64, tA + 96};
    if constexpr (kTwt) {
        cf f[16], h[16];
        net::stage_factors<L>(bs, f, h);
        tmem_store16(tt.a2, f);
        tmem_store16(tt.a3, h);
    }
    auto FWD = [&](cf* vv) {
        if constexpr (kTwt) net::fwd_p<L>(vv, E, tt, t);
        else net::fwd<L>(vv, E, bs, t);
    };
    auto INV = [&](cf* vv) {
        if constexpr (kTwt) net::inv_t_p<L>(vv, E, tt, t);
        else net::inv_t<L>(vv, E, bs, t);
    };
    const int pt = net::perm<L>(t);
    const int te = pt == 0 ? 0 : net::perm_inv<L>(T - pt);
    const int to = net::perm_inv<L>(T - 1 - pt);
    const cf wt = reg::ld_tw(tw, t);
    cf v[16];
    auto load_col = [&](const cf* zs) {
        const cf* zc = zs + (size_t)tile * slab + c;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int n = t + r * T;
            v[r] = n < nx ? ld2(zc + (size_t)n * kTW) : mk(0.f, 0.f);
        }
    };
    auto twist_to = [&](const Stash<L>& st) {
#pragma unroll
        for (int g4 = 0; g4 < 4; ++g4) {
            cf y[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) y[e] = cmul(v[4 * g4 + e], reg::twist(wt, 4 * g4 + e));
            st.store4(g4, y);
        }
        st.store_done();
    };
    // g_x: even-half products into A, odd-half products into C (twisted column via B)
    load_col(zx);
    twist_to(sB);
    FWD(v);
    adj_products<L, 0>(v, se, t, pt, te, 0, (const Stash<L>*)nullptr);
    sA.store16(v);
    sB.load16(v);
    __syncthreads();  // fwd then fwd on one buffer
    FWD(v);
    adj_products<L, 1>(v, so, t, pt, to, 0, (const Stash<L>*)nullptr);
    sC.store16(v);
    // g_y: add its products, transform back
    load_col(zy);
    twist_to(sB);
    __syncthreads();
    FWD(v);
    adj_products<L, 0>(v, se, t, pt, te, 1, &sA);
    INV(v);
    sA.store16(v);  // u_even
    sB.load16(v);
    __syncthreads();
    FWD(v);
    adj_products<L, 1>(v, so, t, pt, to, 1, &sC);
    INV(v);
    // u = conj(u_even + W_2L^n u_odd), cropped to the grid
    {
        const cf wtc = reg::ld_tw(tw, (2 * L - t) & (2 * L - 1));
#pragma unroll
        for (int g4 = 0; g4 < 4; ++g4) {
            cf ue[4];
            sA.load4(g4, ue);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int r = 4 * g4 + e;
                const int n = t + r * T;
                v[r] = n < nx ? conjg(ue[e] + cmulc(v[r], reg::untwist(wtc, r))) : mk(0.f, 0.f);
            }
        }
    }
    const int nact = nx >> 4;
    cf* gc = g + (size_t)tile * slab + c;
    if (solve) {
        // natural-strided -> chunks through xb, x solve, rows 16 t + r stored at r (nx/16) + t
        __syncthreads();  // every thread is done with its stash C slots in xb
#pragma unroll
        for (int r = 0; r < 16; ++r) xb[pad(t + r * T)] = v[r];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = xb[pad(16 * t + r)];
        solve_chunk<cf>(v, t, nact, T, edge, solve);
        if (store && t < nact) {
#pragma unroll
            for (int r = 0; r < 16; ++r) gc[(size_t)(r * nact + t) * kTW] = v[r];
        }
    } else if (store) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int n = t + r * T;
            if (n < nx) gc[(size_t)((n & 15) * nact + (n >> 4)) * kTW] = v[r];
        }
    }
}

template <int L>
__global__ void __launch_bounds__(L / 16, 2)
    k_net_cols_adj(const cf* __restrict__ zx, const cf* __restrict__ zy, int nx, int solve,
                   const cf* __restrict__ nb, const cf* __restrict__ tw, const float2* __restrict__ spec,
                   cf* __restrict__ g) {
    constexpr int T = L / 16;
    constexpr int BUF = net::Cfg<L>::BUF;
    constexpr bool kTm = Stash<L>::kTmem;
    constexpr unsigned kCols = cols_twiddles_in_tmem<L>() ? 256 : (T > 128 ? 128 : 64);
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned* tslot = reinterpret_cast<unsigned*>(reinterpret_cast<cf*>(smem_raw) + 2 * BUF + edge_slots<T>());
    const int t = threadIdx.x;
    if constexpr (kTm) {
        if (t < 32) tmem_alloc(tslot, kCols);
    }
    cols_adj_item<L>(smem_raw, t, blockIdx.x, true, zx, zy, nx, solve, nb, tw, spec, g, tslot);
    if constexpr (kTm) {
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
        if (t < 32) tmem_dealloc(*tslot, kCols);
    }
}

template <int L>
constexpr size_t cols_adj_smem_bytes() {
    constexpr int T = L / 16, BUF = net::Cfg<L>::BUF;
    return (size_t)(2 * BUF) * sizeof(cf) + edge_slots<T>() * sizeof(cf) + 16 +
           (Stash<L>::kTmem ? 0 : (size_t)2 * 16 * T * sizeof(cf));
}

// pass C of the adjoint: persistent over rows i of G (stored at the chunk-permuted row
// positions); inverse row transform, crop to ny, y solve, coalesced store of the row
template <int L>
__global__ void __launch_bounds__(L / 16, 3)
    k_net_rows_inv_adj(const __grid_constant__ CUtensorMap gmap, const cf* __restrict__ g, int nx, int ny,
                       int solve, const cf* __restrict__ nb, const cf* __restrict__ tw, float* __restrict__ out,
                       int* __restrict__ err) {
    constexpr int T = L / 16;
    constexpr int BUF = net::Cfg<L>::BUF;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    cf* S = reinterpret_cast<cf*>(smem_raw);
    cf* E = reinterpret_cast<cf*>(smem_raw + inv_e_offset<L>());
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(E + BUF);
    float* edge = reinterpret_cast<float*>(bar + 1);
    const int t = threadIdx.x;
    int i = blockIdx.x;
    if (i >= nx) return;
    const int nq = nx >> 4;
    auto rowpos = [&](int row) { return (row & 15) * nq + (row >> 4); };
    auto issue = [&](int row) {
        mbar_expect_tx(bar, (unsigned)(L * sizeof(cf)));
#pragma unroll 1
        for (int b = 0; b < L / 2 / kBox; ++b) tma_load_4d(S + 2 * b * kBox, &gmap, 0, rowpos(row), b * kBox, 0, bar);
        S[L] = ld2(g + (size_t)(L / 2) * nx * kTW + (size_t)rowpos(row) * kTW);  // read back by thread 0 only
    };
    if (t == 0) mbar_init(bar, 1);
    __syncthreads();
    if (t == 0) issue(i);
    const net::Bases bs = net::load_bases<L>(nb, t);
    const cf wt = reg::ld_tw(tw, t);
    const int pt = net::perm<L>(t);
    const int nact = ny >> 4;
    unsigned ph = 0;
    for (; i < nx; i += gridDim.x, ph ^= 1u) {
        const int ok = __syncthreads_and(mbar_wait(bar, ph) ? 1 : 0);
        if (!ok) {
            if (t == 0) flag_error(err, TDG_ERR_TIMEOUT);
            mbar_wait(bar, ph);
            return;
        }
        cf v[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int k = t + T * r;
            v[r] = conjg(pack_c2r(S[k], S[L - k], reg::twist(wt, r)));
        }
        net::fwd<L>(v, E, bs, t);  // its barrier: every thread is done with S
        if (t == 0 && i + (int)gridDim.x < nx) issue(i + gridDim.x);
        __syncthreads();  // every half-warp is done with its slab of E
#pragma unroll
        for (int ka = 0; ka < 8; ++ka) E[pad(pt + T * ka)] = conjg(v[ka]);
        __syncthreads();
        float* row = out + (size_t)i * ny;
        if (solve) {
            // pairs 8 t .. 8 t + 7 = reals 16 t .. 16 t + 15 of the row
            float x[16];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const cf o = E[pad(8 * t + j)];
                x[2 * j] = o.x;
                x[2 * j + 1] = o.y;
            }
            solve_chunk<float>(x, t, nact, T, edge, solve);  // its barrier: E is read before the next fwd
            if (t < nact) {
                float4* dst = reinterpret_cast<float4*>(row) + 4 * t;
#pragma unroll
                for (int q = 0; q < 4; ++q) dst[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
            }
        } else {
            float2* dst = reinterpret_cast<float2*>(row);
#pragma unroll
            for (int c2 = 0; c2 < 8; ++c2) {
                const int n = t + T * c2;
                const cf o = E[pad(n)];
                if (2 * n < ny) dst[n] = make_float2(o.x, o.y);
            }
        }
    }
}

template <int L>
size_t inv_adj_bytes() {
    return (size_t)inv_e_offset<L>() + net::Cfg<L>::BUF * sizeof(cf) + 16 + edge_slots<L / 16>() * sizeof(float);
}

// ---------------------------------------------------------------------------------------
// The batched persistent kernel on the network item bodies.  Blocks of 64 threads take
// items in list order from an atomic ticket (every row item of every grid, then every column
// item, then every inverse-row item); a column item of grid d waits until all of d's row
// items are finished, an inverse-row item until all its column items are (bounded, about a
// second, then TDG_ERR_TIMEOUT and the item is skipped).  A 1024-length item runs on both
// warps; a 512-length item runs one transform per warp (rows 2 j, 2 j + 1, and likewise).
// The column stashes live in tensor memory: 64 columns a block, warp w on lanes 32 w ...
// ---------------------------------------------------------------------------------------
constexpr int kNetBatchThreads = 64;
constexpr long long kNetSpinLimit = 1000000;  // ~1 s with 1 us naps

template <int L>
constexpr size_t batch_item_bytes() {  // shared memory of one transform's item, any pass
    constexpr size_t a = (size_t)2 * net::Cfg<L>::BUF * sizeof(cf) + edge_slots<L / 16>() * sizeof(float);
    constexpr size_t b = (size_t)2 * net::Cfg<L>::BUF * sizeof(cf) + edge_slots<L / 16>() * sizeof(cf) + 16;
    constexpr size_t c = (size_t)inv_e_offset<L>() + net::Cfg<L>::BUF * sizeof(cf);
    return ((std::max(a, std::max(b, c)) + 1023) / 1024) * 1024;
}
constexpr size_t kNetBatchSmem = std::max(batch_item_bytes<1024>(),
                                          std::max(2 * batch_item_bytes<512>(), 4 * batch_item_bytes<256>()));

__device__ __forceinline__ int find_grid(const int* pref, int count, int item) {
    int lo = 0, hi = count;  // pref[lo] <= item < pref[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (pref[mid] <= item) lo = mid;
        else hi = mid;
    }
    return lo;
}

constexpr int kNetBatchMaxGrids = 256;  // grids whose item prefix sums stay in shared memory

// one out-of-line function per item kind, each running the item's units u0 .. u1 - 1: each
// gets its own register allocation instead of the union of all six in the loop
__device__ __noinline__ void bitem_rows1024(unsigned char* sm, const NetDisk& g, int u0, int u1) {
    for (int u = u0; u < u1; ++u) {
        if (u > u0) __syncthreads();  // the previous unit is done with shared memory
        rows_item<1024, -1>(sm, threadIdx.x, u, g.sigma, g.ny, g.ord, g.ord != 0, g.nx,
                            reinterpret_cast<const cf*>(g.nby), reinterpret_cast<const cf*>(g.twy),
                            reinterpret_cast<cf*>(g.z));
    }
}
__device__ __noinline__ void bitem_rows512(unsigned char* sm, const NetDisk& g, int u0, int u1) {
    const int w = threadIdx.x >> 5;
    for (int u = u0; u < u1; ++u) {
        if (u > u0) __syncthreads();
        rows_item<512, -1>(sm + w * batch_item_bytes<512>(), threadIdx.x & 31, 2 * u + w, g.sigma, g.ny, g.ord,
                           g.ord != 0, g.nx, reinterpret_cast<const cf*>(g.nby), reinterpret_cast<const cf*>(g.twy),
                           reinterpret_cast<cf*>(g.z));
    }
}
__device__ __noinline__ void bitem_cols1024(unsigned char* sm, const NetDisk& g, int u0, int u1, const unsigned* tm) {
    for (int u = u0; u < u1; ++u) {
        if (u > u0) {
            tmem_fence_before();
            __syncthreads();
            tmem_fence_after();
        }
        cols_item<1024, -1, true>(sm, threadIdx.x, u, u, reinterpret_cast<const cf*>(g.z), g.nx, g.nx, g.ord,
                                  reinterpret_cast<const cf*>(g.nbx), reinterpret_cast<const cf*>(g.twx),
                                  reinterpret_cast<const float2*>(g.spec), reinterpret_cast<cf*>(g.gx),
                                  reinterpret_cast<cf*>(g.gy), tm);
    }
}
__device__ __noinline__ void bitem_cols512(unsigned char* sm, const NetDisk& g, int u0, int u1, const unsigned* tm) {
    const int w = threadIdx.x >> 5;
    for (int u = u0; u < u1; ++u) {
        if (u > u0) {
            tmem_fence_before();
            __syncthreads();
            tmem_fence_after();
        }
        const int col = 2 * u + w;  // hy is odd: the second warp of the last unit stores nothing
        const bool real = col < g.hy;
        const int c = real ? col : g.hy - 1;
        cols_item<512, -1, true>(sm + w * batch_item_bytes<512>(), threadIdx.x & 31, c, c,
                                 reinterpret_cast<const cf*>(g.z), g.nx, real ? g.nx : 0, g.ord,
                                 reinterpret_cast<const cf*>(g.nbx), reinterpret_cast<const cf*>(g.twx),
                                 reinterpret_cast<const float2*>(g.spec), reinterpret_cast<cf*>(g.gx),
                                 reinterpret_cast<cf*>(g.gy), tm);
    }
}
__device__ __noinline__ void bitem_inv1024(unsigned char* sm, const NetDisk& g, int u0, int u1) {
    for (int u = u0; u < u1; ++u) {
        if (u > u0) __syncthreads();
        const int comp = u / g.nx, i = u - comp * g.nx;
        inv_item<1024>(sm, threadIdx.x, i, reinterpret_cast<const cf*>(comp ? g.gy : g.gx), g.nx, g.ny,
                       reinterpret_cast<const cf*>(g.nby), reinterpret_cast<const cf*>(g.twy), comp ? g.fy : g.fx);
    }
}
__device__ __noinline__ void bitem_inv512(unsigned char* sm, const NetDisk& g, int u0, int u1) {
    const int w = threadIdx.x >> 5;
    for (int u = u0; u < u1; ++u) {
        if (u > u0) __syncthreads();
        const int rc = 2 * u + w, comp = rc / g.nx, i = rc - comp * g.nx;
        inv_item<512>(sm + w * batch_item_bytes<512>(), threadIdx.x & 31, i,
                      reinterpret_cast<const cf*>(comp ? g.gy : g.gx), g.nx, g.ny, reinterpret_cast<const cf*>(g.nby),
                      reinterpret_cast<const cf*>(g.twy), comp ? g.fy : g.fx);
    }
}

// 256-length lines: one per half-warp, four per unit
__device__ __noinline__ void bitem_rows256(unsigned char* sm, const NetDisk& g, int u0, int u1) {
    const int q = threadIdx.x >> 4;
    for (int u = u0; u < u1; ++u) {
        if (u > u0) __syncthreads();
        rows_item<256, -1>(sm + q * batch_item_bytes<256>(), threadIdx.x & 15, 4 * u + q, g.sigma, g.ny, g.ord,
                           g.ord != 0, g.nx, reinterpret_cast<const cf*>(g.nby), reinterpret_cast<const cf*>(g.twy),
                           reinterpret_cast<cf*>(g.z));
    }
}
__device__ __noinline__ void bitem_cols256(unsigned char* sm, const NetDisk& g, int u0, int u1, const unsigned* tm) {
    const int q = threadIdx.x >> 4;
    for (int u = u0; u < u1; ++u) {
        if (u > u0) {
            tmem_fence_before();
            __syncthreads();
            tmem_fence_after();
        }
        const int col = 4 * u + q;  // past the last column: computed again, not stored
        const bool real = col < g.hy;
        const int c = real ? col : g.hy - 1;
        cols_item<256, -1, true>(sm + q * batch_item_bytes<256>(), threadIdx.x & 15, c, c,
                                 reinterpret_cast<const cf*>(g.z), g.nx, real ? g.nx : 0, g.ord,
                                 reinterpret_cast<const cf*>(g.nbx), reinterpret_cast<const cf*>(g.twx),
                                 reinterpret_cast<const float2*>(g.spec), reinterpret_cast<cf*>(g.gx),
                                 reinterpret_cast<cf*>(g.gy), tm);
    }
}
__device__ __noinline__ void bitem_inv256(unsigned char* sm, const NetDisk& g, int u0, int u1) {
    const int q = threadIdx.x >> 4;
    for (int u = u0; u < u1; ++u) {
        if (u > u0) __syncthreads();
        const int rc = 4 * u + q, comp = rc / g.nx, i = rc - comp * g.nx;
        inv_item<256>(sm + q * batch_item_bytes<256>(), threadIdx.x & 15, i,
                      reinterpret_cast<const cf*>(comp ? g.gy : g.gx), g.nx, g.ny, reinterpret_cast<const cf*>(g.nby),
                      reinterpret_cast<const cf*>(g.twy), comp ? g.fy : g.fx);
    }
}

__global__ void __launch_bounds__(kNetBatchThreads, 6) k_batched_net(NetBatchDev b) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ int s_item, s_ok;
    __shared__ unsigned s_tmem;
    const int t = threadIdx.x;
    if (t < 32) tmem_alloc(&s_tmem, 64);
    // the items' prefix sums after the dynamic shared memory, when the batch is small enough
    const int nstart = 3 * (b.count + 1) + 3 * b.count;  // prefix sums, then the orders
    int* sstart = reinterpret_cast<int*>(smem_raw + kNetBatchSmem);
    const bool local = b.count <= kNetBatchMaxGrids;
    if (local)
        for (int i = t; i < nstart; i += kNetBatchThreads) sstart[i] = b.start[i];
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const int* st = local ? sstart : b.start;
    const int* startA = st;
    const int* startB = st + (b.count + 1);
    const int* startC = st + 2 * (b.count + 1);
    const int totA = startA[b.count], totB = startB[b.count];
    for (;;) {
        if (t == 0) s_item = atomicAdd(b.ticket, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= b.total) break;
        int phase, local_item;
        const int* pref;
        if (item < totA) {
            phase = 0;
            local_item = item;
            pref = startA;
        } else if (item < totA + totB) {
            phase = 1;
            local_item = item - totA;
            pref = startB;
        } else {
            phase = 2;
            local_item = item - totA - totB;
            pref = startC;
        }
        const int pos = find_grid(pref, b.count, local_item);
        const int idx = local_item - pref[pos];
        const int d = st[3 * (b.count + 1) + phase * b.count + pos];
        const NetDisk& g = b.disks[d];
        if (t == 0) {
            int ok = 1;
            if (phase > 0) {
                const int need = phase == 1 ? g.nA : g.nB;
                volatile int* cnt = b.done + (phase - 1) * b.count + d;
                volatile int* errw = b.err;
                long long spins = 0;
                while (*cnt < need) {
                    if (++spins > kNetSpinLimit || *errw != 0) {
                        ok = 0;
                        atomicExch(b.err, (int)TDG_ERR_TIMEOUT);
                        break;
                    }
                    __nanosleep(1000);
                }
                __threadfence();
            }
            s_ok = ok;
        }
        __syncthreads();
        if (s_ok) {
            // this item's units: idx * U .. (a unit is one transform of a 1024-length line, two
            // of a 512-length one, four of a 256-length one)
            const int units = phase == 0 ? g.uA : (phase == 1 ? g.uB : g.uC);
            const int u0 = idx * b.units, u1 = min(u0 + b.units, units);
            if (phase == 0) {
                if (g.ly == 1024) bitem_rows1024(smem_raw, g, u0, u1);
                else if (g.ly == 512) bitem_rows512(smem_raw, g, u0, u1);
                else bitem_rows256(smem_raw, g, u0, u1);
            } else if (phase == 1) {
                if (g.lx == 1024) bitem_cols1024(smem_raw, g, u0, u1, &s_tmem);
                else if (g.lx == 512) bitem_cols512(smem_raw, g, u0, u1, &s_tmem);
                else bitem_cols256(smem_raw, g, u0, u1, &s_tmem);
            } else {
                if (g.ly == 1024) bitem_inv1024(smem_raw, g, u0, u1);
                else if (g.ly == 512) bitem_inv512(smem_raw, g, u0, u1);
                else bitem_inv256(smem_raw, g, u0, u1);
            }
        }
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
        if (t == 0) {
            __threadfence();
            if (!(phase == 0 && d == b.withhold)) atomicAdd(b.done + phase * b.count + d, 1);
        }
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (t < 32) tmem_dealloc(s_tmem, 64);
}

// ---------------------------------------------------------------------------------------
// L = 256: a line is half a warp (T = 16), so these kernels run two lines per 32-thread
// block, each half-warp on its own shared-memory region (the item bodies above, thread
// t = threadIdx.x % 16).  Both halves pass the same block barriers; a half with no line of
// its own (an odd count of columns) computes the last column again and stores nothing.
// ---------------------------------------------------------------------------------------
template <size_t B>
constexpr size_t item_stride() {
    return ((B + 127) / 128) * 128;
}

// pass C of the adjoint for one row i of G (stored at its chunk-permuted position) with
// plain 16-byte loads: the body of k_net_rows_inv_adj for the half-warp lines
template <int L>
constexpr size_t inv_adj_item_bytes() {
    return (size_t)inv_e_offset<L>() + net::Cfg<L>::BUF * sizeof(cf) + edge_slots<L / 16>() * sizeof(float);
}

template <int L>
__device__ __forceinline__ void inv_adj_item(unsigned char* smem, int t, int i, const cf* __restrict__ g, int nx,
                                             int ny, int solve, const cf* __restrict__ nb,
                                             const cf* __restrict__ tw, float* __restrict__ out) {
    constexpr int T = L / 16;
    constexpr int BUF = net::Cfg<L>::BUF;
    cf* S = reinterpret_cast<cf*>(smem);
    cf* E = reinterpret_cast<cf*>(smem + inv_e_offset<L>());
    float* edge = reinterpret_cast<float*>(E + BUF);
    const int nq = nx >> 4;
    const cf* gr = g + (size_t)((i & 15) * nq + (i >> 4)) * kTW;
#pragma unroll
    for (int q = 0; q < L / 2 / T; ++q) {
        const int p = t + T * q;
        *reinterpret_cast<float4*>(S + 2 * p) = __ldg(reinterpret_cast<const float4*>(gr + (size_t)p * nx * kTW));
    }
    if (t == 0) S[L] = ld2(gr + (size_t)(L / 2) * nx * kTW);
    __syncthreads();
    const net::Bases bs = net::load_bases<L>(nb, t);
    const cf wt = reg::ld_tw(tw, t);
    const int pt = net::perm<L>(t);
    cf v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int k = t + T * r;
        v[r] = conjg(pack_c2r(S[k], S[L - k], reg::twist(wt, r)));
    }
    net::fwd<L>(v, E, bs, t);
    __syncthreads();  // every half-warp is done with its slab of E
#pragma unroll
    for (int ka = 0; ka < 8; ++ka) E[pad(pt + T * ka)] = conjg(v[ka]);
    __syncthreads();
    float* row = out + (size_t)i * ny;
    if (solve) {
        // pairs 8 t .. 8 t + 7 = reals 16 t .. 16 t + 15 of the row
        const int nact = ny >> 4;
        float x[16];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const cf o = E[pad(8 * t + j)];
            x[2 * j] = o.x;
            x[2 * j + 1] = o.y;
        }
        solve_chunk<float>(x, t, nact, T, edge, solve);
        if (t < nact) {
            float4* dst = reinterpret_cast<float4*>(row) + 4 * t;
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
        }
    } else {
        float2* dst = reinterpret_cast<float2*>(row);
#pragma unroll
        for (int c2 = 0; c2 < 8; ++c2) {
            const int n = t + T * c2;
            const cf o = E[pad(n)];
            if (2 * n < ny) dst[n] = make_float2(o.x, o.y);
        }
    }
}

template <int L>
constexpr size_t rows_h_stride() {
    return item_stride<(size_t)2 * net::Cfg<L>::BUF * sizeof(cf) + edge_slots<L / 16>() * sizeof(float)>();
}
template <int L>
constexpr size_t cols_h_stride() {
    constexpr int T = L / 16, BUF = net::Cfg<L>::BUF;
    return item_stride<(size_t)(2 * BUF) * sizeof(cf) + edge_slots<T>() * sizeof(cf) + 16 +
                       (size_t)2 * 16 * T * sizeof(cf)>();
}
template <int L>
constexpr size_t inv_h_stride() {
    return item_stride<(size_t)inv_e_offset<L>() + net::Cfg<L>::BUF * sizeof(cf)>();
}
template <int L>
constexpr size_t inv_adj_h_stride() {
    return item_stride<inv_adj_item_bytes<L>()>();
}

template <int L, int ORD>
__global__ void __launch_bounds__(32) k_net_rows_h(const float* __restrict__ sigma, int ny, int ord, int rowmap,
                                                   int nx, const cf* __restrict__ nb, const cf* __restrict__ tw,
                                                   cf* __restrict__ z) {
    static_assert(L / 16 == 16, "half-warp lines");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int h = threadIdx.x >> 4;
    rows_item<L, ORD>(smem_raw + h * rows_h_stride<L>(), threadIdx.x & 15, 2 * blockIdx.x + h, sigma, ny, ord,
                      rowmap, nx, nb, tw, z);
}

// columns ky0 .. ky0 + nky - 1 (Z, G_x, G_y hold them from ky0 on)
template <int L, int ORD>
__global__ void __launch_bounds__(32) k_net_cols_h(const cf* __restrict__ z, int nx, int ord, const cf* __restrict__ nb,
                                                   const cf* __restrict__ tw, const float2* __restrict__ spec,
                                                   cf* __restrict__ gx, cf* __restrict__ gy, int ky0, int nky) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int h = threadIdx.x >> 4;
    const int kl = 2 * blockIdx.x + h;
    const bool act = kl < nky;
    const int k = act ? kl : nky - 1;
    cols_item<L, ORD, false>(smem_raw + h * cols_h_stride<L>(), threadIdx.x & 15, k, ky0 + k, z, nx, act ? nx : 0, ord,
                             nb, tw, spec, gx, gy, nullptr);
}

template <int L>
__global__ void __launch_bounds__(32) k_net_rows_inv_h(const cf* __restrict__ g0, const cf* __restrict__ g1, int nx,
                                                       int ny, const cf* __restrict__ nb, const cf* __restrict__ tw,
                                                       float* __restrict__ f0, float* __restrict__ f1) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int h = threadIdx.x >> 4;
    const int w = 2 * blockIdx.x + h;
    const int comp = w / nx, i = w - comp * nx;
    inv_item<L>(smem_raw + h * inv_h_stride<L>(), threadIdx.x & 15, i, comp ? g1 : g0, nx, ny, nb, tw,
                comp ? f1 : f0);
}

template <int L>
__global__ void __launch_bounds__(32) k_net_cols_adj_h(const cf* __restrict__ zx, const cf* __restrict__ zy, int nx,
                                                       int solve, int hy, const cf* __restrict__ nb,
                                                       const cf* __restrict__ tw, const float2* __restrict__ spec,
                                                       cf* __restrict__ g) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int h = threadIdx.x >> 4;
    const int ky = 2 * blockIdx.x + h;
    const bool act = ky < hy;
    cols_adj_item<L>(smem_raw + h * cols_h_stride<L>(), threadIdx.x & 15, act ? ky : hy - 1, act, zx, zy, nx, solve,
                     nb, tw, spec, g, nullptr);
}

template <int L>
__global__ void __launch_bounds__(32) k_net_rows_inv_adj_h(const cf* __restrict__ g, int nx, int ny, int solve,
                                                           const cf* __restrict__ nb, const cf* __restrict__ tw,
                                                           float* __restrict__ out) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int h = threadIdx.x >> 4;
    inv_adj_item<L>(smem_raw + h * inv_adj_h_stride<L>(), threadIdx.x & 15, 2 * blockIdx.x + h, g, nx, ny, solve, nb,
                    tw, out);
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    }
    return fn;
}

// the tiled intermediate(s) as a tensor of floats {2 tw (one tile cell), nx rows, ntile cells,
// ncomp}: strides 8 tw B, nx * 8 tw B, comp_bytes; box {2 tw, 1, min(kBox, cells), 1}
cudaError_t encode_tiles(CUtensorMap* map, void* base, int nx, int ntile, int ncomp, size_t comp_bytes,
                         bool rank4 = false, int tw = kTW, int cells = kBox,
                         CUtensorMapSwizzle swizzle = CU_TENSOR_MAP_SWIZZLE_NONE) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const cuuint32_t rank = (ncomp > 1 || rank4) ? 4 : 3;
    const cuuint64_t cell = (cuuint64_t)tw * 8;
    cuuint64_t dims[4] = {(cuuint64_t)(2 * tw), (cuuint64_t)nx, (cuuint64_t)ntile, (cuuint64_t)ncomp};
    cuuint64_t strides[3] = {cell, (cuuint64_t)nx * cell,
                             (cuuint64_t)(comp_bytes ? comp_bytes : (size_t)ntile * nx * cell)};
    cuuint32_t box[4] = {(cuuint32_t)(2 * tw), 1, (cuuint32_t)std::min(kBox, cells), 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int L>
size_t rows_bytes() {
    return (size_t)2 * net::Cfg<L>::BUF * sizeof(cf) + edge_slots<L / 16>() * sizeof(float);
}

template <int L>
size_t inv_bytes() {
    return (size_t)inv_e_offset<L>() + net::Cfg<L>::BUF * sizeof(cf) + 16;
}

template <int L>
size_t inv2_bytes() {
    return (size_t)inv2_e_offset<L>() + net::Cfg<L>::BUF * sizeof(cf) + 16;
}

// transform length of an axis (P / 2) and the plan's bases tables: x axis first (2 T_x
// values), then y (2 T_y)
int len_x(const Plan& p) { return p.ax.P / 2; }
int len_y(const Plan& p) { return p.ay.P / 2; }
const cf* bases_x(const Plan& p) { return reinterpret_cast<const cf*>(p.net_tw); }
const cf* bases_y(const Plan& p) { return reinterpret_cast<const cf*>(p.net_tw) + len_x(p) / 8; }
// FP32_TC16 plans: the DFT_16 matrix (k_tc_bmat) after the bases, 256-byte aligned
size_t tc_bmat_offset(const Plan& p) { return (((size_t)(len_x(p) / 8 + len_y(p) / 8) * sizeof(cf) + 255) / 256) * 256; }
const float* tc_bmat(const Plan& p) {
    return reinterpret_cast<const float*>(reinterpret_cast<const char*>(p.net_tw) + tc_bmat_offset(p));
}

// Pass A over nx rows: row pairs for the long rows (L >= 2048, a few blocks per SM, 64
// tensor-memory columns each), one row per block below (up to ten blocks per SM there,
// more than tensor memory could stash for)
template <int LY, int OR>
cudaError_t launch_rows(const float* sigma, int ny, int ord, int nx, const cf* nb, const cf* tw, cf* z, int* err,
                        cudaStream_t s) {
    size_t sm = rows_bytes<LY>();
    cudaError_t e;
    if constexpr (LY == 256) {  // two rows per 32-thread block
        sm = 2 * rows_h_stride<LY>();
        if ((e = set_smem(k_net_rows_h<LY, OR>, sm))) return e;
        k_net_rows_h<LY, OR><<<nx / 2, 32, sm, s>>>(sigma, ny, ord, ord != 0, nx, nb, tw, z);
        return cudaGetLastError();
    }
    if constexpr (LY >= 2048) {
        // solved rows of whole 128-byte pieces by TMA: a map of sigma as {32 floats, ny / 32
        // pieces, nx rows}, one row per box, 128-byte swizzle
        CUtensorMap smap;
        int sma = 0;
        if (ord != 0 && ny % 32 == 0 && ((uintptr_t)sigma & 15) == 0) {
            EncodeTiledFn fn = encode_fn();
            if (!fn) return cudaErrorNotSupported;
            cuuint64_t dims[3] = {32, (cuuint64_t)(ny / 32), (cuuint64_t)nx};
            cuuint64_t strides[2] = {128, (cuuint64_t)ny * sizeof(float)};
            cuuint32_t box[3] = {32, (cuuint32_t)(ny / 32), 1};
            cuuint32_t estr[3] = {1, 1, 1};
            if (fn(&smap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(sigma), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return cudaErrorInvalidValue;
            sma = 1;
        } else {
            memset(&smap, 0, sizeof(smap));
        }
        sm = rows2_bytes<LY>();
        if ((e = set_smem(k_net_rows2<LY, OR>, sm))) return e;
        k_net_rows2<LY, OR><<<nx / 2, LY / 16, sm, s>>>(smap, sma, sigma, ny, ord, ord != 0, nx, nb, tw, z, err);
    } else {
        if ((e = set_smem(k_net_rows<LY, OR>, sm))) return e;
        k_net_rows<LY, OR><<<nx, LY / 16, sm, s>>>(sigma, ny, ord, ord != 0, nx, nb, tw, z);
    }
    return cudaGetLastError();
}

// Resident blocks per SM of a kernel launched with `threads` threads and `smem` bytes of
// dynamic shared memory, from its registers (allocated per warp in units of 256) and shared
// memory (plus the 1 KB the driver keeps per block)
template <typename K>
cudaError_t blocks_per_sm(K kernel, int threads, size_t smem, int* per_sm) {
    cudaError_t e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kernel))) return e;
    int dev = 0, regs_sm = 0, smem_sm = 0;
    if ((e = cudaGetDevice(&dev))) return e;
    if ((e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev))) return e;
    if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev))) return e;
    const int warp_regs = ((fa.numRegs * 32 + 255) / 256) * 256;
    const int by_regs = regs_sm / (warp_regs * ((threads + 31) / 32));
    const int by_smem = smem_sm / (int)(fa.sharedSizeBytes + smem + 1024);
    *per_sm = std::max(1, std::min(by_regs, by_smem));
    return cudaSuccess;
}

// Pass C over nx rows of both components of G (g0, g1: [tile][row][2], ntile tiles each):
// persistent, row pairs for the long rows (L >= 2048, two blocks per SM, 64 tensor-memory
// columns each), single rows below
template <int LY>
cudaError_t launch_rows_inv(const cf* g0, const cf* g1, int nx, int ntile, int ny, const cf* nb, const cf* tw,
                            float* fx, float* fy, int* err, cudaStream_t s) {
    cudaError_t e;
    int dev = 0, nsm = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev))) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev))) return e;
    const size_t comp_bytes = (size_t)(g1 - g0) * sizeof(cf);
    if constexpr (LY == 256) {  // two rows per 32-thread block, plain loads
        const size_t sm = 2 * inv_h_stride<LY>();
        if ((e = set_smem(k_net_rows_inv_h<LY>, sm))) return e;
        k_net_rows_inv_h<LY><<<nx, 32, sm, s>>>(g0, g1, nx, ny, nb, tw, fx, fy);
        return cudaGetLastError();
    }
    CUtensorMap gmap;
    if constexpr (LY >= 2048) {
        // pair view: cells of 4 complex (rows 2j and 2j + 1 of one tile), nx / 2 pairs
        // 32-byte pieces under the 32-byte swizzle (the piece is exactly the swizzle span, so
        // the box's footprint in shared memory is its dense size)
        if ((e = encode_tiles(&gmap, const_cast<cf*>(g0), nx / 2, ntile, 2, comp_bytes, false, 2 * kGW, LY / kGW,
                              CU_TENSOR_MAP_SWIZZLE_32B)))
            return e;
        const size_t sm = inv2_bytes<LY>();
        if ((e = set_smem(k_net_rows_inv2<LY>, sm))) return e;
        if ((e = blocks_per_sm(k_net_rows_inv2<LY>, LY / 16, sm, &per_sm))) return e;
        const int grid = std::min(nx, std::min(per_sm, 2) * nsm);
        k_net_rows_inv2<LY><<<grid, LY / 16, sm, s>>>(gmap, g0, g1, nx, ny, nb, tw, fx, fy, err);
    } else {
        if ((e = encode_tiles(&gmap, const_cast<cf*>(g0), nx, ntile, 2, comp_bytes, false, kGW, LY / kGW))) return e;
        const size_t sm = inv_bytes<LY>();
        if ((e = set_smem(k_net_rows_inv<LY>, sm))) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_net_rows_inv<LY>, LY / 16, sm))) return e;
        const int grid = std::min(2 * nx, std::max(1, per_sm) * nsm);
        k_net_rows_inv<LY><<<grid, LY / 16, sm, s>>>(gmap, g0, g1, nx, ny, nb, tw, fx, fy, err);
    }
    return cudaGetLastError();
}

// Pass B over columns ky0 .. ky0 + nky - 1 (FP32 form): one column per block, two per
// 32-thread block for L = 256
template <int LX, int OC>
cudaError_t launch_cols(const cf* z, int nx, int ord, const cf* nb, const cf* tw, const float2* spec, cf* gx, cf* gy,
                        int ky0, int nky, cudaStream_t s) {
    cudaError_t e;
    if constexpr (LX == 256) {
        const size_t sm = 2 * cols_h_stride<LX>();
        if ((e = set_smem(k_net_cols_h<LX, OC>, sm))) return e;
        k_net_cols_h<LX, OC><<<(nky + 1) / 2, 32, sm, s>>>(z, nx, ord, nb, tw, spec, gx, gy, ky0, nky);
    } else {
        const size_t sm = cols_smem_bytes<LX>();
        if ((e = set_smem(k_net_cols<LX, OC>, sm))) return e;
        k_net_cols<LX, OC><<<nky, LX / 16, sm, s>>>(z, nx, ord, nb, tw, spec, gx, gy, ky0);
    }
    return cudaGetLastError();
}

template <int LX, int LY, int ORD>
cudaError_t run_net_o(const Plan& p, const float* sigma, float* fx, float* fy, void* work, cudaStream_t s) {
    const int hy = p.hy;
    const int ntile = (hy + kTW - 1) / kTW;
    const size_t n_el = (size_t)ntile * p.nx * kTW;
    const int ntile_g = (hy + kGW - 1) / kGW;
    const size_t n_el_g = (size_t)ntile_g * p.nx * kGW;
    cf* z = reinterpret_cast<cf*>(work);
    cf* gx = z + n_el;
    cf* gy = gx + n_el_g;
    const cf* twx = reinterpret_cast<const cf*>(p.tw_x);
    const cf* twy = reinterpret_cast<const cf*>(p.tw_y);
    cudaError_t e;
    size_t sm;
    // the order is compiled into the 4096-length kernels (pass B issues faster); shorter
    // lengths share one instance for every order (the batched streams form runs many of
    // them side by side, and one instance keeps their code footprint small)
    constexpr int OR = LY == 4096 ? ORD : -1;
    constexpr int OC = LX == 4096 ? ORD : -1;
    const int ord = solve_order(p);
    mark(p, 0, s);
    if ((e = launch_rows<LY, OR>(sigma, p.ny, ord, p.nx, bases_y(p), twy, z, p.err, s))) return e;
    mark(p, 1, s);
    if constexpr (LX >= 2048) {
        if (p.prec == TDG_FP32_TC16) {
            sm = tc_cols_smem_bytes<LX>();
            if ((e = set_smem(k_net_cols_tc<LX, OC>, sm))) return e;
            k_net_cols_tc<LX, OC><<<hy, LX / 16, sm, s>>>(z, p.nx, ord, bases_x(p), twx,
                                                         reinterpret_cast<const float2*>(p.spec_half), tc_bmat(p),
                                                         gx, gy, p.err);
        }
    }
    if (p.prec != TDG_FP32_TC16) {
        if ((e = launch_cols<LX, OC>(z, p.nx, ord, bases_x(p), twx, reinterpret_cast<const float2*>(p.spec_half), gx,
                                     gy, 0, hy, s)))
            return e;
    }
    if ((e = cudaGetLastError())) return e;
    mark(p, 2, s);
    e = launch_rows_inv<LY>(gx, gy, p.nx, ntile_g, p.ny, bases_y(p), twy, fx, fy, p.err, s);
    mark(p, 3, s);
    return e;
}

// ---------------------------------------------------------------------------------------
// Slab decomposition of one grid (the distribution of Sec. 2.3: the solves and transforms
// split over ranks in slabs, with transposes between them).  A rank's passes are the
// passes above on its share: pass A on its rows (a grid of `nrows` rows), pass B on its
// frequency columns ky0 .. (ky0 even), pass C on its rows again.  Layouts: Z row slab
// [tile][row position], Z column slab [tile - t0][position of all nx rows], G column slab
// [component][tile - t0][row], G row slab [component][tile][row], cells of two columns.
// ---------------------------------------------------------------------------------------
template <int LY, int ORD>
cudaError_t slab_rows_o(const Plan& p, const float* sigma_rows, int nrows, cf* zr, cudaStream_t s) {
    constexpr int OR = LY == 4096 ? ORD : -1;
    return launch_rows<LY, OR>(sigma_rows, p.ny, solve_order(p), nrows, bases_y(p),
                               reinterpret_cast<const cf*>(p.tw_y), zr, p.err, s);
}

template <int LX, int ORD>
cudaError_t slab_cols_o(const Plan& p, const cf* zc, int ky0, int nky, cf* gxc, cf* gyc, cudaStream_t s) {
    constexpr int OC = LX == 4096 ? ORD : -1;
    return launch_cols<LX, OC>(zc, p.nx, solve_order(p), bases_x(p), reinterpret_cast<const cf*>(p.tw_x),
                               reinterpret_cast<const float2*>(p.spec_half), gxc, gyc, ky0, nky, s);
}

template <int LY>
cudaError_t slab_rows_inv_l(const Plan& p, const cf* gr, int nrows, float* fx, float* fy, cudaStream_t s) {
    const int ntile = (p.hy + kGW - 1) / kGW;
    const size_t n_el = (size_t)ntile * nrows * kGW;
    return launch_rows_inv<LY>(gr, gr + n_el, nrows, ntile, p.ny, bases_y(p), reinterpret_cast<const cf*>(p.tw_y),
                               fx, fy, p.err, s);
}

template <int LY>
cudaError_t slab_rows_l(const Plan& p, const float* sigma_rows, int nrows, cf* zr, cudaStream_t s) {
    switch (solve_order(p)) {
        case 3: return slab_rows_o<LY, 3>(p, sigma_rows, nrows, zr, s);
        case 4: return slab_rows_o<LY, 4>(p, sigma_rows, nrows, zr, s);
        case 5: return slab_rows_o<LY, 5>(p, sigma_rows, nrows, zr, s);
        default: return slab_rows_o<LY, 0>(p, sigma_rows, nrows, zr, s);
    }
}

template <int LX>
cudaError_t slab_cols_l(const Plan& p, const cf* zc, int ky0, int nky, cf* gxc, cf* gyc, cudaStream_t s) {
    switch (solve_order(p)) {
        case 3: return slab_cols_o<LX, 3>(p, zc, ky0, nky, gxc, gyc, s);
        case 4: return slab_cols_o<LX, 4>(p, zc, ky0, nky, gxc, gyc, s);
        case 5: return slab_cols_o<LX, 5>(p, zc, ky0, nky, gxc, gyc, s);
        default: return slab_cols_o<LX, 0>(p, zc, ky0, nky, gxc, gyc, s);
    }
}

template <int LX, int LY>
cudaError_t run_net(const Plan& p, const float* sigma, float* fx, float* fy, void* work, cudaStream_t s) {
    switch (solve_order(p)) {
        case 3: return run_net_o<LX, LY, 3>(p, sigma, fx, fy, work, s);
        case 4: return run_net_o<LX, LY, 4>(p, sigma, fx, fy, work, s);
        case 5: return run_net_o<LX, LY, 5>(p, sigma, fx, fy, work, s);
        default: return run_net_o<LX, LY, 0>(p, sigma, fx, fy, work, s);
    }
}

template <int LX, int LY>
cudaError_t run_net_adj(const Plan& p, const float* gxin, const float* gyin, float* gsig, void* work,
                        cudaStream_t s) {
    const int hy = p.hy;
    const int ntile = (hy + kTW - 1) / kTW;
    const size_t n_el = (size_t)ntile * p.nx * kTW;
    cf* zx = reinterpret_cast<cf*>(work);
    cf* zy = zx + n_el;
    cf* g = zy + n_el;
    const cf* twx = reinterpret_cast<const cf*>(p.tw_x);
    const cf* twy = reinterpret_cast<const cf*>(p.tw_y);
    const int solve = solve_order(p);
    cudaError_t e;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev))) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev))) return e;
    mark(p, 0, s);
    if ((e = launch_rows<LY, 0>(gxin, p.ny, 0, p.nx, bases_y(p), twy, zx, p.err, s))) return e;
    if ((e = launch_rows<LY, 0>(gyin, p.ny, 0, p.nx, bases_y(p), twy, zy, p.err, s))) return e;
    mark(p, 1, s);
    size_t sm;
    if constexpr (LX == 256) {  // two columns per 32-thread block
        sm = 2 * cols_h_stride<LX>();
        if ((e = set_smem(k_net_cols_adj_h<LX>, sm))) return e;
        k_net_cols_adj_h<LX><<<(hy + 1) / 2, 32, sm, s>>>(zx, zy, p.nx, solve, hy, bases_x(p), twx,
                                                         reinterpret_cast<const float2*>(p.spec_half), g);
    } else {
        sm = cols_adj_smem_bytes<LX>();
        if ((e = set_smem(k_net_cols_adj<LX>, sm))) return e;
        k_net_cols_adj<LX><<<hy, LX / 16, sm, s>>>(zx, zy, p.nx, solve, bases_x(p), twx,
                                                   reinterpret_cast<const float2*>(p.spec_half), g);
    }
    if ((e = cudaGetLastError())) return e;
    mark(p, 2, s);
    if constexpr (LY == 256) {  // two rows per 32-thread block, plain loads
        sm = 2 * inv_adj_h_stride<LY>();
        if ((e = set_smem(k_net_rows_inv_adj_h<LY>, sm))) return e;
        k_net_rows_inv_adj_h<LY><<<p.nx / 2, 32, sm, s>>>(g, p.nx, p.ny, solve, bases_y(p), twy, gsig);
        e = cudaGetLastError();
        mark(p, 3, s);
        return e;
    }
    CUtensorMap gmap;
    if ((e = encode_tiles(&gmap, g, p.nx, ntile, 1, 0, true))) return e;
    sm = inv_adj_bytes<LY>();
    if ((e = set_smem(k_net_rows_inv_adj<LY>, sm))) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_net_rows_inv_adj<LY>, LY / 16, sm)))
        return e;
    const int grid = std::min(p.nx, std::max(1, per_sm) * nsm);
    k_net_rows_inv_adj<LY><<<grid, LY / 16, sm, s>>>(gmap, g, p.nx, p.ny, solve, bases_y(p), twy, gsig, p.err);
    e = cudaGetLastError();
    mark(p, 3, s);
    return e;
}

template <int LX>
cudaError_t run_net_adj_x(const Plan& p, const float* gx, const float* gy, float* gs, void* work, cudaStream_t s) {
    switch (len_y(p)) {
        case 256: return run_net_adj<LX, 256>(p, gx, gy, gs, work, s);
        case 512: return run_net_adj<LX, 512>(p, gx, gy, gs, work, s);
        case 1024: return run_net_adj<LX, 1024>(p, gx, gy, gs, work, s);
        case 2048: return run_net_adj<LX, 2048>(p, gx, gy, gs, work, s);
        default: return run_net_adj<LX, 4096>(p, gx, gy, gs, work, s);
    }
}

template <int LX>
cudaError_t run_net_x(const Plan& p, const float* sigma, float* fx, float* fy, void* work, cudaStream_t s) {
    switch (len_y(p)) {
        case 256: return run_net<LX, 256>(p, sigma, fx, fy, work, s);
        case 512: return run_net<LX, 512>(p, sigma, fx, fy, work, s);
        case 1024: return run_net<LX, 1024>(p, sigma, fx, fy, work, s);
        case 2048: return run_net<LX, 2048>(p, sigma, fx, fy, work, s);
        default: return run_net<LX, 4096>(p, sigma, fx, fy, work, s);
    }
}

template <int L>
cudaError_t build_axis(cf* tab, cudaStream_t s) {
    k_net_bases<L><<<(L / 16 + 255) / 256, 256, 0, s>>>(tab);
    return cudaGetLastError();
}

cudaError_t build_bases(cf* tab, int n, cudaStream_t s) {
    switch (n) {
        case 256: return build_axis<256>(tab, s);
        case 512: return build_axis<512>(tab, s);
        case 1024: return build_axis<1024>(tab, s);
        case 2048: return build_axis<2048>(tab, s);
        default: return build_axis<4096>(tab, s);
    }
}

template <int L>
cudaError_t spectra_axis(const Plan& p, cudaStream_t s) {
    const long total = (long)p.hy * 2 * (L / 2 + 2);
    k_net_spectra<L><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(reinterpret_cast<const float*>(p.spec), p.hy,
                                                                        reinterpret_cast<float2*>(p.spec_half));
    return cudaGetLastError();
}

}  // namespace

int net_fp32_length(int n) {
    if (n < 128 || n > 4096 || n % 16 != 0) return 0;
    int L = 256;
    while (L < n) L *= 2;
    return L;
}

bool net_fp32_eligible(const Plan& p) {
    return (p.prec == TDG_FP32 || (p.prec == TDG_FP32_TC16 && len_x(p) >= 2048)) &&
           net_fp32_length(p.nx) == len_x(p) && net_fp32_length(p.ny) == len_y(p) &&
           encode_fn() != nullptr;
}

size_t net_fp32_table_bytes(const Plan& p) {
    return p.prec == TDG_FP32_TC16 ? tc_bmat_offset(p) + kTcBFloats * sizeof(float)
                                   : (size_t)(len_x(p) / 8 + len_y(p) / 8) * sizeof(cf);
}

size_t net_fp32_spec_bytes(const Plan& p) { return (size_t)p.hy * 2 * (len_x(p) / 2 + 2) * sizeof(float2); }

cudaError_t launch_net_tables(const Plan& p, cudaStream_t s) {
    cudaError_t e;
    cf* tab = reinterpret_cast<cf*>(p.net_tw);
    if ((e = build_bases(tab, len_x(p), s))) return e;
    if ((e = build_bases(tab + len_x(p) / 8, len_y(p), s))) return e;
    if (p.prec == TDG_FP32_TC16) {
        k_tc_bmat<<<4, 256, 0, s>>>(const_cast<float*>(tc_bmat(p)));
        if ((e = cudaGetLastError())) return e;
    }
    switch (len_x(p)) {
        case 256: return spectra_axis<256>(p, s);
        case 512: return spectra_axis<512>(p, s);
        case 1024: return spectra_axis<1024>(p, s);
        case 2048: return spectra_axis<2048>(p, s);
        default: return spectra_axis<4096>(p, s);
    }
}

cudaError_t launch_adjoint_net(const Plan& p, const float* gx, const float* gy, float* gsig, void* work,
                               cudaStream_t s) {
    switch (len_x(p)) {
        case 256: return run_net_adj_x<256>(p, gx, gy, gsig, work, s);
        case 512: return run_net_adj_x<512>(p, gx, gy, gsig, work, s);
        case 1024: return run_net_adj_x<1024>(p, gx, gy, gsig, work, s);
        case 2048: return run_net_adj_x<2048>(p, gx, gy, gsig, work, s);
        default: return run_net_adj_x<4096>(p, gx, gy, gsig, work, s);
    }
}

cudaError_t launch_slab_rows(const Plan& p, const float* sigma_rows, int nrows, void* zr, cudaStream_t s) {
    cf* z = reinterpret_cast<cf*>(zr);
    switch (len_y(p)) {
        case 256: return slab_rows_l<256>(p, sigma_rows, nrows, z, s);
        case 512: return slab_rows_l<512>(p, sigma_rows, nrows, z, s);
        case 1024: return slab_rows_l<1024>(p, sigma_rows, nrows, z, s);
        case 2048: return slab_rows_l<2048>(p, sigma_rows, nrows, z, s);
        default: return slab_rows_l<4096>(p, sigma_rows, nrows, z, s);
    }
}

cudaError_t launch_slab_cols(const Plan& p, const void* zc, int ky0, int nky, int ntiles, void* gc, cudaStream_t s) {
    const cf* z = reinterpret_cast<const cf*>(zc);
    cf* gx = reinterpret_cast<cf*>(gc);
    cf* gy = gx + (size_t)ntiles * p.nx * kGW;
    switch (len_x(p)) {
        case 256: return slab_cols_l<256>(p, z, ky0, nky, gx, gy, s);
        case 512: return slab_cols_l<512>(p, z, ky0, nky, gx, gy, s);
        case 1024: return slab_cols_l<1024>(p, z, ky0, nky, gx, gy, s);
        case 2048: return slab_cols_l<2048>(p, z, ky0, nky, gx, gy, s);
        default: return slab_cols_l<4096>(p, z, ky0, nky, gx, gy, s);
    }
}

cudaError_t launch_slab_rows_inv(const Plan& p, const void* gr, int nrows, float* fx, float* fy, cudaStream_t s) {
    const cf* g = reinterpret_cast<const cf*>(gr);
    switch (len_y(p)) {
        case 256: return slab_rows_inv_l<256>(p, g, nrows, fx, fy, s);
        case 512: return slab_rows_inv_l<512>(p, g, nrows, fx, fy, s);
        case 1024: return slab_rows_inv_l<1024>(p, g, nrows, fx, fy, s);
        case 2048: return slab_rows_inv_l<2048>(p, g, nrows, fx, fy, s);
        default: return slab_rows_inv_l<4096>(p, g, nrows, fx, fy, s);
    }
}

int net_batch_units(const Plan& p, int pass) {
    if (!net_fp32_eligible(p) || p.prec != TDG_FP32 || len_x(p) > 1024 || len_y(p) > 1024) return 0;
    // lines per unit: one of 1024 points, two of 512, four of 256 (a 64-thread block)
    const int per_y = 1024 / len_y(p), per_x = 1024 / len_x(p);
    if (pass == 0) return p.nx / per_y;
    if (pass == 1) return (p.hy + per_x - 1) / per_x;
    return 2 * p.nx / per_y;
}

size_t net_batch_smem() { return kNetBatchSmem + (3 * (kNetBatchMaxGrids + 1) + 3 * kNetBatchMaxGrids) * sizeof(int); }

cudaError_t net_batch_blocks(int device, int* blocks) {
    cudaError_t e;
    if ((e = set_smem(k_batched_net, net_batch_smem()))) return e;
    // resident blocks per SM from the kernel's registers (per warp, in units of 256) and
    // shared memory (plus the 1 KB the driver keeps per block), and 64 of the 512
    // tensor-memory columns per block
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, k_batched_net))) return e;
    int nsm = 0, regs_sm = 0, smem_sm = 0;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device))) return e;
    if ((e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, device))) return e;
    if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device))) return e;
    const int warp_regs = ((fa.numRegs * 32 + 255) / 256) * 256;
    const int by_regs = regs_sm / (warp_regs * (kNetBatchThreads / 32));
    const int by_smem = smem_sm / (int)(fa.sharedSizeBytes + net_batch_smem() + 1024);
    const int per = std::min(std::min(by_regs, by_smem), 8);
    *blocks = std::max(1, per) * nsm;
    return cudaSuccess;
}

cudaError_t launch_batched_net(const NetBatchDev& d, int blocks, cudaStream_t s) {
    cudaError_t e;
    if ((e = set_smem(k_batched_net, net_batch_smem()))) return e;
    k_batched_net<<<blocks, kNetBatchThreads, net_batch_smem(), s>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_forward_net(const Plan& p, const float* sigma, float* fx, float* fy, void* work,
                               cudaStream_t s) {
    switch (len_x(p)) {
        case 256: return run_net_x<256>(p, sigma, fx, fy, work, s);
        case 512: return run_net_x<512>(p, sigma, fx, fy, work, s);
        case 1024: return run_net_x<1024>(p, sigma, fx, fy, work, s);
        case 2048: return run_net_x<2048>(p, sigma, fx, fy, work, s);
        default: return run_net_x<4096>(p, sigma, fx, fy, work, s);
    }
}

}  // namespace tdg
