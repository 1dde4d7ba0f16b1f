// Register-resident FFT of one line of length L = 16 * R1 * 16 (R1 in {4, 8, 16}) by T =
// L / 16 threads, 16 complex values per thread, two exchanges through padded shared memory.
//
// Data distribution at entry and exit: thread t holds element t + r * T in v[r], r < 16
// ("natural strided").  Three Stockham stages (radix 16, R1, 16); the last stage leaves its
// outputs exactly where the first stage of the next transform reads its inputs, so a
// forward transform, a pointwise product and an inverse transform chain without any
// reordering.  The inverse transform is conj(FFT(conj(x))).
//
// Shared buffer per line: L + L/16 complex values; element i lives at i + i/16 (the pad
// spreads the stride-16 stores of the first stage over all banks).
#pragma once

#include <cuda_fp16.h>

#include "tdg_internal.cuh"

namespace tdg {
namespace reg {

typedef cpx<float> cf;

__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }

__device__ __forceinline__ cf ld_tw(const cf* tw, int i) {
    float2 v = __ldg(reinterpret_cast<const float2*>(tw) + i);
    return mk(v.x, v.y);
}

__device__ __forceinline__ cf mul_w16(cf a, int q) {
    // exp(-2 pi i q / 16)
    const float c1 = 0.923879532511286756f, s1 = 0.382683432365089772f, h = 0.707106781186547524f;
    switch (q & 15) {
        case 0: return a;
        case 1: return mk(a.x * c1 + a.y * s1, a.y * c1 - a.x * s1);
        case 2: return mk(h * (a.x + a.y), h * (a.y - a.x));
        case 3: return mk(a.x * s1 + a.y * c1, a.y * s1 - a.x * c1);
        case 4: return mk(a.y, -a.x);
        case 6: return mk(h * (a.y - a.x), -h * (a.x + a.y));
        case 9: return mk(-a.x * c1 - a.y * s1, a.x * s1 - a.y * c1);
        default: {
            float sn, cs;
            sincospif(-2.0f * (float)q / 16.0f, &sn, &cs);
            return mk(a.x * cs - a.y * sn, a.x * sn + a.y * cs);
        }
    }
}

__device__ __forceinline__ void dft2(cf& a, cf& b) {
    cf t = a - b;
    a = a + b;
    b = t;
}

// forward DFT_4 in place on (a0, a1, a2, a3)
__device__ __forceinline__ void dft4(cf& a0, cf& a1, cf& a2, cf& a3) {
    cf t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3, t3 = a1 - a3;
    t3 = mk(t3.y, -t3.x);  // * (-i)
    a0 = t0 + t2;
    a2 = t0 - t2;
    a1 = t1 + t3;
    a3 = t1 - t3;
}

// forward DFT_8 in place on a[0..7] (stride s in the register array)
template <int S>
__device__ __forceinline__ void dft8(cf* a) {
    cf e0 = a[0], e1 = a[2 * S], e2 = a[4 * S], e3 = a[6 * S];
    cf o0 = a[S], o1 = a[3 * S], o2 = a[5 * S], o3 = a[7 * S];
    dft4(e0, e1, e2, e3);
    dft4(o0, o1, o2, o3);
    o1 = mul_w16(o1, 2);
    o2 = mul_w16(o2, 4);
    o3 = mul_w16(o3, 6);
    a[0] = e0 + o0;
    a[4 * S] = e0 - o0;
    a[S] = e1 + o1;
    a[5 * S] = e1 - o1;
    a[2 * S] = e2 + o2;
    a[6 * S] = e2 - o2;
    a[3 * S] = e3 + o3;
    a[7 * S] = e3 - o3;
}

// forward DFT_16 in place on a[0..15]: n = 4 n1 + n2, k = k1 + 4 k2
__device__ __forceinline__ void dft16(cf* a) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4(a[n2], a[4 + n2], a[8 + n2], a[12 + n2]);
    // now a[4 k1 + n2] = B[n2][k1]; twiddle W16^(n2 k1)
    a[5] = mul_w16(a[5], 1);
    a[6] = mul_w16(a[6], 2);
    a[7] = mul_w16(a[7], 3);
    a[9] = mul_w16(a[9], 2);
    a[10] = mul_w16(a[10], 4);
    a[11] = mul_w16(a[11], 6);
    a[13] = mul_w16(a[13], 3);
    a[14] = mul_w16(a[14], 6);
    a[15] = mul_w16(a[15], 9);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4(a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]);
    // a[4 k1 + k2] = A[k1 + 4 k2]: transpose 4 x 4 into natural order
    cf t;
    t = a[1]; a[1] = a[4]; a[4] = t;
    t = a[2]; a[2] = a[8]; a[8] = t;
    t = a[3]; a[3] = a[12]; a[12] = t;
    t = a[6]; a[6] = a[9]; a[9] = t;
    t = a[7]; a[7] = a[13]; a[13] = t;
    t = a[11]; a[11] = a[14]; a[14] = t;
}

// ---------------------------------------------------------------------------------------
// Tensor-core DFT_16 (the TC16 form): the 32 butterflies of a warp as one real product
//   [Yr; Yi] = [[C, S], [-S, C]] [Xr; Xi],  C = cos(2 pi r k / 16), S = sin(2 pi r k / 16)
// on mma.sync.m16n8k16 (FP16 operands, FP32 accumulation).  Operands are split into
// FP16 hi + lo parts and three products are accumulated (hi.hi + hi.lo + lo.hi), after a
// power-of-two scale that brings the warp's largest value near 1.
// ---------------------------------------------------------------------------------------
struct TcConst {
    unsigned c_hi[4], c_lo[4], s_hi[4], s_lo[4], n_hi[4], n_lo[4];  // A fragments of C, S, -S
};

__device__ __forceinline__ unsigned pack_h2(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<unsigned*>(&h);
}

__device__ __forceinline__ void split_h2(float a, float b, unsigned& hi, unsigned& lo) {
    __half2 h = __floats2half2_rn(a, b);
    float2 f = __half22float2(h);
    __half2 l = __floats2half2_rn(a - f.x, b - f.y);
    hi = *reinterpret_cast<unsigned*>(&h);
    lo = *reinterpret_cast<unsigned*>(&l);
}

// A fragments (row-major 16 x 16) of this lane for the DFT_16 matrices
__device__ __forceinline__ TcConst make_tc_const(int lane) {
    TcConst k;
    const int g = lane >> 2, q = lane & 3;
    const int rows[4] = {g, g + 8, g, g + 8};
    const int cols[4] = {2 * q, 2 * q, 2 * q + 8, 2 * q + 8};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float c[2], sn[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            int rk = (rows[i] * (cols[i] + e)) & 15;
            sincospif((float)rk / 8.0f, &sn[e], &c[e]);
        }
        split_h2(c[0], c[1], k.c_hi[i], k.c_lo[i]);
        split_h2(sn[0], sn[1], k.s_hi[i], k.s_lo[i]);
        split_h2(-sn[0], -sn[1], k.n_hi[i], k.n_lo[i]);
    }
    return k;
}

__device__ __forceinline__ void mma16816(float* d, const unsigned* a, unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int kTcRow = 17;  // complex values per butterfly row of the warp scratch (16 + pad)
constexpr int kTcWarpScratch = 32 * kTcRow;

// DFT_16 of this thread's butterfly v[0..15]; ws: this warp's scratch (kTcWarpScratch)
__device__ __forceinline__ void dft16_tc(cf* v, cf* ws, const TcConst& K) {
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, q = lane & 3;
    float m = 0.f;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        ws[lane * kTcRow + r] = v[r];
        m = fmaxf(m, fmaxf(fabsf(v[r].x), fabsf(v[r].y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    // scale = 2^-e with 2^(e-1) <= m < 2^e: scaled values below 1
    int e = m > 0.f ? ((__float_as_int(m) >> 23) & 255) - 126 : 0;
    const float sc = __int_as_float((127 - e) << 23), inv = __int_as_float((127 + e) << 23);
    __syncwarp();
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const int n = nt * 8 + g;  // butterfly (column) of this lane's B fragment
        const cf x0 = ws[n * kTcRow + 2 * q], x1 = ws[n * kTcRow + 2 * q + 1];
        const cf x8 = ws[n * kTcRow + 2 * q + 8], x9 = ws[n * kTcRow + 2 * q + 9];
        unsigned rh0, rl0, rh1, rl1, ih0, il0, ih1, il1;
        split_h2(x0.x * sc, x1.x * sc, rh0, rl0);
        split_h2(x8.x * sc, x9.x * sc, rh1, rl1);
        split_h2(x0.y * sc, x1.y * sc, ih0, il0);
        split_h2(x8.y * sc, x9.y * sc, ih1, il1);
        float yr[4] = {0.f, 0.f, 0.f, 0.f}, yi[4] = {0.f, 0.f, 0.f, 0.f};
        mma16816(yr, K.c_hi, rh0, rh1);
        mma16816(yr, K.c_hi, rl0, rl1);
        mma16816(yr, K.c_lo, rh0, rh1);
        mma16816(yr, K.s_hi, ih0, ih1);
        mma16816(yr, K.s_hi, il0, il1);
        mma16816(yr, K.s_lo, ih0, ih1);
        mma16816(yi, K.n_hi, rh0, rh1);
        mma16816(yi, K.n_hi, rl0, rl1);
        mma16816(yi, K.n_lo, rh0, rh1);
        mma16816(yi, K.c_hi, ih0, ih1);
        mma16816(yi, K.c_hi, il0, il1);
        mma16816(yi, K.c_lo, ih0, ih1);
        __syncwarp();  // every lane has read this tile's inputs
        const int n0 = nt * 8 + 2 * q;  // output columns n0, n0 + 1; rows g and g + 8
        ws[n0 * kTcRow + g] = mk(yr[0] * inv, yi[0] * inv);
        ws[(n0 + 1) * kTcRow + g] = mk(yr[1] * inv, yi[1] * inv);
        ws[n0 * kTcRow + g + 8] = mk(yr[2] * inv, yi[2] * inv);
        ws[(n0 + 1) * kTcRow + g + 8] = mk(yr[3] * inv, yi[3] * inv);
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = ws[lane * kTcRow + r];
    __syncwarp();
}

// radix-R butterflies of one stage on the thread's 16 values; butterfly b uses
// v[b * R .. b * R + R - 1] (element r at v[b * R + r])
template <int R, bool TC = false>
__device__ __forceinline__ void butterflies(cf* v, cf* ws = nullptr, const TcConst* K = nullptr) {
    if constexpr (R == 16 && TC) {
        dft16_tc(v, ws, *K);
    } else if constexpr (R == 16) {
        dft16(v);
    } else if constexpr (R == 8) {
        dft8<1>(v);
        dft8<1>(v + 8);
    } else if constexpr (R == 2) {
#pragma unroll
        for (int m = 0; m < 8; ++m) dft2(v[2 * m], v[2 * m + 1]);
    } else {
        dft4(v[0], v[1], v[2], v[3]);
        dft4(v[4], v[5], v[6], v[7]);
        dft4(v[8], v[9], v[10], v[11]);
        dft4(v[12], v[13], v[14], v[15]);
    }
}

// One exchange: registers (outputs of a stage of radix RA with stride NSA) -> shared ->
// registers (inputs of the next stage of radix RB).  tw: W_L^m at tw[m * TS].
template <int L, int RA, int NSA, int RB>
__device__ __forceinline__ void exchange(cf* v, cf* buf, int t) {
    constexpr int T = L / 16;
    constexpr int BA = 16 / RA;
#pragma unroll
    for (int b = 0; b < BA; ++b) {
        int j = t + T * b;
        int base = (j / NSA) * NSA * RA + (j % NSA);
#pragma unroll
        for (int r = 0; r < RA; ++r) buf[pad(base + r * NSA)] = v[b * RA + r];
    }
    __syncthreads();
    constexpr int BB = 16 / RB;
#pragma unroll
    for (int b = 0; b < BB; ++b) {
        int j = t + T * b;
#pragma unroll
        for (int r = 0; r < RB; ++r) v[b * RB + r] = buf[pad(j + r * (L / RB))];
    }
    __syncthreads();
}

// exp(-2 pi i r / 32), r < 32: the factors W_2L^(r T) = W_32^r of the per-element twists
struct W32 {
    float c, s;
};
__device__ __forceinline__ cf w32(int r) {
    constexpr W32 tab[32] = {
    {1.00000000000000000e+00f, -0.00000000000000000e+00f},
    {9.80785280403230431e-01f, -1.95090322016128248e-01f},
    {9.23879532511286738e-01f, -3.82683432365089782e-01f},
    {8.31469612302545236e-01f, -5.55570233019602178e-01f},
    {7.07106781186547573e-01f, -7.07106781186547462e-01f},
    {5.55570233019602289e-01f, -8.31469612302545236e-01f},
    {3.82683432365089837e-01f, -9.23879532511286738e-01f},
    {1.95090322016128331e-01f, -9.80785280403230431e-01f},
    {6.12323399573676604e-17f, -1.00000000000000000e+00f},
    {-1.95090322016128193e-01f, -9.80785280403230431e-01f},
    {-3.82683432365089726e-01f, -9.23879532511286738e-01f},
    {-5.55570233019601956e-01f, -8.31469612302545458e-01f},
    {-7.07106781186547462e-01f, -7.07106781186547573e-01f},
    {-8.31469612302545347e-01f, -5.55570233019602178e-01f},
    {-9.23879532511286738e-01f, -3.82683432365089893e-01f},
    {-9.80785280403230431e-01f, -1.95090322016128609e-01f},
    {-1.00000000000000000e+00f, -1.22464679914735321e-16f},
    {-9.80785280403230431e-01f, 1.95090322016128359e-01f},
    {-9.23879532511286850e-01f, 3.82683432365089671e-01f},
    {-8.31469612302545458e-01f, 5.55570233019601956e-01f},
    {-7.07106781186547684e-01f, 7.07106781186547462e-01f},
    {-5.55570233019602178e-01f, 8.31469612302545236e-01f},
    {-3.82683432365090337e-01f, 9.23879532511286516e-01f},
    {-1.95090322016128664e-01f, 9.80785280403230320e-01f},
    {-1.83697019872102969e-16f, 1.00000000000000000e+00f},
    {1.95090322016128304e-01f, 9.80785280403230431e-01f},
    {3.82683432365090004e-01f, 9.23879532511286627e-01f},
    {5.55570233019601845e-01f, 8.31469612302545458e-01f},
    {7.07106781186547351e-01f, 7.07106781186547684e-01f},
    {8.31469612302545236e-01f, 5.55570233019602178e-01f},
    {9.23879532511286516e-01f, 3.82683432365090392e-01f},
    {9.80785280403230320e-01f, 1.95090322016128720e-01f}
    };
    return mk(tab[r & 31].c, tab[r & 31].s);
}

// v[r] *= w^r for r < R, from the loaded w^1 (and w^4, w^8 for R >= 8): each power is at
// most four chained products from a table entry and is applied as soon as it is formed,
// so only a handful of factors are live at once
template <int R>
__device__ __forceinline__ void apply_powers(cf* v, cf w1, cf w4, cf w8) {
    v[1] = cmul(v[1], w1);
    if constexpr (R > 2) {
        cf w2 = cmul(w1, w1);
        cf w3 = cmul(w2, w1);
        v[2] = cmul(v[2], w2);
        v[3] = cmul(v[3], w3);
        if constexpr (R > 4) {
            cf w5 = cmul(w4, w1);
            cf w6 = cmul(w4, w2);
            cf w7 = cmul(w4, w3);
            v[4] = cmul(v[4], w4);
            v[5] = cmul(v[5], w5);
            v[6] = cmul(v[6], w6);
            v[7] = cmul(v[7], w7);
            if constexpr (R > 8) {
                v[8] = cmul(v[8], w8);
                v[9] = cmul(v[9], cmul(w8, w1));
                v[10] = cmul(v[10], cmul(w8, w2));
                v[11] = cmul(v[11], cmul(w8, w3));
                v[12] = cmul(v[12], cmul(w8, w4));
                v[13] = cmul(v[13], cmul(w8, w5));
                v[14] = cmul(v[14], cmul(w8, w6));
                v[15] = cmul(v[15], cmul(w8, w7));
            }
        }
    }
}

// Twiddle bases of one thread, loaded once per kernel and reused by every transform the
// thread runs (they depend only on t): for the middle stage (radix R1, NS = 16) and the
// last stage (radix 16, NS = L/16) the table entries W^e, W^4e, W^8e of each butterfly.
template <int L, int R1>
struct TwBase {
    static constexpr int B1 = 16 / R1;
    cf m1[B1], m4[B1], m8[B1];
    cf l1, l4, l8;
};

template <int L, int R1, int TS>
__device__ __forceinline__ TwBase<L, R1> load_tw_base(const cf* tw, int t) {
    constexpr int T = L / 16;
    constexpr int STEP1 = L / (16 * R1);
    TwBase<L, R1> b;
#pragma unroll
    for (int q = 0; q < TwBase<L, R1>::B1; ++q) {
        const int e = ((t + T * q) % 16) * STEP1;
        b.m1[q] = ld_tw(tw, e * TS);
        b.m4[q] = R1 > 4 ? ld_tw(tw, ((4 * e) % L) * TS) : b.m1[q];
        b.m8[q] = R1 > 8 ? ld_tw(tw, ((8 * e) % L) * TS) : b.m1[q];
    }
    b.l1 = ld_tw(tw, t * TS);
    b.l4 = ld_tw(tw, ((4 * t) % L) * TS);
    b.l8 = ld_tw(tw, ((8 * t) % L) * TS);
    return b;
}

// W_2L^(t + r T) for r < 16, from the table entry W_2L^t (tw has W_2L^m at tw[m]) and the
// constants W_2L^(r T) = W_32^r (T = L / 16)
__device__ __forceinline__ cf twist(cf wt, int r) { return cmul(wt, w32(r)); }

// W_2L^-(t + r T) from the table entry W_2L^(2L - t) (= W_2L^-t) and conj(W_32^r).  Written
// from a different table entry than twist() on purpose: the compiler cannot merge the two,
// so the factors are not kept alive across the transforms in between.
__device__ __forceinline__ cf untwist(cf wtc, int r) { return cmulc(wtc, w32(r)); }

// Forward FFT of length L = 16 * R1 * 16; v natural strided in and out.  buf: this line's
// shared buffer (L + L/16 values).  tb: the thread's twiddle bases (load_tw_base).
// With TC, every radix-16 stage runs on the tensor cores (ws: the warp's scratch, K: the
// lane's DFT_16 fragments); other radices stay on the FP32 pipes.
template <int L, int R1, bool TC = false>
__device__ __forceinline__ void fft(cf* v, cf* buf, const TwBase<L, R1>& tb, int t, cf* ws = nullptr,
                                    const TcConst* K = nullptr) {
    static_assert(16 * R1 * 16 == L, "L = 16 * R1 * 16");
    butterflies<16, TC>(v, ws, K);
    exchange<L, 16, 1, R1>(v, buf, t);
#pragma unroll
    for (int q = 0; q < TwBase<L, R1>::B1; ++q) apply_powers<R1>(v + q * R1, tb.m1[q], tb.m4[q], tb.m8[q]);
    butterflies<R1, TC>(v, ws, K);
    exchange<L, R1, 16, 16>(v, buf, t);
    apply_powers<16>(v, tb.l1, tb.l4, tb.l8);
    butterflies<16, TC>(v, ws, K);
}

template <int L, int R1, bool TC = false>
__device__ __forceinline__ void ifft(cf* v, cf* buf, const TwBase<L, R1>& tb, int t, cf* ws = nullptr,
                                     const TcConst* K = nullptr) {
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = conjg(v[r]);
    fft<L, R1, TC>(v, buf, tb, t, ws, K);
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = conjg(v[r]);
}

template <int L> struct Mid;
template <> struct Mid<1024> { static constexpr int R1 = 4; };
template <> struct Mid<2048> { static constexpr int R1 = 8; };
template <> struct Mid<4096> { static constexpr int R1 = 16; };

}  // namespace reg
}  // namespace tdg
