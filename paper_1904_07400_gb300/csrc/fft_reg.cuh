// Register butterflies and twiddle helpers of the transform network (fft_net.cuh): radix
// 1, 2, 4, 8 and 16 DFTs on a thread's 16 complex values, powers of a twiddle base, the
// per-element twist W_2L^(t + r T) of the padded column transform, and the padded
// shared-memory index.
#pragma once

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

// radix-R butterflies of one stage on the thread's 16 values; butterfly b uses
// v[b * R .. b * R + R - 1] (element r at v[b * R + r])
template <int R>
__device__ __forceinline__ void butterflies(cf* v) {
    if constexpr (R == 1) {
        // radix 1: nothing to do (the 16 * 1 * 16 network has no middle stage)
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

// W_2L^(t + r T) for r < 16, from the table entry W_2L^t (tw has W_2L^m at tw[m]) and the
// constants W_2L^(r T) = W_32^r (T = L / 16)
__device__ __forceinline__ cf twist(cf wt, int r) { return cmul(wt, w32(r)); }

// W_2L^-(t + r T) from the table entry W_2L^(2L - t) (= W_2L^-t) and conj(W_32^r).  Written
// from a different table entry than twist() on purpose: the compiler cannot merge the two,
// so the factors are not kept alive across the transforms in between.
__device__ __forceinline__ cf untwist(cf wtc, int r) { return cmulc(wtc, w32(r)); }

}  // namespace reg
}  // namespace tdg
