// Register FFT network of length L = 16 * R * 16 (R in {1, 2, 4, 8, 16}) run by T = L / 16
// threads with 16 complex values each, with ONE block barrier per transform.  For R = 1
// (L = 256, one half-warp) the first exchange and the middle stage are the identity: the
// barrier stays (callers rely on it to order their own uses of the buffer), the data stay
// in registers.
//
// Index decomposition: n = a + 16 b + 16 R c and k = k_c + 16 k_b + 16 R k_a
// (a, k_a < 16; b, k_b < R; c, k_c < 16).  Three stages of butterflies:
//   1. DFT_16 over c                      (thread t = a + 16 b holds c = 0..15)
//   2. twiddle W_{16R}^(b k_c), DFT_R over b (thread t = a + 16 j holds k_c = j + R m, all b)
//   3. twiddle W_L^(a (k_c + 16 k_b)), DFT_16 over a
//      (thread t = 16 j + s, s = k_b + R m, holds all a)
// The exchange before stage 2 crosses warps and goes through a shared buffer with one
// __syncthreads.  The exchange before stage 3 stays inside a half-warp: half-warp j holds
// every (a, k_c = j + R m) pair and every stage-3 group with the same k_c, so the 16 x 16
// transpose runs in the half-warp's own slab of the same buffer with __syncwarp only.
//
// Layouts:
//   NS ("natural strided"):  thread t holds x[t + T r] in v[r]
//   SP ("spectral permuted"): thread t holds X[perm(t) + T r] in v[r],
//        perm(t) = j + R m + 16 k_b  with j = t / 16, s = t % 16, k_b = s % R, m = s / R
// fwd() maps NS to SP (the forward DFT).  inv_t() is the transposed network, SP to NS with
// the same forward kernels; the inverse DFT (unnormalised) is conj(inv_t(conj(X))).
//
// Shared buffer: R slabs of 272 complex values (slab j: the stage-2 inputs of half-warp j,
// 256 values, reused for its 16 x 17 padded transpose).  Hazards between calls:
//   * fwd then inv_t on the same buffer: only each half-warp's own slab is touched between
//     the two barriers, so nothing more is needed;
//   * any other pair of calls on the same buffer needs a __syncthreads between them (or a
//     second buffer), because the later call writes slabs that other warps may still read.
#pragma once

#include "fft_reg.cuh"

namespace tdg {
namespace net {

using reg::cf;

template <int L>
struct Cfg {
    static constexpr int R = L / 256;
    static constexpr int T = L / 16;
    static constexpr int NM = 16 / R;  // stage-2 groups per thread
    static constexpr int SLAB = 272;
    static constexpr int BUF = R * SLAB;  // complex values per exchange buffer
    static_assert(R == 1 || R == 2 || R == 4 || R == 8 || R == 16, "L in {256, 512, 1024, 2048, 4096}");
};

template <int L>
__host__ __device__ constexpr int perm(int t) {
    constexpr int R = Cfg<L>::R;
    const int j = t >> 4, s = t & 15;
    return j + R * (s / R) + 16 * (s % R);
}

template <int L>
__host__ __device__ constexpr int perm_inv(int p) {
    constexpr int R = Cfg<L>::R;
    const int kb = p >> 4, rem = p & 15;
    return 16 * (rem % R) + kb + R * (rem / R);
}

// per-thread twiddle bases: b2 = W_{16R}^(t / 16) (stage 2), b3 = W_L^perm(t) (stage 3)
struct Bases {
    cf b2, b3;
};

// table layout: [0, T) the stage-3 bases by thread, [T, 2T) the stage-2 bases by thread
template <int L>
__device__ __forceinline__ Bases load_bases(const cf* __restrict__ tab, int t) {
    Bases b;
    b.b3 = reg::ld_tw(tab, t);
    b.b2 = reg::ld_tw(tab, Cfg<L>::T + t);
    return b;
}

__device__ __forceinline__ cf csq(cf a) { return mk(a.x * a.x - a.y * a.y, 2.0f * a.x * a.y); }

// stage-2 twiddles: group m multiplies v[m R + b] by (W_{16R}^(j + R m))^b
template <int L>
__device__ __forceinline__ void tw2(cf* v, cf b2) {
    constexpr int R = Cfg<L>::R;
    if constexpr (R == 1) {
        // W_16^(0 k_c) = 1
    } else if constexpr (R == 16) {
        const cf w4 = csq(csq(b2));
        reg::apply_powers<16>(v, b2, w4, csq(w4));
    } else if constexpr (R == 8) {
        // W_{16R}^(R m) = W_16^m
        const cf w1b = reg::mul_w16(b2, 1);
        reg::apply_powers<8>(v, b2, csq(csq(b2)), b2);
        reg::apply_powers<8>(v + 8, w1b, csq(csq(w1b)), w1b);
    } else if constexpr (R == 4) {
#pragma unroll
        for (int m = 0; m < 4; ++m) reg::apply_powers<4>(v + 4 * m, reg::mul_w16(b2, m), b2, b2);
    } else {
        // R = 2: W_32^(j + 2 m) = W_32^j W_16^m, one factor per pair
#pragma unroll
        for (int m = 1; m < 8; ++m) v[2 * m + 1] = cmul(v[2 * m + 1], reg::mul_w16(b2, m));
        v[1] = cmul(v[1], b2);
    }
}

// stage-3 twiddles: v[a] *= b3^a
__device__ __forceinline__ void tw3(cf* v, cf b3) {
    const cf w4 = csq(csq(b3));
    reg::apply_powers<16>(v, b3, w4, csq(w4));
}

// twiddle providers of the network: Bases forms the powers from the two bases at every
// stage; a kernel may pass any type with apply2(v) / apply3(v) (e.g. powers kept in
// tensor memory)
template <int L>
struct GenTw {
    Bases b;
    __device__ __forceinline__ void apply2(cf* v) const { tw2<L>(v, b.b2); }
    __device__ __forceinline__ void apply3(cf* v) const { tw3(v, b.b3); }
};

// the 16 stage-2 factors (group m, b at v[m R + b]) and the 16 stage-3 factors (v[a]) of
// thread t, for kernels that keep them
template <int L>
__device__ __forceinline__ void stage_factors(const Bases& bs, cf* f2, cf* f3) {
#pragma unroll
    for (int i = 0; i < 16; ++i) f2[i] = f3[i] = mk(1.f, 0.f);
    tw2<L>(f2, bs.b2);
    tw3(f3, bs.b3);
}

// butterfly providers of the network: stage<R>(v) runs the radix-R butterflies of one stage
// on the thread's 16 values (R = 16: one DFT_16).  The default runs them on the FP32 pipes;
// a kernel may pass another provider (e.g. DFT_16 as tensor-core products).
struct CoreDft {
    template <int R>
    __device__ __forceinline__ void stage(cf* v) {
        reg::butterflies<R>(v);
    }
};

// forward DFT, NS in, SP out
template <int L, typename TW, typename DF = CoreDft>
__device__ __forceinline__ void fwd_p(cf* v, cf* buf, const TW& tw, int t, DF&& df = DF{}) {
    constexpr int R = Cfg<L>::R, NM = Cfg<L>::NM;
    df.template stage<16>(v);
    const int a = t & 15;
    cf* slab = buf + (t >> 4) * 272;
    if constexpr (R > 1) {
#pragma unroll
        for (int kc = 0; kc < 16; ++kc) buf[(kc % R) * 272 + (kc / R) * 16 * R + t] = v[kc];
        __syncthreads();
#pragma unroll
        for (int m = 0; m < NM; ++m)
#pragma unroll
            for (int b = 0; b < R; ++b) v[m * R + b] = slab[m * 16 * R + b * 16 + a];
    } else {
        __syncthreads();
    }
    tw.apply2(v);
    df.template stage<R>(v);
    __syncwarp();
#pragma unroll
    for (int s = 0; s < 16; ++s) slab[s * 17 + a] = v[s];
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = slab[a * 17 + i];
    tw.apply3(v);
    df.template stage<16>(v);
}

template <int L>
__device__ __forceinline__ void fwd(cf* v, cf* buf, const Bases& bs, int t) {
    fwd_p<L>(v, buf, GenTw<L>{bs}, t);
}

// transposed network, SP in, NS out (forward kernels): the unnormalised inverse DFT is
// conj(inv_t(conj(X)))
template <int L, typename TW, typename DF = CoreDft>
__device__ __forceinline__ void inv_t_p(cf* v, cf* buf, const TW& tw, int t, DF&& df = DF{}) {
    constexpr int R = Cfg<L>::R, NM = Cfg<L>::NM;
    df.template stage<16>(v);
    tw.apply3(v);
    const int a = t & 15;
    cf* slab = buf + (t >> 4) * 272;
    __syncwarp();  // a preceding fwd() on this buffer may still read the slab
#pragma unroll
    for (int i = 0; i < 16; ++i) slab[a * 17 + i] = v[i];
    __syncwarp();
#pragma unroll
    for (int s = 0; s < 16; ++s) v[s] = slab[s * 17 + a];
    df.template stage<R>(v);
    tw.apply2(v);
    if constexpr (R > 1) {
        __syncwarp();
#pragma unroll
        for (int m = 0; m < NM; ++m)
#pragma unroll
            for (int b = 0; b < R; ++b) slab[m * 16 * R + b * 16 + a] = v[m * R + b];
        __syncthreads();
#pragma unroll
        for (int kc = 0; kc < 16; ++kc) v[kc] = buf[(kc % R) * 272 + (kc / R) * 16 * R + t];
    } else {
        __syncthreads();
    }
    df.template stage<16>(v);
}

template <int L>
__device__ __forceinline__ void inv_t(cf* v, cf* buf, const Bases& bs, int t) {
    inv_t_p<L>(v, buf, GenTw<L>{bs}, t);
}

}  // namespace net
}  // namespace tdg
