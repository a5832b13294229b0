// Register-resident complex FFTs of compile-time length (sm_103a, FP32).
//
// One thread owns one length-N line in registers; the bit-reversal permutation
// and every twiddle index are resolved at compile time, trivial twiddles
// (1, -i, -1, i) cost no multiply, the rest come from a constant-memory table
// exp(-2 pi i t / 128) filled on the host in FP64.  Transforms are
// unnormalised: forward X_k = sum_j x_j e^{-2 pi i jk/N}, inverse with e^{+}.
#pragma once

#include <cuda_runtime.h>

namespace boltz_dev {

__constant__ float2 c_twiddle[128];

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
__host__ __device__ constexpr int bitrev(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

// a * exp(-+ 2 pi i t / 128), t in [0, 128) known at compile time after unrolling.
template <bool INV>
__device__ __forceinline__ float2 twiddle_mul(float2 a, int t) {
    if (t == 0) return a;
    if (t == 64) return make_float2(-a.x, -a.y);
    if (t == 32) return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
    if (t == 96) return INV ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
    float2 w = c_twiddle[t];
    if (INV) w.y = -w.y;
    return cmul(a, w);
}

// Bit-reversal permutation with indices fixed at compile time (template
// recursion), so the register array is never indexed dynamically.
template <int N, int I>
struct BitRevSwap {
    static __device__ __forceinline__ void run(float2 (&x)[N]) {
        constexpr int J = bitrev(I, ilog2(N));
        if constexpr (J > I) {
            const float2 t = x[I];
            x[I] = x[J];
            x[J] = t;
        }
        BitRevSwap<N, I + 1>::run(x);
    }
};
template <int N>
struct BitRevSwap<N, N> {
    static __device__ __forceinline__ void run(float2 (&)[N]) {}
};

// One radix-2 stage (butterfly span m = 2^S); trip counts are compile-time
// constants so the whole transform unrolls into straight-line register code.
template <int N, int S, bool INV>
struct Radix2Stage {
    static __device__ __forceinline__ void run(float2 (&x)[N]) {
        constexpr int m = 1 << S, h = m >> 1;
#pragma unroll
        for (int i = 0; i < N; i += m) {
#pragma unroll
            for (int k = 0; k < h; ++k) {
                const float2 u = x[i + k];
                const float2 t = twiddle_mul<INV>(x[i + k + h], k * (128 / m));
                x[i + k] = cadd(u, t);
                x[i + k + h] = csub(u, t);
            }
        }
        if constexpr (m < N) Radix2Stage<N, S + 1, INV>::run(x);
    }
};

// In-place radix-2 decimation-in-time FFT of N (power of two, <= 128) points.
template <int N, bool INV>
__device__ __forceinline__ void fft_reg(float2 (&x)[N]) {
    BitRevSwap<N, 0>::run(x);
    Radix2Stage<N, 1, INV>::run(x);
}

}  // namespace boltz_dev
