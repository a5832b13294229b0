// Register-resident complex FFTs of compile-time length (sm_103a).
//
// One thread owns one length-N line in registers; the bit-reversal permutation
// and every twiddle index are resolved at compile time, trivial twiddles
// (1, -i, -1, i) cost no multiply, the rest come from constant-memory tables
// exp(-2 pi i t / 128) and exp(-2 pi i t / 48) filled on the host in FP64.
// Transforms are unnormalised: forward X_k = sum_j x_j e^{-2 pi i jk/N},
// inverse with e^{+}.  The element type is float2 (the FP32 path) or double2
// (the FP64 check build); both run the same code.
#pragma once

#include <cuda_runtime.h>

namespace boltz_dev {

__constant__ float2 c_twiddle[128];
__constant__ float2 c_twiddle48[48];     // exp(-2 pi i t / 48), for the lengths 3 * 2^k
__constant__ double2 c_twiddle_d[128];
__constant__ double2 c_twiddle48_d[48];

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// Real type R, its complex pair C and the twiddle tables of that precision.
template <typename R>
struct Prec;
template <>
struct Prec<float> {
    using C = float2;
    static __device__ __forceinline__ C mk(float x, float y) { return make_float2(x, y); }
    static __device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
    static __device__ __forceinline__ C tw128(int t) { return c_twiddle[t]; }
    static __device__ __forceinline__ C tw48(int t) { return c_twiddle48[t]; }
};
template <>
struct Prec<double> {
    using C = double2;
    static __device__ __forceinline__ C mk(double x, double y) { return make_double2(x, y); }
    static __device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
    static __device__ __forceinline__ C tw128(int t) { return c_twiddle_d[t]; }
    static __device__ __forceinline__ C tw48(int t) { return c_twiddle48_d[t]; }
};

// real type of a complex pair
template <typename C>
struct RealOf;
template <>
struct RealOf<float2> {
    using R = float;
};
template <>
struct RealOf<double2> {
    using R = double;
};

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
__host__ __device__ constexpr int bitrev(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

// a * exp(-+ 2 pi i t / 128), t in [0, 128) known at compile time after unrolling.
template <bool INV, typename C>
__device__ __forceinline__ C twiddle_mul(C a, int t) {
    using P = Prec<typename RealOf<C>::R>;
    if (t == 0) return a;
    if (t == 64) return P::mk(-a.x, -a.y);
    if (t == 32) return INV ? P::mk(-a.y, a.x) : P::mk(a.y, -a.x);
    if (t == 96) return INV ? P::mk(a.y, -a.x) : P::mk(-a.y, a.x);
    C w = P::tw128(t);
    if (INV) w.y = -w.y;
    return cmul(a, w);
}

// Bit-reversal permutation with indices fixed at compile time (template
// recursion), so the register array is never indexed dynamically.
template <int N, int I, typename C>
struct BitRevSwap {
    static __device__ __forceinline__ void run(C (&x)[N]) {
        constexpr int J = bitrev(I, ilog2(N));
        if constexpr (J > I) {
            const C t = x[I];
            x[I] = x[J];
            x[J] = t;
        }
        BitRevSwap<N, I + 1, C>::run(x);
    }
};
template <int N, typename C>
struct BitRevSwap<N, N, C> {
    static __device__ __forceinline__ void run(C (&)[N]) {}
};

// Radix-2 butterfly (u, v) <- (u + w v, u - w v), w = exp(-+ 2 pi i t / 128).
// A trivial twiddle (t = 0, 32, 64, 96) costs additions only.  Otherwise the
// sum is formed with four fused multiply-adds and the difference as
// 2 u - (u + w v), one more fused multiply-add per component: 6 instructions
// instead of the 8 of a complex multiply followed by two complex additions.
// The difference carries one rounding of the sum, an error of at most one
// unit in the last place of max(|u|, |w v|), the same order as the plain form.
template <bool INV, typename C>
__device__ __forceinline__ void butterfly(C& u, C& v, int t) {
    using R = typename RealOf<C>::R;
    using P = Prec<R>;
    if (t == 0 || t == 32 || t == 64 || t == 96) {
        const C a = u, b = twiddle_mul<INV>(v, t);
        u = cadd(a, b);
        v = csub(a, b);
        return;
    }
    C w = P::tw128(t);
    if (INV) w.y = -w.y;
    const R sr = P::fma_(w.x, v.x, P::fma_(-w.y, v.y, u.x));
    const R si = P::fma_(w.x, v.y, P::fma_(w.y, v.x, u.y));
    v = P::mk(P::fma_(R(2), u.x, -sr), P::fma_(R(2), u.y, -si));
    u = P::mk(sr, si);
}

// One radix-2 stage (butterfly span m = 2^S); trip counts are compile-time
// constants so the whole transform unrolls into straight-line register code.
template <int N, int S, bool INV, typename C>
struct Radix2Stage {
    static __device__ __forceinline__ void run(C (&x)[N]) {
        constexpr int m = 1 << S, h = m >> 1;
#pragma unroll
        for (int i = 0; i < N; i += m) {
#pragma unroll
            for (int k = 0; k < h; ++k) butterfly<INV>(x[i + k], x[i + k + h], k * (128 / m));
        }
        if constexpr (m < N) Radix2Stage<N, S + 1, INV, C>::run(x);
    }
};

// In-place radix-2 decimation-in-time FFT of N (power of two, <= 128) points.
template <int N, bool INV, typename C>
__device__ __forceinline__ void fft_pow2(C (&x)[N]) {
    BitRevSwap<N, 0, C>::run(x);
    Radix2Stage<N, 1, INV, C>::run(x);
}

// a * exp(-+ 2 pi i t / 48), t in [0, 48) known at compile time.
template <bool INV, typename C>
__device__ __forceinline__ C twiddle48_mul(C a, int t) {
    using P = Prec<typename RealOf<C>::R>;
    if (t == 0) return a;
    if (t == 24) return P::mk(-a.x, -a.y);
    if (t == 12) return INV ? P::mk(-a.y, a.x) : P::mk(a.y, -a.x);
    if (t == 36) return INV ? P::mk(a.y, -a.x) : P::mk(-a.y, a.x);
    C w = P::tw48(t);
    if (INV) w.y = -w.y;
    return cmul(a, w);
}

// Mixed radix for N = 3 * 2^k (24, 48): one radix-3 decimation-in-time step
// over three power-of-two transforms of the subsequences x[3m + r]:
//   X[k + jM] = sum_r w3^{jr} W_N^{rk} Y_r[k],  M = N/3, w3 = exp(-+ 2 pi i/3).
template <int N, bool INV, typename C>
__device__ __forceinline__ void fft_radix3(C (&x)[N]) {
    using R = typename RealOf<C>::R;
    using P = Prec<R>;
    constexpr int M = N / 3;
    static_assert(48 % N == 0, "radix-3 lengths are divisors of 48");
    C y0[M], y1[M], y2[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        y0[m] = x[3 * m];
        y1[m] = x[3 * m + 1];
        y2[m] = x[3 * m + 2];
    }
    fft_pow2<M, INV>(y0);
    fft_pow2<M, INV>(y1);
    fft_pow2<M, INV>(y2);
    const R S3 = R(0.86602540378443864676);               // sqrt(3)/2
    const R HALF = R(0.5);
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const C t1 = twiddle48_mul<INV>(y1[k], k * (48 / N));
        const C t2 = twiddle48_mul<INV>(y2[k], 2 * k * (48 / N));
        const C s = cadd(t1, t2), d = csub(t1, t2);
        const C base = P::mk(y0[k].x - HALF * s.x, y0[k].y - HALF * s.y);
        // forward: w3 t1 + w3^2 t2 = -s/2 - i (sqrt3/2) d ; inverse flips the sign of the i term
        const C id = INV ? P::mk(-S3 * d.y, S3 * d.x) : P::mk(S3 * d.y, -S3 * d.x);
        x[k] = cadd(y0[k], s);
        x[k + M] = cadd(base, id);
        x[k + 2 * M] = csub(base, id);
    }
}

// FFT of a register-resident line of N points: powers of two up to 128, and 24, 48.
template <int N, bool INV, typename C>
__device__ __forceinline__ void fft_reg(C (&x)[N]) {
    if constexpr (N % 3 == 0) fft_radix3<N, INV>(x);
    else fft_pow2<N, INV>(x);
}

}  // namespace boltz_dev
