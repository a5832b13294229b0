// Two-dimensional grids with N = 128: each 128-point line is transformed by a
// group of 4 consecutive lanes (a line does not fit one thread's registers).
//
// Cooperative transform: lane l of a group holds the decimated subsequence
// x[4m + l], m = 0..31.  Each lane runs a register 32-point FFT, multiplies by
// W_128^{l k'}, and a radix-4 butterfly across the group (warp shuffles)
// leaves lane q holding X[32 q + k'], k' = 0..31 — natural order:
//   X[k' + 32 q] = sum_l (W_128^{l k'} Y_l[k']) W_4^{l q}.
// The kernels mirror k_synth / k_analysis / k_output for d = 2 with two
// fields per CTA (256 threads each).
#pragma once

#include "kernels.cuh"

namespace boltz_dev {

constexpr int kW = 128;          // line length
constexpr int kWH = 64;          // N/2
constexpr int kWNH = 65;         // half-axis length
constexpr int kWRS = 65;         // smem row stride (complex)
constexpr int kWTPF = 256;       // threads per field: 64 lines x 4 lanes
constexpr int kWFPC = 2;         // fields per CTA
constexpr size_t kWSMEM = size_t(kWFPC) * kW * kWRS * sizeof(float2) + kW * sizeof(float2);

// tw: shared table exp(-2 pi i t / 128); l: lane within the group; gbase: first lane of the group
template <bool INV>
__device__ __forceinline__ void fft128_coop(float2 (&y)[32], int l, int gbase, const float2* tw) {
    fft_reg<32, INV>(y);
#pragma unroll
    for (int k = 1; k < 32; ++k) {
        float2 w = tw[l * k];
        if (INV) w.y = -w.y;
        y[k] = cmul(y[k], w);
    }
    const unsigned mask = 0xffffffffu;
    const int q = l;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        float2 z[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            z[s].x = __shfl_sync(mask, y[k].x, gbase + s);
            z[s].y = __shfl_sync(mask, y[k].y, gbase + s);
        }
        const float2 a = cadd(z[0], z[2]), b = csub(z[0], z[2]), c = cadd(z[1], z[3]), d = csub(z[1], z[3]);
        // forward: X1 = b - i d, X3 = b + i d; inverse swaps the signs of i
        const float2 md = INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);     // -+ i d
        float2 out;
        if (q == 0) out = cadd(a, c);
        else if (q == 1) out = cadd(b, md);
        else if (q == 2) out = csub(a, c);
        else out = csub(b, md);
        y[k] = out;
    }
}

template <int MODE>
__global__ void __launch_bounds__(kWTPF * kWFPC) k_synth_w128(SynParams P) {
    using G = Geo<kW, 2>;
    extern __shared__ float2 smem[];
    float2* tw = smem + kWFPC * kW * kWRS;
    const int grp = threadIdx.x / kWTPF, lt = threadIdx.x % kWTPF;
    const int f = blockIdx.x * kWFPC + grp;
    const bool active = f < P.n_fields;
    float2* s = smem + grp * kW * kWRS;
    for (int i = threadIdx.x; i < kW; i += blockDim.x) tw[i] = c_twiddle[i];
    int input = 0, node = P.id_node;
    bool use_gm = false;
    if (active) {
        const int jj = f % P.n_c;
        input = P.inputs[jj];
        if (MODE == SYN_SHIFT) {
            const int t = f / P.n_c, p = t % P.M, qq = t / P.M;
            node = (P.q0 + qq) * P.M + p;
        } else {
            use_gm = f >= P.n_c;
        }
    }
    __syncthreads();
    const float2* __restrict__ src = P.spectra + (size_t)input * G::half;
    const float2* __restrict__ ph = P.phase + (size_t)node * 2 * kW;
    const int line = lt >> 2, l = lt & 3, gbase = (threadIdx.x & 31) & ~3;
    float2 y[32];
    // axis 0: column k1 = line (< 64), lane l holds k0 = 4m + l
    if (active) {
        const int k1 = line;
        const float2 w1 = __ldg(&ph[kW + k1]);
#pragma unroll
        for (int m = 0; m < 32; ++m) {
            const int k0 = 4 * m + l;
            float2 v = cmul(__ldg(&src[k0 * kWNH + k1]), cmul(w1, __ldg(&ph[k0])));
            if (MODE == SYN_PREP && use_gm) {
                const int a = wrapk(k0, kW);
                v = cscale(v, P.gm_full ? __ldg(&P.gm_full[k0 * kWNH + k1]) : __ldg(&P.gm[a * a + k1 * k1]));
            }
            y[m] = v;
        }
    }
    fft128_coop<true>(y, l, gbase, tw);            // all lanes take part (shuffles)
    if (active) {
#pragma unroll
        for (int k = 0; k < 32; ++k) s[(32 * l + k) * kWRS + line] = y[k];
    }
    __syncthreads();
    // axis 1: complex-to-real of rows i0 = line and line + 64; lane l holds positions 4m + l
    if (active) {
        const float2* r1 = s + line * kWRS;
        const float2* r2 = s + (line + kWH) * kWRS;
#pragma unroll
        for (int m = 0; m < 32; ++m) {
            const int k = 4 * m + l;
            if (k == 0) y[m] = make_float2(r1[0].x, r2[0].x);
            else if (k == kWH) y[m] = make_float2(0.f, 0.f);
            else if (k < kWH) {
                const float2 a = r1[k], b = r2[k];
                y[m] = make_float2(a.x - b.y, a.y + b.x);
            } else {
                const float2 a = r1[kW - k], b = r2[kW - k];
                y[m] = make_float2(a.x + b.y, b.x - a.y);
            }
        }
    }
    fft128_coop<true>(y, l, gbase, tw);
    if (active) {
        auto row_ptr = [&](int r) -> float* {
            if (MODE == SYN_SHIFT) return shifted_field_row<kW, 2>(P.out, f / P.n_c, f % P.n_c, P.n_c, r * kW);
            return P.out + (size_t)f * G::n + (size_t)r * kW;
        };
        float4* o1 = reinterpret_cast<float4*>(row_ptr(line) + 32 * l);
        float4* o2 = reinterpret_cast<float4*>(row_ptr(line + kWH) + 32 * l);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            o1[c] = make_float4(y[4 * c].x, y[4 * c + 1].x, y[4 * c + 2].x, y[4 * c + 3].x);
            o2[c] = make_float4(y[4 * c].y, y[4 * c + 1].y, y[4 * c + 2].y, y[4 * c + 3].y);
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(kWTPF * kWFPC) k_analysis_w128(AnaParams P) {
    using G = Geo<kW, 2>;
    extern __shared__ float2 smem[];
    float2* tw = smem + kWFPC * kW * kWRS;
    const int grp = threadIdx.x / kWTPF, lt = threadIdx.x % kWTPF;
    const int f = blockIdx.x * kWFPC + grp;
    const bool active = f < P.n_fields;
    float2* s = smem + grp * kW * kWRS;
    float2* __restrict__ dst = P.out + (size_t)f * G::half;
    for (int i = threadIdx.x; i < kW; i += blockDim.x) tw[i] = c_twiddle[i];
    __syncthreads();
    const int line = lt >> 2, l = lt & 3, lane = threadIdx.x & 31, gbase = lane & ~3;
    float2 y[32];
    const int n_iter = (MODE == ANA_ACCUM) ? P.nq : 1;
    for (int qq = 0; qq < n_iter; ++qq) {
        const float* __restrict__ src =
            (MODE == ANA_ACCUM) ? P.in + ((size_t)qq * P.U + f) * G::n : P.in + (size_t)f * G::n;
        const float* __restrict__ ct = P.ctab + (size_t)(P.q0 + qq) * (G::SMAX + 1);
        // rows line and line + 64 packed as one complex line
        if (active) {
#pragma unroll
            for (int m = 0; m < 32; ++m) {
                const int k = 4 * m + l;
                y[m] = make_float2(__ldg(&src[line * kW + k]), __ldg(&src[(line + kWH) * kW + k]));
            }
        }
        fft128_coop<false>(y, l, gbase, tw);
        // split: X1 = (Z_k + conj Z_{N-k})/2, X2 = (Z_k - conj Z_{N-k})/(2i); Z_{N-k} lives in lane 3-l
        // (index 32-k') or, for k' = 0, in lane (4-l)%4 (index 0)
        float2 zc[32];
        {
            const float zx = __shfl_sync(0xffffffffu, y[0].x, gbase + ((4 - l) & 3));
            const float zy = __shfl_sync(0xffffffffu, y[0].y, gbase + ((4 - l) & 3));
            zc[0] = make_float2(zx, zy);
        }
#pragma unroll
        for (int k = 1; k < 32; ++k) {
            zc[k].x = __shfl_sync(0xffffffffu, y[32 - k].x, gbase + 3 - l);
            zc[k].y = __shfl_sync(0xffffffffu, y[32 - k].y, gbase + 3 - l);
        }
        if (active) {
            float2* r1 = s + line * kWRS;
            float2* r2 = s + (line + kWH) * kWRS;
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const int kk = 32 * l + k;
                if (kk <= kWH) {
                    const float2 z = y[k], c = zc[k];
                    r1[kk] = make_float2(0.5f * (z.x + c.x), 0.5f * (z.y - c.y));
                    r2[kk] = make_float2(0.5f * (z.y + c.y), -0.5f * (z.x - c.x));
                }
            }
        }
        __syncthreads();
        // axis 0: columns k1 = 0..64 (65 columns over 64 groups: group 0 also takes column 64)
        for (int pass = 0; pass < 2; ++pass) {
            const int k1 = pass == 0 ? line : kWH;
            const bool col_active = active && (pass == 0 || line == 0);
            if (pass == 1 && __syncthreads_or(col_active) == 0) break;
            if (col_active) {
#pragma unroll
                for (int m = 0; m < 32; ++m) y[m] = s[(4 * m + l) * kWRS + k1];
            }
            fft128_coop<false>(y, l, gbase, tw);
            if (col_active) {
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    const int k0 = 32 * l + k;
                    const int idx = k0 * kWNH + k1;
                    const int par = (k0 + k1) & 1;
                    if (MODE == ANA_SPECTRUM) {
                        const bool nyq = (k0 == kWH) || (k1 == kWH);
                        const float sc = nyq ? 0.f : (par ? -P.inv_n : P.inv_n);
                        dst[idx] = cscale(y[k], sc);
                    } else {
                        const int a = wrapk(k0, kW);
                        const float c0 = __ldg(&ct[a * a + k1 * k1]);
                        const float sc = par ? -c0 : c0;
                        const float2 old = dst[idx];
                        dst[idx] = make_float2(fmaf(y[k].x, sc, old.x), fmaf(y[k].y, sc, old.y));
                    }
                }
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kWTPF * kWFPC) k_output_w128(OutParams P) {
    using G = Geo<kW, 2>;
    extern __shared__ float2 smem[];
    float2* tw = smem + kWFPC * kW * kWRS;
    const int grp = threadIdx.x / kWTPF, lt = threadIdx.x % kWTPF;
    const int u = blockIdx.x * kWFPC + grp;
    const bool active = u < P.U;
    float2* s = smem + grp * kW * kWRS;
    const float2* __restrict__ src = P.qhat + (size_t)u * G::half;
    for (int i = threadIdx.x; i < kW; i += blockDim.x) tw[i] = c_twiddle[i];
    __syncthreads();
    const int line = lt >> 2, l = lt & 3, lane = threadIdx.x & 31, gbase = lane & ~3;
    float2 y[32];
    // axis 0 over all columns k1 = 0..64, sign (-1)^k from the index parity
    for (int pass = 0; pass < 2; ++pass) {
        const int k1 = pass == 0 ? line : kWH;
        const bool col_active = active && (pass == 0 || line == 0);
        if (pass == 1 && __syncthreads_or(col_active) == 0) break;
        if (col_active) {
#pragma unroll
            for (int m = 0; m < 32; ++m) {
                const int k0 = 4 * m + l;
                const float2 v = src[k0 * kWNH + k1];
                y[m] = ((k0 + k1) & 1) ? make_float2(-v.x, -v.y) : v;
            }
        }
        fft128_coop<true>(y, l, gbase, tw);
        if (col_active) {
#pragma unroll
            for (int k = 0; k < 32; ++k) s[(32 * l + k) * kWRS + k1] = y[k];
        }
    }
    __syncthreads();
    if (active) {
        const float2* r1 = s + line * kWRS;
        const float2* r2 = s + (line + kWH) * kWRS;
#pragma unroll
        for (int m = 0; m < 32; ++m) {
            const int k = 4 * m + l;
            if (k == 0) y[m] = make_float2(r1[0].x, r2[0].x);
            else if (k == kWH) y[m] = make_float2(r1[kWH].x, r2[kWH].x);
            else if (k < kWH) {
                const float2 a = r1[k], b = r2[k];
                y[m] = make_float2(a.x - b.y, a.y + b.x);
            } else {
                const float2 a = r1[kW - k], b = r2[kW - k];
                y[m] = make_float2(a.x + b.y, b.x - a.y);
            }
        }
    }
    fft128_coop<true>(y, l, gbase, tw);
    if (!active) return;
    bool bad = false;
    for (int o = P.out_start[u]; o < P.out_start[u + 1]; ++o) {
        const int4 e = P.outs[o];
        const size_t off1 = (size_t)line * kW + 32 * l, off2 = (size_t)(line + kWH) * kW + 32 * l;
        const float4* f1 = reinterpret_cast<const float4*>(P.fN + (size_t)e.z * G::n + off1);
        const float4* f2 = reinterpret_cast<const float4*>(P.fN + (size_t)e.z * G::n + off2);
        const float4* l1 = reinterpret_cast<const float4*>(P.lam + (size_t)e.y * G::n + off1);
        const float4* l2 = reinterpret_cast<const float4*>(P.lam + (size_t)e.y * G::n + off2);
        float4* q1 = reinterpret_cast<float4*>(P.Q + (size_t)e.x * G::n + off1);
        float4* q2 = reinterpret_cast<float4*>(P.Q + (size_t)e.x * G::n + off2);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float4 a = __ldg(&f1[c]), b = __ldg(&l1[c]), a2 = __ldg(&f2[c]), b2 = __ldg(&l2[c]);
            const float4 v1 = make_float4(fmaf(-a.x, b.x, y[4 * c].x), fmaf(-a.y, b.y, y[4 * c + 1].x),
                                          fmaf(-a.z, b.z, y[4 * c + 2].x), fmaf(-a.w, b.w, y[4 * c + 3].x));
            const float4 v2 = make_float4(fmaf(-a2.x, b2.x, y[4 * c].y), fmaf(-a2.y, b2.y, y[4 * c + 1].y),
                                          fmaf(-a2.z, b2.z, y[4 * c + 2].y), fmaf(-a2.w, b2.w, y[4 * c + 3].y));
            bad |= nonfinite4(v1) || nonfinite4(v2);
            q1[c] = v1;
            q2[c] = v2;
        }
    }
    if (bad) atomicOr(P.err, kErrNonFinite);
}

}  // namespace boltz_dev
