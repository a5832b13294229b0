// sm_103a kernels of the separated fast-spectral collision operator.
//
// The single-CTA field kernels, the sigma-contraction and the CUDA-core
// projection are templates on the real type R: float for the product path,
// double for the FP64 check build of the small grids (same code, same
// schedule).  The cluster kernels (3D 32^3, 48^3, 64^3) are FP32 only.
//
// Field layout (all kernels): a physical field is float [N]^D, C order, axis
// 0 slowest; a spectrum is the real-to-complex half spectrum float2
// [N]^(D-1) x [N/2+1] (last axis k = 0..N/2, other axes in DFT index order).
// A CTA holds FPC fields at once, TPF threads per field; every 1-D transform
// along an axis is done by one thread in registers (fft_reg), the transposes
// between axes go through shared memory whose rows are padded to N/2+1
// complex entries so that both row- and column-wise accesses are free of bank
// conflicts.  The real-to-complex and complex-to-real steps along the last
// axis pack two real lines into one complex line.
//
// Sign and scale conventions: with v_j = -L + j dv the synthesis
// sum_k F_k exp(i pi k.v_j / L) equals sum_k F_k (-1)^k exp(2 pi i k.j / N),
// so the (-1)^k factor is folded into the phase tables (synthesis) or applied
// from the index parity (analysis, output); the 1/N^D of the analysis is
// folded into the radial table.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "async.cuh"
#include "fft.cuh"

namespace boltz_dev {

template <int N, int D>
struct Geo {
    static constexpr int H = N / 2;
    static constexpr int NH = H + 1;                             // half-axis length
    static constexpr int RS = H + 1;                             // smem row stride (float2)
    static constexpr int n = (D == 3) ? N * N * N : N * N;       // real points
    static constexpr int half = (D == 3) ? N * N * NH : N * NH;  // half-spectrum entries
    static constexpr int TPF = (D == 3) ? N * H : H;             // threads per field
    static constexpr int SMEM_F = (D == 3) ? N * N * RS : N * RS;
    static constexpr int COLS = (D == 3) ? N * NH : NH;          // columns incl. the half-axis Nyquist
    static constexpr int SMAX = D * H * H;                       // largest |k|^2
    // shifted fields are stored voxel-chunk-major (see shifted_field_row)
    // voxels per chunk: 256 for power-of-two sizes, 288 (a whole number of rows) for N = 24, 48
    static constexpr int VCH = n < 256 ? n : (N % 3 == 0 ? 288 : 256);
    static constexpr int NCH = n / VCH;                          // chunks per field
};

// Layout of the shifted-field buffer: for slot s = qq*M + p (node in the
// block, direction) and chunk-local input jj, voxel v of the field is stored at
//   out[((s * NCH + v / VCH) * n_c + jj) * VCH + v % VCH],
// so the rows of all inputs of one (slot, voxel chunk) are one contiguous
// block that the contraction fetches with a single bulk copy.
template <int N, int D, typename R>
__device__ __forceinline__ R* shifted_field_row(R* out, int slot, int jj, int n_c, int v) {
    using G = Geo<N, D>;
    return out + (((size_t)slot * G::NCH + v / G::VCH) * n_c + jj) * G::VCH + (v % G::VCH);
}

__device__ __forceinline__ int wrapk(int i, int N) { return i < N / 2 ? i : i - N; }

// ------------------------------------------------------------------ synthesis
// Spectra -> real fields.  SHIFT: the shifted fields A_{q,p,j}(v) =
// g_j,N(v - rho_q sigma_p / 2) for every (node in the q-block, direction,
// chunk input); PREP: f_N (identity node) and Lambda_g (identity node times
// the loss multiplier G-(|l|^2)) for every chunk input.
// MULT: the Carleman-form fields IDFT(m_s * ghat) for every (slot s, chunk input)
// with real per-mode multiplier tables m_s (which carry the (-1)^k grid sign
// and are zero at the Nyquist indices).
enum { SYN_SHIFT = 0, SYN_PREP = 1, SYN_MULT = 2 };

template <typename R>
struct SynParamsT {
    using C = typename Prec<R>::C;
    const C* spectra;       // [n_inputs][half]
    const int* inputs;      // chunk-local -> global input index [n_c]
    const C* phase;         // [nodes][D][N]: (-1)^k exp(-i pi k s_a / L), zero at the Nyquist index
    const R* gm;            // [SMAX+1] loss multiplier (function of |l|^2)
    const R* gm_full;       // PREP: [half] loss multiplier per mode, or null (then gm)
    const R* mult;          // MULT: [slots][half] multipliers
    R* out;                 // SHIFT: [nq][M][n_c][n]; MULT: [slots][n_c][n]; PREP: [2][n_c][n]
    int n_c, M, q0, id_node, n_fields;
};
using SynParams = SynParamsT<float>;

// Two real rows of N values to and from the two halves of a complex register
// line (x[c].x <-> row a, x[c].y <-> row b) with 16-byte accesses.
template <int N>
__device__ __forceinline__ void store_two_rows(float* a, float* b, const float2 (&x)[N]) {
    float4* o1 = reinterpret_cast<float4*>(a);
    float4* o2 = reinterpret_cast<float4*>(b);
#pragma unroll
    for (int c = 0; c < N / 4; ++c) {
        o1[c] = make_float4(x[4 * c].x, x[4 * c + 1].x, x[4 * c + 2].x, x[4 * c + 3].x);
        o2[c] = make_float4(x[4 * c].y, x[4 * c + 1].y, x[4 * c + 2].y, x[4 * c + 3].y);
    }
}
template <int N>
__device__ __forceinline__ void store_two_rows(double* a, double* b, const double2 (&x)[N]) {
    double2* o1 = reinterpret_cast<double2*>(a);
    double2* o2 = reinterpret_cast<double2*>(b);
#pragma unroll
    for (int c = 0; c < N / 2; ++c) {
        o1[c] = make_double2(x[2 * c].x, x[2 * c + 1].x);
        o2[c] = make_double2(x[2 * c].y, x[2 * c + 1].y);
    }
}
template <int N>
__device__ __forceinline__ void load_two_rows(const float* a, const float* b, float2 (&x)[N]) {
    const float4* a4 = reinterpret_cast<const float4*>(a);
    const float4* b4 = reinterpret_cast<const float4*>(b);
#pragma unroll
    for (int c = 0; c < N / 4; ++c) {
        const float4 p = __ldg(&a4[c]), q = __ldg(&b4[c]);
        x[4 * c] = make_float2(p.x, q.x);
        x[4 * c + 1] = make_float2(p.y, q.y);
        x[4 * c + 2] = make_float2(p.z, q.z);
        x[4 * c + 3] = make_float2(p.w, q.w);
    }
}
template <int N>
__device__ __forceinline__ void load_two_rows(const double* a, const double* b, double2 (&x)[N]) {
    const double2* a2 = reinterpret_cast<const double2*>(a);
    const double2* b2 = reinterpret_cast<const double2*>(b);
#pragma unroll
    for (int c = 0; c < N / 2; ++c) {
        const double2 p = __ldg(&a2[c]), q = __ldg(&b2[c]);
        x[2 * c] = make_double2(p.x, q.x);
        x[2 * c + 1] = make_double2(p.y, q.y);
    }
}

template <int N, int D, int FPC, int MODE, typename R = float>
__global__ void __launch_bounds__(Geo<N, D>::TPF * FPC) k_synth(SynParamsT<R> P) {
    using G = Geo<N, D>;
    using PR = Prec<R>;
    using C = typename PR::C;
    constexpr int H = G::H, RS = G::RS;
    extern __shared__ __align__(16) unsigned char fsm_raw[];
    const int grp = threadIdx.x / G::TPF, lt = threadIdx.x % G::TPF;
    const int f = blockIdx.x * FPC + grp;
    const bool active = f < P.n_fields;
    C* s = reinterpret_cast<C*>(fsm_raw) + grp * G::SMEM_F;

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
    const C* __restrict__ src = P.spectra + (size_t)input * G::half;
    const C* __restrict__ ph = P.phase + (size_t)node * D * N;
    // start of row r of this field in the output (rows never straddle a voxel chunk)
    auto row_ptr = [&](int r) -> R* {
        if (MODE != SYN_PREP) return shifted_field_row<N, D>(P.out, f / P.n_c, f % P.n_c, P.n_c, r * N);
        return P.out + (size_t)f * G::n + (size_t)r * N;
    };
    const R* __restrict__ mu = (MODE == SYN_MULT) ? P.mult + (size_t)(active ? f / P.n_c : 0) * G::half : nullptr;
    C x[N];

    if (D == 3) {
        // axis 0: columns (k1, k2), k2 < N/2 (the input's half-axis Nyquist is zero)
        if (active) {
            const int k1 = lt / H, k2 = lt % H;
            const C w12 = cmul(__ldg(&ph[N + k1]), __ldg(&ph[2 * N + k2]));
#pragma unroll
            for (int k0 = 0; k0 < N; ++k0) {
                const int idx = (k0 * N + k1) * G::NH + k2;
                C v;
                if constexpr (MODE == SYN_MULT) {
                    v = cscale(__ldg(&src[idx]), __ldg(&mu[idx]));
                } else {
                    v = cmul(__ldg(&src[idx]), cmul(w12, __ldg(&ph[k0])));
                    if (MODE == SYN_PREP && use_gm) {
                        const int a = wrapk(k0, N), b = wrapk(k1, N);
                        v = cscale(v, P.gm_full ? __ldg(&P.gm_full[idx]) : __ldg(&P.gm[a * a + b * b + k2 * k2]));
                    }
                }
                x[k0] = v;
            }
            fft_reg<N, true>(x);
#pragma unroll
            for (int i0 = 0; i0 < N; ++i0) s[(i0 * N + k1) * RS + k2] = x[i0];
        }
        __syncthreads();
        // axis 1
        if (active) {
            const int i0 = lt / H, k2 = lt % H;
#pragma unroll
            for (int k1 = 0; k1 < N; ++k1) x[k1] = s[(i0 * N + k1) * RS + k2];
            fft_reg<N, true>(x);
#pragma unroll
            for (int i1 = 0; i1 < N; ++i1) s[(i0 * N + i1) * RS + k2] = x[i1];
        }
        __syncthreads();
        // axis 2: complex-to-real of rows (i0, i1) and (i0, i1 + N/2) together
        if (active) {
            const int i0 = lt / H, i1 = lt % H;
            const C* r1 = s + (i0 * N + i1) * RS;
            const C* r2 = s + (i0 * N + i1 + H) * RS;
            x[0] = PR::mk(r1[0].x, r2[0].x);
            x[H] = PR::mk(R(0), R(0));
#pragma unroll
            for (int k = 1; k < H; ++k) {
                const C a = r1[k], b = r2[k];
                x[k] = PR::mk(a.x - b.y, a.y + b.x);
                x[N - k] = PR::mk(a.x + b.y, b.x - a.y);
            }
            fft_reg<N, true>(x);
            store_two_rows<N>(row_ptr(i0 * N + i1), row_ptr(i0 * N + i1 + H), x);
        }
    } else {
        // axis 0: columns k1 < N/2
        if (active) {
            const int k1 = lt;
            const C w1 = __ldg(&ph[N + k1]);
#pragma unroll
            for (int k0 = 0; k0 < N; ++k0) {
                const int idx = k0 * G::NH + k1;
                C v;
                if constexpr (MODE == SYN_MULT) {
                    v = cscale(__ldg(&src[idx]), __ldg(&mu[idx]));
                } else {
                    v = cmul(__ldg(&src[idx]), cmul(w1, __ldg(&ph[k0])));
                    if (MODE == SYN_PREP && use_gm) {
                        const int a = wrapk(k0, N);
                        v = cscale(v, P.gm_full ? __ldg(&P.gm_full[idx]) : __ldg(&P.gm[a * a + k1 * k1]));
                    }
                }
                x[k0] = v;
            }
            fft_reg<N, true>(x);
#pragma unroll
            for (int i0 = 0; i0 < N; ++i0) s[i0 * RS + k1] = x[i0];
        }
        __syncthreads();
        // axis 1: complex-to-real of rows i0 and i0 + N/2
        if (active) {
            const int i0 = lt;
            const C* r1 = s + i0 * RS;
            const C* r2 = s + (i0 + H) * RS;
            x[0] = PR::mk(r1[0].x, r2[0].x);
            x[H] = PR::mk(R(0), R(0));
#pragma unroll
            for (int k = 1; k < H; ++k) {
                const C a = r1[k], b = r2[k];
                x[k] = PR::mk(a.x - b.y, a.y + b.x);
                x[N - k] = PR::mk(a.x + b.y, b.x - a.y);
            }
            fft_reg<N, true>(x);
            store_two_rows<N>(row_ptr(i0), row_ptr(i0 + H), x);
        }
    }
}

// ------------------------------------------------------------------ analysis
// Real fields -> half spectra.  SPECTRUM: the input spectra (x (-1)^k / n,
// Nyquist entries written as zero).  ACCUM: for every gain slot u and node q
// of the q-block, Qhat+_u += c_q(|k|^2) (-1)^k DFT[P_{q,u}]  (c_q includes 1/n).
enum { ANA_SPECTRUM = 0, ANA_ACCUM = 1 };

template <typename R>
struct AnaParamsT {
    using C = typename Prec<R>::C;
    const R* in;         // SPECTRUM: [n_fields][n]; ACCUM: [nq][U][n]
    C* out;              // [n_fields][half]
    const R* ctab;       // [N_rho][SMAX+1]
    int n_fields, nq, q0, U;
    R inv_n;
};
using AnaParams = AnaParamsT<float>;

template <int N, int D, int FPC, int MODE, typename R = float>
__global__ void __launch_bounds__(Geo<N, D>::TPF * FPC) k_analysis(AnaParamsT<R> P) {
    using G = Geo<N, D>;
    using PR = Prec<R>;
    using C = typename PR::C;
    constexpr int H = G::H, RS = G::RS, NH = G::NH;
    extern __shared__ __align__(16) unsigned char fsm_raw[];
    const int grp = threadIdx.x / G::TPF, lt = threadIdx.x % G::TPF;
    const int f = blockIdx.x * FPC + grp;
    const bool active = f < P.n_fields;
    C* s = reinterpret_cast<C*>(fsm_raw) + grp * G::SMEM_F;
    C* __restrict__ dst = P.out + (size_t)f * G::half;
    C x[N];
    const int n_iter = (MODE == ANA_ACCUM) ? P.nq : 1;
    const R HALF = R(0.5);

    for (int qq = 0; qq < n_iter; ++qq) {
        const R* __restrict__ src =
            (MODE == ANA_ACCUM) ? P.in + ((size_t)qq * P.U + f) * G::n : P.in + (size_t)f * G::n;
        const R* __restrict__ ct = P.ctab + (size_t)(P.q0 + qq) * (G::SMAX + 1);
        // last axis: real-to-complex of two rows at once
        if (active) {
            const int row = (D == 3) ? (lt / H) * N + (lt % H) : lt;   // (i0, i1) or i0
            load_two_rows<N>(src + row * N, src + (row + H) * N, x);
            fft_reg<N, false>(x);
            C* r1 = s + row * RS;
            C* r2 = s + (row + H) * RS;
#pragma unroll
            for (int k = 0; k <= H; ++k) {
                const C z = x[k], zc = x[(N - k) % N];
                // X1 = (Z_k + conj Z_{N-k}) / 2,  X2 = (Z_k - conj Z_{N-k}) / (2i)
                r1[k] = PR::mk(HALF * (z.x + zc.x), HALF * (z.y - zc.y));
                r2[k] = PR::mk(HALF * (z.y + zc.y), -HALF * (z.x - zc.x));
            }
        }
        __syncthreads();
        if (D == 3) {
            // axis 1
            if (active) {
                for (int c = lt; c < G::COLS; c += G::TPF) {
                    const int i0 = c / NH, k2 = c % NH;
#pragma unroll
                    for (int k1 = 0; k1 < N; ++k1) x[k1] = s[(i0 * N + k1) * RS + k2];
                    fft_reg<N, false>(x);
#pragma unroll
                    for (int k1 = 0; k1 < N; ++k1) s[(i0 * N + k1) * RS + k2] = x[k1];
                }
            }
            __syncthreads();
        }
        // axis 0, then scale and store
        if (active) {
            for (int c = lt; c < G::COLS; c += G::TPF) {
                const int k1 = (D == 3) ? c / NH : 0, k2 = (D == 3) ? c % NH : c;
#pragma unroll
                for (int k0 = 0; k0 < N; ++k0) x[k0] = s[(D == 3 ? (k0 * N + k1) * RS : k0 * RS) + k2];
                fft_reg<N, false>(x);
#pragma unroll
                for (int k0 = 0; k0 < N; ++k0) {
                    const int idx = (D == 3) ? (k0 * N + k1) * NH + k2 : k0 * NH + k2;
                    const int par = (k0 + k1 + k2) & 1;
                    if (MODE == ANA_SPECTRUM) {
                        const bool nyq = (k0 == H) || (k2 == H) || (D == 3 && k1 == H);
                        const R sc = nyq ? R(0) : (par ? -P.inv_n : P.inv_n);
                        dst[idx] = cscale(x[k0], sc);
                    } else {
                        const int a = wrapk(k0, N), b = (D == 3) ? wrapk(k1, N) : 0;
                        const R c0 = __ldg(&ct[a * a + b * b + k2 * k2]);
                        const R sc = par ? -c0 : c0;
                        const C old = dst[idx];
                        dst[idx] = PR::mk(PR::fma_(x[k0].x, sc, old.x), PR::fma_(x[k0].y, sc, old.y));
                    }
                }
            }
        }
        __syncthreads();
    }
}

// Outputs of the output kernels: gain field of every slot (complex-to-real of
// Qhat+ with all modes, Nyquist included) minus the loss f_N(l) * Lambda(j),
// written for every ordered pair (e, j, l) that maps to the slot.
template <typename R>
struct OutParamsT {
    using C = typename Prec<R>::C;
    const C* qhat;        // [U][half]
    const R* fN;          // [n_c][n]
    const R* lam;         // [n_c][n]
    const int* out_start; // [U+1]
    const int4* outs;     // (e, jloc, lloc, 0)
    R* Q;                 // [n_pairs][n]
    int* err;             // device error word: kErrNonFinite when a written value is not finite
    int U;
};
using OutParams = OutParamsT<float>;

// True when any of the values is NaN or infinite (NaN fails every comparison).
__device__ __forceinline__ bool nonfinite4(const float4& v) {
    return !(fabsf(v.x) <= 3.402823466e38f && fabsf(v.y) <= 3.402823466e38f && fabsf(v.z) <= 3.402823466e38f &&
             fabsf(v.w) <= 3.402823466e38f);
}
__device__ __forceinline__ bool nonfinite2(const double2& v) {
    return !(fabs(v.x) <= 1.7976931348623157e308 && fabs(v.y) <= 1.7976931348623157e308);
}

// ------------------------------------------------------------------ 3D field kernels on a CTA cluster
// Same transforms as k_synth / k_analysis / k_output for d = 3, with one field
// spread over a cluster of CL CTAs: CTA r holds the PP = N/CL planes i0 in
// [r PP, r PP + PP) in shared memory (for 32^3 the synthesis runs on four
// CTAs of 37 KB, six per SM, the analysis and output on two CTAs of 73 KB,
// three per SM; 48^3 on eight CTAs of 60 KB; 64^3 on sixteen CTAs of 71 KB,
// a cluster size beyond the portable 8).  The transform along axis 0
// is the only one that crosses planes; it reads or writes the other CTAs'
// planes through distributed shared memory, between cluster barriers.  A
// CTA's part of a real field is one contiguous block of global memory; it is
// moved through a staging copy in shared memory (rows padded to N+4 floats)
// so that every warp reads or writes 512 contiguous bytes with 16-byte
// accesses, and the node's three phase rows are staged once per CTA.  Complex
// rows have an even stride (N/2 + 2 entries), so the real-to-complex and
// complex-to-real passes move two entries per 16-byte access.  Planes are
// padded by 8 complex entries so that the plane groups a warp touches fall on
// different banks, except for 32^3, where the two planes a warp touches need
// two wavefronts anyway and the padding would cost the sixth CTA per SM.
namespace cg = cooperative_groups;

template <int N, int CL>
struct ClusterGeo {
    static constexpr int H = N / 2;
    static constexpr int PP = N / CL;            // planes per CTA
    static constexpr int RS = H + 2;             // complex row stride (even: rows start on 16 bytes)
    static constexpr int PS = N * RS + (N == 32 ? 0 : 8);   // complex plane stride
    static constexpr int RR = N + 4;             // staged real row stride (floats, 16-byte rows)
    static constexpr int NT = PP * H;            // threads per CTA
    static constexpr int PART_N = PP * N * N;    // floats of a field held by one CTA
    static constexpr int COLS = PP * (H + 1);    // columns of a CTA incl. the half-axis Nyquist
    static constexpr size_t SMEM = size_t(PP) * PS * sizeof(float2) + 3 * N * sizeof(float2);
    static constexpr int MINB = (SMEM <= (37u << 10)) ? 6 : ((SMEM <= (74u << 10)) ? 3 : 1);
    static_assert(size_t(PP) * N * RR * sizeof(float) <= size_t(PP) * PS * sizeof(float2), "staging fits");
    static_assert((4 * NT) % N == 0 && (4 * NT) % Geo<N, 3>::VCH == 0 && PART_N % (4 * NT) == 0, "copy strides");
};

// pointers to the plane buffers of every CTA of the cluster (index = rank)
template <int CL>
__device__ __forceinline__ void cluster_planes(cg::cluster_group& cluster, float2* smem, float2* (&pl)[CL]) {
#pragma unroll
    for (int r = 0; r < CL; ++r) pl[r] = cluster.map_shared_rank(smem, r);
}

// Coalesced move of this CTA's part of a real field between a staging area in
// shared memory (rows of N floats padded to RR) and global memory, 16 bytes a
// thread: thread lt moves floats L = 4 lt + 4 NT it; both addresses advance
// by constants.
template <int N, int CL, bool TO_GLOBAL>
__device__ __forceinline__ void staged_copy(float* stg, float* gptr, size_t g_step, int lt) {
    using CG = ClusterGeo<N, CL>;
    constexpr int ITER = CG::PART_N / (4 * CG::NT);
    constexpr int S_STEP = (4 * CG::NT / N) * CG::RR;
    const int L0 = 4 * lt;
    float* sp = stg + (L0 / N) * CG::RR + (L0 % N);
#pragma unroll 8
    for (int it = 0; it < ITER; ++it) {
        float4* g = reinterpret_cast<float4*>(gptr + it * g_step);
        float4* sm = reinterpret_cast<float4*>(sp + it * S_STEP);
        if (TO_GLOBAL) *g = *sm;
        else *sm = __ldg(g);
    }
}

// Two rows of N reals staged in shared memory (16-byte aligned) into the two
// halves of a complex register line: x[c] = (a[c], b[c]).
template <int N>
__device__ __forceinline__ void load_two_rows_smem(const float* a, const float* b, float2 (&x)[N]) {
    const float4* a4 = reinterpret_cast<const float4*>(a);
    const float4* b4 = reinterpret_cast<const float4*>(b);
#pragma unroll
    for (int c = 0; c < N / 4; ++c) {
        const float4 p = a4[c], q = b4[c];
        x[4 * c] = make_float2(p.x, q.x);
        x[4 * c + 1] = make_float2(p.y, q.y);
        x[4 * c + 2] = make_float2(p.z, q.z);
        x[4 * c + 3] = make_float2(p.w, q.w);
    }
}

// Complex-to-real input line from two half-spectrum rows r1, r2 (entries
// 0..N/2, read 16 bytes at a time): x[k] = r1[k] + i r2[k] and
// x[N-k] = conj(r1[k]) + i conj(r2[k]), so that one complex inverse transform
// gives row 1 in the real and row 2 in the imaginary parts.  The Nyquist
// entries r[N/2] are read only when NYQ (they are zero in the shifted fields).
template <int N, bool NYQ>
__device__ __forceinline__ void c2r_pack_rows(const float2* r1, const float2* r2, float2 (&x)[N]) {
    constexpr int H = N / 2;
    const float4* a4 = reinterpret_cast<const float4*>(r1);
    const float4* b4 = reinterpret_cast<const float4*>(r2);
#pragma unroll
    for (int c = 0; c < H / 2; ++c) {
        const float4 a = a4[c], b = b4[c];           // entries k = 2c and 2c + 1 of both rows
        const int k = 2 * c;
        if (k == 0) {
            x[0] = make_float2(a.x, b.x);
        } else {
            x[k] = make_float2(a.x - b.y, a.y + b.x);
            x[N - k] = make_float2(a.x + b.y, b.x - a.y);
        }
        x[k + 1] = make_float2(a.z - b.w, a.w + b.z);
        x[N - k - 1] = make_float2(a.z + b.w, b.z - a.w);
    }
    x[H] = NYQ ? make_float2(r1[H].x, r2[H].x) : make_float2(0.f, 0.f);
}

template <int N, int CL, int MODE>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(ClusterGeo<N, CL>::NT, ClusterGeo<N, CL>::MINB)
    k_synth_cl(SynParams P) {
    using G = Geo<N, 3>;
    using CG = ClusterGeo<N, CL>;
    constexpr int H = CG::H, PP = CG::PP, RS = CG::RS, PS = CG::PS, RR = CG::RR, NT = CG::NT;
    extern __shared__ float2 smem[];             // [PP][PS] planes | [3][N] phase rows
    float2* phs = smem + PP * PS;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    float2* pl[CL];
    cluster_planes<CL>(cluster, smem, pl);
    const int f = blockIdx.x / CL;
    const bool active = f < P.n_fields;          // same for every CTA of the cluster
    const int lt = threadIdx.x;
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
    const float2* __restrict__ src = P.spectra + (size_t)input * G::half;
    for (int i = lt; i < 3 * N; i += NT) phs[i] = __ldg(&P.phase[(size_t)node * 3 * N + i]);
    __syncthreads();
    float2 x[N];
    // axis 0: columns (k1, k2), k1 in this CTA's range, k2 < N/2
    if (active) {
        const int k1 = rank * PP + lt / H, k2 = lt % H;
        const float2 w12 = cmul(phs[N + k1], phs[2 * N + k2]);
        const float* __restrict__ mu = (MODE == SYN_MULT) ? P.mult + (size_t)(f / P.n_c) * G::half : nullptr;
#pragma unroll
        for (int k0 = 0; k0 < N; ++k0) {
            const int idx = (k0 * N + k1) * G::NH + k2;
            float2 v;
            if constexpr (MODE == SYN_MULT) {
                v = cscale(__ldg(&src[idx]), __ldg(&mu[idx]));
            } else {
                v = cmul(__ldg(&src[idx]), cmul(w12, phs[k0]));
                if (MODE == SYN_PREP && use_gm) {
                    const int a = wrapk(k0, N), b = wrapk(k1, N);
                    v = cscale(v, P.gm_full ? __ldg(&P.gm_full[idx]) : __ldg(&P.gm[a * a + b * b + k2 * k2]));
                }
            }
            x[k0] = v;
        }
        fft_reg<N, true>(x);
#pragma unroll
        for (int i0 = 0; i0 < N; ++i0) pl[i0 / PP][(i0 % PP) * PS + k1 * RS + k2] = x[i0];
    }
    cluster.sync();
    // axis 1 on this CTA's planes
    if (active) {
        const int p0 = lt / H, k2 = lt % H;
#pragma unroll
        for (int k1 = 0; k1 < N; ++k1) x[k1] = smem[p0 * PS + k1 * RS + k2];
        fft_reg<N, true>(x);
#pragma unroll
        for (int i1 = 0; i1 < N; ++i1) smem[p0 * PS + i1 * RS + k2] = x[i1];
    }
    __syncthreads();
    // axis 2: complex-to-real of rows (p0, i1) and (p0, i1 + N/2)
    const int p0 = lt / H, i1 = lt % H;
    if (active) {
        c2r_pack_rows<N, false>(smem + p0 * PS + i1 * RS, smem + p0 * PS + (i1 + H) * RS, x);
        fft_reg<N, true>(x);
    }
    __syncthreads();                              // every row is read before staging overwrites the planes
    float* stg = reinterpret_cast<float*>(smem);
    if (active) store_two_rows<N>(stg + (p0 * N + i1) * RR, stg + (p0 * N + i1 + H) * RR, x);
    __syncthreads();
    if (active) {
        const int v0 = rank * CG::PART_N + 4 * lt;
        if (MODE != SYN_PREP)
            staged_copy<N, CL, true>(stg, shifted_field_row<N, 3>(P.out, f / P.n_c, f % P.n_c, P.n_c, v0),
                                     (size_t)(4 * NT / G::VCH) * P.n_c * G::VCH, lt);
        else
            staged_copy<N, CL, true>(stg, P.out + (size_t)f * G::n + v0, 4 * NT, lt);
    }
}

template <int N, int CL, int MODE>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(ClusterGeo<N, CL>::NT, (ClusterGeo<N, CL>::MINB > 1 ? 2 : 1))
    k_analysis_cl(AnaParams P) {
    using G = Geo<N, 3>;
    using CG = ClusterGeo<N, CL>;
    constexpr int H = CG::H, PP = CG::PP, RS = CG::RS, PS = CG::PS, RR = CG::RR, NT = CG::NT, NH = G::NH;
    constexpr int COLS = CG::COLS;
    extern __shared__ float2 smem[];              // [PP][PS] planes (or the staged real rows)
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    float2* pl[CL];
    cluster_planes<CL>(cluster, smem, pl);
    const int f = blockIdx.x / CL;
    const bool active = f < P.n_fields;
    const int lt = threadIdx.x;
    float2* __restrict__ dst = P.out + (size_t)f * G::half;
    float* stg = reinterpret_cast<float*>(smem);
    float2 x[N];
    const int n_iter = (MODE == ANA_ACCUM) ? P.nq : 1;
    for (int qq = 0; qq < n_iter; ++qq) {
        const float* src =
            ((MODE == ANA_ACCUM) ? P.in + ((size_t)qq * P.U + f) * G::n : P.in + (size_t)f * G::n) +
            (size_t)rank * CG::PART_N;
        const float* __restrict__ ct = P.ctab + (size_t)(P.q0 + qq) * (G::SMAX + 1);
        // stage this CTA's part of the real field (coalesced), then R2C along the last axis
        if (active) staged_copy<N, CL, false>(stg, const_cast<float*>(src) + 4 * lt, 4 * NT, lt);
        __syncthreads();
        const int p0 = lt / H, i1 = lt % H;
        if (active) load_two_rows_smem<N>(stg + (p0 * N + i1) * RR, stg + (p0 * N + i1 + H) * RR, x);
        __syncthreads();                          // staged rows consumed before the planes are written
        if (active) {
            fft_reg<N, false>(x);
            // half spectra of the two rows: R1[k] = (X[k] + conj X[N-k]) / 2,
            // R2[k] = (X[k] - conj X[N-k]) / 2i, entries k and k + 1 stored together
            float4* r1 = reinterpret_cast<float4*>(smem + p0 * PS + i1 * RS);
            float4* r2 = reinterpret_cast<float4*>(smem + p0 * PS + (i1 + H) * RS);
#pragma unroll
            for (int c = 0; c < H / 2; ++c) {
                const int k = 2 * c;
                const float2 z = x[k], zc = x[(N - k) % N], w = x[k + 1], wc = x[N - k - 1];
                r1[c] = make_float4(0.5f * (z.x + zc.x), 0.5f * (z.y - zc.y), 0.5f * (w.x + wc.x), 0.5f * (w.y - wc.y));
                r2[c] = make_float4(0.5f * (z.y + zc.y), -0.5f * (z.x - zc.x), 0.5f * (w.y + wc.y), -0.5f * (w.x - wc.x));
            }
            const float2 z = x[H];
            reinterpret_cast<float2*>(r1)[H] = make_float2(z.x, 0.f);
            reinterpret_cast<float2*>(r2)[H] = make_float2(z.y, 0.f);
        }
        __syncthreads();
        // axis 1 on this CTA's planes
        if (active) {
            for (int c = lt; c < COLS; c += NT) {
                const int q0 = c / NH, k2 = c % NH;
#pragma unroll
                for (int k1 = 0; k1 < N; ++k1) x[k1] = smem[q0 * PS + k1 * RS + k2];
                fft_reg<N, false>(x);
#pragma unroll
                for (int k1 = 0; k1 < N; ++k1) smem[q0 * PS + k1 * RS + k2] = x[k1];
            }
        }
        cluster.sync();
        // axis 0: columns (k1, k2), k1 in this CTA's range; planes from every CTA
        if (active) {
            for (int c = lt; c < COLS; c += NT) {
                const int k1 = rank * PP + c / NH, k2 = c % NH;
#pragma unroll
                for (int i0 = 0; i0 < N; ++i0) x[i0] = pl[i0 / PP][(i0 % PP) * PS + k1 * RS + k2];
                fft_reg<N, false>(x);
#pragma unroll
                for (int k0 = 0; k0 < N; ++k0) {
                    const int idx = (k0 * N + k1) * NH + k2;
                    const int par = (k0 + k1 + k2) & 1;
                    if (MODE == ANA_SPECTRUM) {
                        const bool nyq = (k0 == H) || (k1 == H) || (k2 == H);
                        const float sc = nyq ? 0.f : (par ? -P.inv_n : P.inv_n);
                        dst[idx] = cscale(x[k0], sc);
                    } else {
                        const int a = wrapk(k0, N), b = wrapk(k1, N);
                        const float c0 = __ldg(&ct[a * a + b * b + k2 * k2]);
                        const float sc = par ? -c0 : c0;
                        const float2 old = dst[idx];
                        dst[idx] = make_float2(fmaf(x[k0].x, sc, old.x), fmaf(x[k0].y, sc, old.y));
                    }
                }
            }
        }
        cluster.sync();      // the other CTAs have finished reading these planes
    }
}

template <int N, int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(ClusterGeo<N, CL>::NT, 1) k_output_cl(OutParams P) {
    using G = Geo<N, 3>;
    using CG = ClusterGeo<N, CL>;
    constexpr int H = CG::H, PP = CG::PP, RS = CG::RS, PS = CG::PS, RR = CG::RR, NT = CG::NT, NH = G::NH;
    constexpr int COLS = CG::COLS;
    extern __shared__ float2 smem[];
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    float2* pl[CL];
    cluster_planes<CL>(cluster, smem, pl);
    const int u = blockIdx.x / CL;
    const bool active = u < P.U;
    const int lt = threadIdx.x;
    const float2* __restrict__ src = P.qhat + (size_t)u * G::half;
    float2 x[N];
    // axis 0 over every column (k1 in this CTA's range, k2 = 0..N/2), sign (-1)^k from the index parity
    if (active) {
        for (int c = lt; c < COLS; c += NT) {
            const int k1 = rank * PP + c / NH, k2 = c % NH;
#pragma unroll
            for (int k0 = 0; k0 < N; ++k0) {
                const float2 v = src[(k0 * N + k1) * NH + k2];
                x[k0] = ((k0 + k1 + k2) & 1) ? make_float2(-v.x, -v.y) : v;
            }
            fft_reg<N, true>(x);
#pragma unroll
            for (int i0 = 0; i0 < N; ++i0) pl[i0 / PP][(i0 % PP) * PS + k1 * RS + k2] = x[i0];
        }
    }
    cluster.sync();
    // axis 1 on this CTA's planes
    if (active) {
        for (int c = lt; c < COLS; c += NT) {
            const int q0 = c / NH, k2 = c % NH;
#pragma unroll
            for (int k1 = 0; k1 < N; ++k1) x[k1] = smem[q0 * PS + k1 * RS + k2];
            fft_reg<N, true>(x);
#pragma unroll
            for (int i1 = 0; i1 < N; ++i1) smem[q0 * PS + i1 * RS + k2] = x[i1];
        }
    }
    __syncthreads();
    const int p0 = lt / H, i1 = lt % H;
    if (active) {
        c2r_pack_rows<N, true>(smem + p0 * PS + i1 * RS, smem + p0 * PS + (i1 + H) * RS, x);
        fft_reg<N, true>(x);
    }
    __syncthreads();
    float* stg = reinterpret_cast<float*>(smem);  // gain rows of this CTA's part
    if (active) store_two_rows<N>(stg + (p0 * N + i1) * RR, stg + (p0 * N + i1 + H) * RR, x);
    __syncthreads();
    if (!active) return;
    constexpr int ITER = CG::PART_N / (4 * NT);
    constexpr int S_STEP = (4 * NT / N) * RR;
    const int L0 = 4 * lt;
    const float* sp = stg + (L0 / N) * RR + (L0 % N);
    const size_t v0 = (size_t)rank * CG::PART_N + L0;
    bool bad = false;
    for (int o = P.out_start[u]; o < P.out_start[u + 1]; ++o) {
        const int4 e = P.outs[o];
        const float* fl = P.fN + (size_t)e.z * G::n + v0;
        const float* lj = P.lam + (size_t)e.y * G::n + v0;
        float* q = P.Q + (size_t)e.x * G::n + v0;
#pragma unroll 4
        for (int it = 0; it < ITER; ++it) {
            const float4 g4 = *reinterpret_cast<const float4*>(sp + it * S_STEP);
            const float4 a = __ldg(reinterpret_cast<const float4*>(fl + (size_t)it * 4 * NT));
            const float4 b = __ldg(reinterpret_cast<const float4*>(lj + (size_t)it * 4 * NT));
            const float4 v =
                make_float4(fmaf(-a.x, b.x, g4.x), fmaf(-a.y, b.y, g4.y), fmaf(-a.z, b.z, g4.z), fmaf(-a.w, b.w, g4.w));
            bad |= nonfinite4(v);
            *reinterpret_cast<float4*>(q + (size_t)it * 4 * NT) = v;
        }
    }
    if (bad) atomicOr(P.err, kErrNonFinite);
}

// ------------------------------------------------------------------ output (single-CTA fields)


// Gain minus loss for two rows: q = x.(x|y) - f * lam, 16-byte accesses.
template <int N>
__device__ __forceinline__ void gain_minus_loss_rows(const float* f1, const float* f2, const float* l1,
                                                     const float* l2, float* q1, float* q2, const float2 (&x)[N],
                                                     bool& bad) {
    const float4* F1 = reinterpret_cast<const float4*>(f1);
    const float4* F2 = reinterpret_cast<const float4*>(f2);
    const float4* L1 = reinterpret_cast<const float4*>(l1);
    const float4* L2 = reinterpret_cast<const float4*>(l2);
    float4* Q1 = reinterpret_cast<float4*>(q1);
    float4* Q2 = reinterpret_cast<float4*>(q2);
#pragma unroll
    for (int c = 0; c < N / 4; ++c) {
        const float4 a = __ldg(&F1[c]), b = __ldg(&L1[c]), a2 = __ldg(&F2[c]), b2 = __ldg(&L2[c]);
        const float4 v1 = make_float4(fmaf(-a.x, b.x, x[4 * c].x), fmaf(-a.y, b.y, x[4 * c + 1].x),
                                      fmaf(-a.z, b.z, x[4 * c + 2].x), fmaf(-a.w, b.w, x[4 * c + 3].x));
        const float4 v2 = make_float4(fmaf(-a2.x, b2.x, x[4 * c].y), fmaf(-a2.y, b2.y, x[4 * c + 1].y),
                                      fmaf(-a2.z, b2.z, x[4 * c + 2].y), fmaf(-a2.w, b2.w, x[4 * c + 3].y));
        bad |= nonfinite4(v1) || nonfinite4(v2);
        Q1[c] = v1;
        Q2[c] = v2;
    }
}
template <int N>
__device__ __forceinline__ void gain_minus_loss_rows(const double* f1, const double* f2, const double* l1,
                                                     const double* l2, double* q1, double* q2,
                                                     const double2 (&x)[N], bool& bad) {
    const double2* F1 = reinterpret_cast<const double2*>(f1);
    const double2* F2 = reinterpret_cast<const double2*>(f2);
    const double2* L1 = reinterpret_cast<const double2*>(l1);
    const double2* L2 = reinterpret_cast<const double2*>(l2);
    double2* Q1 = reinterpret_cast<double2*>(q1);
    double2* Q2 = reinterpret_cast<double2*>(q2);
#pragma unroll
    for (int c = 0; c < N / 2; ++c) {
        const double2 a = __ldg(&F1[c]), b = __ldg(&L1[c]), a2 = __ldg(&F2[c]), b2 = __ldg(&L2[c]);
        const double2 v1 = make_double2(fma(-a.x, b.x, x[2 * c].x), fma(-a.y, b.y, x[2 * c + 1].x));
        const double2 v2 = make_double2(fma(-a2.x, b2.x, x[2 * c].y), fma(-a2.y, b2.y, x[2 * c + 1].y));
        bad |= nonfinite2(v1) || nonfinite2(v2);
        Q1[c] = v1;
        Q2[c] = v2;
    }
}

template <int N, int D, int FPC, typename R = float>
__global__ void __launch_bounds__(Geo<N, D>::TPF * FPC) k_output(OutParamsT<R> P) {
    using G = Geo<N, D>;
    using PR = Prec<R>;
    using C = typename PR::C;
    constexpr int H = G::H, RS = G::RS, NH = G::NH;
    extern __shared__ __align__(16) unsigned char fsm_raw[];
    const int grp = threadIdx.x / G::TPF, lt = threadIdx.x % G::TPF;
    const int u = blockIdx.x * FPC + grp;
    const bool active = u < P.U;
    C* s = reinterpret_cast<C*>(fsm_raw) + grp * G::SMEM_F;
    const C* __restrict__ src = P.qhat + (size_t)u * G::half;
    C x[N];
    // axis 0 (all columns, Nyquist included), sign (-1)^k from the index parity
    if (active) {
        for (int c = lt; c < G::COLS; c += G::TPF) {
            const int k1 = (D == 3) ? c / NH : 0, k2 = (D == 3) ? c % NH : c;
#pragma unroll
            for (int k0 = 0; k0 < N; ++k0) {
                const int idx = (D == 3) ? (k0 * N + k1) * NH + k2 : k0 * NH + k2;
                const C v = src[idx];
                x[k0] = ((k0 + k1 + k2) & 1) ? PR::mk(-v.x, -v.y) : v;
            }
            fft_reg<N, true>(x);
#pragma unroll
            for (int i0 = 0; i0 < N; ++i0) s[(D == 3 ? (i0 * N + k1) * RS : i0 * RS) + k2] = x[i0];
        }
    }
    __syncthreads();
    if (D == 3) {
        if (active) {
            for (int c = lt; c < G::COLS; c += G::TPF) {
                const int i0 = c / NH, k2 = c % NH;
#pragma unroll
                for (int k1 = 0; k1 < N; ++k1) x[k1] = s[(i0 * N + k1) * RS + k2];
                fft_reg<N, true>(x);
#pragma unroll
                for (int i1 = 0; i1 < N; ++i1) s[(i0 * N + i1) * RS + k2] = x[i1];
            }
        }
        __syncthreads();
    }
    if (!active) return;
    const int row = (D == 3) ? (lt / H) * N + (lt % H) : lt;
    {
        const C* r1 = s + row * RS;
        const C* r2 = s + (row + H) * RS;
        x[0] = PR::mk(r1[0].x, r2[0].x);
        x[H] = PR::mk(r1[H].x, r2[H].x);
#pragma unroll
        for (int k = 1; k < H; ++k) {
            const C a = r1[k], b = r2[k];
            x[k] = PR::mk(a.x - b.y, a.y + b.x);
            x[N - k] = PR::mk(a.x + b.y, b.x - a.y);
        }
        fft_reg<N, true>(x);
    }
    bool bad = false;
    for (int o = P.out_start[u]; o < P.out_start[u + 1]; ++o) {
        const int4 e = P.outs[o];
        const R* fl = P.fN + (size_t)e.z * G::n;
        const R* lj = P.lam + (size_t)e.y * G::n;
        R* q = P.Q + (size_t)e.x * G::n;
        gain_minus_loss_rows<N>(fl + row * N, fl + (row + H) * N, lj + row * N, lj + (row + H) * N, q + row * N,
                                q + (row + H) * N, x, bad);
    }
    if (bad) atomicOr(P.err, kErrNonFinite);
}

// ------------------------------------------------------------------ sigma-contraction
// P_{q,u}(v) = sum_p w_p A_{q,p,j_u}(v) A_{q,antipode(p),l_u}(v) for the slots of a tile:
//   TRI  (TJ = TL = T): all (j0+a, j0+b), a <= b   -> slot0 + a*T - a(a-1)/2 + (b-a)
//   FULL (TJ x TL)    : all (j0+a, l0+b)           -> slot0 + a*TL + b
//   LIST (T = 16)     : (ja[t], lb[t]) for t < count -> slot0 + t
// The direction sum runs over antipodal pairs (p, p'): with c = A_p', a = w A_p
// (w_p = w_p'), the two terms of a pair are a_j c_l + c_j a_l, so every field
// value loaded serves both directions of the pair.
enum { TILE_TRI = 0, TILE_FULL = 1, TILE_LIST = 2 };

struct Tile {
    int ja[16];
    int lb[16];
    int slot0;
    int count;
    int j0, l0;
};

template <typename R>
struct ConParamsT {
    const R* A;            // [nq][M][n_c][n]
    R* P;                  // [nq][U][n]; the asymmetric sum: [n_split][U][n] partial sums
    const Tile* tiles;
    const R* w;            // [M/2] weight of each antipodal direction pair
    const int2* dpair;     // [M/2] (p, antipode(p)) with p < antipode(p)
    int* err;              // device error word
    int n_dpair, M, n_c, U, n;
    int n_split;           // asymmetric sum: direction pairs split over gridDim.z = n_split blocks (>= 1)
};
using ConParams = ConParamsT<float>;

// A CTA owns VC consecutive voxels (one per thread); for
// every antipodal pair one warp issues 1-D bulk copies of the 2 x NR field
// rows (VC floats each) into a ring of shared-memory stages, and all threads
// read their voxel's column from shared memory.  The copies of STAGES pairs
// are in flight while the FMAs of the current pair run.
template <int KIND, int TJ, int TL>
struct ContractShape {
    static constexpr int NR = (KIND == TILE_TRI) ? TJ : (KIND == TILE_FULL ? TJ + TL : 2 * TJ);
    static constexpr int ROWS = 2 * NR;                           // A_p rows then A_p' rows
    static constexpr int NACC = (KIND == TILE_TRI) ? TJ * (TJ + 1) / 2 : (KIND == TILE_FULL ? TJ * TL : TJ);
};

// The asymmetric sum reads only the g-side j rows of slot x and the f-side l
// rows of slot y: TJ + TL rows per stage (FULL) or 2 TJ (LIST).
template <int KIND, int TJ, int TL>
struct ContractShapeA {
    static constexpr int ROWS = (KIND == TILE_FULL) ? TJ + TL : 2 * TJ;
    static constexpr int NACC = (KIND == TILE_FULL) ? TJ * TL : TJ;
};

// ASYM (the Carleman form): slot x of a direction pair holds the g-side fields
// and slot y the f-side fields, and only P[j,l] += w A_x[j] A_y[l] is summed
// (FULL and LIST tiles; every ordered pair has its own gain slot).
template <int KIND, int TJ, int TL, int VC, int STAGES, typename R = float, bool ASYM = false>
__global__ void __launch_bounds__(VC, 1) k_contract_pipe(ConParamsT<R> C) {
    using CS = ContractShape<KIND, TJ, TL>;
    using CA = ContractShapeA<KIND, TJ, TL>;
    using PR = Prec<R>;
    static_assert(!ASYM || KIND != TILE_TRI, "the asymmetric sum has no triangular tiles");
    constexpr int NR = CS::NR, ROWS = ASYM ? CA::ROWS : CS::ROWS, NACC = ASYM ? CA::NACC : CS::NACC;
    constexpr uint32_t STAGE_BYTES = ROWS * VC * sizeof(R);
    extern __shared__ __align__(128) unsigned char csm_raw[];
    R* sbuf = reinterpret_cast<R*>(csm_raw);                      // [STAGES][ROWS][VC]
    __shared__ uint64_t bars[STAGES];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const Tile& tl = C.tiles[blockIdx.y];
    const int nch = C.n / VC;                                     // VC is the layout's voxel chunk
    const size_t blk = (size_t)C.n_c * VC;                        // one (slot, chunk) block
    // radial node of the block: the last node first, since its fields were the
    // last ones written and are the likeliest to still be in L2.  The
    // asymmetric sum has no radial nodes: blockIdx.z selects its share
    // [k0, k1) of the direction pairs instead, summed into partial P block z.
    const int qz = ASYM ? 0 : (int)(gridDim.z - 1 - blockIdx.z);
    // block of (slot = qz*M + p, chunk = blockIdx.x)
    auto block_of = [&](int p) -> const R* {
        return C.A + (((size_t)qz * C.M + p) * nch + blockIdx.x) * blk;
    };
    const int k0 = ASYM ? (int)(((long long)C.n_dpair * blockIdx.z) / gridDim.z) : 0;
    const int npairs = ASYM ? (int)(((long long)C.n_dpair * (blockIdx.z + 1)) / gridDim.z) : C.n_dpair;
    if (t == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
        mbar_init_fence();
    }
    __syncthreads();
    // rows of one direction: TRI j0..j0+TJ; FULL j0..j0+TJ then l0..l0+TL; LIST ja[], lb[]
    auto issue = [&](int k) {                                     // warp 0 only
        const int s = (k - k0) % STAGES;
        const int2 d = C.dpair[k];
        R* dstp = sbuf + (size_t)s * ROWS * VC;
        if (lane == 0) mbar_arrive_expect_tx(&bars[s], STAGE_BYTES);
        __syncwarp();
        if constexpr (ASYM) {
            // rows [0, TJ): slot x (g side) rows j; then slot y (f side) rows l
            if (KIND == TILE_LIST) {
                for (int r = lane; r < ROWS; r += 32) {
                    const int row = r < TJ ? tl.ja[r] : tl.lb[r - TJ];
                    bulk_g2s(dstp + (size_t)r * VC, block_of(r < TJ ? d.x : d.y) + (size_t)row * VC,
                             VC * sizeof(R), &bars[s]);
                }
            } else if (lane == 0) {
                bulk_g2s(dstp, block_of(d.x) + (size_t)tl.j0 * VC, TJ * VC * sizeof(R), &bars[s]);
                bulk_g2s(dstp + TJ * VC, block_of(d.y) + (size_t)tl.l0 * VC, TL * VC * sizeof(R), &bars[s]);
            }
        } else if (KIND == TILE_LIST) {
            for (int r = lane; r < ROWS; r += 32) {
                const int i = r < NR ? r : r - NR;
                const int row = i < TJ ? tl.ja[i] : tl.lb[i - TJ];
                bulk_g2s(dstp + (size_t)r * VC, block_of(r < NR ? d.x : d.y) + (size_t)row * VC,
                         VC * sizeof(R), &bars[s]);
            }
        } else if (lane < 2) {
            const R* b = block_of(lane == 0 ? d.x : d.y);
            R* o = dstp + (size_t)lane * NR * VC;
            bulk_g2s(o, b + (size_t)tl.j0 * VC, TJ * VC * sizeof(R), &bars[s]);
            if (KIND == TILE_FULL) bulk_g2s(o + TJ * VC, b + (size_t)tl.l0 * VC, TL * VC * sizeof(R), &bars[s]);
        }
    };
    if (warp == 0)
        for (int k = k0; k < k0 + STAGES && k < npairs; ++k) issue(k);
    R acc[NACC];
#pragma unroll
    for (int i = 0; i < NACC; ++i) acc[i] = R(0);
    for (int k = k0; k < npairs; ++k) {
        const int s = (k - k0) % STAGES;
        const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((k - k0) / STAGES) & 1u);
        if (__syncthreads_or(!ok)) {
            // a copy did not land: record it, wait (bounded) for the copies still in flight, leave
            if (t == 0) {
                atomicOr(C.err, kErrTimeout);
                for (int k2 = k; k2 < npairs && k2 < k + STAGES; ++k2)
                    (void)mbar_wait_bounded(&bars[(k2 - k0) % STAGES], (uint32_t)((k2 - k0) / STAGES) & 1u);
            }
            __syncthreads();
            return;
        }
        const R* __restrict__ xs = sbuf + (size_t)s * ROWS * VC + t;
        const R wk = __ldg(&C.w[k]);
        if constexpr (ASYM) {
            constexpr int NL = (KIND == TILE_FULL) ? TL : TJ;
            R xj[TJ], xl[NL];
#pragma unroll
            for (int i = 0; i < TJ; ++i) xj[i] = wk * xs[i * VC];
#pragma unroll
            for (int i = 0; i < NL; ++i) xl[i] = xs[(TJ + i) * VC];
            if (KIND == TILE_FULL) {
#pragma unroll
                for (int x = 0; x < TJ; ++x)
#pragma unroll
                    for (int y = 0; y < NL; ++y) acc[x * NL + y] = PR::fma_(xj[x], xl[y], acc[x * NL + y]);
            } else {
#pragma unroll
                for (int i = 0; i < TJ; ++i) acc[i] = PR::fma_(xj[i], xl[i], acc[i]);
            }
        } else {
        R xp[NR], xq[NR];
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            xp[i] = wk * xs[i * VC];
            xq[i] = xs[(NR + i) * VC];
        }
        if (KIND == TILE_TRI) {
            int i = 0;
#pragma unroll
            for (int x = 0; x < TJ; ++x)
#pragma unroll
                for (int y = x; y < TJ; ++y) {
                    acc[i] = PR::fma_(xp[x], xq[y], PR::fma_(xq[x], xp[y], acc[i]));
                    ++i;
                }
        } else if (KIND == TILE_FULL) {
#pragma unroll
            for (int x = 0; x < TJ; ++x)
#pragma unroll
                for (int y = 0; y < TL; ++y)
                    acc[x * TL + y] = PR::fma_(xp[x], xq[TJ + y], PR::fma_(xq[x], xp[TJ + y], acc[x * TL + y]));
        } else {
#pragma unroll
            for (int i = 0; i < TJ; ++i) acc[i] = PR::fma_(xp[i], xq[TJ + i], PR::fma_(xq[i], xp[TJ + i], acc[i]));
        }
        }
        __syncthreads();                                          // stage s fully read
        if (warp == 0 && k + STAGES < npairs) {
            fence_proxy_async_smem();
            issue(k + STAGES);
        }
    }
    const size_t n = (size_t)C.n;
    R* __restrict__ Pq = C.P + (size_t)(ASYM ? blockIdx.z : qz) * C.U * n + (size_t)blockIdx.x * VC + t;
    const int cnt = (KIND == TILE_LIST) ? tl.count : NACC;
#pragma unroll
    for (int i = 0; i < NACC; ++i)
        if (i < cnt) Pq[(size_t)(tl.slot0 + i) * n] = acc[i];
}

// ------------------------------------------------------------------ Carleman-form output
// Q[e](v) = P[u](v) - f_N[l](v) Lambda[j](v) for every ordered pair e = (j, l)
// of slot u (no forward transform: the gain's grid values are the weighted sum
// of products itself), P the sum of the n_split partial blocks [z][U][n] of
// the contraction.  Blocks (voxel quarter-chunk, slot).
__global__ void __launch_bounds__(256) k_carleman_output(const float* __restrict__ Pg, const float* __restrict__ fN,
                                                          const float* __restrict__ lam,
                                                          const int* __restrict__ out_start,
                                                          const int4* __restrict__ outs, float* __restrict__ Q, int n,
                                                          int* __restrict__ err, int n_split = 1, int U = 0) {
    const int u = blockIdx.y;
    const int v4 = blockIdx.x * 256 + threadIdx.x;           // float4 index
    if (v4 * 4 >= n) return;
    float4 p = __ldg(reinterpret_cast<const float4*>(Pg + (size_t)u * n) + v4);
    for (int z = 1; z < n_split; ++z) {                      // partial sums of the direction splits, in order
        const float4 q = __ldg(reinterpret_cast<const float4*>(Pg + ((size_t)z * U + u) * n) + v4);
        p = make_float4(p.x + q.x, p.y + q.y, p.z + q.z, p.w + q.w);
    }
    for (int o = out_start[u]; o < out_start[u + 1]; ++o) {
        const int4 e = outs[o];
        const float4 a = __ldg(reinterpret_cast<const float4*>(fN + (size_t)e.z * n) + v4);
        const float4 b = __ldg(reinterpret_cast<const float4*>(lam + (size_t)e.y * n) + v4);
        const float4 v = make_float4(fmaf(-a.x, b.x, p.x), fmaf(-a.y, b.y, p.y), fmaf(-a.z, b.z, p.z),
                                     fmaf(-a.w, b.w, p.w));
        if (nonfinite4(v)) atomicOr(err, kErrNonFinite);
        reinterpret_cast<float4*>(Q + (size_t)e.x * n)[v4] = v;
    }
}

// ------------------------------------------------------------------ FP64 moment sums
// out[f][0] = dv^D sum_v Q_f(v), out[f][1+a] = dv^D sum_v v_a Q_f(v),
// out[f][D+1] = dv^D sum_v |v|^2 Q_f(v)  (paper Sec. 1: mass, momentum,
// energy), accumulated in FP64 with a fixed-order block reduction.
template <int D>
__global__ void __launch_bounds__(256) k_moments(const float* __restrict__ Q, double* __restrict__ out, int N,
                                                 double L, double dv) {
    const int f = blockIdx.x;
    const int n = (D == 3) ? N * N * N : N * N;
    const float* q = Q + (size_t)f * n;
    double acc[D + 2];
#pragma unroll
    for (int i = 0; i < D + 2; ++i) acc[i] = 0.0;
    for (int v = threadIdx.x; v < n; v += 256) {
        const double x = (double)q[v];
        int rem = v;
        double r2 = 0.0;
        double c[D];
#pragma unroll
        for (int a = D - 1; a >= 0; --a) {
            c[a] = -L + (rem % N) * dv;
            rem /= N;
            r2 += c[a] * c[a];
        }
        acc[0] += x;
#pragma unroll
        for (int a = 0; a < D; ++a) acc[1 + a] += c[a] * x;
        acc[D + 1] += r2 * x;
    }
    __shared__ double red[256];
    const double vol = pow(dv, (double)D);
    for (int i = 0; i < D + 2; ++i) {
        red[threadIdx.x] = acc[i];
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[(size_t)f * (D + 2) + i] = vol * red[0];
        __syncthreads();
    }
}

// out[0] = dv^D sum_f sum_v v_1^2 Q_f(v): the v_1^2 moment (v_1 = velocity axis 0)
// summed over n_fields fields, FP64, one CTA, fixed order (paper Sec. 4.2).
template <int D>
__global__ void __launch_bounds__(256) k_axis0_second_moment(const float* __restrict__ Q, int n_fields, int N,
                                                             double L, double dv, double* __restrict__ out) {
    const int n = (D == 3) ? N * N * N : N * N;
    const int plane = n / N;
    double acc = 0.0;
    for (int f = 0; f < n_fields; ++f) {
        const float* q = Q + (size_t)f * n;
        for (int v = threadIdx.x; v < n; v += 256) {
            const double v0 = -L + (v / plane) * dv;
            acc = fma(v0 * v0, (double)q[v], acc);
        }
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = pow(dv, (double)D) * red[0];
}

// ------------------------------------------------------------------ failure-path self-test
// One CTA announces an incoming transfer on an mbarrier and never issues it:
// the bounded wait runs out, the kernel records a timeout in the error word
// and returns normally, leaving the context usable.
__global__ void k_selftest_wait_timeout(int* err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 16);    // 16 bytes that never arrive
    const bool ok = mbar_wait_bounded(&bar, 0);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(err, kErrTimeout);
}

// ------------------------------------------------------------------ projection
// partial[vs][k][pr] = sum_{v in slice vs} V_k(v) Q_pr(v); the reduce kernel sums
// the slices in a fixed order and applies dv^D (midpoint rule).
template <int PB, int RT, typename R = float>
__global__ void __launch_bounds__(256) k_project(const R* __restrict__ V, const R* __restrict__ Q,
                                                 R* __restrict__ partial, int r, int n, int n_slices) {
    using PR = Prec<R>;
    const int pr0 = blockIdx.x * PB, vs = blockIdx.y, k0 = blockIdx.z * RT;
    const int r2 = r * r;
    const int v0 = (int)((long long)n * vs / n_slices), v1 = (int)((long long)n * (vs + 1) / n_slices);
    R acc[PB][RT];
#pragma unroll
    for (int i = 0; i < PB; ++i)
#pragma unroll
        for (int j = 0; j < RT; ++j) acc[i][j] = R(0);
    for (int v = v0 + threadIdx.x; v < v1; v += 256) {
        R q[PB], w[RT];
#pragma unroll
        for (int i = 0; i < PB; ++i) q[i] = (pr0 + i < r2) ? __ldg(&Q[(size_t)(pr0 + i) * n + v]) : R(0);
#pragma unroll
        for (int j = 0; j < RT; ++j) w[j] = (k0 + j < r) ? __ldg(&V[(size_t)(k0 + j) * n + v]) : R(0);
#pragma unroll
        for (int i = 0; i < PB; ++i)
#pragma unroll
            for (int j = 0; j < RT; ++j) acc[i][j] = PR::fma_(q[i], w[j], acc[i][j]);
    }
    __shared__ R red[8][PB * RT];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < PB; ++i)
#pragma unroll
        for (int j = 0; j < RT; ++j) {
            R t = acc[i][j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) red[warp][i * RT + j] = t;
        }
    __syncthreads();
    for (int e = threadIdx.x; e < PB * RT; e += 256) {
        R t = R(0);
#pragma unroll
        for (int w = 0; w < 8; ++w) t += red[w][e];
        const int i = e / RT, j = e % RT;
        if (pr0 + i < r2 && k0 + j < r) partial[((size_t)vs * r + k0 + j) * r2 + pr0 + i] = t;
    }
}

template <typename R = float>
__global__ void k_project_reduce(const R* __restrict__ partial, R* __restrict__ T, int count, int n_slices,
                                 R scale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    R t = R(0);
    for (int s = 0; s < n_slices; ++s) t += partial[(size_t)s * count + i];
    T[i] = t * scale;
}

}  // namespace boltz_dev
