// Split-precision shifted fields: the DFT-as-GEMM variant of the synthesis
// step on the fifth-generation tensor cores (sm_103a).
//
// A shifted field is a separable product of per-axis shifts of the input's
// band-limited interpolant (Sec. 2.1, the values of g_N on the grid):
//   A_{q,p}(v) = g_N(v - s),  s = rho_q sigma_p / 2,
//   A = (S(s_0) x S(s_1) x S(s_2)) g,
//   S(s)[i][m] = (1/N) sum_{|k| < N/2} exp(i pi k ((i - m) dv - s) / L)   (real),
// so the three inverse transforms of the FFT path become three GEMM passes of
// N x N matrices over the field's N^2 lines.  Operands are split into BF16
// pairs x = hi + lo and each product is hi*hi + lo*hi + hi*lo (lo*lo, ~2^-17
// relative, is dropped), accumulated in FP32 in tensor memory.  The pair of
// an element is stored as one 32-bit word (hi in the low half), so the K
// dimension of every GEMM is 2N interleaved values, and the B operand is
//   B'[n][2m] = S_hi[n][m], B'[n][2m+1] = S_hi[n][m]   (n < N)
//   B'[n][2m] = S_lo[n-N][m], B'[n][2m+1] = 0           (n >= N)
// whose two column blocks of D sum to the three-term product.
//
// A cluster of CL CTAs owns one field at a time; CTA r holds 1/CL of the
// field's lines in every pass (N = 32: CL = 1, the whole field one 128 KB
// operand -- two CTAs per field also work but ran slower; N = 64: CL = 8,
// 128 KB per CTA).  With PP = N / CL:
//   pass 1: lines (i0, i1) along i2, CTA r owns i0 in [r PP, r PP + PP),
//           local line i0l N + i1;
//   pass 2: lines (i2, i0) along i1, same i0 slab, local line i2 PP + i0l;
//   pass 3: lines (i1, i2) along i0, CTA r owns i1 in [r PP, r PP + PP),
//           local line i1l N + i2.
// Between passes every thread reads its TMEM lane (one line) and writes the
// line's N results, split and packed, into the next pass's A operand; from
// pass 1 to 2 that stays in the CTA, from pass 2 to 3 result c goes to the
// CTA owning i1 = c (distributed shared memory, between cluster barriers).
// From pass 1 to 2 the lanes of a warp write 32 consecutive k of one line;
// the A layout puts the 16-byte core columns 16 bytes out of step (K-core
// stride = lines/8 * 128 + 16), so those stores hit 32 different banks.
#pragma once

#include <cuda_bf16.h>

#include "async.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace boltz_dev {

template <int N, int CL>
struct SplitGeo {
    static constexpr int PP = N / CL;                   // planes (slab width) per CTA
    static constexpr int LINES = N * N / CL;            // local lines of one pass
    static constexpr int TILES = LINES / 128;           // 128-line M tiles
    static constexpr int KP = 2 * N;                    // interleaved hi/lo K
    static constexpr int KCORES = KP / 8;               // 16-byte core columns along K
    static constexpr int RG = LINES / 8;                // 8-line row groups
    static constexpr uint32_t LBO = RG * 128 + 16;      // K-core stride of A (skewed)
    static constexpr uint32_t A_BYTES = KCORES * LBO;   // the CTA's part of a field
    static constexpr int NB = 2 * N;                    // rows of B'
    static constexpr uint32_t B_AXIS_BYTES = NB * KP * 2;
    static constexpr uint32_t B_BYTES = 3 * B_AXIS_BYTES;    // axes 0, 1, 2
    static constexpr int TMEM_COLS = TILES * NB;
    static constexpr int KSTEPS = KP / 16;              // BF16 MMAs take K = 16
    static constexpr size_t SMEM = size_t(A_BYTES) + B_BYTES;
    static_assert(TMEM_COLS == 256 || TMEM_COLS == 512, "tensor memory allocation");
    static_assert(PP % 8 == 0 && LINES % 128 == 0, "slabs of whole row groups and tiles");
    static_assert(SMEM + 1024 <= (227u << 10), "operands fit in shared memory");
};

// Byte offset of the packed pair of element k of local line R in the A operand.
template <int N, int CL>
__device__ __forceinline__ uint32_t split_a_offset(int R, int k) {
    using S = SplitGeo<N, CL>;
    return (uint32_t)(k >> 2) * S::LBO + (uint32_t)(R >> 3) * 128u + (uint32_t)(R & 7) * 16u + (uint32_t)(k & 3) * 4u;
}

// x -> (bf16(x), bf16(x - bf16(x))) packed hi | lo << 16 (one paired
// conversion re-rounds x to the same hi).
__device__ __forceinline__ uint32_t split_pack(float x) {
    const float r = x - __bfloat162float(__float2bfloat16_rn(x));
    const __nv_bfloat162 p = __floats2bfloat162_rn(x, r);
    return *reinterpret_cast<const uint32_t*>(&p);
}

// Orders this thread's generic-proxy shared-memory writes (local or to other
// CTAs of the cluster) before later async-proxy (tensor core) reads.
__device__ __forceinline__ void fence_proxy_async_all() { asm volatile("fence.proxy.async;" ::: "memory"); }

// Pre-split inputs: img[jj][r] = CTA r's pass-1 A operand of f_N of chunk
// input jj (element k = i2 of local line (i0 - r PP) N + i1), written once per
// chunk and copied into shared memory for every node.
template <int N, int CL>
__global__ void __launch_bounds__(256) k_split_input(const float* __restrict__ fN, uint8_t* __restrict__ img,
                                                     int n_c) {
    using S = SplitGeo<N, CL>;
    constexpr int n = N * N * N;
    const size_t total = (size_t)n_c * n;
    for (size_t e = (size_t)blockIdx.x * 256 + threadIdx.x; e < total; e += (size_t)gridDim.x * 256) {
        const int jj = (int)(e / n), v = (int)(e % n);
        const int i0 = v / (N * N), r = i0 / S::PP, R = (i0 % S::PP) * N + (v / N) % N;
        const uint32_t w = split_pack(__ldg(&fN[e]));
        *reinterpret_cast<uint32_t*>(img + ((size_t)jj * CL + r) * S::A_BYTES + split_a_offset<N, CL>(R, v % N)) = w;
    }
}

struct SplitParams {
    const uint8_t* img;     // [n_c][CL][A_BYTES] pre-split chunk inputs
    const uint8_t* smat;    // [nodes][B_BYTES] split shift matrices (axes 0, 1, 2)
    float* out;             // shifted fields, voxel-chunk-major layout (shifted_field_row)
    int* err;               // device error word
    int n_c, M, q0, n_fields;
};

constexpr int kSplitThreads = 512;    // 16 warps; warps w, w + 4, w + 8, w + 12 share TMEM lanes 32 (w % 4) ...

// Cluster-wide barrier with release/acquire semantics (a no-op for CL = 1).
template <int CL>
__device__ __forceinline__ void split_cluster_sync() {
    if constexpr (CL > 1) {
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    } else {
        __syncthreads();
    }
}

template <int N, int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(kSplitThreads, 1) k_shift_split(SplitParams P) {
    using S = SplitGeo<N, CL>;
    constexpr int PP = S::PP;
    extern __shared__ __align__(1024) uint8_t ssm[];
    uint8_t* A = ssm;                                   // [A_BYTES]
    uint8_t* Bm = ssm + S::A_BYTES;                     // [3][B_AXIS_BYTES]
    __shared__ uint64_t bar_in, bar_mma;
    __shared__ uint32_t tmem_base;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int q = warp & 3, h = warp >> 2;              // lane quarter, tile phase
    constexpr int TSTEP = kSplitThreads / 128;
    int rank = 0;
    if constexpr (CL > 1) rank = (int)cg::this_cluster().block_rank();
    const int cid = blockIdx.x / CL, ncl = gridDim.x / CL;
    const int f0 = (int)((long long)P.n_fields * cid / ncl);
    const int f1 = (int)((long long)P.n_fields * (cid + 1) / ncl);
    auto node_of = [&](int f) { return P.q0 * P.M + f / P.n_c; };   // slot = f / n_c = qq*M + p
    // shared-memory base of the A operand of every CTA of the cluster (generic addresses)
    uint8_t* Ar[CL];
#pragma unroll
    for (int r = 0; r < CL; ++r) {
        if constexpr (CL > 1) Ar[r] = cg::this_cluster().map_shared_rank(A, r);
        else Ar[r] = A;
    }
    if (t == 0) {
        mbar_init(&bar_in, 1);
        mbar_init(&bar_mma, 1);
        mbar_init_fence();
    }
    if (warp == 0) tc_alloc<S::TMEM_COLS>(&tmem_base);
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = tmem_base;
    constexpr uint32_t IDESC = tc_instr_desc(1, 128, S::NB);
    constexpr uint32_t SBO_A = 128, SBO_B = S::KCORES * 128;
    // loads of this CTA's part of the input image (and the node's matrices when the node changes)
    auto issue_load = [&](int f, bool with_b) {
        const uint32_t bytes = S::A_BYTES + (with_b ? S::B_BYTES : 0u);
        mbar_arrive_expect_tx(&bar_in, bytes);
        bulk_g2s(A, P.img + ((size_t)(f % P.n_c) * CL + rank) * S::A_BYTES, S::A_BYTES, &bar_in);
        if (with_b) bulk_g2s(Bm, P.smat + (size_t)node_of(f) * S::B_BYTES, S::B_BYTES, &bar_in);
    };
    auto issue_mmas = [&](int axis) {                   // one pass over this CTA's lines (thread 0)
        tc_fence_after_sync();
        const uint32_t b0 = smem_u32(Bm) + (uint32_t)axis * S::B_AXIS_BYTES;
#pragma unroll 1
        for (int tile = 0; tile < S::TILES; ++tile) {
#pragma unroll
            for (int ks = 0; ks < S::KSTEPS; ++ks) {
                const uint64_t ad = tc_smem_desc(smem_u32(A) + (uint32_t)(2 * ks) * S::LBO + (uint32_t)tile * 16u * 128u,
                                                 S::LBO, SBO_A);
                const uint64_t bd = tc_smem_desc(b0 + (uint32_t)(2 * ks) * 128u, 128, SBO_B);
                tc_mma_bf16(tmem + (uint32_t)(tile * S::NB), ad, bd, IDESC, ks > 0 ? 1u : 0u);
            }
        }
        tc_commit(&bar_mma);
    };
    uint32_t ph_in = 0, ph_mma = 0;
    bool pending_in = false, pending_mma = false, ok = true;
    if (t == 0 && f0 < f1) issue_load(f0, true);
    pending_in = f0 < f1;
    // Every CTA of a cluster walks the same fields and passes the same cluster
    // barriers; after a failed wait a CTA stops working but keeps passing them.
    for (int f = f0; f < f1; ++f) {
        if (ok) {
            ok = mbar_wait_bounded(&bar_in, ph_in);
            ok = __syncthreads_and(ok);
            if (ok) {
                ph_in ^= 1u;
                pending_in = false;
            }
        }
        for (int pass = 0; pass < 3; ++pass) {
            if (ok) {
                if (t == 0) issue_mmas(2 - pass);       // axis 2, 1, 0
                pending_mma = true;
                ok = mbar_wait_bounded(&bar_mma, ph_mma);
                ok = __syncthreads_and(ok);
                if (ok) {
                    ph_mma ^= 1u;
                    pending_mma = false;
                }
                tc_fence_after_sync();
            }
            // pass 2 -> 3 writes into other CTAs' operands: they must have finished their pass-2 MMAs
            if (pass == 1) split_cluster_sync<CL>();
            if (ok && pass == 2 && f + 1 < f1) {
                // A and B are free (the MMAs are done): fetch the next field while this one is written out
                if (t == 0) issue_load(f + 1, node_of(f + 1) != node_of(f));
                pending_in = true;
            }
            if (ok) {
                // the tiles h, h + TSTEP, ... of lanes 32q..32q+31; result c of local line R is
                // D[R][c] + D[R][N + c]
#pragma unroll 1
                for (int tile = h; tile < S::TILES; tile += TSTEP) {
                    const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(tile * S::NB);
                    const int R = tile * 128 + 32 * q + lane;
#pragma unroll
                    for (int c0 = 0; c0 < N; c0 += 16) {
                        uint32_t u[16], w[16];
                        tc_ld16(taddr + c0, u);
                        tc_ld16(taddr + N + c0, w);
                        tc_wait_ld();
                        if (pass == 0) {
                            // line (i0l, i1) -> element k = i1 of local line c PP + i0l
                            uint8_t* dst = A + split_a_offset<N, CL>(R / N, R % N);
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const float x = __uint_as_float(u[j]) + __uint_as_float(w[j]);
                                *reinterpret_cast<uint32_t*>(dst + (c0 + j) * (PP / 8) * 128) = split_pack(x);
                            }
                        } else if (pass == 1) {
                            // line (i2, i0l) -> element k = rank PP + i0l of line (c % PP) N + i2 of CTA c / PP
                            const uint32_t off = split_a_offset<N, CL>(R / PP, rank * PP + R % PP);
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const int c = c0 + j;
                                const float x = __uint_as_float(u[j]) + __uint_as_float(w[j]);
                                *reinterpret_cast<uint32_t*>(Ar[c / PP] + off + (c % PP) * (N / 8) * 128) =
                                    split_pack(x);
                            }
                        } else {
                            // line (i1l, i2) -> voxel c N^2 + rank PP N + R, c N^2 n_c floats apart
                            float* dst = shifted_field_row<N, 3>(P.out, f / P.n_c, f % P.n_c, P.n_c, rank * PP * N + R);
                            const size_t cstride = (size_t)N * N * P.n_c;
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                dst[(size_t)(c0 + j) * cstride] = __uint_as_float(u[j]) + __uint_as_float(w[j]);
                        }
                    }
                }
                if (pass < 2) fence_proxy_async_all();  // re-staged operand -> tensor core reads
                tc_fence_before_sync();
            }
            // pass 1 -> 2 is local; pass 2 -> 3 must have landed in every CTA before pass 3
            if (pass == 1) split_cluster_sync<CL>();
            else __syncthreads();
        }
    }
    if (!ok && t == 0) {
        atomicOr(P.err, kErrTimeout);
        // let transfers and MMAs still in flight land before the CTA exits
        if (pending_mma) (void)mbar_wait_bounded(&bar_mma, ph_mma);
        if (pending_in) (void)mbar_wait_bounded(&bar_in, ph_in);
    }
    tc_fence_before_sync();
    // no CTA leaves while another may still write into its shared memory
    split_cluster_sync<CL>();
    if (warp == 0) tc_dealloc<S::TMEM_COLS>(tmem);
}

}  // namespace boltz_dev
