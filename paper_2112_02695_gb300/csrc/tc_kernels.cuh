// Tensor-core (tcgen05) kernels.
//
// k_project_tc: the r^3 projection T_{k,(j,l)} = dv^d sum_v V_k(v) Q_{jl}(v) as
// a GEMM D = Q V^T (M = r^2 pair rows, N = r padded to NP, K = N^d voxels) on
// the fifth-generation tensor cores, with both operands split as
// x = hi + lo (hi = x rounded to TF32, lo = x - hi) and
// D = Qhi Vhi + Qhi Vlo + Qlo Vhi accumulated in FP32 in tensor memory, which
// keeps FP32 accuracy (the dropped lo*lo term is ~2^-22 relative).  A CTA owns
// one 128-row M tile and a slice of K; partial sums per slice are reduced by
// k_project_reduce in a fixed order.
#pragma once

#include "tc.cuh"

namespace boltz_dev {

constexpr int kProjKC = 128;          // voxels per staged K chunk

template <int NP>
struct ProjTcShape {
    static constexpr int TMEM_COLS = NP <= 32 ? 32 : (NP <= 64 ? 64 : 128);
    static constexpr size_t A_BYTES = size_t(128) * kProjKC * 4;     // one of hi / lo
    static constexpr size_t B_BYTES = size_t(NP) * kProjKC * 4;
    static constexpr size_t SMEM = 2 * A_BYTES + 2 * B_BYTES;
};

// Stage rows [row0, row0 + nrows) x voxels [v0, v0 + kProjKC) of a row-major
// [rows][n] matrix as TF32 hi and lo parts in the K-major core-matrix layout
// (rows beyond `valid_rows` are zero).  Each warp writes 512 contiguous bytes.
template <int NROWS>
__device__ __forceinline__ void stage_tf32_split(const float* __restrict__ src, int row0, int valid_rows, int n,
                                                 int v0, uint8_t* hi, uint8_t* lo, int t, int nthreads) {
    constexpr int KC4 = kProjKC / 4;                       // cores along K (16 B = 4 floats each)
#pragma unroll 8
    for (int e = t; e < NROWS * KC4; e += nthreads) {
        const int r8 = e & 7, k4 = (e >> 3) % KC4, mb = e / (8 * KC4);
        const int row = mb * 8 + r8;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row0 + row < valid_rows)
            x = __ldg(reinterpret_cast<const float4*>(src + (size_t)(row0 + row) * n + v0 + 4 * k4));
        const float4 h = make_float4(to_tf32(x.x), to_tf32(x.y), to_tf32(x.z), to_tf32(x.w));
        const float4 l = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
        const int off = (mb * KC4 + k4) * 128 + r8 * 16;
        *reinterpret_cast<float4*>(hi + off) = h;
        *reinterpret_cast<float4*>(lo + off) = l;
    }
}

constexpr int kProjThreads = 256;     // 8 warps stage operands; warps 0-3 read the 128 TMEM lanes

template <int NP>
__global__ void __launch_bounds__(kProjThreads, 1) k_project_tc(const float* __restrict__ V, const float* __restrict__ Q,
                                                        float* __restrict__ partial, int r, int n, int kpc,
                                                        int* err) {
    using S = ProjTcShape<NP>;
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t* a_hi = sm;
    uint8_t* a_lo = sm + S::A_BYTES;
    uint8_t* b_hi = sm + 2 * S::A_BYTES;
    uint8_t* b_lo = b_hi + S::B_BYTES;
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int r2 = r * r;
    const int m0 = blockIdx.y * 128;                       // first pair row of this M tile
    const int vbeg = blockIdx.x * kpc;
    if (t == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
    }
    if (warp == 0) tc_alloc<S::TMEM_COLS>(&tmem_base);
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = tmem_base;
    constexpr uint32_t IDESC = tc_instr_desc(2, 128, NP);
    constexpr uint32_t SBO_A = (kProjKC / 4) * 128, SBO_B = (kProjKC / 4) * 128;
    bool ok = true;
    const int nchunks = kpc / kProjKC;
    for (int c = 0; c < nchunks && ok; ++c) {
        const int v0 = vbeg + c * kProjKC;
        stage_tf32_split<128>(Q, m0, r2, n, v0, a_hi, a_lo, t, kProjThreads);
        stage_tf32_split<NP>(V, 0, r, n, v0, b_hi, b_lo, t, kProjThreads);
        fence_proxy_async_smem();
        __syncthreads();
        if (t == 0) {
            tc_fence_after_sync();
#pragma unroll 1
            for (int ks = 0; ks < kProjKC / 8; ++ks) {      // K = 8 TF32 per MMA = 2 cores of 16 bytes
                const uint32_t koff = ks * 256;
                const uint64_t ah = tc_smem_desc(smem_u32(a_hi) + koff, 128, SBO_A);
                const uint64_t al = tc_smem_desc(smem_u32(a_lo) + koff, 128, SBO_A);
                const uint64_t bh = tc_smem_desc(smem_u32(b_hi) + koff, 128, SBO_B);
                const uint64_t bl = tc_smem_desc(smem_u32(b_lo) + koff, 128, SBO_B);
                tc_mma_tf32(tmem, ah, bh, IDESC, (c > 0 || ks > 0) ? 1u : 0u);
                tc_mma_tf32(tmem, ah, bl, IDESC, 1u);
                tc_mma_tf32(tmem, al, bh, IDESC, 1u);
            }
            tc_commit(&bar);
        }
        ok = mbar_wait_bounded(&bar, (uint32_t)c & 1u);   // MMAs done: the stage can be refilled
        ok = __syncthreads_and(ok);
        tc_fence_after_sync();
    }
    if (!ok) {
        if (t == 0) atomicOr(err, kErrTimeout);
    } else if (warp < 4) {
        // rows m0 + 32 warp + lane, columns k = 0..NP-1 of D
        const int pr = m0 + warp * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        const int slice = blockIdx.x;
#pragma unroll
        for (int c0 = 0; c0 < NP; c0 += 16) {
            uint32_t v[16];
            tc_ld16(lane_addr + c0, v);
            tc_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int k = c0 + j;
                if (pr < r2 && k < r) partial[((size_t)slice * r + k) * r2 + pr] = __uint_as_float(v[j]);
            }
        }
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tc_dealloc<S::TMEM_COLS>(tmem);
}

}  // namespace boltz_dev
