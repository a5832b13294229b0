// Kernels of the low-rank step pieces that consume the collision batch
// (paper Sec. 2, eqs. "eqn:K-step detailed" and "eqn:L-step detailed";
// Sec. 2.4, the fully discrete scheme; Sec. 3.2, dropping basis).
//
// Functions of x or v are rows: K [r][n_x], V [r][n_v]; r <= 64.
//   k_kstep_collision   C_j(x) = sum_{m,n} T_jmn K_m(x) K_n(x)            (FP32)
//   k_lstep_collision   G_i(v) = sum_{p,q} C_ipq Q_{p r + q}(v)             (FP32)
//   Cholesky-QR2        W_j = sum_i Y_i R_ij, <Y_i, Y_k> = w sum Y_i Y_k = delta  (FP64;
//                       Fukaya et al., "CholeskyQR2", 2014: Gram matrix,
//                       Cholesky factor, triangular solve, done twice)
//   k_svd_jacobi_f64    S = U Sigma Q^T by one-sided (Hestenes) Jacobi rotations
//                       in round-robin pair order, singular values sorted
//                       descending; r' = #{sigma >= drop_tol}               (FP64;
//                       k_svd_small_f64: the same in one warp for r <= 16)
//   k_rotate_f64        X_bar_k = sum_i X_i U_ik, k < r'                    (FP64)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace boltz_dev {

constexpr int kLrThreads = 256;

// ---------------------------------------------------------------- K-step collision term
// One thread per cell; K_m(x) of the cell in registers; block row y takes the
// output slices j in chunks of jt (T[j0 .. j0 + jt) staged in shared memory,
// jt r^2 floats <= 48 KB), chunks y, y + gridDim.y, ...
template <int RMAX>
__global__ void __launch_bounds__(kLrThreads) k_kstep_collision(const float* __restrict__ T,
                                                               const float* __restrict__ K, float* __restrict__ out,
                                                               int r, int n, int jt) {
    extern __shared__ float lr_smem[];
    const int x = blockIdx.x * kLrThreads + threadIdx.x;
    float k[RMAX];
#pragma unroll
    for (int m = 0; m < RMAX; ++m) k[m] = (m < r && x < n) ? __ldg(&K[(size_t)m * n + x]) : 0.f;
    const int rr = r * r;
    for (int j0 = blockIdx.y * jt; j0 < r; j0 += gridDim.y * jt) {
        const int jn = min(jt, r - j0);
        __syncthreads();
        for (int e = threadIdx.x; e < jn * rr; e += kLrThreads) lr_smem[e] = __ldg(&T[(size_t)j0 * rr + e]);
        __syncthreads();
        for (int jj = 0; jj < jn; ++jj) {
            const float* Tj = lr_smem + jj * rr;
            float acc = 0.f;
#pragma unroll
            for (int m = 0; m < RMAX; ++m) {
                if (m < r) {
                    float inner = 0.f;
#pragma unroll
                    for (int q = 0; q < RMAX; ++q)
                        if (q < r) inner = fmaf(Tj[m * r + q], k[q], inner);
                    acc = fmaf(k[m], inner, acc);
                }
            }
            if (x < n) out[(size_t)(j0 + jj) * n + x] = acc;
        }
    }
}

// ---------------------------------------------------------------- L-step collision term
// A block owns 64 voxels; its 256 threads split the r^2 pair index into
// LSL = 4 interleaved slices (thread = voxel + 64 slice), each accumulating
// the r outputs of its voxel over its slice in registers; the slices are
// summed through shared memory in a fixed order.  C is staged in chunks of
// 64 pair columns; every Q value is read once, by 64-voxel coalesced loads.
constexpr int kLstepPC = 64;
constexpr int kLstepVB = 64;
constexpr int kLstepSL = kLrThreads / kLstepVB;

template <int RMAX>
constexpr size_t lstep_smem() {
    return (size_t(RMAX) * kLstepPC + size_t(kLstepSL - 1) * kLstepVB * RMAX) * sizeof(float);
}

template <int RMAX>
__global__ void __launch_bounds__(kLrThreads) k_lstep_collision(const float* __restrict__ Q,
                                                               const float* __restrict__ C, float* __restrict__ out,
                                                               int r, int n) {
    extern __shared__ float lst_smem[];
    float* Cs = lst_smem;                                     // [RMAX][PC]
    float* red = lst_smem + RMAX * kLstepPC;                  // [SL-1][RMAX][VB]
    const int lv = threadIdx.x % kLstepVB, sl = threadIdx.x / kLstepVB;
    const int v = blockIdx.x * kLstepVB + lv;
    const int rr = r * r;
    float acc[RMAX];
#pragma unroll
    for (int i = 0; i < RMAX; ++i) acc[i] = 0.f;
    for (int pq0 = 0; pq0 < rr; pq0 += kLstepPC) {
        const int pn = min(kLstepPC, rr - pq0);
        __syncthreads();
        for (int e = threadIdx.x; e < r * kLstepPC; e += kLrThreads) {
            const int i = e / kLstepPC, c = e % kLstepPC;
            Cs[i * kLstepPC + c] = c < pn ? __ldg(&C[(size_t)i * rr + pq0 + c]) : 0.f;
        }
        __syncthreads();
        if (v < n) {
#pragma unroll 4
            for (int c = sl; c < pn; c += kLstepSL) {
                const float qv = __ldg(&Q[(size_t)(pq0 + c) * n + v]);
#pragma unroll
                for (int i = 0; i < RMAX; ++i)
                    if (i < r) acc[i] = fmaf(Cs[i * kLstepPC + c], qv, acc[i]);
            }
        }
    }
    if (sl > 0) {
#pragma unroll
        for (int i = 0; i < RMAX; ++i) red[((sl - 1) * RMAX + i) * kLstepVB + lv] = acc[i];
    }
    __syncthreads();
    if (sl == 0 && v < n) {
#pragma unroll
        for (int i = 0; i < RMAX; ++i) {
            if (i < r) {
                float t = acc[i];
#pragma unroll
                for (int k = 0; k < kLstepSL - 1; ++k) t += red[(k * RMAX + i) * kLstepVB + lv];
                out[(size_t)i * n + v] = t;
            }
        }
    }
}

// ---------------------------------------------------------------- r^4 couplings of the S- and L-steps
// Block i: M_i[m][n] = sum_l ( sum_k E_ikl S_km ) S_ln  (the same form as the
// L-step's C_ipq = sum_n (sum_m E_imn S_mp) S_nq, with E symmetric in its
// last two indices), staged in shared memory; C_out[i] = M_i.  When T is
// given, also D[i][j] = sum_{m,n} T_jmn M_i[m][n] (the S-step collision term).
constexpr size_t kCouplingSmem = 3 * 64 * 64 * sizeof(float);

__global__ void __launch_bounds__(kLrThreads) k_lr_coupling(const float* __restrict__ E, const float* __restrict__ S,
                                                           const float* __restrict__ T, int r,
                                                           float* __restrict__ C_out, float* __restrict__ D) {
    extern __shared__ float cp_smem[];
    float* Ei = cp_smem;                 // [r][r]  E_i k l
    float* Ss = cp_smem + 64 * 64;       // [r][r]
    float* In = cp_smem + 2 * 64 * 64;   // [r][r]  inner[m][l]
    const int i = blockIdx.x, rr = r * r;
    for (int e = threadIdx.x; e < rr; e += kLrThreads) {
        Ei[e] = __ldg(&E[(size_t)i * rr + e]);
        Ss[e] = __ldg(&S[e]);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rr; e += kLrThreads) {      // inner[m][l] = sum_k E_ikl S_km
        const int m = e / r, l = e % r;
        float a = 0.f;
        for (int k = 0; k < r; ++k) a = fmaf(Ei[k * r + l], Ss[k * r + m], a);
        In[e] = a;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rr; e += kLrThreads) {      // M[m][n] = sum_l inner[m][l] S_ln
        const int m = e / r, n = e % r;
        float a = 0.f;
        for (int l = 0; l < r; ++l) a = fmaf(In[m * r + l], Ss[l * r + n], a);
        Ei[e] = a;                                          // E_i is no longer needed
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rr; e += kLrThreads) C_out[(size_t)i * rr + e] = Ei[e];
    if (T) {
        for (int j = threadIdx.x; j < r; j += kLrThreads) {
            float a = 0.f;
            for (int e = 0; e < rr; ++e) a = fmaf(__ldg(&T[(size_t)j * rr + e]), Ei[e], a);
            D[(size_t)i * r + j] = a;
        }
    }
}

// ---------------------------------------------------------------- Cholesky-QR2 (FP64)
constexpr int kGramVT = 32;         // staged columns of W per step

// part[slice][a][b] = sum_{v in slice} W_a(v) W_b(v)  (both triangles written)
__global__ void __launch_bounds__(kLrThreads) k_gram_f64(const double* __restrict__ W, int r, int n, int nslices,
                                                        double* __restrict__ part) {
    __shared__ double Ws[64 * kGramVT];
    const int s = blockIdx.x;
    const int v0 = (int)((long long)n * s / nslices), v1 = (int)((long long)n * (s + 1) / nslices);
    const int npairs = r * (r + 1) / 2;
    constexpr int PT = (64 * 65 / 2 + kLrThreads - 1) / kLrThreads;     // pairs per thread (max)
    double acc[PT];
    int pa[PT], pb[PT];
#pragma unroll
    for (int k = 0; k < PT; ++k) {
        acc[k] = 0.0;
        int e = threadIdx.x + k * kLrThreads, a = 0;
        if (e < npairs) {
            while (e >= r - a) {               // e -> (a, b), a <= b, row-major upper triangle
                e -= r - a;
                ++a;
            }
        }
        pa[k] = a;
        pb[k] = a + e;
    }
    for (int c0 = v0; c0 < v1; c0 += kGramVT) {
        const int cn = min(kGramVT, v1 - c0);
        __syncthreads();
        for (int e = threadIdx.x; e < r * kGramVT; e += kLrThreads) {
            const int a = e / kGramVT, c = e % kGramVT;
            Ws[a * kGramVT + c] = c < cn ? __ldg(&W[(size_t)a * n + c0 + c]) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PT; ++k) {
            if (threadIdx.x + k * kLrThreads >= npairs) break;
            const double* wa = Ws + pa[k] * kGramVT;
            const double* wb = Ws + pb[k] * kGramVT;
            double t = acc[k];
#pragma unroll 8
            for (int c = 0; c < kGramVT; ++c) t = fma(wa[c], wb[c], t);
            acc[k] = t;
        }
    }
#pragma unroll
    for (int k = 0; k < PT; ++k) {
        if (threadIdx.x + k * kLrThreads >= npairs) break;
        part[((size_t)s * r + pa[k]) * r + pb[k]] = acc[k];
        part[((size_t)s * r + pb[k]) * r + pa[k]] = acc[k];
    }
}

// One CTA: G = w sum_s part[s] (fixed order), G = R^T R (R upper, positive
// diagonal), Rinv = R^-1; when Rprev is given, Rout = R Rprev (the factor of
// the two passes; Rout must not alias Rprev), else Rout = R.  When pivot k is
// not positive, info (zeroed by the caller) receives k + 1 unless an earlier
// pass already failed, and R, Rinv are NaN.
constexpr size_t kCholSmem = 3 * 64 * 64 * sizeof(double);

constexpr int kCholThreads = 1024;

__global__ void __launch_bounds__(kCholThreads) k_chol_f64(const double* __restrict__ part, int nslices, int r, double w,
                                                          const double* __restrict__ Rprev, double* __restrict__ Rout,
                                                          double* __restrict__ Rinv, int* __restrict__ info) {
    extern __shared__ double chol_smem[];
    double* G = chol_smem;                         // [64 * 64] each
    double* Rs = chol_smem + 64 * 64;
    double* Xs = chol_smem + 2 * 64 * 64;
    __shared__ int bad;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    constexpr int NW = kCholThreads / 32;
    if (t == 0) bad = 0;
    // G = w sum_s part[s]: one warp per entry, lanes over the slices, fixed-order tree
    for (int e = warp; e < r * r; e += NW) {
        double g = 0.0;
        for (int s = lane; s < nslices; s += 32) g += part[(size_t)s * r * r + e];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g += __shfl_down_sync(0xffffffffu, g, o);
        if (lane == 0) {
            G[e] = w * g;
            Rs[e] = 0.0;
        }
    }
    __syncthreads();
    for (int k = 0; k < r; ++k) {
        if (t == 0) {
            double d = G[k * r + k];
            for (int i = 0; i < k; ++i) d -= Rs[i * r + k] * Rs[i * r + k];
            if (!(d > 0.0)) {
                bad = k + 1;
                d = 0.0;
            }
            Rs[k * r + k] = sqrt(d);
        }
        __syncthreads();
        if (bad) break;
        for (int j = k + 1 + t; j < r; j += kCholThreads) {
            double a = G[k * r + j];
            for (int i = 0; i < k; ++i) a -= Rs[i * r + k] * Rs[i * r + j];
            Rs[k * r + j] = a / Rs[k * r + k];
        }
        __syncthreads();
    }
    if (bad) {
        if (t == 0 && *info == 0) *info = bad;     // the first failing pass is reported
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        for (int e = t; e < r * r; e += kCholThreads) {
            Rout[e] = nan;
            Rinv[e] = nan;
        }
        return;
    }
    // Rinv by back substitution, one column per thread: R X = I
    for (int j = t; j < r; j += kCholThreads) {
        for (int i = r - 1; i >= 0; --i) {
            double a = (i == j) ? 1.0 : 0.0;
            for (int k = i + 1; k <= j; ++k) a -= Rs[i * r + k] * Xs[k * r + j];
            Xs[i * r + j] = (i <= j) ? a / Rs[i * r + i] : 0.0;
        }
    }
    __syncthreads();
    for (int e = t; e < r * r; e += kCholThreads) {
        Rinv[e] = Xs[e];
        const int i = e / r, j = e % r;
        double o = Rs[e];
        if (Rprev) {
            o = 0.0;
            for (int k = i; k <= j; ++k) o += Rs[i * r + k] * Rprev[k * r + j];
        }
        Rout[e] = o;
    }
}

// Y_k(v) = sum_{i <= k} W_i(v) Rinv_ik; in place allowed (Y == W): each
// thread reads its voxel's r values before writing.
template <int RMAX>
__global__ void __launch_bounds__(kLrThreads) k_apply_rinv_f64(const double* W, const double* __restrict__ Rinv,
                                                              int r, int n, double* Y) {
    __shared__ double Ri[64 * 64];
    for (int e = threadIdx.x; e < r * r; e += kLrThreads) Ri[e] = Rinv[e];
    __syncthreads();
    const int v = blockIdx.x * kLrThreads + threadIdx.x;
    if (v >= n) return;
    double w[RMAX];
#pragma unroll
    for (int i = 0; i < RMAX; ++i) w[i] = (i < r) ? W[(size_t)i * n + v] : 0.0;
#pragma unroll 4
    for (int k = 0; k < RMAX; ++k) {
        if (k >= r) break;
        double y = 0.0;
#pragma unroll
        for (int i = 0; i < RMAX; ++i)
            if (i <= k) y = fma(w[i], Ri[i * r + k], y);
        Y[(size_t)k * n + v] = y;
    }
}

// ---------------------------------------------------------------- Cholesky-QR2 over many CTAs (FP64)
// The same factorisation for r <= kQrSpreadR rows of n <= kQrSpreadMaxN
// entries (e.g. the K and L factors of a low-rank step).  FP64 issues at a
// small fraction of the FP32 rate on this GPU, so the Gram sums and the R^-1
// applications are spread over up to 152 CTAs (a block of at most 256
// entries each), and the small factorisations run in whichever CTA finishes
// its block last (a ticket counter: nothing waits):
//   pass 0: partial Gram of W; last CTA: G = w sum of the partials in CTA
//           order, G = R1^T R1, X1 = R1^-1;
//   pass 1: W X1 written to Y, its partial Gram; last CTA: R2, X2 = R2^-1,
//           R = R2 R1;
//   then Y <- Y X2 (k_qr_spread_apply).
// A Cholesky factorisation that meets a pivot d <= 0 records k + 1 in info
// (the first failure) and writes NaN to R and to the inverse, so that Y
// comes out NaN, as on the multi-kernel path.
constexpr int kQrSpreadR = 16, kQrSpreadThreads = 256, kQrSpreadRows = 256, kQrSpreadCtas = 152;
constexpr int kQrSpreadMaxN = kQrSpreadCtas * kQrSpreadRows;
constexpr int kQrSpreadPairs = kQrSpreadR * (kQrSpreadR + 1) / 2;

// entries per CTA: at least 16, so that small blocks use few CTAs
__host__ __device__ inline int qr_spread_rows(int n) {
    const int rows = (n + kQrSpreadCtas - 1) / kQrSpreadCtas;
    return rows < 16 ? 16 : rows;
}

// workspace: partial Grams [ctas][kQrSpreadPairs], X1, X2, R1 [16 * 16] each, then room for two
// tickets (used when the caller passes none of its own)
__host__ __device__ constexpr size_t qr_spread_ticket_offset() {
    return (size_t(kQrSpreadCtas) * kQrSpreadPairs + 3 * kQrSpreadR * kQrSpreadR) * sizeof(double);
}
__host__ __device__ constexpr size_t qr_spread_bytes() { return qr_spread_ticket_offset() + 64; }

// G = R^T R (R upper, r <= 32) and X = R^-1 by one warp, lane j owning column
// j; returns 0 or the 1-based index of the first pivot that is not positive.
__device__ inline int chol_inv_warp(const double* G, int r, double* Rs, double* Xs, double* Dinv) {
    const int lane = threadIdx.x & 31;
    for (int e = lane; e < r * r; e += 32) {
        Rs[e] = 0.0;
        Xs[e] = 0.0;
    }
    __syncwarp();
    for (int k = 0; k < r; ++k) {
        double a = 0.0;
        if (lane >= k && lane < r) {
            a = G[k * r + lane];
            for (int i = 0; i < k; ++i) a = fma(-Rs[i * r + k], Rs[i * r + lane], a);
        }
        const double d = __shfl_sync(0xffffffffu, a, k);
        if (!(d > 0.0)) return k + 1;                      // the same value in every lane
        const double inv = rsqrt(d);
        if (lane >= k && lane < r) Rs[k * r + lane] = lane == k ? d * inv : a * inv;
        if (lane == 0) Dinv[k] = inv;
        __syncwarp();
    }
    if (lane < r) {                                        // column j of R^-1, bottom up
        const int j = lane;
        for (int i = j; i >= 0; --i) {
            double a = i == j ? 1.0 : 0.0;
            for (int k = i + 1; k <= j; ++k) a = fma(-Rs[i * r + k], Xs[k * r + j], a);
            Xs[i * r + j] = a * Dinv[i];
        }
    }
    __syncwarp();
    return 0;
}

// ticket: two counters, zero before the first launch and left at zero.
template <int PASS>
__global__ void __launch_bounds__(kQrSpreadThreads) k_qr_spread_f64(const double* W, int r, int n, double w, int rows,
                                                                   double* Y, double* __restrict__ R,
                                                                   double* __restrict__ ws, unsigned* __restrict__ ticket,
                                                                   int* __restrict__ info) {
    __shared__ double Ws[kQrSpreadR * kQrSpreadRows];     // this CTA's entries, [row i][entry]
    __shared__ double Xin[kQrSpreadR * kQrSpreadR];
    __shared__ double G[kQrSpreadR * kQrSpreadR], Rs[kQrSpreadR * kQrSpreadR], Xs[kQrSpreadR * kQrSpreadR];
    __shared__ double Dinv[kQrSpreadR];
    __shared__ int last;
    double* part = ws;
    double* X1 = ws + size_t(kQrSpreadCtas) * kQrSpreadPairs;
    double* X2 = X1 + kQrSpreadR * kQrSpreadR;
    double* R1 = X2 + kQrSpreadR * kQrSpreadR;
    const int t = threadIdx.x, v0 = blockIdx.x * rows, nr = min(rows, n - v0);
    const int npairs = r * (r + 1) / 2;
    if (PASS == 1) {
        for (int e = t; e < r * r; e += kQrSpreadThreads) Xin[e] = X1[e];
        __syncthreads();
    }
    if (t < nr) {
        double x[kQrSpreadR];
#pragma unroll
        for (int i = 0; i < kQrSpreadR; ++i) x[i] = i < r ? W[(size_t)i * n + v0 + t] : 0.0;
        if (PASS == 1) {                                   // row of W X1 (upper-triangular X1)
#pragma unroll
            for (int k = kQrSpreadR - 1; k >= 0; --k) {
                if (k >= r) continue;
                double y = 0.0;
#pragma unroll
                for (int i = 0; i <= k; ++i) y = fma(x[i], Xin[i * r + k], y);
                x[k] = y;
            }
#pragma unroll
            for (int i = 0; i < kQrSpreadR; ++i)
                if (i < r) Y[(size_t)i * n + v0 + t] = x[i];
        }
#pragma unroll
        for (int i = 0; i < kQrSpreadR; ++i)
            if (i < r) Ws[i * kQrSpreadRows + t] = x[i];
    }
    __syncthreads();
    if (t < npairs) {                                      // entry t = (a, b), a <= b, row-major upper triangle
        int e = t, a = 0;
        while (e >= r - a) {
            e -= r - a;
            ++a;
        }
        const int b = a + e;
        double g = 0.0;
        for (int c = 0; c < nr; ++c) g = fma(Ws[a * kQrSpreadRows + c], Ws[b * kQrSpreadRows + c], g);
        part[(size_t)blockIdx.x * kQrSpreadPairs + t] = g;
    }
    __threadfence();
    __syncthreads();
    if (t == 0) last = atomicAdd(&ticket[PASS], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    {   // G = w sum of the partials.  An FP64 instruction costs a warp the same for one lane as for 32, so
        // thread (slice, entry) sums the CTAs c = slice, slice + S, ... of one entry (whole warps busy),
        // then one thread per entry adds the S slice sums in order.
        __shared__ double sl[kQrSpreadThreads];
        const int pad = (npairs + 31) & ~31, S = kQrSpreadThreads / pad;     // slices (>= 1: pad <= 160)
        const int slice = t / pad, e = t % pad;
        if (slice < S) {
            double g = 0.0;
            if (e < npairs)
                for (int c = slice; c < (int)gridDim.x; c += S) g += __ldcg(&part[(size_t)c * kQrSpreadPairs + e]);
            sl[slice * pad + e] = g;
        }
        __syncthreads();
        if (t < npairs) {
            double g = 0.0;
            for (int k = 0; k < S; ++k) g += sl[k * pad + t];
            int ee = t, a = 0;
            while (ee >= r - a) {
                ee -= r - a;
                ++a;
            }
            const int b = a + ee;
            G[a * r + b] = w * g;
            G[b * r + a] = w * g;
        }
    }
    __syncthreads();
    __shared__ int bad;
    if (t < 32) {
        const int bk = chol_inv_warp(G, r, Rs, Xs, Dinv);
        if (t == 0) bad = bk;
    }
    __syncthreads();
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    if (bad && t == 0 && *info == 0) *info = bad;
    double* Xout = PASS == 0 ? X1 : X2;
    for (int e = t; e < r * r; e += kQrSpreadThreads) {
        Xout[e] = bad ? nan : Xs[e];
        if (PASS == 0) {
            R1[e] = bad ? nan : Rs[e];
        } else {
            const int i = e / r, j = e % r;
            double o = 0.0;
            for (int k = i; k <= j; ++k) o = fma(Rs[i * r + k], __ldcg(&R1[k * r + j]), o);
            R[e] = bad ? nan : o;
        }
    }
    if (t == 0) ticket[PASS] = 0u;
}

// Y <- Y X2 in place, one entry per thread (the last step of the spread QR)
__global__ void __launch_bounds__(kQrSpreadThreads) k_qr_spread_apply(double* Y, int r, int n,
                                                                     const double* __restrict__ ws) {
    __shared__ double Xs[kQrSpreadR * kQrSpreadR];
    const double* X2 = ws + size_t(kQrSpreadCtas) * kQrSpreadPairs + kQrSpreadR * kQrSpreadR;
    for (int e = threadIdx.x; e < r * r; e += kQrSpreadThreads) Xs[e] = X2[e];
    __syncthreads();
    const int v = blockIdx.x * kQrSpreadThreads + threadIdx.x;
    if (v >= n) return;
    double x[kQrSpreadR];
#pragma unroll
    for (int i = 0; i < kQrSpreadR; ++i) x[i] = i < r ? Y[(size_t)i * n + v] : 0.0;
#pragma unroll
    for (int k = kQrSpreadR - 1; k >= 0; --k) {
        if (k >= r) continue;
        double y = 0.0;
#pragma unroll
        for (int i = 0; i <= k; ++i) y = fma(x[i], Xs[i * r + k], y);
        x[k] = y;
    }
#pragma unroll
    for (int i = 0; i < kQrSpreadR; ++i)
        if (i < r) Y[(size_t)i * n + v] = x[i];
}

// ---------------------------------------------------------------- one-sided Jacobi SVD (FP64)
// One CTA of 32 warps: in every round of a sweep the columns are paired by
// the round-robin schedule and warp p rotates pair p (lanes split the r
// entries, dot products by shuffles, the rotation computed in one lane).  A
// sweep without a rotation ends the iteration.  FP64 issues at a small
// fraction of the FP32 rate on this GPU, so the sweeps first run in FP32 on a
// rounded copy; the accumulated rotations are re-orthonormalised in FP64
// (V <- V (I - E/2), E = V^T V - I, twice) and the FP64 sweeps then start from
// A = S V, which is already diagonal to FP32 accuracy.
constexpr int kSvdMaxSweeps = 40;
constexpr size_t kSvdSmem = 2 * 64 * 64 * sizeof(double) + 2 * 64 * 64 * sizeof(float) + 64 * 64 * sizeof(double);

template <typename T>
__device__ __forceinline__ T jac_rsqrt(T x);
template <>
__device__ __forceinline__ float jac_rsqrt(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double jac_rsqrt(double x) { return rsqrt(x); }

// Sweeps on column-major A, V (column c at c*64) until no pair has
// |a_p . a_q| > tol * |a_p| |a_q|; returns whether that happened.
template <typename T>
__device__ bool jacobi_sweeps(T* A, T* V, int r, T tol, int max_sweeps) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = (r + 1) & ~1;                   // even number of columns (one idle column if r is odd)
    const T tol2 = tol * tol;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        int rotated = 0;
        for (int round = 0; round < m - 1; ++round) {
            if (warp < m / 2) {
                auto slot = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + round) % (m - 1); };
                int p = slot(warp), q = slot(m - 1 - warp);
                if (p > q) {
                    const int tmp = p;
                    p = q;
                    q = tmp;
                }
                if (q < r) {
                    T al = T(0), be = T(0), ga = T(0);
                    for (int i = lane; i < r; i += 32) {
                        const T x = A[p * 64 + i], y = A[q * 64 + i];
                        al = fma(x, x, al);
                        be = fma(y, y, be);
                        ga = fma(x, y, ga);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const T a2 = __shfl_down_sync(0xffffffffu, al, o);
                        const T b2 = __shfl_down_sync(0xffffffffu, be, o);
                        const T g2 = __shfl_down_sync(0xffffffffu, ga, o);
                        if (lane < o && lane + o < r) {
                            al += a2;
                            be += b2;
                            ga += g2;
                        }
                    }
                    T c = T(1), s = T(0);
                    int rot = 0;
                    if (lane == 0 && ga != T(0) && ga * ga > tol2 * (al * be)) {
                        const T zeta = (be - al) / (T(2) * ga);
                        const T tt = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(fma(zeta, zeta, T(1))));
                        c = jac_rsqrt(fma(tt, tt, T(1)));
                        s = c * tt;
                        rot = 1;
                    }
                    rot = __shfl_sync(0xffffffffu, rot, 0);
                    if (rot) {
                        c = __shfl_sync(0xffffffffu, c, 0);
                        s = __shfl_sync(0xffffffffu, s, 0);
                        for (int i = lane; i < r; i += 32) {
                            const T x = A[p * 64 + i], y = A[q * 64 + i];
                            A[p * 64 + i] = c * x - s * y;
                            A[q * 64 + i] = s * x + c * y;
                            const T vx = V[p * 64 + i], vy = V[q * 64 + i];
                            V[p * 64 + i] = c * vx - s * vy;
                            V[q * 64 + i] = s * vx + c * vy;
                        }
                        rotated = 1;
                    }
                }
            }
            __syncthreads();
        }
        if (!__syncthreads_or(rotated)) return true;
    }
    return false;
}

// drop_tol_dev, when not null, replaces drop_tol (a value written to device
// memory before the launch, as in a replayed graph).
__global__ void __launch_bounds__(1024) k_svd_jacobi_f64(const double* __restrict__ S, int r, double drop_tol,
                                                        double* __restrict__ U, double* __restrict__ sigma,
                                                        double* __restrict__ Qm, int* __restrict__ r_keep,
                                                        int* __restrict__ info,
                                                        const double* __restrict__ drop_tol_dev = nullptr) {
    extern __shared__ double svd_smem[];
    double* A = svd_smem;                          // column-major: column c at c*64
    double* V = svd_smem + 64 * 64;
    float* Af = reinterpret_cast<float*>(svd_smem + 2 * 64 * 64);
    float* Vf = Af + 64 * 64;
    double* E = svd_smem + 2 * 64 * 64 + 64 * 64;  // after the two float arrays (64*64 doubles' room)
    __shared__ double sv[64];
    __shared__ int order[64];
    const int t = threadIdx.x;
    for (int e = t; e < 64 * 64; e += 1024) {
        const int c = e / 64, i = e % 64;
        Af[e] = (c < r && i < r) ? (float)S[i * r + c] : 0.f;
        Vf[e] = (c == i && c < r) ? 1.f : 0.f;
    }
    __syncthreads();
    (void)jacobi_sweeps<float>(Af, Vf, r, 1e-6f, kSvdMaxSweeps);
    // V = Vf re-orthonormalised in FP64: V <- V (I - E/2), E = V^T V - I, twice
    for (int e = t; e < 64 * 64; e += 1024) V[e] = (double)Vf[e];
    __syncthreads();
    for (int it = 0; it < 2; ++it) {
        for (int e = t; e < r * r; e += 1024) {
            const int a = e / r, b = e % r;
            double g = 0.0;
            for (int i = 0; i < r; ++i) g = fma(V[a * 64 + i], V[b * 64 + i], g);
            E[a * 64 + b] = g - (a == b ? 1.0 : 0.0);
        }
        __syncthreads();
        for (int e = t; e < r * r; e += 1024) {          // new column c, row i
            const int c = e / r, i = e % r;
            double v = V[c * 64 + i];
            for (int k = 0; k < r; ++k) v = fma(-0.5 * V[k * 64 + i], E[k * 64 + c], v);
            A[c * 64 + i] = v;                               // A as scratch for the new V
        }
        __syncthreads();
        for (int e = t; e < r * r; e += 1024) {
            const int c = e / r, i = e % r;
            V[c * 64 + i] = A[c * 64 + i];
        }
        __syncthreads();
    }
    // A = S V, then the FP64 sweeps
    for (int e = t; e < 64 * 64; e += 1024) {
        const int c = e / 64, i = e % 64;
        double a = 0.0;
        if (c < r && i < r)
            for (int k = 0; k < r; ++k) a = fma(S[i * r + k], V[c * 64 + k], a);
        A[e] = a;
    }
    for (int e = t; e < 64 * 64; e += 1024) {
        const int c = e / 64, i = e % 64;
        if (c >= r || i >= r) V[e] = 0.0;
    }
    __syncthreads();
    const bool converged = jacobi_sweeps<double>(A, V, r, 1e-15, kSvdMaxSweeps);
    // singular values = column norms; sort descending (one thread, r <= 64)
    if (t < r) {
        double nn = 0.0;
        for (int i = 0; i < r; ++i) nn = fma(A[t * 64 + i], A[t * 64 + i], nn);
        sv[t] = sqrt(nn);
    }
    __syncthreads();
    if (t == 0) {
        for (int i = 0; i < r; ++i) order[i] = i;
        for (int i = 0; i < r; ++i) {
            int best = i;
            for (int j = i + 1; j < r; ++j)
                if (sv[order[j]] > sv[order[best]]) best = j;
            const int tmp = order[i];
            order[i] = order[best];
            order[best] = tmp;
        }
        const double tol = drop_tol_dev ? *drop_tol_dev : drop_tol;
        int keep = 0;
        for (int i = 0; i < r; ++i) keep += sv[order[i]] >= tol ? 1 : 0;
        *r_keep = keep;
        *info = converged ? 0 : 1;
    }
    __syncthreads();
    for (int e = t; e < r * r; e += 1024) {
        const int i = e / r, k = e % r;          // row i, output column k
        const int c = order[k];
        const double s = sv[c];
        U[e] = s > 0.0 ? A[c * 64 + i] / s : 0.0;
        Qm[e] = V[c * 64 + i];
        if (i == 0) sigma[k] = s;
    }
}

// The same SVD for r <= 16 in one warp: eight lane groups of four, group g
// rotating pair g of each round (its lanes split the r entries, sums by two
// xor shuffles, every lane of the group computing the same rotation), and
// __syncwarp between rounds instead of a CTA barrier.  The steps are those of
// k_svd_jacobi_f64: FP32 sweeps, FP64 re-orthonormalisation of the rotations,
// FP64 sweeps from A = S V, then the sorted column norms.
constexpr int kSvdSmallR = 16;

// Jacobi rotation (c, s) that zeroes <a_p, a_q> = ga given |a_p|^2 = al and
// |a_q|^2 = be: tan = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta =
// (be - al) / (2 ga), written as tan = +-|h| / (|d| + sqrt(d^2 + h^2)) with
// d = be - al, h = 2 ga.
__device__ __forceinline__ void jac_rotation(float al, float be, float ga, float& c, float& s) {
    const float zeta = (be - al) / (2.f * ga);
    const float tt = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
    c = rsqrtf(fmaf(tt, tt, 1.f));
    s = c * tt;
}
// FP64: FP64 divisions and square roots are slow on this GPU, so the angle
// comes from FP32 arithmetic on d and h scaled by a power of two (exact), and
// (c, s) is then normalised in FP64 by two terms of the series of
// (c^2 + s^2)^(-1/2) around 1 (error ~ (c^2 + s^2 - 1)^3).  An angle good to
// FP32 accuracy leaves ~1e-7 of the pair's inner product, which the next
// sweep removes; every rotation is orthogonal to FP64 rounding.
__device__ __forceinline__ void jac_rotation(double al, double be, double ga, double& c, double& s) {
    const double d = be - al, h = 2.0 * ga;
    int ex;
    (void)frexp(fmax(fabs(d), fabs(h)), &ex);
    const double sc = ldexp(1.0, -ex);
    const float df = (float)(d * sc), hf = (float)(h * sc);
    const float sg = (d == 0.0 || (d > 0.0) == (h > 0.0)) ? 1.f : -1.f;
    const float tf = sg * fabsf(hf) / (fabsf(df) + sqrtf(fmaf(df, df, hf * hf)));
    const float cf = rsqrtf(fmaf(tf, tf, 1.f));
    double cd = (double)cf, sd = (double)(cf * tf);
    const double e = fma(cd, cd, fma(sd, sd, -1.0));
    const double corr = fma(e, fma(e, 0.375, -0.5), 1.0);
    c = cd * corr;
    s = sd * corr;
}

// Lane groups of LG lanes (8 for r <= 8, 4 for r <= 16), group g rotating
// pair g of a round.  FP64: a sweep in which no pair had |<a_p, a_q>| above
// 1e-8 |a_p| |a_q| and every rotation was small (|sin| <= 1e-7) ends the
// iteration: each rotation leaves its own pair near 1e-15 of the norms (the
// FP32 angle is good to ~1e-7) and moves the other pairs' inner products by
// at most |sin| times theirs, which saves the checking sweep.  (Columns of
// nearly equal norm rotate by ~45 degrees however small their inner product,
// so such sweeps run to the check.)
template <typename T, int LG>
__device__ bool small_sweeps(T* A, T* V, int r, T tol, int max_sweeps) {
    const int lane = threadIdx.x & 31, g = lane / LG, u = lane % LG;
    const int m = (r + 1) & ~1;
    const T tol2 = tol * tol;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        int rotated = 0, big = 0;
        for (int round = 0; round < m - 1; ++round) {
            int p = 0, q = r;                                // groups past m / 2 stay idle (q >= r)
            if (g < m / 2) {
                auto slot = [&](int pos) {
                    int x = pos - 1 + round;
                    if (x >= m - 1) x -= m - 1;
                    return pos == 0 ? 0 : 1 + x;
                };
                p = slot(g);
                q = slot(m - 1 - g);
                if (p > q) {
                    const int tmp = p;
                    p = q;
                    q = tmp;
                }
            }
            T al = T(0), be = T(0), ga = T(0);
            if (q < r) {
                for (int i = u; i < r; i += LG) {
                    const T x = A[p * kSvdSmallR + i], y = A[q * kSvdSmallR + i];
                    al = fma(x, x, al);
                    be = fma(y, y, be);
                    ga = fma(x, y, ga);
                }
            }
#pragma unroll
            for (int o = 1; o < LG; o <<= 1) {               // every lane takes part
                al += __shfl_xor_sync(0xffffffffu, al, o);
                be += __shfl_xor_sync(0xffffffffu, be, o);
                ga += __shfl_xor_sync(0xffffffffu, ga, o);
            }
            const T g2 = ga * ga, ab = al * be;
            if (q < r && ga != T(0) && g2 > tol2 * ab) {
                T c, sn;
                jac_rotation(al, be, ga, c, sn);
                if (sizeof(T) == 8 && (g2 > T(1e-16) * ab || fabs(sn) > T(1e-7))) big = 1;
                for (int i = u; i < r; i += LG) {
                    const T x = A[p * kSvdSmallR + i], y = A[q * kSvdSmallR + i];
                    A[p * kSvdSmallR + i] = c * x - sn * y;
                    A[q * kSvdSmallR + i] = sn * x + c * y;
                    const T vx = V[p * kSvdSmallR + i], vy = V[q * kSvdSmallR + i];
                    V[p * kSvdSmallR + i] = c * vx - sn * vy;
                    V[q * kSvdSmallR + i] = sn * vx + c * vy;
                }
                rotated = 1;
            }
            __syncwarp();
        }
        if (!__any_sync(0xffffffffu, rotated)) return true;
        if (sizeof(T) == 8 && !__any_sync(0xffffffffu, big)) return true;
    }
    return false;
}

__global__ void __launch_bounds__(32) k_svd_small_f64(const double* __restrict__ S, int r, double drop_tol,
                                                     double* __restrict__ U, double* __restrict__ sigma,
                                                     double* __restrict__ Qm, int* __restrict__ r_keep,
                                                     int* __restrict__ info,
                                                     const double* __restrict__ drop_tol_dev = nullptr) {
    constexpr int R = kSvdSmallR;
    __shared__ double A[R * R], V[R * R], E[R * R], Sm[R * R];   // column-major: column c at c*R
    __shared__ float Af[R * R], Vf[R * R];
    __shared__ double sv[R];
    __shared__ int order[R];
    const int t = threadIdx.x;
    for (int e = t; e < R * R; e += 32) {
        const int c = e / R, i = e % R;
        const double x = (c < r && i < r) ? S[i * r + c] : 0.0;
        Sm[e] = x;                                   // Sm[c * R + i] = S[i][c]
        Af[e] = (float)x;
        Vf[e] = (c == i && c < r) ? 1.f : 0.f;
    }
    __syncwarp();
    if (r <= 8) (void)small_sweeps<float, 8>(Af, Vf, r, 1e-6f, kSvdMaxSweeps);
    else (void)small_sweeps<float, 4>(Af, Vf, r, 1e-6f, kSvdMaxSweeps);
    for (int e = t; e < R * R; e += 32) V[e] = (double)Vf[e];
    __syncwarp();
    for (int it = 0; it < 2; ++it) {                 // V <- V (I - E/2), E = V^T V - I
        for (int e = t; e < r * r; e += 32) {
            const int a = e / r, b = e % r;
            double g = 0.0;
            for (int i = 0; i < r; ++i) g = fma(V[a * R + i], V[b * R + i], g);
            E[a * R + b] = g - (a == b ? 1.0 : 0.0);
        }
        __syncwarp();
        for (int e = t; e < r * r; e += 32) {
            const int c = e / r, i = e % r;
            double v = V[c * R + i];
            for (int k = 0; k < r; ++k) v = fma(-0.5 * V[k * R + i], E[k * R + c], v);
            A[c * R + i] = v;
        }
        __syncwarp();
        for (int e = t; e < r * r; e += 32) {
            const int c = e / r, i = e % r;
            V[c * R + i] = A[c * R + i];
        }
        __syncwarp();
    }
    for (int e = t; e < r * r; e += 32) {            // A = S V (only the leading r x r block is used)
        const int c = e / r, i = e % r;
        double a = 0.0;
        for (int k = 0; k < r; ++k) a = fma(Sm[k * R + i], V[c * R + k], a);
        A[c * R + i] = a;
    }
    __syncwarp();
    const bool converged = r <= 8 ? small_sweeps<double, 8>(A, V, r, 1e-15, kSvdMaxSweeps)
                                  : small_sweeps<double, 4>(A, V, r, 1e-15, kSvdMaxSweeps);
    __shared__ double inv_sv[R];
    if (t < r) {
        double nn = 0.0;
        for (int i = 0; i < r; ++i) nn = fma(A[t * R + i], A[t * R + i], nn);
        sv[t] = sqrt(nn);
        inv_sv[t] = sv[t] > 0.0 ? 1.0 / sv[t] : 0.0;
    }
    __syncwarp();
    if (t == 0) {
        for (int i = 0; i < r; ++i) order[i] = i;
        for (int i = 0; i < r; ++i) {
            int best = i;
            for (int j = i + 1; j < r; ++j)
                if (sv[order[j]] > sv[order[best]]) best = j;
            const int tmp = order[i];
            order[i] = order[best];
            order[best] = tmp;
        }
        const double tol = drop_tol_dev ? *drop_tol_dev : drop_tol;
        int keep = 0;
        for (int i = 0; i < r; ++i) keep += sv[order[i]] >= tol ? 1 : 0;
        *r_keep = keep;
        *info = converged ? 0 : 1;
    }
    __syncwarp();
    for (int e = t; e < r * r; e += 32) {
        const int i = e / r, k = e % r;
        const int c = order[k];
        U[e] = A[c * R + i] * inv_sv[c];
        Qm[e] = V[c * R + i];
        if (i == 0) sigma[k] = sv[c];
    }
}

// X_bar_k(x) = sum_i X_i(x) U_ik, k < r_new (U row-major r x r, ld r).
// r_new_dev, when not null, replaces r_new; skip, when not null and set,
// makes the kernel write nothing (both read from device memory, as in a
// replayed graph whose earlier kernels decide them).
template <int RMAX>
__global__ void __launch_bounds__(kLrThreads) k_rotate_f64(const double* __restrict__ X, const double* __restrict__ U,
                                                          int r, int r_new, int n, double* __restrict__ out,
                                                          const int* __restrict__ r_new_dev = nullptr,
                                                          const int* __restrict__ skip = nullptr) {
    if (skip && *skip) return;
    if (r_new_dev) r_new = min(max(*r_new_dev, 0), r);
    __shared__ double Us[64 * 64];
    for (int e = threadIdx.x; e < r * r; e += kLrThreads) Us[e] = U[e];
    __syncthreads();
    const int x = blockIdx.x * kLrThreads + threadIdx.x;
    if (x >= n) return;
    double xv[RMAX];
#pragma unroll
    for (int i = 0; i < RMAX; ++i) xv[i] = (i < r) ? __ldg(&X[(size_t)i * n + x]) : 0.0;
    for (int k = 0; k < r_new; ++k) {
        double y = 0.0;
#pragma unroll
        for (int i = 0; i < RMAX; ++i)
            if (i < r) y = fma(xv[i], Us[i * r + k], y);
        out[(size_t)k * n + x] = y;
    }
}

}  // namespace boltz_dev
