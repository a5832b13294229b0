// Kernels of the 1D normal-shock solver (paper Sec. 2.3: first-order upwind
// transport and the projected inflow boundary; Sec. 2.4: the fully discrete
// K-S-L scheme; Sec. 3: adding and dropping basis).  The factor algebra is
// FP64; the collision terms come from the FP32 collision batch.
//
// Storage: functions of x or v are rows, X [r][n_x], K [r][n_x], V [r][n_v],
// L [r][n_v]; small matrices are row-major.  Inner products are the midpoint
// rules <a, b>_x = dx sum_x a b and <a, b>_v = w sum_v a b (w = dv^d).
// Upwind differences with boundary values g_L, g_R (one per row):
//   D+ K(x_p) = (K(x_p) - K(x_{p-1})) / dx,  D- K(x_p) = (K(x_{p+1}) - K(x_p)) / dx,
//   K(x_0) = g_L, K(x_{N+1}) = g_R.
// Every reduction runs in a fixed order (run-to-run identical results).
#pragma once

#include <cuda_runtime.h>

namespace boltz_dev {

constexpr int kShT = 256;

// Sum of one double per thread over a block of kShT threads, fixed order;
// the result is valid in thread 0.
__device__ __forceinline__ double sh_block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < kShT / 32; ++k) s += red[k];
    return s;
}

__global__ void k_sh_to_f32(const double* __restrict__ in, float* __restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

// Full-tensor forward-Euler upwind step (Sec. 2.3, eq. "scheme:fullupwind"):
//   g = f - dt/dx (v1+ (f - f_left) + v1- (f_right - f)) + dt Q,
// ghost cells f_L (left) and f_R (right).
__global__ void k_sh_full(const double* __restrict__ f, const float* __restrict__ Q, const double* __restrict__ fL,
                          const double* __restrict__ fR, const double* __restrict__ v1, int n_x, int n_v, double dt,
                          double dx, double* __restrict__ g) {
    const size_t total = (size_t)n_x * n_v;
    const double cfl = dt / dx;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(t / n_v), v = (int)(t % n_v);
        const double c = f[t];
        const double l = p > 0 ? f[t - n_v] : fL[v];
        const double r = p < n_x - 1 ? f[t + n_v] : fR[v];
        const double a = v1[v], ap = fmax(a, 0.0), am = fmin(a, 0.0);
        g[t] = c - cfl * (ap * (c - l) + am * (r - c)) + dt * (double)Q[t];
    }
}

// out_j = sum_i coef(i, j) in_i for j < r_out, coef(i, j) = A[i][j] (A_ROWS false:
// out = A^T in) or A[j][i] (A_ROWS true: out = A in); A has leading dimension lda.
template <bool A_ROWS>
__global__ void k_sh_comb(const double* __restrict__ in, int r_in, int n, const double* __restrict__ A, int lda,
                          int r_out, double* __restrict__ out) {
    const size_t total = (size_t)r_out * n;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / n), x = (int)(t % n);
        double acc = 0.0;
        for (int i = 0; i < r_in; ++i) acc = fma(A_ROWS ? A[(size_t)j * lda + i] : A[(size_t)i * lda + j], in[(size_t)i * n + x], acc);
        out[t] = acc;
    }
}

// Velocity Gram matrices and boundary projections, block (j, l):
//   l < r:  Ap[j][l] = w sum v1+ V_j V_l,  Am[j][l] = w sum v1- V_j V_l,
//           Pl[j][l] = w sum 1{v1 <= 0} V_j V_l,  Pr[j][l] = w sum 1{v1 >= 0} V_j V_l
//   l == r: bl[j] = w sum f_L 1{v1 > 0} V_j,  br[j] = w sum f_R 1{v1 < 0} V_j
__global__ void __launch_bounds__(kShT) k_sh_vgram(const double* __restrict__ V, int r, int n_v,
                                                  const double* __restrict__ v1, const double* __restrict__ fL,
                                                  const double* __restrict__ fR, double w, double* Ap, double* Am,
                                                  double* Pl, double* Pr, double* bl, double* br) {
    __shared__ double red[kShT / 32];
    const int j = blockIdx.x, l = blockIdx.y;
    const double* Vj = V + (size_t)j * n_v;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    if (l < r) {
        const double* Vl = V + (size_t)l * n_v;
        for (int v = threadIdx.x; v < n_v; v += kShT) {
            const double a = v1[v], p = Vj[v] * Vl[v];
            s0 = fma(fmax(a, 0.0), p, s0);
            s1 = fma(fmin(a, 0.0), p, s1);
            s2 += a <= 0.0 ? p : 0.0;
            s3 += a >= 0.0 ? p : 0.0;
        }
    } else {
        for (int v = threadIdx.x; v < n_v; v += kShT) {
            const double a = v1[v];
            s0 = fma(a > 0.0 ? fL[v] : 0.0, Vj[v], s0);
            s1 = fma(a < 0.0 ? fR[v] : 0.0, Vj[v], s1);
        }
    }
    s0 = sh_block_sum(s0, red);
    s1 = sh_block_sum(s1, red);
    if (l < r) {
        s2 = sh_block_sum(s2, red);
        s3 = sh_block_sum(s3, red);
        if (threadIdx.x == 0) {
            Ap[j * r + l] = w * s0;
            Am[j * r + l] = w * s1;
            Pl[j * r + l] = w * s2;
            Pr[j * r + l] = w * s3;
        }
    } else if (threadIdx.x == 0) {
        bl[j] = w * s0;
        br[j] = w * s1;
    }
}

// Boundary values of K (Sec. 2.3, eq. "boundary general"; outflow part from
// the first interior cell): g_L[j] = bl[j] + sum_l K_l(x_1) Pl[l][j],
// g_R[j] = br[j] + sum_l K_l(x_N) Pr[l][j].  Computed by the kernels that use
// them, thread j of the block (r <= 64), into shared memory.
__device__ __forceinline__ void sh_ghost_values(const double* __restrict__ K, int r, int n_x,
                                                const double* __restrict__ Pl, const double* __restrict__ Pr,
                                                const double* __restrict__ bl, const double* __restrict__ br,
                                                double* gL, double* gR) {
    for (int j = threadIdx.x; j < r; j += blockDim.x) {
        double a = bl[j], b = br[j];
        for (int l = 0; l < r; ++l) {
            a = fma(K[(size_t)l * n_x], Pl[l * r + j], a);
            b = fma(K[(size_t)l * n_x + n_x - 1], Pr[l * r + j], b);
        }
        gL[j] = a;
        gR[j] = b;
    }
    __syncthreads();
}

// dx D+ K_l(x) and dx D- K_l(x): the differences only (FP64 division is slow;
// callers apply 1/dx once, or not at all where a factor dx cancels it)
__device__ __forceinline__ double sh_diff_plus(const double* K, int n_x, const double* gL, int l, int x) {
    const double* Kl = K + (size_t)l * n_x;
    return Kl[x] - (x > 0 ? Kl[x - 1] : gL[l]);
}
__device__ __forceinline__ double sh_diff_minus(const double* K, int n_x, const double* gR, int l, int x) {
    const double* Kl = K + (size_t)l * n_x;
    return (x < n_x - 1 ? Kl[x + 1] : gR[l]) - Kl[x];
}

// K-step Euler update (Sec. 2.4, K-step (b), upwind form of Sec. 2.3):
//   K1_j(x) = K_j(x) - dt sum_l (Ap[j][l] D+ K_l(x) + Am[j][l] D- K_l(x)) + dt C_j(x)
__global__ void k_sh_kupdate(const double* __restrict__ K, const float* __restrict__ C, const double* __restrict__ Ap,
                             const double* __restrict__ Am, const double* __restrict__ Pl,
                             const double* __restrict__ Pr, const double* __restrict__ bl,
                             const double* __restrict__ br, int r, int n_x, double dt, double dx,
                             double* __restrict__ K1) {
    __shared__ double gL[64], gR[64];
    sh_ghost_values(K, r, n_x, Pl, Pr, bl, br, gL, gR);
    const size_t total = (size_t)r * n_x;
    const double cfl = dt / dx;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / n_x), x = (int)(t % n_x);
        double tr = 0.0;
        for (int l = 0; l < r; ++l)
            tr = fma(Ap[j * r + l], sh_diff_plus(K, n_x, gL, l, x),
                     fma(Am[j * r + l], sh_diff_minus(K, n_x, gR, l, x), tr));
        K1[t] = K[t] - cfl * tr + dt * (double)C[t];
    }
}

// Space Gram matrices of the transport, block (i, l):
//   Bp[i][l] = dx sum_x X_i(x) D+ K_l(x),  Bm[i][l] = dx sum_x X_i(x) D- K_l(x)
// (the factor dx cancels the 1/dx of the differences)
__global__ void __launch_bounds__(kShT) k_sh_xgram(const double* __restrict__ X, const double* __restrict__ K,
                                                  const double* __restrict__ Pl, const double* __restrict__ Pr,
                                                  const double* __restrict__ bl, const double* __restrict__ br,
                                                  int r, int n_x, double* Bp, double* Bm) {
    __shared__ double red[kShT / 32];
    __shared__ double gL[64], gR[64];
    sh_ghost_values(K, r, n_x, Pl, Pr, bl, br, gL, gR);
    const int i = blockIdx.x, l = blockIdx.y;
    const double* Xi = X + (size_t)i * n_x;
    double sp = 0.0, sm = 0.0;
    for (int x = threadIdx.x; x < n_x; x += kShT) {
        sp = fma(Xi[x], sh_diff_plus(K, n_x, gL, l, x), sp);
        sm = fma(Xi[x], sh_diff_minus(K, n_x, gR, l, x), sm);
    }
    sp = sh_block_sum(sp, red);
    sm = sh_block_sum(sm, red);
    if (threadIdx.x == 0) {
        Bp[i * r + l] = sp;
        Bm[i * r + l] = sm;
    }
}

__global__ void k_sh_transpose(const double* __restrict__ in, int rows, int cols, double* __restrict__ out) {
    const size_t total = (size_t)rows * cols;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(t / cols), b = (int)(t % cols);
        out[(size_t)b * rows + a] = in[t];
    }
}

// Triple products E[i][m][n] = dx sum_x X_i X_m X_n (FP32 result for the r^4
// coupling kernel).  Block (i, m); warp w takes n = w, w + 8, ..., its lanes
// stride over the cells (coalesced rows) and reduce by shuffles.
__global__ void __launch_bounds__(kShT) k_sh_triple(const double* __restrict__ X, int r, int n_x, double dx,
                                                   float* __restrict__ E) {
    const int i = blockIdx.x, m = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double* Xi = X + (size_t)i * n_x;
    const double* Xm = X + (size_t)m * n_x;
    for (int n = warp; n < r; n += kShT / 32) {
        const double* Xn = X + (size_t)n * n_x;
        double acc = 0.0;
        for (int x = lane; x < n_x; x += 32) acc = fma(Xi[x] * Xm[x], Xn[x], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) E[((size_t)i * r + m) * r + n] = (float)(dx * acc);
    }
}

// S-step Euler update (Sec. 2.4, S-step (a)):
//   S2[i][j] = S1[i][j] + dt sum_l (Ap[j][l] Bp[i][l] + Am[j][l] Bm[i][l]) - dt D[i][j]
__global__ void k_sh_supdate(const double* __restrict__ S1, const double* __restrict__ Ap, const double* __restrict__ Am,
                             const double* __restrict__ Bp, const double* __restrict__ Bm, const float* __restrict__ D,
                             int r, double dt, double* __restrict__ S2) {
    for (int t = threadIdx.x; t < r * r; t += blockDim.x) {
        const int i = t / r, j = t % r;
        double tr = 0.0;
        for (int l = 0; l < r; ++l) tr = fma(Ap[j * r + l], Bp[i * r + l], fma(Am[j * r + l], Bm[i * r + l], tr));
        S2[t] = S1[t] + dt * tr - dt * (double)D[t];
    }
}

// L-step Euler update (Sec. 2.4, L-step (b), upwind form of Sec. 2.3):
//   L1_i(v) = L_i(v) - dt (v1+ sum_l Bp[i][l] V_l(v) + v1- sum_l Bm[i][l] V_l(v)) + dt G_i(v)
__global__ void k_sh_lupdate(const double* __restrict__ L, const double* __restrict__ V, const double* __restrict__ v1,
                             const double* __restrict__ Bp, const double* __restrict__ Bm, const float* __restrict__ G,
                             int r, int n_v, double dt, double* __restrict__ L1) {
    const size_t total = (size_t)r * n_v;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / n_v), v = (int)(t % n_v);
        double sp = 0.0, sm = 0.0;
        for (int l = 0; l < r; ++l) {
            const double Vl = V[(size_t)l * n_v + v];
            sp = fma(Bp[i * r + l], Vl, sp);
            sm = fma(Bm[i * r + l], Vl, sm);
        }
        const double a = v1[v];
        L1[t] = L[t] - dt * (fmax(a, 0.0) * sp + fmin(a, 0.0) * sm) + dt * (double)G[t];
    }
}

// Gram-Schmidt pieces of the basis augmentation (Sec. 3.1):
//   c[j] = w sum_v V_j(v) b(v)        (block j)
__global__ void __launch_bounds__(kShT) k_sh_rowdots(const double* __restrict__ V, int n, const double* __restrict__ b,
                                                    double w, double* __restrict__ c) {
    __shared__ double red[kShT / 32];
    const double* Vj = V + (size_t)blockIdx.x * n;
    double s = 0.0;
    for (int v = threadIdx.x; v < n; v += kShT) s = fma(Vj[v], b[v], s);
    s = sh_block_sum(s, red);
    if (threadIdx.x == 0) c[blockIdx.x] = w * s;
}

//   b(v) -= sum_{j < r} c[j] V_j(v)
__global__ void k_sh_subtract(double* __restrict__ b, const double* __restrict__ V, const double* __restrict__ c, int r,
                              int n) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        double s = b[v];
        for (int j = 0; j < r; ++j) s = fma(-c[j], V[(size_t)j * n + v], s);
        b[v] = s;
    }
}

//   b /= sqrt(w sum b^2) (one block; a zero vector stays zero)
__global__ void __launch_bounds__(kShT) k_sh_normalize(double* __restrict__ b, int n, double w) {
    __shared__ double red[kShT / 32];
    __shared__ double scale;
    double s = 0.0;
    for (int v = threadIdx.x; v < n; v += kShT) s = fma(b[v], b[v], s);
    s = sh_block_sum(s, red);
    if (threadIdx.x == 0) scale = s > 0.0 ? 1.0 / sqrt(w * s) : 0.0;
    __syncthreads();
    for (int v = threadIdx.x; v < n; v += kShT) b[v] *= scale;
}

// The basis augmentation (Sec. 3.1) spread over up to kAugCtas CTAs (FP64
// issues slowly on this GPU, so the inner products use many SMs).  Boundary
// vector k goes to column rh = rh0 + k of Vh: b = src, two Gram-Schmidt passes
// against the columns before it (c_j = w <V_j, b>, b -= sum_j c_j V_j), kept
// when |b|^2 after > 1e-20 |b|^2 before, then scaled to unit w-norm.  Each
// launch ends with the CTA that finishes last (a ticket counter, left at zero;
// nothing waits) summing the per-CTA partial sums in CTA order:
//   k_aug_start   b = src (after scaling column rh - 1, the previous vector);
//                 partials of |src|^2 and <V_j, b>; last: c, nrm[2k]
//   k_aug_update  b -= sum c_j V_j; PASS 0: partials of <V_j, b>, last: c;
//                 PASS 1: partial |b|^2, last: nrm[2k + 1], the keep decision,
//                 the scale, skip bit 1 if not kept (when skip is not null)
//   k_aug_scale   b *= scale (the last vector)
// Thread t of CTA c owns the entries v = c kAugT + t + e kAugT G (G CTAs), the
// same in every launch, so b needs no other synchronisation.
constexpr int kAugT = 128, kAugCtas = 128, kAugR = 32, kAugSlots = kAugR + 1;

struct AugState {                  // device scratch of the augmentation
    double part[kAugCtas][kAugSlots];
    double coef[kAugR];            // w <V_j, b> of the last pass
    double scale;                  // scale of the vector finished last (1 if not kept)
    unsigned ticket;
};

// block sums of acc[0..nj) (and of x when with_x) into part[blockIdx.x][.]
template <int RM>
__device__ __forceinline__ void aug_partials(const double (&acc)[RM], int nj, double x, bool with_x, AugState* S) {
    __shared__ double red[kAugT / 32][kAugSlots];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < RM; ++j) {
        double y = acc[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(0xffffffffu, y, o);
        if (lane == 0 && j < nj) red[warp][j] = y;
    }
    if (with_x) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp][kAugR] = x;
    }
    __syncthreads();
    const int t = threadIdx.x;
    const int slot = t < nj ? t : (t == kAugT - 1 && with_x ? kAugR : -1);
    if (slot >= 0) {
        double y = 0.0;
#pragma unroll
        for (int w = 0; w < kAugT / 32; ++w) y += red[w][slot];
        S->part[blockIdx.x][slot] = y;
    }
}

// true in the CTA that finished last (every CTA has written its partials)
__device__ __forceinline__ bool aug_last(AugState* S) {
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&S->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// sum over the CTAs of slot j, by warp j % 4 with lanes over CTAs (fixed order)
__device__ __forceinline__ double aug_total(AugState* S, int j) {
    const int lane = threadIdx.x & 31;
    double y = 0.0;
    for (int c = lane; c < (int)gridDim.x; c += 32) y += __ldcg(&S->part[c][j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(0xffffffffu, y, o);
    return __shfl_sync(0xffffffffu, y, 0);
}

template <int RM>
__global__ void __launch_bounds__(kAugT) k_aug_start(double* Vh, int rh, int n, double w,
                                                      const double* __restrict__ src, int scale_prev,
                                                      double* __restrict__ nrm, int k, AugState* S) {
    const int G = gridDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double sp = scale_prev ? __ldcg(&S->scale) : 1.0;
    double* b = Vh + (size_t)rh * n;
    double acc[RM];
#pragma unroll
    for (int j = 0; j < RM; ++j) acc[j] = 0.0;
    double x2 = 0.0;
    for (int v = blockIdx.x * kAugT + threadIdx.x; v < n; v += G * kAugT) {
        if (scale_prev) Vh[(size_t)(rh - 1) * n + v] *= sp;
        const double bv = src[v];
        b[v] = bv;
        x2 = fma(bv, bv, x2);
#pragma unroll
        for (int j = 0; j < RM; ++j)
            if (j < rh) acc[j] = fma(Vh[(size_t)j * n + v], bv, acc[j]);
    }
    aug_partials<RM>(acc, rh, x2, true, S);
    if (!aug_last(S)) return;
    for (int j = warp; j <= kAugR; j += kAugT / 32) {
        if (j < rh || j == kAugR) {
            const double y = aug_total(S, j);
            if (lane == 0) {
                if (j < rh) S->coef[j] = w * y;
                else nrm[2 * k] = y;
            }
        }
    }
    if (threadIdx.x == 0) S->ticket = 0u;
}

template <int RM, int PASS>
__global__ void __launch_bounds__(kAugT) k_aug_update(double* Vh, int rh, int n, double w, double* __restrict__ nrm,
                                                       int k, int* __restrict__ skip, AugState* S) {
    __shared__ double c[kAugR];
    const int G = gridDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < rh) c[threadIdx.x] = __ldcg(&S->coef[threadIdx.x]);
    __syncthreads();
    double* b = Vh + (size_t)rh * n;
    double acc[RM];
#pragma unroll
    for (int j = 0; j < RM; ++j) acc[j] = 0.0;
    double x2 = 0.0;
    for (int v = blockIdx.x * kAugT + threadIdx.x; v < n; v += G * kAugT) {
        double Vv[RM];
#pragma unroll
        for (int j = 0; j < RM; ++j) Vv[j] = j < rh ? Vh[(size_t)j * n + v] : 0.0;
        double bv = b[v];
#pragma unroll
        for (int j = 0; j < RM; ++j)
            if (j < rh) bv = fma(-c[j], Vv[j], bv);
        b[v] = bv;
        if (PASS == 0) {
#pragma unroll
            for (int j = 0; j < RM; ++j)
                if (j < rh) acc[j] = fma(Vv[j], bv, acc[j]);
        } else {
            x2 = fma(bv, bv, x2);
        }
    }
    aug_partials<RM>(acc, PASS == 0 ? rh : 0, x2, PASS == 1, S);
    if (!aug_last(S)) return;
    if (PASS == 0) {
        for (int j = warp; j < rh; j += kAugT / 32) {
            const double y = aug_total(S, j);
            if (lane == 0) S->coef[j] = w * y;
        }
    } else if (warp == 0) {
        const double n1 = aug_total(S, kAugR);
        if (lane == 0) {
            const double n0 = nrm[2 * k];
            const bool kept = n1 > 1e-20 * n0;
            nrm[2 * k + 1] = n1;
            S->scale = kept && n1 > 0.0 ? 1.0 / sqrt(w * n1) : 1.0;
            if (skip && !kept) *skip |= 1;
        }
    }
    if (threadIdx.x == 0) S->ticket = 0u;
}

__global__ void __launch_bounds__(kAugT) k_aug_scale(double* Vh, int rh, int n, const AugState* S) {
    const double sc = __ldcg(&S->scale);
    for (int v = blockIdx.x * kAugT + threadIdx.x; v < n; v += gridDim.x * kAugT) Vh[(size_t)rh * n + v] *= sc;
}

// Change of f over a low-rank step (Sec. 5.1, eqs. "err low rank1" and "err low rank2"):
//   err^2 = sum_j |dK_j|^2 + sum_ij dS_ij^2 + sum_i |dL_i|^2
//           + 2 sum_ij P_ij dS_ij + 2 sum_ij dS_ij Qd_ij + 2 sum_ij P_ij Qd_ij,
// P_ij = <dK_j, X'_i>_x (Pk[i][j]), Qd_ij = <dL_i, V_j>_v (stored as Gv[j][i]),
// dS = S2 - S1, err >= 0.  One launch of 2 r + 2 r^2 blocks, one inner product
// each: block b < r: nk[b] = dx |K1_b - K0_b|^2; b < 2 r: nl = wv |L1 - L0|^2;
// then Pk[i][j] = dx <X1_i, K1_j - K0_j>, then Gv[i][j] = wv <Vh_i, L1_j - L0_j>.
// The block that finishes last (a ticket counter, reset to zero afterwards;
// nothing waits) forms err from them.
__global__ void __launch_bounds__(kShT) k_sh_change(const double* __restrict__ K1, const double* __restrict__ K0,
                                                   const double* __restrict__ X1, const double* __restrict__ L1,
                                                   const double* __restrict__ L0, const double* __restrict__ Vh,
                                                   int r, int n_x, int n_v, double dx, double wv,
                                                   const double* __restrict__ S1, const double* __restrict__ S2,
                                                   double* nk, double* nl, double* Pk, double* Gv,
                                                   unsigned* __restrict__ ticket, double* __restrict__ err) {
    __shared__ double red[kShT / 32];
    __shared__ int last;
    int b = blockIdx.x;
    const double *A = nullptr, *B1, *B0;
    double w;
    int n;
    double* out;
    if (b < r) {
        B1 = K1 + (size_t)b * n_x, B0 = K0 + (size_t)b * n_x, n = n_x, w = dx, out = nk + b;
    } else if ((b -= r) < r) {
        B1 = L1 + (size_t)b * n_v, B0 = L0 + (size_t)b * n_v, n = n_v, w = wv, out = nl + b;
    } else if ((b -= r) < r * r) {
        const int i = b / r, j = b % r;
        A = X1 + (size_t)i * n_x, B1 = K1 + (size_t)j * n_x, B0 = K0 + (size_t)j * n_x, n = n_x, w = dx, out = Pk + b;
    } else {
        b -= r * r;
        const int i = b / r, j = b % r;
        A = Vh + (size_t)i * n_v, B1 = L1 + (size_t)j * n_v, B0 = L0 + (size_t)j * n_v, n = n_v, w = wv, out = Gv + b;
    }
    double acc = 0.0;
    for (int k = threadIdx.x; k < n; k += kShT) {
        const double d = B1[k] - B0[k];
        acc = fma(A ? A[k] : d, d, acc);
    }
    acc = sh_block_sum(acc, red);
    if (threadIdx.x == 0) *out = w * acc;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    double e = 0.0;
    for (int t = threadIdx.x; t < r * r; t += kShT) {
        const int i = t / r, j = t % r;
        const double ds = S2[t] - S1[t], q = __ldcg(&Gv[j * r + i]), pk = __ldcg(&Pk[t]);
        e += ds * ds + 2.0 * pk * ds + 2.0 * ds * q + 2.0 * pk * q;
        if (i == j) e += __ldcg(&nk[i]) + __ldcg(&nl[i]);
    }
    e = sh_block_sum(e, red);
    if (threadIdx.x == 0) {
        *err = sqrt(fmax(e, 0.0));
        *ticket = 0u;
    }
}

// S = diag(sigma[:r]) (packed [r][r]); r_dev and skip as in k_rotate_f64
__global__ void k_sh_diag(const double* __restrict__ sigma, int r, double* __restrict__ S,
                          const int* __restrict__ r_dev = nullptr, const int* __restrict__ skip = nullptr) {
    if (skip && *skip) return;
    if (r_dev) r = *r_dev;
    for (int t = threadIdx.x; t < r * r; t += blockDim.x) S[t] = (t / r == t % r) ? sigma[t / r] : 0.0;
}

// Keep/drop decision of an appended boundary vector made on the device: it
// is kept when its squared norm after Gram-Schmidt, nrm[1], is more than
// 1e-20 of its squared norm before, nrm[0].  A replayed graph assumes that
// both boundary vectors are kept; skip[0] records that one was not, and the
// kernels that write the step's outputs then do nothing (the host reruns the
// step without the graph).
__global__ void k_sh_keep_check(const double* __restrict__ nrm, int* __restrict__ skip) {
    if (threadIdx.x == 0 && !(nrm[1] > 1e-20 * nrm[0])) *skip |= 1;
}

// After the drop: a QR that met linearly dependent rows (info[0], info[1]) or
// no singular value kept (info[2] < 1) sets skip bit 2, so that the outputs
// stay as they were, as the host-driven step leaves them on that error.
__global__ void k_sh_step_check(const int* __restrict__ info, int* __restrict__ skip) {
    if (threadIdx.x == 0 && (info[0] != 0 || info[1] != 0 || info[2] < 1)) *skip |= 2;
}

// f[x][v] = sum_i X_i(x) L_i(v)
__global__ void k_sh_outer(const double* __restrict__ X, const double* __restrict__ L, int r, int n_x, int n_v,
                           double* __restrict__ f) {
    const size_t total = (size_t)n_x * n_v;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(t / n_v), v = (int)(t % n_v);
        double acc = 0.0;
        for (int i = 0; i < r; ++i) acc = fma(X[(size_t)i * n_x + x], L[(size_t)i * n_v + v], acc);
        f[t] = acc;
    }
}

}  // namespace boltz_dev
