// Batched collision operator on 3D 32^3 grids as one persistent kernel with
// shared partial transforms ("pencil" schedule, sm_103a).
//
// What it computes is the separated fast-spectral gain of the batched form
// (Sec. 2.1: for every radial node q and direction p the shifted fields
// A_{q,p,j}(v) = g_j,N(v - rho_q sigma_p / 2), their products summed over
// the directions with the weights w_p, one forward transform per node times
// the radial multiplier c_q(|k|), accumulated over q) for chunks of at most
// 16 inputs and the used ones of their 136 unordered pairs each.  A batch of
// more inputs is split into chunks on the host; chunks of one shape (the same
// input count and used slots) run in one launch, as one list of radial nodes
// (node q of the launch is node q % n_rho of chunk q / n_rho).  How it
// computes it:
//
// * The phase of a shifted field separates over the axes,
//   phi(k) = phi_0(k_0; s_0) phi_1(k_1; s_1) phi_2(k_2; s_2), s = rho sigma / 2,
//   and the inverse transform runs axis 0, then axis 1, then the
//   complex-to-real transform along axis 2.  After the axis-0 pass a field
//   depends on the direction only through sigma_0, after the axis-1 pass only
//   through (sigma_0, sigma_1).  The 38-point rule has 9 distinct sigma_0 and
//   25 distinct (sigma_0, sigma_1) values, so computing each partial
//   transform once per distinct value does the axis-0 work 9 times and the
//   axis-1 work 25 times per (node, input) instead of 38 times each.
// * TREE items (node q, input j, block of 4 k_2 columns, group of sigma_0
//   values): the axis-0 pass of its columns for each sigma_0, then the axis-1
//   pass for every (sigma_0, sigma_1) below it, written as "X blocks" laid
//   out for the consumer: X[s01][line block][j][k_2][4 lines].  The axes 0
//   and 1 never mix k_2 columns, so a block of columns is an independent
//   problem.
// * FUSED items (node q, line block of 4 lines (i0, i1) = 128 voxels): for
//   every direction, the axis-2 complex-to-real transform of the X block of
//   its (sigma_0, sigma_1) with the phase phi_2(s_2) into shared memory, and
//   at once the sigma-contraction
//   P[j,l](v) += w_p (A_{p,j}(v) A_{p',l}(v) + A_{p',j}(v) A_{p,l}(v)) over
//   antipodal pairs (p, p').  Thread t owns voxel t; its 136 accumulators
//   live in tensor memory (TMEM lane t, 128 columns) and registers (the last
//   8).  The shifted fields never leave the SM.  At the end the item applies
//   the first pass of the forward transform (real-to-complex along axis 2)
//   to its 136 gain fields and writes half spectra of its lines ("Pt planes").
// * RADIAL items (node q, gain slot u): for each block of 4 k_2 columns, the
//   forward axis-1 and axis-0 passes of the slot's Pt plane columns and the
//   multiplier c_q(|k|) (-1)^k, accumulated into Qhat+[u] (node by node, in
//   order) in a packed layout copied in and out of shared memory in one piece;
//   the last node writes the finished sums in the standard half-spectrum
//   layout the output kernel reads.  The k_2 = 0 and k_2 = N/2 planes of a
//   real field are real in (i0, i1): they travel as one complex column
//   (re = k_2 0, im = k_2 N/2), and so do their running sums, separated with
//   the conjugate-symmetry identity at the end.
//
// Scheduling: a fixed list of items, stage by stage (stage s: tree items of
// node s, fused items of node s-2, radial items of node s-4), claimed in order
// from an atomic counter by persistent CTAs (three per SM: 128 threads, at
// most 168 registers, 67 KB of shared memory and 128 TMEM columns each).  A
// CTA claims its next item when it starts the current one (the claim's round
// trip is hidden behind the work; claiming further ahead delays claimed items
// behind long ones and stalls the items that depend on them).  Every dependency
// points to an item earlier in the list (fused(q) needs all tree(q) and the
// Pt buffer free; tree(q) needs its X buffer free; radial(q) needs fused(q)
// and radial(q-1) of its chunk's slot), so the lowest unfinished item can always run:
// progress needs no co-residency.  The two-stage lags give every dependency a
// stage of slack.  Each wait is a bounded poll (about one second of device
// time); a wait that gives up records a timeout in the error word and raises
// an abort flag, after which every CTA drains the list without working, so the
// launch always ends.  X has four node buffers (~56 MB each) and Pt four
// (~18 MB each); together they exceed the L2, so most of their lines make one
// round trip to DRAM, which carries under half of its bandwidth.
// (Dropping consumed lines from L2 with discard.global.L2 saves their
// write-back but was measured 6% slower overall.)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "async.cuh"
#include "fft.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace boltz_dev {
namespace pencil {

constexpr int N = 32;
constexpr int H = 16;
constexpr int NH = H + 1;
constexpr int HALF = N * N * NH;               // half-spectrum entries of a 32^3 field
constexpr int SMAX = 3 * H * H;                // largest |k|^2
constexpr int NT = 128;                        // threads per CTA
constexpr int NJ = 16;                         // inputs of a batch
constexpr int NSLOT = NJ * (NJ + 1) / 2;       // unordered gain slots: 136
constexpr int NTSLOT = 128;                    // slots accumulated in TMEM (columns 0..127)
constexpr int NRSLOT = NSLOT - NTSLOT;         // slots accumulated in registers: 8
constexpr int KB = 4;                          // k2 columns per tree / radial item
constexpr int NKB = H / KB;                    // column blocks: k2 = 0..15 (k2 = 16 rides in column 0)
constexpr int NLB = N * N / 4;                 // line blocks per field (4 lines, 128 voxels): 256
constexpr int XJS = H * 4 + 2;                 // float2 per input in an X block (+2: bank spread)
constexpr int XBLK = NJ * XJS;                 // float2 per X block: 1056 (8448 B = 66 L2 lines)
constexpr int PRS = N * KB + 4;                // plane row stride in float2 (+4: bank spread)
constexpr int PLANE = N * PRS;                 // float2 per plane: 4224 (33792 B = 264 L2 lines)
constexpr int AJS = 4 * N + 4;                 // floats per input in the A buffer (+4: bank spread)
constexpr int ADS = NJ * AJS;                  // floats per direction slot of a step
constexpr int PSS = 4 * N + 4;                 // floats per slot in the epilogue transpose
constexpr int MAX_ROWS = 32;                   // phase rows a tree item stages (1 + children)
constexpr int MAX_S = 96;                      // sigma_0 and (sigma_0, sigma_1) values (M <= 86)
constexpr int MAX_STEP = 24;                   // fused-item steps (M/2 antipodal pairs, two a step)
constexpr int NXB = 4;                         // X node buffers
constexpr int NPB = 4;                         // Pt node buffers
constexpr int FLAG = 2;                        // fused items of node s - FLAG run in stage s
constexpr int RLAG = 4;                        // radial items of node s - RLAG run in stage s
constexpr uint32_t TMEM_COLS = 128;            // per CTA (three CTAs use 384 of the SM's 512 columns)
constexpr int CTAS_PER_SM = 3;

// dynamic shared memory (bytes).  Fused: two stages, each holding the X
// blocks of one step, then that step's A buffer (its shifted fields) in the
// same place once the X values are in registers, while the next step's X
// blocks land in the other stage; the epilogue transposes 64 slots at a time
// in stage 0.  Tree and radial: one plane.  Sized so that at most three CTAs
// share an SM (their TMEM columns must fit the SM's 512).
constexpr int SM_STAGE = 4 * XBLK * 8;                // 33792 B
constexpr int SM_PH2 = 2 * SM_STAGE;                  // [2 stages][4 slots][H] float2 phase rows
constexpr int SM_TPH = PLANE * 8;                     // tree: phase rows after the plane
constexpr int QBLK = N * N * KB;                      // float2 of one (slot, column block) of Qhat+
constexpr int SM_QS = PLANE * 8;                      // radial: that Qhat+ block after the plane
constexpr int SM_TOTAL = SM_PH2 + 2 * 4 * H * 8;       // 68608 B: three CTAs with their static tables fit 228 KB
static_assert(4 * ADS * 4 <= SM_STAGE, "A overlays the X blocks of its stage");
static_assert(64 * PSS * 4 <= SM_STAGE, "64 epilogue slots fit a stage");
static_assert(SM_PH2 + 2 * 4 * H * 8 <= SM_TOTAL, "phase rows fit");
static_assert(SM_TPH + MAX_ROWS * N * 8 <= SM_TOTAL, "tree phase rows fit");
static_assert(SM_QS + QBLK * 8 <= SM_TOTAL, "radial Qhat+ block fits");
static_assert((CTAS_PER_SM + 1) * (SM_TOTAL + 4096) > 228 * 1024, "at most three CTAs per SM");
static_assert(CTAS_PER_SM * (SM_TOTAL + 4096) <= 228 * 1024, "three CTAs per SM");

// Direction structure of the rule (node independent), built on the host.
struct Tree {
    int n_s0, n_s01, n_grp, n_step;
    const int* grp;          // host grouping of the sigma_0 values (kept for the plan layout)
    const int* s0_dir;       // [n_s0]: a direction with this sigma_0
    const int* s0_child;     // [n_s0 + 1]: ranges of its (sigma_0, sigma_1) values
    const int* s01_dir;      // [n_s01]: a direction with this (sigma_0, sigma_1) = X block index
    const int4* step_blk;    // [n_step]: X block of stage slot 0..3 (-1 unused)
    const int4* step_dir;    // [n_step]: direction of slot 0..3 (-1 unused); (0,1), (2,3) antipodal
    const int4* step_sel;    // [n_step]: stage slot (0..3) of the X block that slot d reads
    const float2* step_w;    // [n_step]: weights w_p of the pairs (0,1) and (2,3)
};

struct Params {
    const float2* spectra;   // [n_inputs][HALF]
    const int* inputs;       // [n_chunk][n_c]: chunk-local -> global input
    const float2* phase;     // [(n_rho M + 1)][3][N]: (-1)^k exp(-i pi k s_a / L), zero at Nyquist
    const float* ctab;       // [n_rho][SMAX + 1]: c_q(|k|^2) including 1/n
    float2* X;               // [NXB][n_s01][NLB][XBLK]
    float2* Pt;              // [NPB][NSLOT][NKB][PLANE]
    float2* qhat;            // [n_chunk][n_used][NKB][QBLK]: running Qhat+ sums of the used slots, packed:
                             // [kb][k0][k1][c],
                             // k2 = 4 kb + c, column 0 holding Y = A + i B of the planes k2 = 0, N/2
    float2* qstd;            // [n_chunk][n_used][HALF]: the final Qhat+ in the standard half-spectrum
                             // layout, written by the last node's radial items
    const int* slots;        // [n_used]: slots whose gain is needed (the same in every chunk)
    unsigned used[5];        // the same slots as a bit set (slot u: bit u % 32 of word u / 32),
                             // one set for every chunk of the launch
    int* ctr;                // counters, zeroed before the launch (layout in ctr_*)
    int* err;                // device error word
    Tree tr;
    int n_c, M, n_rho, n_used;   // per chunk: inputs, directions, radial nodes, used slots
    int n_node;                  // radial nodes of the launch: chunks x n_rho (node q of the
                                 // launch is node q % n_rho of chunk q / n_rho)
};

// counters: [0] claim, [1] abort, then per node of the launch: tree done,
// fused done, radial done, then per used slot of every chunk the nodes
// accumulated into its Qhat+
__host__ __device__ constexpr int ctr_tree(int n_node, int q) { return 2 + q; }
__host__ __device__ constexpr int ctr_fused(int n_node, int q) { return 2 + n_node + q; }
__host__ __device__ constexpr int ctr_radial(int n_node, int q) { return 2 + 2 * n_node + q; }
__host__ __device__ constexpr int ctr_acc(int n_node, int i) { return 2 + 3 * n_node + i; }
__host__ __device__ constexpr int ctr_count(int n_node, int n_slots) { return 2 + 3 * n_node + n_slots; }

// TRI16 slot of the unordered pair (a <= b)
__host__ __device__ constexpr int tri_slot(int a, int b) { return a * NJ - a * (a - 1) / 2 + (b - a); }

// Accumulator columns of a fused item.  Column pair (2i, 2i + 1), i < 64, holds
// the slots (x, y) and (x, y + 1) with y even, so that one packed two-lane FMA
// updates both from the natural input pairs (2h, 2h + 1); row x runs over
// y = x (x even) or x + 1 (x odd) .. 15.  The 8 diagonal slots (x, x) of odd x
// left over are kept in registers (column 128 + (x - 1) / 2).
struct PairTable {
    int x[NTSLOT / 2], yh[NTSLOT / 2];   // pair i: row x, columns y = 2 yh, 2 yh + 1
};
__host__ __device__ constexpr PairTable make_pair_table() {
    PairTable t{};
    int i = 0;
    for (int a = 0; a < NJ; ++a)
        for (int b = (a + 1) & ~1; b < NJ; b += 2) {
            t.x[i] = a;
            t.yh[i] = b / 2;
            ++i;
        }
    return t;
}
constexpr PairTable kPair = make_pair_table();

// TRI16 slot of accumulator column c (for the epilogue's runtime index)
struct ColSlots {
    int u[NSLOT];
};
__host__ __device__ constexpr ColSlots make_col_slots() {
    ColSlots cs{};
    const PairTable pt = make_pair_table();
    for (int i = 0; i < NTSLOT / 2; ++i) {
        cs.u[2 * i] = tri_slot(pt.x[i], 2 * pt.yh[i]);
        cs.u[2 * i + 1] = tri_slot(pt.x[i], 2 * pt.yh[i] + 1);
    }
    for (int k = 0; k < NRSLOT; ++k) cs.u[NTSLOT + k] = tri_slot(2 * k + 1, 2 * k + 1);
    return cs;
}
__constant__ ColSlots kColSlots = make_col_slots();

enum { IT_FUSED = 0, IT_TREE = 1, IT_RADIAL = 2, IT_END = 3 };

struct Item {
    int kind, q, local;
};

__host__ __device__ inline int tree_items(int n_c, int n_grp) { return n_c * NKB * n_grp; }

// Items of stage s in list order: tree items of node s, fused items of node
// s - FLAG, radial items of node s - RLAG.
__host__ __device__ inline void stage_counts(int s, int n_node, int nT, int nR, int& t, int& f, int& r) {
    t = (s < n_node) ? nT : 0;
    f = (s >= FLAG && s < n_node + FLAG) ? NLB : 0;
    r = (s >= RLAG && s < n_node + RLAG) ? nR : 0;
}

// First item of stage s: every stage has nT tree, NLB fused and nR radial
// items while its node index is in range, so the offset is a closed form.
__device__ __forceinline__ int stage_offset(int s, int nn, int nT, int nR) {
    auto cl = [nn](int v) { return v < 0 ? 0 : (v > nn ? nn : v); };
    return nT * cl(s) + NLB * cl(s - FLAG) + nR * cl(s - RLAG);
}

// Item idx of the stage-ordered list.  `stage` is the caller's cursor: its
// claims increase, so the search resumes where the previous one ended.
__device__ __noinline__ Item decode_item(const Params& P, int& stage, int idx) {
    const int nn = P.n_node, nT = tree_items(P.n_c, P.tr.n_grp), nR = P.n_used;
    const int ns = nn + RLAG;
    if (idx >= stage_offset(ns, nn, nT, nR)) return {IT_END, 0, 0};
    while (idx >= stage_offset(stage + 1, nn, nT, nR)) ++stage;
    int t, f, r;
    stage_counts(stage, nn, nT, nR, t, f, r);
    int k = idx - stage_offset(stage, nn, nT, nR);
    if (k < t) return {IT_TREE, stage, k};
    k -= t;
    if (k < f) return {IT_FUSED, stage - FLAG, k};
    return {IT_RADIAL, stage - RLAG, k - f};
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(int* p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Orders generic-proxy accesses to global memory with async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Bounded wait (one thread) until *c1 >= t1 and *c2 >= t2 (c2 may be null).
// Both counters are read at once, so a satisfied dependency costs one memory
// round trip.  False when about one second of device time passed or another
// CTA has raised the abort flag.
__device__ __noinline__ bool wait_at_least(const int* c1, int t1, const int* c2, int t2, const int* abort) {
    int v1 = ld_acquire(c1);
    int v2 = c2 ? ld_acquire(c2) : t2;
    if (v1 >= t1 && v2 >= t2) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t i = 0; i < kSpinLimit; ++i) {
        __nanosleep(128);
        if (v1 < t1) v1 = ld_acquire(c1);
        if (v2 < t2) v2 = ld_acquire(c2);
        if (v1 >= t1 && v2 >= t2) return true;
        if ((i & 15u) == 15u) {
            if (*reinterpret_cast<const volatile int*>(abort)) return false;
            if (global_timer_ns() - t0 > kWaitNs) return false;
        }
    }
    return false;
}

// TMEM: 32 consecutive 32-bit columns of this thread's lane (warp w owns lanes 32w..32w+31)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
        "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
        "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Waits for this thread's TMEM loads.  The registers they fill are in/out
// operands, so that no use of them can be scheduled before the wait.
__device__ __forceinline__ void tmem_wait_ld32(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// Tables of the direction tree, copied to shared memory once per CTA.
struct TreeSmem {
    int grp[MAX_S + 1], s0_dir[MAX_S], s0_child[MAX_S + 1], s01_dir[MAX_S];
    int4 step_blk[MAX_STEP], step_dir[MAX_STEP], step_sel[MAX_STEP];
    float2 step_w[MAX_STEP];
};

// ------------------------------------------------------------------ tree item
// Columns (k1 = t/4, k2 = 4 kb + c) of input jj, for the sigma_0 values of
// group g: the axis-0 inverse pass of each, then for each of its
// (sigma_0, sigma_1) children the axis-1 inverse pass of the lines
// (i0 = t/4, k2), stored into the X block of line block (i0, m) for m = 0..7
// with lines ordered (i1 = 2m, 2m+16, 2m+1, 2m+17).  The column stays in
// registers for the whole group; the group's phase rows are staged at once.
__device__ void tree_item(const Params& P, const TreeSmem& ts, int q, int local, unsigned char* smem) {
    const int t = threadIdx.x;
    const int ng = P.tr.n_grp;
    const int g = local % ng, kb = (local / ng) % NKB, jj = local / (ng * NKB);
    float2* S0 = reinterpret_cast<float2*>(smem);                  // [N][PRS]: (i0, k1, c)
    float2* ph = reinterpret_cast<float2*>(smem + SM_TPH);         // [rows][N]
    const int k1 = t >> 2, c = t & 3;
    const int ql = q % P.n_rho, ch = q / P.n_rho;                  // node of chunk ch
    const float2* __restrict__ src =
        P.spectra + (size_t)__ldg(&P.inputs[ch * P.n_c + jj]) * HALF + k1 * NH + KB * kb + c;
    float2 col[N];
#pragma unroll
    for (int k0 = 0; k0 < N; ++k0) col[k0] = __ldg(src + k0 * N * NH);
    // phase rows of the group: for each sigma_0 its axis-0 row, then its children's axis-1 rows
    const int i0b = ts.grp[g], i0e = ts.grp[g + 1];
    const int cb0 = ts.s0_child[i0b], rows = (i0e - i0b) + (ts.s0_child[i0e] - cb0);
    for (int e = t; e < rows * N; e += NT) {
        const int r = e / N, k = e % N;
        // row r: the sigma_0 values of the group occupy rows (i - i0b) + (s0_child[i] - cb0)
        int i = i0b;
        while (i + 1 < i0e && r >= (i + 1 - i0b) + (ts.s0_child[i + 1] - cb0)) ++i;
        const int rr = r - ((i - i0b) + (ts.s0_child[i] - cb0));
        const int dir = rr == 0 ? ts.s0_dir[i] : ts.s01_dir[ts.s0_child[i] + rr - 1];
        ph[e] = __ldg(&P.phase[((size_t)(ql * P.M + dir) * 3 + (rr == 0 ? 0 : 1)) * N + k]);
    }
    __syncthreads();
    float2* Xn = P.X + (size_t)(q % NXB) * P.tr.n_s01 * NLB * XBLK;
    const int i0 = t >> 2;
    for (int i = i0b; i < i0e; ++i) {
        const int cb = ts.s0_child[i], ce = ts.s0_child[i + 1];
        const float2* p0 = ph + ((i - i0b) + (cb - cb0)) * N;
        float2 x[N];
#pragma unroll
        for (int k0 = 0; k0 < N; ++k0) {
            x[k0] = cmul(col[k0], p0[k0]);
            if ((k0 & 7) == 7) asm volatile("" ::: "memory");
        }
        fft_reg<N, true>(x);
#pragma unroll
        for (int r0 = 0; r0 < N; ++r0) S0[r0 * PRS + k1 * KB + c] = x[r0];
        __syncthreads();
        for (int ch = cb; ch < ce; ++ch) {
            const float2* p1 = p0 + (1 + ch - cb) * N;
            // loads in groups of eight: with the column held in registers, all
            // sixty-four in flight at once would not fit the register budget
#pragma unroll
            for (int kk = 0; kk < N; ++kk) {
                x[kk] = cmul(S0[i0 * PRS + kk * KB + c], p1[kk]);
                if ((kk & 7) == 7) asm volatile("" ::: "memory");
            }
            fft_reg<N, true>(x);
            float2* xb = Xn + ((size_t)ch * NLB + i0 * 8) * XBLK + jj * XJS + (KB * kb + c) * 4;
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                float4* o = reinterpret_cast<float4*>(xb + m * XBLK);
                o[0] = make_float4(x[2 * m].x, x[2 * m].y, x[2 * m + H].x, x[2 * m + H].y);
                o[1] = make_float4(x[2 * m + 1].x, x[2 * m + 1].y, x[2 * m + 1 + H].x, x[2 * m + 1 + H].y);
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ fused item
// Stage slot k (0..3) of step st: its X block and axis-2 phase row into the
// stage.  Issued by lane 0 of warp k, one of the four arrivals on the stage's
// mbarrier, so that no single thread pays for all eight copies of a step.
__device__ __forceinline__ void fused_issue(const Params& P, const TreeSmem& ts, const float2* Xn, int q, int st,
                                            int k, float2* Xs, float2* ph2, uint64_t* bar) {   // Xs, ph2: the stage
    const int4 blk = ts.step_blk[st];
    const int4 dir = ts.step_dir[st];
    const int bl = k == 0 ? blk.x : k == 1 ? blk.y : k == 2 ? blk.z : blk.w;
    const int dr = k == 0 ? dir.x : k == 1 ? dir.y : k == 2 ? dir.z : dir.w;
    const uint32_t bytes = (bl >= 0 ? XBLK * 8 : 0) + (dr >= 0 ? H * 8 : 0);
    mbar_arrive_expect_tx(bar, bytes);
    if (bl >= 0) bulk_g2s(Xs + k * XBLK, Xn + (size_t)bl * NLB * XBLK, XBLK * 8, bar);
    if (dr >= 0) bulk_g2s(ph2 + k * H, P.phase + ((size_t)((q % P.n_rho) * P.M + dr) * 3 + 2) * N, H * 8, bar);
}

// Two FP32 lanes in one 64-bit register, and the packed FMA of sm_100+.
__device__ __forceinline__ uint64_t f2pack(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2unpack(uint64_t r, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// acc(x, y) += a[x] c[y] + c[x] a[y] for the 16 column pairs of TMEM chunk CH
// (two slots per packed FMA; a2, c2: the natural pairs (2h, 2h + 1) of a, c)
template <int CH>
__device__ __forceinline__ void contract_chunk(uint32_t (&r)[32], const float (&a)[NJ], const float (&cc)[NJ],
                                               const uint64_t (&a2)[NJ / 2], const uint64_t (&c2)[NJ / 2]) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        constexpr PairTable pt = kPair;
        const int x = pt.x[CH * 16 + k], yh = pt.yh[CH * 16 + k];
        uint64_t v = f2pack(__uint_as_float(r[2 * k]), __uint_as_float(r[2 * k + 1]));
        v = ffma2(f2pack(a[x], a[x]), c2[yh], ffma2(f2pack(cc[x], cc[x]), a2[yh], v));
        float lo, hi;
        f2unpack(v, lo, hi);
        r[2 * k] = __float_as_uint(lo);
        r[2 * k + 1] = __float_as_uint(hi);
    }
}

// Returns false when a bulk copy did not land in time (the caller aborts).
// DIAG: every used gain slot is a diagonal (j, j) (the cells of a full tensor
// grid, Q(f_x, f_x)): the 16 diagonal accumulators stay in registers, tensor
// memory is not used, and the epilogue transforms those 16 slots only.
template <bool DIAG>
__device__ bool fused_item(const Params& P, const TreeSmem& ts, int q, int lb, unsigned char* smem, uint64_t* bars,
                           uint32_t& par, uint32_t tmem) {
    const int t = threadIdx.x, warp = t >> 5;
    const int nst = P.tr.n_step;
    const float2* Xn = P.X + (size_t)(q % NXB) * P.tr.n_s01 * NLB * XBLK + (size_t)lb * XBLK;
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);    // this warp's 32 TMEM lanes
    auto stage_x = [&](int b) { return reinterpret_cast<float2*>(smem + b * SM_STAGE); };
    auto stage_ph = [&](int b) { return reinterpret_cast<float2*>(smem + SM_PH2) + b * 4 * H; };
    if ((t & 31) == 0) {
        fence_proxy_async_global();
        fence_proxy_async_smem();
        fused_issue(P, ts, Xn, q, 0, warp, stage_x(0), stage_ph(0), &bars[0]);
        if (nst > 1) fused_issue(P, ts, Xn, q, 1, warp, stage_x(1), stage_ph(1), &bars[1]);
    }
    if constexpr (!DIAG) {
        uint32_t z[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) z[k] = 0u;
#pragma unroll
        for (int ch = 0; ch < NTSLOT / 32; ++ch) tmem_st32(tl + 32 * ch, z);
        tmem_wait_st();
    }
    constexpr int NREG = DIAG ? NJ : NRSLOT;
    float racc[NREG];                          // DIAG: slot (x, x) in racc[x]; else the odd diagonals
#pragma unroll
    for (int k = 0; k < NREG; ++k) racc[k] = 0.f;
    const int d = warp, lp = (t >> 4) & 1, j = t & 15;
#pragma unroll 1
    for (int st = 0; st < nst; ++st) {
        const int b = st & 1;
        const bool ok = mbar_wait_bounded(&bars[b], (par >> b) & 1u);
        par ^= 1u << b;
        if (__syncthreads_or(!ok)) {
            // leave no copy in flight: the other stage may still be landing
            if (t == 0) {
                (void)mbar_wait_bounded(&bars[b], ((par >> b) & 1u) ^ 1u);
                if (st + 1 < nst) (void)mbar_wait_bounded(&bars[b ^ 1], (par >> (b ^ 1)) & 1u);
            }
            return false;
        }
        const float2* Xs = stage_x(b);
        float* A = reinterpret_cast<float*>(smem + b * SM_STAGE);  // overlays Xs once X is in registers
        const int4 dir4 = ts.step_dir[st];
        const int dir = d == 0 ? dir4.x : d == 1 ? dir4.y : d == 2 ? dir4.z : dir4.w;
        const int sel = d == 0 ? ts.step_sel[st].x : d == 1 ? ts.step_sel[st].y : d == 2 ? ts.step_sel[st].z
                                                                                       : ts.step_sel[st].w;
        // X lines of this thread's line pair (i1 = 2m + lp, 2m + lp + 16), input j, with the
        // axis-2 phase, packed for one complex-to-real transform.  Every thread transforms
        // (an unused slot or input reads stale stage data and its result is not stored):
        // a branch here costs the register allocator ~40 registers.
        const bool work = dir >= 0 && j < P.n_c;
        float2 x[N];
        {
            const float2* xb = Xs + (sel & 3) * XBLK + j * XJS + lp * 2;
            const float2* pr = stage_ph(b) + d * H;
            {
                const float4 v = *reinterpret_cast<const float4*>(xb);
                x[0] = make_float2(v.x, v.z);
                x[H] = make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int k = 1; k < H; ++k) {
                const float4 v = *reinterpret_cast<const float4*>(xb + 4 * k);
                const float2 w = pr[k];
                const float2 a = cmul(make_float2(v.x, v.y), w), e = cmul(make_float2(v.z, v.w), w);
                x[k] = make_float2(a.x - e.y, a.y + e.x);
                x[N - k] = make_float2(a.x + e.y, e.x - a.y);
            }
            fft_reg<N, true>(x);
        }
        // the X values are in registers: A may overwrite the stage
        __syncthreads();
        float* Ad = A + d * ADS + j * AJS + lp * 2 * N;
        if (work) {
            store_two_rows<N>(Ad, Ad + N, x);
        } else if (dir >= 0) {
            float4* z = reinterpret_cast<float4*>(Ad);
#pragma unroll
            for (int c = 0; c < N / 2; ++c) z[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        // sigma-contraction of the step's two antipodal pairs, voxel v = t
        const float2 w2 = ts.step_w[st];
#pragma unroll 1
        for (int pi = 0; pi < 2; ++pi) {
            const int da = pi == 0 ? dir4.x : dir4.z;
            if (da < 0) continue;
            const float w = pi == 0 ? w2.x : w2.y;
            const float* Aa = A + (2 * pi) * ADS + t;
            const float* Ac = A + (2 * pi + 1) * ADS + t;
            float a[NJ], cc[NJ];
#pragma unroll
            for (int xx = 0; xx < NJ; ++xx) {
                a[xx] = w * Aa[xx * AJS];
                cc[xx] = Ac[xx * AJS];
            }
            if constexpr (DIAG) {
#pragma unroll
                for (int xx = 0; xx < NJ; ++xx) racc[xx] = fmaf(a[xx], cc[xx], fmaf(cc[xx], a[xx], racc[xx]));
                continue;
            }
            uint64_t a2[NJ / 2], c2[NJ / 2];
#pragma unroll
            for (int h = 0; h < NJ / 2; ++h) {
                a2[h] = f2pack(a[2 * h], a[2 * h + 1]);
                c2[h] = f2pack(cc[2 * h], cc[2 * h + 1]);
            }
            uint32_t r[32];
            tmem_ld32(tl + 0, r);
            tmem_wait_ld32(r);
            contract_chunk<0>(r, a, cc, a2, c2);
            tmem_st32(tl + 0, r);
            tmem_ld32(tl + 32, r);
            tmem_wait_ld32(r);
            contract_chunk<1>(r, a, cc, a2, c2);
            tmem_st32(tl + 32, r);
            tmem_ld32(tl + 64, r);
            tmem_wait_ld32(r);
            contract_chunk<2>(r, a, cc, a2, c2);
            tmem_st32(tl + 64, r);
            tmem_ld32(tl + 96, r);
            tmem_wait_ld32(r);
            contract_chunk<3>(r, a, cc, a2, c2);
            tmem_st32(tl + 96, r);
#pragma unroll
            for (int k = 0; k < NRSLOT; ++k) {
                const int xx = 2 * k + 1;                          // diagonal slot (x, x), x odd
                racc[k] = fmaf(a[xx], cc[xx], fmaf(cc[xx], a[xx], racc[k]));
            }
            tmem_wait_st();
        }
        __syncthreads();                                           // A consumed: stage b is free
        if ((t & 31) == 0 && st + 2 < nst) {
            fence_proxy_async_smem();
            fused_issue(P, ts, Xn, q, st + 2, warp, stage_x(b), stage_ph(b), &bars[b]);
        }
    }
    // epilogue: the gain fields of the 128 voxels, 64 slots at a time, through
    // shared memory, then the forward real-to-complex pass along axis 2 of
    // every (slot, line pair)
    float* Pst = reinterpret_cast<float*>(smem);                   // [64][PSS] in stage 0
    float2* Ptn = P.Pt + (size_t)(q % NPB) * NSLOT * NKB * PLANE;
    const int i0 = lb >> 3, m = lb & 7;
#pragma unroll 1
    for (int rnd = 0; rnd < (DIAG ? 1 : 3); ++rnd) {
        const int u0 = 64 * rnd;
        const int nsl = DIAG ? NJ : rnd < 2 ? 64 : NRSLOT;
        if (DIAG) {
#pragma unroll
            for (int k = 0; k < NREG; ++k) Pst[k * PSS + t] = racc[k];
        } else if (rnd < 2) {
            uint32_t r[32];
            tmem_ld32(tl + u0, r);
            tmem_wait_ld32(r);
#pragma unroll
            for (int k = 0; k < 32; ++k) Pst[k * PSS + t] = __uint_as_float(r[k]);
            tmem_ld32(tl + u0 + 32, r);
            tmem_wait_ld32(r);
#pragma unroll
            for (int k = 0; k < 32; ++k) Pst[(32 + k) * PSS + t] = __uint_as_float(r[k]);
        } else {
#pragma unroll
            for (int k = 0; k < NREG; ++k) Pst[k * PSS + t] = racc[k];
        }
        __syncthreads();
        for (int task = t; task < 2 * nsl; task += NT) {
            const int lp2 = task / nsl, us = task % nsl;
            const int u = DIAG ? tri_slot(us, us) : kColSlots.u[u0 + us];
            if (!((P.used[u >> 5] >> (u & 31)) & 1u)) continue;      // no radial item reads this slot
            const float* r1 = Pst + us * PSS + lp2 * 2 * N;           // rows i1 = 2m + lp2 and i1 + 16
            float2 x[N];
            load_two_rows_smem<N>(r1, r1 + N, x);
            fft_reg<N, false>(x);
            const int i1a = 2 * m + lp2;
            float2* oa = Ptn + (size_t)u * NKB * PLANE + i0 * PRS + i1a * KB;
            float2* ob = oa + H * KB;                                 // row i1a + 16
#pragma unroll
            for (int kb = 0; kb < NKB; ++kb) {
                float2 r1v[KB], r2v[KB];
#pragma unroll
                for (int c = 0; c < KB; ++c) {
                    const int k = KB * kb + c;
                    if (k == 0) {
                        // column 0 carries (DC, Nyquist) of each row, both real
                        r1v[c] = make_float2(x[0].x, x[H].x);
                        r2v[c] = make_float2(x[0].y, x[H].y);
                    } else {
                        const float2 z = x[k], zc = x[N - k];
                        r1v[c] = make_float2(0.5f * (z.x + zc.x), 0.5f * (z.y - zc.y));
                        r2v[c] = make_float2(0.5f * (z.y + zc.y), -0.5f * (z.x - zc.x));
                    }
                }
                float4* pa = reinterpret_cast<float4*>(oa + kb * PLANE);
                float4* pb = reinterpret_cast<float4*>(ob + kb * PLANE);
                pa[0] = make_float4(r1v[0].x, r1v[0].y, r1v[1].x, r1v[1].y);
                pa[1] = make_float4(r1v[2].x, r1v[2].y, r1v[3].x, r1v[3].y);
                pb[0] = make_float4(r2v[0].x, r2v[0].y, r2v[1].x, r2v[1].y);
                pb[1] = make_float4(r2v[2].x, r2v[2].y, r2v[3].x, r2v[3].y);
            }
        }
        __syncthreads();
    }
    return true;
}

// ------------------------------------------------------------------ radial item
// 1-D bulk copy of `bytes` from this CTA's shared memory to global memory, as
// one bulk async-group of this thread.
__device__ __forceinline__ void bulk_s2g(void* dst_gmem, const void* src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
                 "r"(smem_u32(src_smem)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Waits until this thread's bulk stores have read their shared-memory sources.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// Slot u, column block by column block: the Pt plane's forward axis-1 pass
// (thread = line (i0, c)), forward axis-0 pass (thread = column (k1, c)), then
// Qhat+[u](k) (+)= c_q(|k|^2) (-1)^(k0+k1+k2) DFT[P_q,u](k), with the block of
// Qhat+ copied into shared memory and back in one piece each way.
__device__ bool radial_item(const Params& P, int q, int ui, unsigned char* smem, uint64_t* bars, uint32_t& par) {
    const int t = threadIdx.x;
    const int ql = q % P.n_rho, gi = (q / P.n_rho) * P.n_used + ui;   // node of the chunk, slot of the launch
    const int u = __ldg(&P.slots[ui]);
    float2* S = reinterpret_cast<float2*>(smem);
    float2* Qs = reinterpret_cast<float2*>(smem + SM_QS);          // [k0][k1][c]
    const bool first = (ql == 0);
    const float* __restrict__ ct = P.ctab + (size_t)ql * (SMAX + 1);
    const int c = t & 3, k1 = t >> 2;
    const int b = wrapk(k1, N), k1m = (N - k1) % N;
    const float2* src0 = P.Pt + (size_t)((q % NPB) * NSLOT + u) * NKB * PLANE;
    float2* qblk0 = P.qhat + (size_t)gi * NKB * QBLK;
    // the plane (bars[2]) and the running-sum block (bars[3]) of a column block travel
    // separately: each is copied in as soon as its buffer is free, the plane of the
    // next block while this block accumulates, the sums while the next plane transforms
    if (t == 0) {
        fence_proxy_async_global();
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bars[2], PLANE * 8);
        bulk_g2s(S, src0, PLANE * 8, &bars[2]);
        if (!first) {
            mbar_arrive_expect_tx(&bars[3], QBLK * 8);
            bulk_g2s(Qs, qblk0, QBLK * 8, &bars[3]);
        }
    }
#pragma unroll 1
    for (int kb = 0; kb < NKB; ++kb) {
        float2* qblk = qblk0 + (size_t)kb * QBLK;
        bool ok = mbar_wait_bounded(&bars[2], (par >> 2) & 1u);
        par ^= 4u;
        if (__syncthreads_or(!ok)) {
            if (t == 0) {
                (void)mbar_wait_bounded(&bars[2], ((par >> 2) & 1u) ^ 1u);   // the copy that was late
                if (!first) (void)mbar_wait_bounded(&bars[3], (par >> 3) & 1u);
                bulk_wait_all();
            }
            return false;
        }
        float2 x[N];
        {
            const int i0 = t >> 2;
#pragma unroll
            for (int i1 = 0; i1 < N; ++i1) x[i1] = S[i0 * PRS + i1 * KB + c];
            fft_reg<N, false>(x);
#pragma unroll
            for (int kk = 0; kk < N; ++kk) S[i0 * PRS + kk * KB + c] = x[kk];
        }
        __syncthreads();
#pragma unroll
        for (int i0 = 0; i0 < N; ++i0) x[i0] = S[i0 * PRS + k1 * KB + c];
        fft_reg<N, false>(x);
        // the packed column (block 0, c = 0) needs its values at the mirrored frequency
        const bool packed = (kb == 0 && c == 0);
        __syncthreads();
        if (packed) {
#pragma unroll
            for (int k0 = 0; k0 < N; ++k0) S[k0 * PRS + k1 * KB] = x[k0];
        }
        if (!first) {
            ok = mbar_wait_bounded(&bars[3], (par >> 3) & 1u);
            par ^= 8u;
        } else if (t == 0) {
            bulk_wait_read();                                   // the previous block's store has read Qs
        }
        if (__syncthreads_or(!ok)) {
            if (t == 0) {
                (void)mbar_wait_bounded(&bars[3], ((par >> 3) & 1u) ^ 1u);
                bulk_wait_all();
            }
            return false;
        }
        const int k2 = KB * kb + c;
#pragma unroll
        for (int k0 = 0; k0 < N; ++k0) {
            const int a = wrapk(k0, N);
            float2 v;
            if (!packed) {
                const float c0 = __ldg(&ct[a * a + b * b + k2 * k2]);
                const float sc = ((k0 + k1 + k2) & 1) ? -c0 : c0;
                v = make_float2(x[k0].x * sc, x[k0].y * sc);
            } else {
                // Z = F[A] + i F[B] of the real planes A (k2 = 0) and B (k2 = N/2); the packed sum
                // is Y = c0 F[A] + i c16 F[B] = ((c0 + c16) Z + (c0 - c16) conj Z(-k)) / 2
                const float2 z = x[k0], zm = S[((N - k0) % N) * PRS + k1m * KB];
                const float sg = ((k0 + k1) & 1) ? -0.5f : 0.5f;      // (-1)^(k0+k1+k2) / 2, k2 = 0 or N/2
                const float c0 = __ldg(&ct[a * a + b * b]), c16 = __ldg(&ct[a * a + b * b + H * H]);
                const float p = sg * (c0 + c16), m = sg * (c0 - c16);
                v = make_float2(fmaf(p, z.x, m * zm.x), fmaf(p, z.y, -m * zm.y));
            }
            float2* o = Qs + (k0 * N + k1) * KB + c;
            if (!first) v = make_float2(v.x + o->x, v.y + o->y);
            *o = v;
        }
        if (ql < P.n_rho - 1) {
            fence_proxy_async_smem();
            __syncthreads();                                    // Qs complete, S read for the last time
            if (t == 0) {
                bulk_s2g(qblk, Qs, QBLK * 8);
                if (kb + 1 < NKB) {
                    mbar_arrive_expect_tx(&bars[2], PLANE * 8);
                    bulk_g2s(S, src0 + (size_t)(kb + 1) * PLANE, PLANE * 8, &bars[2]);
                    if (!first) {
                        bulk_wait_read();                       // the store has read Qs
                        mbar_arrive_expect_tx(&bars[3], QBLK * 8);
                        bulk_g2s(Qs, qblk + QBLK, QBLK * 8, &bars[3]);
                    }
                }
            }
        } else {
            // last node: the finished sums in the standard half-spectrum layout,
            // the packed column split back into its k2 = 0 and k2 = N/2 planes
            __syncthreads();
            if (t == 0 && kb + 1 < NKB) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bars[2], PLANE * 8);
                bulk_g2s(S, src0 + (size_t)(kb + 1) * PLANE, PLANE * 8, &bars[2]);
            }
            float2* qs = P.qstd + (size_t)gi * HALF;
#pragma unroll 4
            for (int k0 = 0; k0 < N; ++k0) {
                const float2 y = Qs[(k0 * N + k1) * KB + c];
                if (kb != 0 || c != 0) {
                    qs[(k0 * N + k1) * NH + k2] = y;
                } else {
                    const float2 ym = Qs[(((N - k0) % N) * N + k1m) * KB];
                    qs[(k0 * N + k1) * NH] = make_float2(0.5f * (y.x + ym.x), 0.5f * (y.y - ym.y));
                    qs[(k0 * N + k1) * NH + H] = make_float2(0.5f * (y.y + ym.y), -0.5f * (y.x - ym.x));
                }
            }
            fence_proxy_async_smem();
            __syncthreads();                                    // Qs read
            if (t == 0 && kb + 1 < NKB && !first) {
                mbar_arrive_expect_tx(&bars[3], QBLK * 8);
                bulk_g2s(Qs, qblk + QBLK, QBLK * 8, &bars[3]);
            }
        }
    }
    if (t == 0) {
        bulk_wait_all();
        fence_proxy_async_global();
    }
    return true;
}

// ------------------------------------------------------------------ persistent kernel
// Publishes a finished item: its global writes (generic stores of every
// thread, ordered by the CTA barrier that ended the item, and bulk stores that
// thread 0 waited for) become visible with release semantics, then the item
// is counted.
__device__ __forceinline__ void publish(const Params& P, const Item& it) {
    fence_proxy_async_global();
    const int nn = P.n_node;
    if (it.kind == IT_TREE) red_release_add(P.ctr + ctr_tree(nn, it.q), 1);
    else if (it.kind == IT_FUSED) red_release_add(P.ctr + ctr_fused(nn, it.q), 1);
    else {
        red_release_add(P.ctr + ctr_acc(nn, (it.q / P.n_rho) * P.n_used + it.local), 1);
        red_release_add(P.ctr + ctr_radial(nn, it.q), 1);
    }
}

template <bool DIAG>
__global__ void __launch_bounds__(NT, CTAS_PER_SM) k_pencil(Params P) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ TreeSmem ts;
    __shared__ uint64_t bars[4];
    __shared__ uint32_t tmem_base;
    __shared__ Item s_it[2];
    __shared__ int s_ok;
    const int t = threadIdx.x, warp = t >> 5;
    const int nT = tree_items(P.n_c, P.tr.n_grp), nR = P.n_used;
    // direction tree tables and the list's stage offsets into shared memory
    for (int e = t; e <= P.tr.n_grp; e += NT) ts.grp[e] = __ldg(&P.tr.grp[e]);
    for (int e = t; e < P.tr.n_s0; e += NT) ts.s0_dir[e] = __ldg(&P.tr.s0_dir[e]);
    for (int e = t; e <= P.tr.n_s0; e += NT) ts.s0_child[e] = __ldg(&P.tr.s0_child[e]);
    for (int e = t; e < P.tr.n_s01; e += NT) ts.s01_dir[e] = __ldg(&P.tr.s01_dir[e]);
    for (int e = t; e < P.tr.n_step; e += NT) {
        ts.step_blk[e] = __ldg(&P.tr.step_blk[e]);
        ts.step_dir[e] = __ldg(&P.tr.step_dir[e]);
        ts.step_sel[e] = __ldg(&P.tr.step_sel[e]);
        ts.step_w[e] = __ldg(&P.tr.step_w[e]);
    }
    int stage = 0;                                     // thread 0: decoding cursor
    if (t == 0) {
        mbar_init(&bars[0], 4);                        // fused stages: one arrival per warp
        mbar_init(&bars[1], 4);
        mbar_init(&bars[2], 1);                        // radial: Pt planes
        mbar_init(&bars[3], 1);                        // radial: running-sum blocks
        mbar_init_fence();
        s_it[0] = decode_item(P, stage, atomicAdd(P.ctr, 1));
    }
    if (!DIAG && warp == 0) tc_alloc<TMEM_COLS>(&tmem_base);
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = DIAG ? 0u : tmem_base;
    uint32_t par = 0;                                  // parity bits of the next phases of bars[0..3]
    int* abort_flag = P.ctr + 1;
    Item prev{IT_END, 0, 0};
    for (int i = 0;; ++i) {
        const Item it = s_it[i & 1];
        // lane 0 of warp 1 publishes the previous item while thread 0 claims the
        // next one and waits for this one's dependencies
        if (t == 32 && prev.kind != IT_END) publish(P, prev);
        if (it.kind == IT_END) break;
        int next = 0;
        if (t == 0) {
            // the next item is claimed now; it is decoded and stored once this item is done
            next = atomicAdd(P.ctr, 1);
            const int nn = P.n_node;
            bool ok = true;
            if (it.kind == IT_TREE && it.q >= NXB)
                ok = wait_at_least(P.ctr + ctr_fused(nn, it.q - NXB), NLB, nullptr, 0, abort_flag);
            else if (it.kind == IT_FUSED)
                ok = wait_at_least(P.ctr + ctr_tree(nn, it.q), nT,
                                   it.q >= NPB ? P.ctr + ctr_radial(nn, it.q - NPB) : nullptr, nR, abort_flag);
            else if (it.kind == IT_RADIAL)   // the slot's sums hold the chunk's earlier nodes
                ok = wait_at_least(P.ctr + ctr_fused(nn, it.q), NLB,
                                   P.ctr + ctr_acc(nn, (it.q / P.n_rho) * P.n_used + it.local), it.q % P.n_rho,
                                   abort_flag);
            if (!ok && *reinterpret_cast<volatile int*>(abort_flag) == 0) {
                atomicOr(P.err, kErrTimeout);
                atomicExch(abort_flag, 1);
            }
            // after an abort no item works (the CTA whose item failed may hold
            // stale copy-stage parities)
            s_ok = ok && *reinterpret_cast<volatile int*>(abort_flag) == 0;
        }
        __syncthreads();
        if (s_ok) {
            bool done = true;
            if (it.kind == IT_TREE) tree_item(P, ts, it.q, it.local, smem);
            else if (it.kind == IT_FUSED) done = fused_item<DIAG>(P, ts, it.q, it.local, smem, bars, par, tmem);
            else done = radial_item(P, it.q, it.local, smem, bars, par);
            if (!done && t == 0) {
                atomicOr(P.err, kErrTimeout);
                atomicExch(abort_flag, 1);
            }
        }
        if (t == 0) s_it[(i + 1) & 1] = decode_item(P, stage, next);
        __syncthreads();                               // every thread's writes of the item are done
        prev = it;
    }
    tc_fence_before_sync();
    __syncthreads();
    if (!DIAG && warp == 0) tc_dealloc<TMEM_COLS>(tmem);
}

}  // namespace pencil
}  // namespace boltz_dev
