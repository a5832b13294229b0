/*
 * boltz.h -- C ABI of the GB300 (sm_103a) fast-spectral Boltzmann collision library.
 *
 * The library evaluates the bilinear collision operator of the paper's Sec. 1
 * (eq. "eqn:collision_operator", post-collision velocities eq.
 * "eqn:collision velocity") as a discrete-velocity method (Sec. 2.1): values of
 * h1, h2 on a uniform grid of [-L, L]^d in, values of Q(h1, h2) on the same
 * grid out.  The collision kernel is the truncated VHS kernel
 * B = b |q|^gamma for |q| <= R, q = v - v_*.  The integral is evaluated by the
 * separated fast-spectral quadrature: Gauss-Legendre radial nodes rho_q on
 * [0, R] times a centrally symmetric direction rule sigma_p on S^{d-1}; for
 * every node both functions are phase-shifted in Fourier space, transformed
 * back, multiplied and summed over directions, then one forward transform per
 * radial node applies the exact omega-average
 * F_3(s) = 4 pi sin(s)/s, F_2(s) = 2 pi J0(s), s = pi rho_q |k| / (2L).
 * Batches follow Sec. 2 and Sec. 2.4: the r^2 basis pairs Q(V_m, V_n) of the
 * K-, S- and L-steps and the projection <V_j, Q(V_m, V_n)>_v, or one
 * evaluation per spatial cell for the full tensor grid.
 *
 * Conventions (all fixed by this header):
 *   grid        v_j = -L + j * dv, dv = 2L/N, j = 0..N-1 along every axis; a
 *               physical field is float32 [N]^d, C order, axis 0 slowest.
 *   spectra     fhat_k = N^-d sum_j f(v_j) exp(-i pi k.v_j / L), k_a in
 *               [-N/2, N/2).  Stored as the real-to-complex half spectrum:
 *               complex64 (float2 re, im) [N]^(d-1) x [N/2 + 1], last axis
 *               holding k = 0..N/2, other axes in DFT index order
 *               (index i <-> k = i for i < N/2, i - N otherwise).
 *               Entries with any k_a = -N/2 (index N/2) are the Nyquist modes;
 *               they are IGNORED on input (treated as zero), and
 *               boltz_spectrum writes them as zero.
 *   kernel      b defaults to 1/|S^{d-1}| (1/(2 pi) in 2D, 1/(4 pi) in 3D).
 *   loss        Q-(g,f)(v) = f_N(v) * sum_l G-(l) ghat_l exp(i pi l.v / L),
 *               G-(l) = b |S^{d-1}| sum_q w_q rho_q^(gamma+d-1) F_d(pi rho_q |l| / L).
 *   pairs       evaluation e computes Q(g, f) with g = input pair_j[e] and
 *               f = input pair_l[e]; the gain part is symmetric in (g, f),
 *               the loss part is not.
 *
 * Memory: every data pointer marked "device" is caller-owned device memory
 * (for example a torch tensor's data_ptr) that must stay valid until the work
 * queued on `stream` has completed; the library reads and writes it
 * asynchronously on that stream.  Pointers marked "host" are read or written
 * synchronously during the call.  The library owns only the grid handle, its
 * tables and its workspace, allocated on the device that is current when the
 * grid is created; all later calls must be made with that device current.
 *
 * Errors: every entry point returns a boltz_status and never throws.  Argument
 * checks are synchronous and leave device memory untouched.  BOLTZ_ECUDA
 * reports a failed CUDA call (launch or allocation); a context error is
 * sticky in CUDA, so the grid should then be destroyed.  Conditions found by
 * the kernels (a bounded wait that gave up, a non-finite output value) are
 * recorded in a device error word and reported by boltz_sync_status.
 *
 * Fault injection (for testing callers' error handling; host side only): the
 * environment variable BOLTZ_FAULT, read at every call, set to "alloc" makes
 * every workspace allocation fail (BOLTZ_ENOMEM), "badplan" makes batch
 * planning reject every batch (BOLTZ_EINVAL), "nan" marks every collision
 * batch queued by boltz_collide_batched as having produced a non-finite value
 * (boltz_sync_status reports BOLTZ_ENONFINITE).  Unset, nothing is injected.
 *
 * Threading: a grid handle is not thread safe; distinct handles are
 * independent.  Calls on one handle must not overlap on different streams
 * (they share the handle's workspace).
 */
#ifndef BOLTZ_H
#define BOLTZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BOLTZ_ABI_VERSION 1

typedef struct boltz_grid_s* boltz_grid;

typedef enum {
    BOLTZ_OK = 0,
    BOLTZ_EINVAL = 1,        /* bad argument (size, pointer, index)            */
    BOLTZ_ENOMEM = 2,        /* host or device allocation failed               */
    BOLTZ_ECUDA = 3,         /* a CUDA runtime call failed                     */
    BOLTZ_ETIMEOUT = 4,      /* a bounded device wait gave up                  */
    BOLTZ_EUNSUPPORTED = 5,  /* valid request the library does not implement  */
    BOLTZ_ENONFINITE = 6     /* non-finite value detected                      */
} boltz_status;

/* Evaluation forms of boltz_collide_batched. */
typedef enum {
    /* Batched form: every distinct input's shifted fields are computed once
     * per node and shared by all pairs that use it (the f-side field of
     * direction p is the g-side field of the antipodal direction), and the
     * symmetric gain is computed once per unordered pair.  FP32 arithmetic. */
    BOLTZ_FORM_BATCHED = 0,
    /* Plain per-evaluation form: two inverse transforms per (rho, sigma) node
     * and evaluation, nothing shared between evaluations.  FP32.  Same result
     * up to FP32 rounding; kept as the comparison baseline. */
    BOLTZ_FORM_PLAIN = 1,
    /* Batched form with split-precision shifted fields: each shifted field
     * g_N(v - rho sigma / 2) is computed as three per-axis GEMMs with the
     * N x N shift-interpolation matrices of the grid (the DFT-as-GEMM form of
     * the inverse transforms) on the tensor cores, with both operands split
     * into BF16 pairs x = hi + lo, three products per pair (hi*hi, lo*hi,
     * hi*lo) and FP32 accumulation.  Every other step is the FP32 batched
     * form.  Error against an FP64 evaluation ~1e-5 of the result scale
     * (gate 1e-3).  Built for d_v = 3, N = 32; other grids return
     * BOLTZ_EUNSUPPORTED.  The first call on a grid builds its per-node
     * matrices (24 KB per (rho, sigma) node, device memory kept until the
     * grid is destroyed). */
    BOLTZ_FORM_SPLIT_BF16 = 2,
    /* Carleman form (the Mouhot-Pareschi fast spectral method the paper's
     * experiments use; Sec. 2.1, Sec. 5), defined for gamma = d_v - 2 only
     * (2D Maxwell molecules, 3D hard spheres): with x = v' - v, y = v'_* - v
     * the gain is int int 2^{d-1} b delta(x.y) g(v+y) f(v+x) dx dy over
     * |x|, |y| <= R (a different truncation from the other forms' |q| <= R),
     * split over one direction e_p of every antipodal pair of the grid's rule
     * (M/2 directions) into the product of the g-side multiplier
     * psi(pi |l - (l.e_p)e_p| / L) and the f-side multiplier
     * phi(pi m.e_p / L) (closed forms), so that no radial quadrature is
     * needed: 2 inverse transforms per direction and input and no forward
     * transform.  The loss uses the same discrete kernel at m = l (mass is
     * conserved to rounding).  N_rho of the grid is unused.  FP32.
     * gamma != d_v - 2: BOLTZ_EINVAL; the 2D 128^2 grid: BOLTZ_EUNSUPPORTED.
     * The first call builds per-mode tables (M + 1 real values per spectral
     * mode, device memory kept until the grid is destroyed). */
    BOLTZ_FORM_CARLEMAN = 3
} boltz_form;

typedef struct {
    double b;              /* kernel constant; <= 0 selects 1/|S^{d-1}|              */
    size_t workspace_max;  /* cap on device workspace in bytes; 0 = library default */
    int field_budget_mb;   /* shifted-field memory per radial block, MB; 0 = 96 MB
                              (the schedule boltz_autotune chooses between)        */
    int schedule;          /* schedule of the batched FP32 form:
                              BOLTZ_SCHEDULE_AUTO (0): the pipelined schedule where
                              it is built (d_v = 3, N = 32, and no group of inputs
                              joined by pairs larger than 16), the node-block
                              schedule elsewhere;
                              BOLTZ_SCHEDULE_NODE_BLOCKS (1): always the node-block
                              schedule (the comparison baseline)                   */
    int loss;              /* loss weight G-(l) of the separated forms (batched,
                              plain, split, FP64 check build):
                              BOLTZ_LOSS_EXACT (0): b |S^{d-1}| sum_q w_q rho_q^{gamma+d-1}
                              F_d(pi rho_q |l| / L), the exact sigma- and omega-average;
                              BOLTZ_LOSS_MASS_CONSISTENT (1): G_sep(l, -l) =
                              b F_d(0) sum_q w_q rho_q^{gamma+d-1} sum_p w_p
                              cos(pi rho_q l.sigma_p / L), the sigma-average taken with
                              the gain's own direction rule, so that the k = 0 mode of
                              Q (its mass) cancels to rounding.  A per-mode table
                              (half-spectrum entries, FP32 and FP64) is built at grid
                              creation.  The Carleman form keeps its own loss.  Other
                              values: BOLTZ_EINVAL                                  */
} boltz_options;

enum { BOLTZ_LOSS_EXACT = 0, BOLTZ_LOSS_MASS_CONSISTENT = 1 };

/*
 * Schedules of the batched FP32 form (same result up to FP32 rounding order):
 *   NODE_BLOCKS  separate launches per block of radial nodes: every shifted
 *                field is synthesised in full (three inverse passes per
 *                direction), written to device memory, read back by the
 *                sigma-contraction, whose per-node gain fields are written and
 *                read back by the radial step.
 *   PIPELINED    one persistent kernel: the axis-0 and axis-1 inverse passes
 *                are computed once per distinct sigma_0 and per distinct
 *                (sigma_0, sigma_1) of the direction rule (9 and 25 of the 38
 *                directions) and kept in L2-sized node buffers, and the last
 *                inverse pass of every direction is fused with the
 *                sigma-contraction and the first forward pass, so the shifted
 *                fields never leave the chip.  The inputs are split into
 *                chunks of at most 16 (each pair's two inputs in one chunk,
 *                e.g. the cells of a full tensor grid Q(f_x, f_x) in chunks of
 *                16 cells); chunks of one shape (input count and used
 *                pairs) run in one launch, at most 64 chunks each.
 */
#define BOLTZ_SCHEDULE_AUTO 0
#define BOLTZ_SCHEDULE_NODE_BLOCKS 1

/* Library ABI version (BOLTZ_ABI_VERSION of the build). */
int boltz_abi_version(void);

/* Human-readable name of a status code (static string, never NULL). */
const char* boltz_status_string(boltz_status s);

/*
 * Create a grid: N points per axis on [-L, L]^d_v, truncation radius R,
 * kernel exponent gamma, N_rho Gauss-Legendre radial nodes on [0, R] and M
 * directions (paper Sec. 2.1: uniform grid, fast spectral collision solver).
 *   N      in {8, 16, 24, 32, 48, 64} for both d_v = 2 and d_v = 3 (24 and 48 use
 *          a mixed radix-3 transform), and 128 for d_v = 2
 *   d_v    2 or 3
 *   M      d_v = 2: even, 2..256 (uniform circle rule theta_p = 2 pi p / M);
 *          d_v = 3: one of 6, 14, 26, 38, 50, 86 (octahedral rules of design
 *          degree 3, 5, 7, 9, 11, 15, derived at init from their moment
 *          equations)
 *   N_rho  1..128;  L > 0;  R > 0;  gamma > -d_v
 *   opt    may be NULL (defaults)
 * Allocates the handle and its device tables on the current device.
 * Errors: BOLTZ_EINVAL (out may be NULL or a value is out of range; *out is
 * left untouched), BOLTZ_EUNSUPPORTED (valid but not built, e.g. d_v = 3 with N = 128),
 * BOLTZ_ENOMEM, BOLTZ_ECUDA.
 */
boltz_status boltz_grid_init(boltz_grid* out, int N, int d_v, double L, double R, double gamma,
                             int N_rho, int M, const boltz_options* opt);

/* Free the handle, its tables and its workspace (synchronises the device first).
 * NULL is accepted and ignored. */
boltz_status boltz_grid_destroy(boltz_grid g);

/*
 * Input spectra of real fields (paper Sec. 2.1: values on the grid are the
 * method's input): spectra_out[i] = half spectrum of f[i] in the convention
 * above, Nyquist entries zero.
 *   f            device float32 [n_inputs][N^d]
 *   spectra_out  device complex64 [n_inputs][N^(d-1) * (N/2+1)]
 * n_inputs = 0 is a no-op.  Errors: BOLTZ_EINVAL (NULL grid/pointer with
 * n_inputs > 0, n_inputs < 0), BOLTZ_ECUDA.
 */
boltz_status boltz_spectrum(boltz_grid g, const float* f, int n_inputs, void* spectra_out,
                            void* stream);

/*
 * Batched collision evaluations (paper Sec. 2.1 interface, batched over the
 * basis pairs of Sec. 2.4's K-, S- and L-steps or over spatial cells):
 *   Q_out[e] = Q(g = input pair_j[e], f = input pair_l[e]) on the grid.
 *   spectra  device complex64 [n_inputs][N^(d-1) * (N/2+1)] (see boltz_spectrum)
 *   pair_j, pair_l  HOST int32 [n_pairs], each in [0, n_inputs)
 *   Q_out    device float32 [n_pairs][N^d]
 *   form     a boltz_form value
 * Work is queued on `stream` (a cudaStream_t, NULL = legacy default stream);
 * the call returns once it is queued.  n_pairs = 0 is a no-op.
 * Device workspace is allocated on first use and grown when a larger batch
 * needs it (cudaMalloc; the grid keeps it until destroyed).
 * Errors: BOLTZ_EINVAL (NULL pointers, n_inputs <= 0 with n_pairs > 0, an
 * index out of range, unknown form), BOLTZ_ENOMEM, BOLTZ_ECUDA.
 */
boltz_status boltz_collide_batched(boltz_grid g, const void* spectra, int n_inputs,
                                   const int32_t* pair_j, const int32_t* pair_l, int n_pairs,
                                   float* Q_out, int form, void* stream);

/*
 * Projection tensor of the K- and S-steps (paper Sec. 2, eq. "eqn:K-step
 * detailed"; Sec. 2.4 evaluates <.,.>_v with the midpoint rule):
 *   T_out[k][j][l] = dv^d sum_v V_k(v) Q_{j*r + l}(v),  k, j, l in [0, r).
 *   V      device float32 [r][N^d]      (physical values of the basis)
 *   Q      device float32 [r*r][N^d]    (pair p = j*r + l, as produced by
 *                                        boltz_collide_batched over all r^2 pairs)
 *   T_out  device float32 [r][r][r]
 * r in 1..64.  Errors: BOLTZ_EINVAL, BOLTZ_ECUDA.
 */
boltz_status boltz_project(boltz_grid g, const float* V, int r, const float* Q, float* T_out,
                           void* stream);

/*
 * FP64 check build of the three calls above (paper Sec. 2.1; the paper fixes
 * no precision): the same kernels, schedule and quadrature instantiated on
 * double, with the grid's tables kept unrounded.  It separates the method's
 * own error (quadrature, truncation, aliasing) from FP32 rounding: against an
 * FP64 evaluation of the same separated quadrature it agrees to ~1e-13
 * relative.  Built for the small single-CTA grids only: d_v = 3 with N in
 * {8, 16} and d_v = 2 with N in {16, 32}; any other grid returns
 * BOLTZ_EUNSUPPORTED (the grid is left usable).  FP64 throughput on this GPU
 * is a small fraction of FP32: these calls are for checking, not for speed.
 *   boltz_spectrum_f64:         f device float64 [n_inputs][N^d];
 *                               spectra_out device complex128 [n_inputs][half]
 *   boltz_collide_batched_f64:  spectra device complex128 [n_inputs][half];
 *                               Q_out device float64 [n_pairs][N^d]; pair
 *                               arrays, form and stream as boltz_collide_batched
 *   boltz_project_f64:          V float64 [r][N^d], Q float64 [r*r][N^d],
 *                               T_out float64 [r][r][r] (device), r in 1..64
 * The FP64 path shares the grid's workspace and cached plan with the FP32
 * path (switching precision rebuilds the plan).  Other errors as for the FP32
 * calls.
 */
boltz_status boltz_spectrum_f64(boltz_grid g, const double* f, int n_inputs, void* spectra_out,
                                void* stream);
boltz_status boltz_collide_batched_f64(boltz_grid g, const void* spectra, int n_inputs,
                                       const int32_t* pair_j, const int32_t* pair_l, int n_pairs,
                                       double* Q_out, int form, void* stream);
boltz_status boltz_project_f64(boltz_grid g, const double* V, int r, const double* Q,
                               double* T_out, void* stream);

/*
 * Autotuner of the batch schedule.  The tunable is the device memory budget
 * for the shifted fields of one radial block (48, 96, 192, 384 or 768 MB):
 * it sets how many inputs share a chunk (so how often shifted fields are
 * recomputed) and how many radial nodes one launch covers (so how long the
 * launch chain is, whether the fields stay in the 126 MB L2, and how evenly
 * the launches' CTAs fill the last wave on the SMs).  Each
 * candidate runs the given batch three times on `stream` (the first untimed)
 * and the fastest is kept in the grid for later calls.  With a cache path,
 * the choice is read from and written to a JSON file keyed by
 * (N, d_v, M, N_rho, n_inputs, n_pairs, form, SM count); a cached key skips
 * the timing.  Q_scratch: device float32 [n_pairs][N^d], overwritten.
 * chosen_mb (HOST, may be NULL) receives the budget.  Synchronises `stream`.
 * Errors: BOLTZ_EINVAL, BOLTZ_ENOMEM (no candidate fits), BOLTZ_ECUDA.
 */
boltz_status boltz_autotune(boltz_grid g, const void* spectra, int n_inputs, const int32_t* pair_j,
                            const int32_t* pair_l, int n_pairs, float* Q_scratch, int form, const char* cache_path,
                            void* stream, int* chosen_mb);

/*
 * Mixed batches under one CUDA graph.  A batch is a set of work items, each
 * on its own grid (grids may differ in N, d_v, quadrature and kernel): an
 * item optionally computes its input spectra from physical fields, then all
 * its pairs, then optionally the r^3 projection.  boltz_batch_plan builds
 * every item's plan, sizes and fills its grid's workspace, and captures all
 * launches into one CUDA graph with one parallel branch per item (the items
 * run concurrently); boltz_batch_run replays it with a single graph launch.
 * Every pointer in the items is baked into the graph: the buffers must stay
 * valid, and the pair lists unchanged, for as long as the batch is used; the
 * host pair arrays are read only by boltz_batch_plan.  While a batch exists,
 * its grids must not be used for other calls with different pair lists
 * (their workspaces hold the batch's plans).
 */
typedef struct boltz_batch_s* boltz_batch;

typedef struct {
    boltz_grid grid;          /* grid of this item; one item per grid                       */
    const float* fields;      /* device float32 [n_inputs][N^d] physical inputs, or NULL     */
    const void* spectra;      /* device complex64 [n_inputs][half]: read, or written from
                                 `fields` when fields != NULL                                */
    int n_inputs;
    const int32_t* pair_j;    /* HOST int32 [n_pairs]                                        */
    const int32_t* pair_l;    /* HOST int32 [n_pairs]                                        */
    int n_pairs;
    float* Q_out;             /* device float32 [n_pairs][N^d]                               */
    const float* V;           /* device float32 [r][N^d] basis to project on, or NULL        */
    int r;                    /* projection rank; r*r == n_pairs when V != NULL              */
    float* T_out;             /* device float32 [r][r][r] when V != NULL                     */
} boltz_work;

/* Errors: BOLTZ_EINVAL (bad item, two items on one grid, unknown form),
 * BOLTZ_ENOMEM, BOLTZ_ECUDA (including a failed capture).  `form` applies to
 * every item. */
boltz_status boltz_batch_plan(boltz_batch* out, const boltz_work* items, int n_items, int form);
/* Queues one replay of the batch's graph on `stream`. */
boltz_status boltz_batch_run(boltz_batch b, void* stream);
/* Number of kernel launches one replay performs. */
boltz_status boltz_batch_kernel_count(boltz_batch b, int* n_kernels);
/* Synchronises the device and frees the graph and its streams.  NULL is ignored. */
boltz_status boltz_batch_destroy(boltz_batch b);

/*
 * Collision invariants of results, in FP64 (paper Sec. 1: mass, momentum and
 * energy moments; Q conserves them up to quadrature accuracy):
 *   out[f][0]      = dv^d sum_v Q_f(v)
 *   out[f][1 + a]  = dv^d sum_v v_a Q_f(v),  a = 0..d-1
 *   out[f][d + 1]  = dv^d sum_v |v|^2 Q_f(v)
 *   Q    device float32 [n_fields][N^d];  out  device float64 [n_fields][d + 2]
 * Summation order is fixed (run-to-run identical).  Errors: BOLTZ_EINVAL, BOLTZ_ECUDA.
 */
boltz_status boltz_moments(boltz_grid g, const float* Q, int n_fields, double* out, void* stream);

/*
 * Mott-Smith strong-shock closure (paper Sec. 4.2, eq. "eqn:alpha"): with
 * input 0 = f_L (upstream) and input 1 = f_R (downstream), drifting along
 * velocity axis 0,
 *   alpha = int v_1^2 ( Q(f_L, f_R) + Q(f_R, f_L) ) dv   (the two cross
 *           evaluations of the batch, then an FP64 moment on the device)
 *   beta  = alpha / ((d_v - 1) rho_L u_L R_gas (T_L - T_R)),
 * so that a(x_1) = 1 / (exp(beta x_1) + 1) in f = a f_L + (1 - a) f_R.
 *   spectra    device complex64 [2][half] (see boltz_spectrum)
 *   Q_scratch  device float32 [2][N^d], receives Q(f_L, f_R), Q(f_R, f_L)
 *   alpha, beta  HOST double
 * Synchronises `stream`.  Errors: BOLTZ_EINVAL (NULL pointers, T_L == T_R or
 * another zero factor in beta's denominator), BOLTZ_ENOMEM, BOLTZ_ECUDA.
 */
boltz_status boltz_mott_smith(boltz_grid g, const void* spectra, double rho_L, double u_L, double T_L,
                              double T_R, double R_gas, float* Q_scratch, double* alpha, double* beta,
                              void* stream);

/*
 * Allocation-free variant of boltz_project (the paper has no counterpart; this
 * is a deployment aid).  Same arguments, layout and result as boltz_project
 * (up to the order of FP32 summation), but it never allocates device memory:
 * its partial sums live in a fixed 2 MiB array in the library's device image
 * (static __device__ storage that every device loading the library holds
 * until the process exits), so it calls no cudaMalloc, cudaFree or
 * allocating library routine.  It is meant for callers that must not
 * allocate device memory while they run: cudaMalloc and cudaFree can
 * synchronise the whole device and stall unrelated streams in a latency-
 * critical solver loop, and a process whose device memory is fully reserved
 * up front by another allocator (a framework's caching pool, a fixed
 * embedded budget) may have no room for a new allocation.
 *   r       1..64 (the partial sums need r^3 x slices floats <= 2^19; the
 *           slice count is reduced to fit).  Larger r: BOLTZ_EINVAL.
 * Each call made outside stream capture resolves the array's device address
 * on the current device with cudaGetSymbolAddress (so a device reset, which
 * reloads the library's device image, is handled); a call made while
 * `stream` is capturing reuses the address the last uncaptured call on that
 * device resolved, so the first call on a device must come before any stream
 * capture (otherwise BOLTZ_ECUDA).  Every call shares the one array: calls
 * that can overlap on the GPU (different streams, or different grids on the
 * same device) race on it and must be serialised by the caller.  Each call
 * writes every partial sum it reads, so no clearing is needed.
 * Errors: BOLTZ_EINVAL, BOLTZ_ECUDA.
 */
boltz_status boltz_project_noalloc(boltz_grid g, const float* V, int r, const float* Q, float* T_out,
                                   void* stream);

/*
 * End-to-end low-rank collision step from host memory: copies the physical
 * basis V (HOST float32 [r][N^d]) to the device, computes its spectra, all r^2
 * pairs Q(V_j, V_l) (batched form) and the projection T, and copies Q (HOST
 * float32 [r*r][N^d], may be NULL to skip the copy) and T (HOST float32
 * [r][r][r]) back.  Synchronises `stream` before returning.  Device staging
 * buffers come from the grid's workspace.  Host buffers that are page-locked
 * (cudaHostAlloc / pinned torch tensors) give full copy bandwidth.
 * Errors: BOLTZ_EINVAL, BOLTZ_ENOMEM, BOLTZ_ECUDA.
 */
boltz_status boltz_lowrank_step_host(boltz_grid g, const float* V_host, int r, float* Q_host,
                                     float* T_host, void* stream);

/*
 * Quadrature the library uses, computed on the host without a GPU (for
 * checking against an independent implementation):
 *   rho, w_rho      HOST double [N_rho]   Gauss-Legendre on [0, R]
 *   sigma, w_sigma  HOST double [M][d_v], [M]   direction rule
 * Errors: BOLTZ_EINVAL (unsupported d_v / M / N_rho, NULL pointer).
 */
boltz_status boltz_host_quadrature(int d_v, int N_rho, int M, double R, double* rho,
                                   double* w_rho, double* sigma, double* w_sigma);

/*
 * Size of the device workspace a batched call would use for this batch, in
 * bytes, without allocating (host-only planning).  Same argument rules as
 * boltz_collide_batched; `bytes` is HOST size_t.
 */
boltz_status boltz_workspace_size(boltz_grid g, int n_inputs, const int32_t* pair_j,
                                  const int32_t* pair_l, int n_pairs, int form, size_t* bytes);

/*
 * Waits for the work queued on `stream` and reports device-detected errors
 * since the last check, then clears them: BOLTZ_ETIMEOUT if a bounded device
 * wait (an asynchronous-copy barrier or a dependency counter) gave up, which
 * leaves the affected results invalid; BOLTZ_ENONFINITE if a collision
 * output value written since the last check was NaN or infinite (a
 * non-finite input propagates to the outputs of every pair that uses it);
 * BOLTZ_ECUDA if a CUDA call failed.  Kernels never trap or spin without a
 * limit; this call is how their failures surface.
 */
boltz_status boltz_sync_status(boltz_grid g, void* stream);

/*
 * Failure-path self-test (not part of the paper's method).  which = 0 runs a
 * one-CTA kernel whose asynchronous-copy barrier is never completed; its
 * bounded wait gives up after about one second, records the timeout and
 * returns, and this call then returns what boltz_sync_status reports:
 * BOLTZ_ETIMEOUT when the failure path works.  The device stays usable.
 * Errors: BOLTZ_EINVAL (NULL grid, unknown `which`), BOLTZ_ECUDA.
 */
boltz_status boltz_selftest(boltz_grid g, int which, void* stream);

/* Kernel classes reported by boltz_profile_read. */
typedef enum {
    BOLTZ_KCLASS_SPECTRUM = 0,  /* input spectra (forward real transforms)                  */
    BOLTZ_KCLASS_PREP = 1,      /* f_N and Lambda_g of a chunk's inputs                       */
    BOLTZ_KCLASS_SHIFT = 2,     /* phase-weighted inverse transforms: the shifted fields      */
    BOLTZ_KCLASS_CONTRACT = 3,  /* sigma-contraction of shifted-field products                */
    BOLTZ_KCLASS_RADIAL = 4,    /* forward transform x radial multiplier, accumulated over q  */
    BOLTZ_KCLASS_OUTPUT = 5,    /* gain synthesis minus loss, written per ordered pair        */
    BOLTZ_KCLASS_PROJECT = 6,   /* projection tensor (two kernels)                            */
    BOLTZ_KCLASS_PIPELINE = 7,  /* pipelined schedule: shifted fields, sigma-contraction and
                                   radial step of all nodes in one persistent kernel          */
    BOLTZ_KCLASS_COUNT = 8
} boltz_kernel_class;

/*
 * Launch accounting and kernel timing (tracing aid; not part of the paper).
 * Every kernel launch is counted per class.  While profiling is enabled, each
 * launch is bracketed by a CUDA event pair recorded on its own stream, so the
 * durations are device times of the kernels themselves (the event records
 * add a few microseconds per launch to a step).
 */
boltz_status boltz_profile_enable(boltz_grid g, int enable);

/*
 * launches: HOST long long [BOLTZ_KCLASS_COUNT] launches since the last reset;
 * ms:       HOST double [BOLTZ_KCLASS_COUNT] summed event durations in
 *           milliseconds of the profiled launches (waits for them to finish).
 * reset != 0 clears both afterwards.  Errors: BOLTZ_EINVAL, BOLTZ_ECUDA.
 */
boltz_status boltz_profile_read(boltz_grid g, int reset, long long* launches, double* ms);

/*
 * ---- Low-rank step consumers of the collision batch (paper Sec. 2, eqs.
 * "eqn:K-step detailed" and "eqn:L-step detailed"; Sec. 2.4, the fully
 * discrete scheme; Sec. 3.2, dropping basis).  They take no grid handle.
 * Functions of x or v are stored as rows ([r][n], r in 1..64); every pointer
 * is device memory; work is queued on `stream`.  Errors: BOLTZ_EINVAL
 * (ranges, NULL pointers), BOLTZ_ECUDA.
 *
 * K-step collision term:  C_out[j][x] = sum_{m,n} T[j][m][n] K[m][x] K[n][x]
 *   T  float32 [r][r][r] (boltz_project's T_out: T[j][m][n] = <V_j Q(V_m,V_n)>_v)
 *   K  float32 [r][n_x]  K_m(x) = sum_i X_i(x) S_im;  C_out float32 [r][n_x]
 */
boltz_status boltz_kstep_collision(const float* T, int r, const float* K, int n_x, float* C_out,
                                   void* stream);

/*
 * L-step collision term:  G_out[i][v] = sum_{p,q} C[i][p][q] Q[p r + q][v]
 *   Q  float32 [r*r][n_v]  (boltz_collide_batched over all ordered pairs (p, q))
 *   C  float32 [r][r][r]   C_ipq = sum_n (sum_m <X_i X_m X_n>_x S_mp) S_nq
 *   G_out float32 [r][n_v]
 */
boltz_status boltz_lstep_collision(const float* Q, int r, const float* C, int n_v, float* G_out,
                                   void* stream);

/*
 * r^4 couplings of the S- and L-steps (Sec. 2.4, S-step (a), L-step (b)):
 *   C_out[i][p][q] = sum_n ( sum_m E[i][m][n] S[m][p] ) S[n][q]
 *   and, when T is not NULL, the S-step collision term
 *   D_out[i][j] = sum_{m,n} T[j][m][n] C_out[i][m][n]
 *               = sum_{m,n} T_jmn sum_l ( sum_k E_ikl S_km ) S_ln.
 *   E  float32 [r][r][r]  E_imn = <X_i X_m X_n>_x;  S float32 [r][r]
 *   T  float32 [r][r][r] or NULL;  C_out float32 [r][r][r];  D_out float32 [r][r]
 * C_out is the coupling boltz_lstep_collision takes.
 */
boltz_status boltz_lowrank_coupling(const float* E, const float* S, int r, const float* T,
                                    float* C_out, float* D_out, void* stream);

/*
 * QR of the K- and L-steps in FP64 (Cholesky-QR2: Gram matrix, Cholesky
 * factor and triangular solve, done twice):  W_j = sum_i Y_i R[i][j] with
 * w sum_x Y_i(x) Y_k(x) = delta_ik (w = the midpoint-rule cell volume) and R
 * upper triangular with a positive diagonal.  For the K-step X = Y, S = R;
 * for the L-step (L_i = sum_j S_ij V_j) V = Y, S = R^T.
 *   W, Y       float64 [r][n] (Y may equal W), n >= r
 *   R          float64 [r][r] row-major
 *   workspace  device bytes from boltz_qr_f64_workspace(r, n)
 *   info       int32: 0, or k + 1 when the k-th pivot was not positive
 *              (the functions are linearly dependent to working precision;
 *              Y and R are then NaN)
 */
boltz_status boltz_qr_f64_workspace(int r, int n, size_t* bytes);
boltz_status boltz_qr_f64(const double* W, int r, int n, double w, double* Y, double* R,
                          void* workspace, int* info, void* stream);

/*
 * Rank truncation of Sec. 3.2 in FP64: S = U diag(sigma) Q^T with sigma
 * descending (one-sided Jacobi), r_keep = the number of sigma >= drop_tol.
 *   S, U, Q  float64 [r][r] row-major (columns of U and Q are the singular
 *            vectors; a column whose sigma is 0 is returned as zeros in U)
 *   sigma    float64 [r];  r_keep, info int32 (info 0 = converged, 1 = the
 *            sweep limit was reached)
 * Then X_bar = X U[:, :r_keep], V_bar = V Q[:, :r_keep] (boltz_basis_rotate_f64)
 * and S_bar = diag(sigma[:r_keep]).
 */
boltz_status boltz_svd_truncate_f64(const double* S, int r, double drop_tol, double* U, double* sigma,
                                    double* Q, int* r_keep, int* info, void* stream);

/*
 * Basis rotation:  X_out[k][x] = sum_i X[i][x] U[i][k], k < r_new <= r.
 *   X float64 [r][n], U float64 [r][r] row-major, X_out float64 [r_new][n]
 *   (must not alias X).
 */
boltz_status boltz_basis_rotate_f64(const double* X, int r, int n, const double* U, int r_new,
                                    double* X_out, void* stream);

/*
 * 1D normal shock solved end to end (paper Sec. 4 problem; Sec. 2.3 upwind
 * transport and projected inflow boundary; Sec. 2.4 fully discrete K-S-L
 * scheme; Sec. 3 adding and dropping basis).  x in [-L_x, L_x] with n_x
 * cells, the velocity grid and collision operator of `g` (form as in
 * boltz_collide_batched), inflow f = f_L for v_1 > 0 at the left end and
 * f = f_R for v_1 < 0 at the right end.  All state is FP64 on the device;
 * the collision terms come from the FP32 collision batch.
 *   boltz_shock_create   f_L, f_R HOST float64 [N^d] (values on the grid);
 *                        r_max in 3..64 bounds the rank after adding the
 *                        boundary basis (r + 2 <= r_max).  Allocates the
 *                        solver's device workspace once.
 *   boltz_shock_full_step  n_steps forward-Euler steps of the full-tensor
 *                        upwind scheme: f DEVICE float64 [n_x][N^d], in place.
 *   boltz_shock_lowrank_step  one adaptive low-rank step: X DEVICE float64
 *                        [r_max][n_x], S DEVICE float64 [r][r] (packed, room
 *                        for r_max^2), V DEVICE float64 [r_max][N^d], *r (HOST)
 *                        the rank in and out; f = sum_ij X_i S_ij V_j with
 *                        dx sum X_i X_k = delta, dv^d sum V_j V_l = delta.
 *                        Adds the boundary Maxwellians to V (Gram-Schmidt,
 *                        twice; a vector keeping under 1e-10 of its norm is
 *                        already in span(V) and is not added), K-, S- and
 *                        L-steps with FP64 Cholesky-QR2, then keeps the
 *                        singular values of S >= drop_tol.  *err (HOST,
 *                        may be NULL) receives ||f^{n+1} - f^n||_{x,v} before
 *                        the drop, from the K, S and L increments and their
 *                        cross terms (Sec. 5.1, eqs. "err low rank1-2"): the
 *                        paper's convergence measure, and its drop_tol =
 *                        c err rule when passed back.  Synchronises `stream`
 *                        (the new rank is read back).  A step called again
 *                        with the same rank, X, S, V pointers and dt, with
 *                        both boundary vectors kept, is captured once as a
 *                        CUDA graph (on a stream of its own) and replayed:
 *                        one host synchronisation per step instead of three
 *                        and no per-kernel launch cost, the same kernels in
 *                        the same order (the same results).  The graph is
 *                        captured again when the grid's workspace moved; a
 *                        replay that finds a boundary vector in span(V)
 *                        writes nothing and the step runs directly, as do
 *                        later steps on those buffers.  The environment
 *                        variable BOLTZ_SHOCK_GRAPH=0 (read at every call)
 *                        turns replays off; so do BOLTZ_FAULT and profiling.
 *   boltz_shock_reconstruct  f DEVICE float64 [n_x][N^d] = X^T S V.
 * Errors: BOLTZ_EINVAL (sizes, r + 2 > r_max or > n_x, non-finite dt),
 * BOLTZ_ENONFINITE (a QR met linearly dependent rows; the factors are then
 * left unchanged), BOLTZ_ENOMEM,
 * BOLTZ_ECUDA.
 */
typedef struct boltz_shock_s* boltz_shock;
boltz_status boltz_shock_create(boltz_grid g, int n_x, double L_x, const double* f_L, const double* f_R,
                                int r_max, int form, boltz_shock* out);
boltz_status boltz_shock_destroy(boltz_shock s);
boltz_status boltz_shock_full_step(boltz_shock s, double* f, int n_steps, double dt, void* stream);
boltz_status boltz_shock_lowrank_step(boltz_shock s, double* X, double* S, double* V, int* r, double dt,
                                      double drop_tol, double* err, void* stream);
boltz_status boltz_shock_reconstruct(boltz_shock s, const double* X, const double* S, const double* V, int r,
                                     double* f, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* BOLTZ_H */
