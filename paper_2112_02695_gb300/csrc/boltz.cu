// C ABI of the GB300 fast-spectral collision library (see include/boltz.h).
//
// Host side: grid creation (quadrature, FP64 tables rounded once to FP32),
// batch planning (chunks of inputs, gain slots, contraction tiles, radial
// node blocks), workspace management and kernel launches.  Every step of the
// collision evaluation runs in the kernels of kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <tuple>
#include <type_traits>
#include <utility>
#include <vector>

#include "boltz.h"
#include "kernels.cuh"
#include "lowrank.cuh"
#include "pencil.cuh"
#include "quadrature.hpp"
#include "shock.cuh"
#include "split.cuh"
#include "tc_kernels.cuh"
#include "wide2d.cuh"

using namespace boltz_dev;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr size_t kDefaultWorkspace = size_t(8) << 30;    // hard cap
constexpr size_t kFieldBudget = size_t(96) << 20;        // shifted fields per radial block

#define BZ_CUDA(call)                                  \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return BOLTZ_ECUDA;     \
    } while (0)

// ------------------------------------------------------------------ plan

struct ChunkPlan {
    std::vector<int> inputs;                      // chunk-local -> global input
    std::vector<Tile> tiles[3];                   // TRI16/TRI8, FULL16/FULL8, LIST16
    int tile_T = 16;                              // block width of TRI/FULL tiles
    std::vector<int> out_start;                   // [U+1]
    std::vector<int4> outs;                       // (e, jloc, lloc, 0)
    int U = 0;
    int split = 1;                                // Carleman form: direction splits of the contraction
    // offsets of this chunk's descriptors inside the device plan buffer (bytes)
    size_t off_inputs = 0, off_tiles[3] = {0, 0, 0}, off_start = 0, off_outs = 0;
};

struct Plan {
    std::vector<ChunkPlan> chunks;
    int nq = 1;
    int max_nc = 0, max_U = 0;
    size_t plan_bytes = 0;
    // workspace layout (byte offsets)
    size_t off_plan = 0, off_A = 0, off_P = 0, off_qhat = 0, off_fN = 0, off_lam = 0, off_img = 0, total = 0;
    // pipelined schedule (pencil.cuh): chunks of at most 16 inputs, gain
    // slots in TRI16 numbering, Qhat+ and the output lists over each chunk's
    // used slots only.  Chunks of one shape share a launch: an entry of
    // `chunks` is then one launch, its inputs and output slots chunk after
    // chunk (U = chunks x used slots per chunk).
    bool pencil = false;
    std::vector<char> pen_blob;           // direction tree + slot lists (device image)
    size_t off_pen_blob = 0, off_X = 0, off_Pt = 0, off_ctr = 0, off_qstd = 0;
    size_t pen_off[8] = {};               // offsets inside the blob: grp, s0_dir, s0_child,
                                          // s01_dir, step_blk, step_dir, step_sel, step_w
    std::vector<int> pen_nchunk;          // per launch: its chunks
    std::vector<size_t> pen_slot_off;     // per launch: its chunks' used-slot list inside the blob
    std::vector<std::array<unsigned, 5>> pen_mask;   // per launch: used TRI16 slots as a bit set
    std::vector<char> pen_diag;           // per launch: every used slot is a diagonal (j, j)
};

// Direction structure of a 3D rule for the pipelined schedule: the distinct
// sigma_0 values (grouped into tree items), the distinct (sigma_0, sigma_1)
// values below each (one X block each), and the steps of the fused items
// (two antipodal pairs each), see pencil.cuh.
struct PencilTree {
    bool ok = false;
    int n_s0 = 0, n_s01 = 0, n_grp = 0;
    std::vector<int> grp, s0_dir, s0_child, s01_dir;
    std::vector<int4> step_blk, step_dir, step_sel;
    std::vector<float2> step_w;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

struct boltz_grid_s {
    int N = 0, D = 0, n_rho = 0, M = 0, device = 0, sms = 1;
    double L = 0, R = 0, gamma = 0, b = 0;
    int n = 0, half = 0, smax = 0;
    std::vector<double> rho, w_rho;
    boltz::DirectionRule dir;
    // device tables
    float2* d_phase = nullptr;   // [(n_rho*M + 1)][D][N]
    float* d_ctab = nullptr;     // [n_rho][smax+1]
    float* d_gm = nullptr;       // [smax+1]
    float* d_gmf = nullptr;      // [half] per-mode loss weight (mass-consistent loss), else null
    float* d_w = nullptr;        // [M/2] weight of each antipodal direction pair
    int2* d_dpair = nullptr;     // [M/2] (p, antipode(p)), p < antipode(p)
    // the same tables unrounded, for the FP64 check build (small grids only)
    double2* d_phase64 = nullptr;
    double* d_ctab64 = nullptr;
    double* d_gm64 = nullptr;
    double* d_gmf64 = nullptr;
    double* d_w64 = nullptr;
    // split-precision form: per-node BF16 shift matrices (built on first use)
    uint8_t* d_smat = nullptr;
    double* d_scalar = nullptr;       // small device results read back by the host (Mott-Smith alpha)
    // Carleman form (gamma = d - 2): per-mode multipliers of the M/2 half-sphere
    // directions (g side, then f side), the per-mode loss table, weights and slot pairs
    float* d_cm_mult = nullptr;       // [M][half]
    float* d_cm_gm = nullptr;         // [half]
    float* d_cm_w = nullptr;          // [M/2]
    int2* d_cm_dpair = nullptr;       // [M/2]
    int split_clusters = 1;           // resident clusters of the split kernel
    int schedule = BOLTZ_SCHEDULE_AUTO;
    int loss = BOLTZ_LOSS_EXACT;
    PencilTree pen_tree;              // 3D N = 32 only
    int pen_ctas = 0;                 // resident CTAs of the pipelined kernel
    int pen_ctas_diag = 0;            // the same for its diagonal-slot variant
    int* d_err = nullptr;        // device error word (bit kErrTimeout: a bounded wait gave up)
    // workspace
    char* d_ws = nullptr;
    size_t ws_cap = 0, ws_max = kDefaultWorkspace;
    size_t field_budget = kFieldBudget;   // shifted-field bytes per radial block (autotuned)
    // last plan (reused when the same pair list comes back)
    std::vector<int32_t> last_j, last_l;
    int last_form = -1, last_n_inputs = -1;
    size_t last_elem = 0;             // bytes per real of the cached plan (4 or 8)
    Plan last_plan;
    bool plan_uploaded = false;
    // side stream for the radial step and the events of the two-buffer pipeline
    cudaStream_t side = nullptr;
    cudaEvent_t ev_ready[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr}, ev_join = nullptr,
                ev_fork = nullptr;
    // profiling: launches per kernel class (always counted) and, when enabled,
    // an event pair around every launch on the launching stream
    bool prof_on = false;
    long long launches[BOLTZ_KCLASS_COUNT] = {};
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_events;
    std::vector<cudaEvent_t> event_pool;
};

namespace {

bool supported_shape(int N, int D) {
    if (D != 2 && D != 3) return false;
    return N == 8 || N == 16 || N == 24 || N == 32 || N == 48 || N == 64 || (D == 2 && N == 128);
}

// Shapes of the FP64 check build: single-CTA fields whose shifted-field
// voxel chunk is 256 (3D 8^3, 16^3; 2D 16^2, 32^2).
bool fp64_shape(int N, int D) { return D == 3 ? (N == 8 || N == 16) : (N == 16 || N == 32); }

// Shapes of the split-precision form: 3D 32^3 (one CTA per field)
// and 64^3 (clusters of 8 CTAs, 1/8 of the field each).
bool split_shape(int N, int D) { return D == 3 && (N == 32 || N == 64); }

#ifndef BOLTZ_SPLIT_CL32
#define BOLTZ_SPLIT_CL32 1
#endif
constexpr int kSplitCL32 = BOLTZ_SPLIT_CL32;   // CTAs per 32^3 field in the split form (1: measured faster than 2)
constexpr int kSplitCL64 = 8;

// Bytes of one pre-split input image (all CTAs' parts) of the split form.
size_t split_image_bytes(int N) {
    return N == 64 ? size_t(kSplitCL64) * SplitGeo<64, kSplitCL64>::A_BYTES
                   : size_t(kSplitCL32) * SplitGeo<32, kSplitCL32>::A_BYTES;
}

bool valid_form(int form) {
    return form == BOLTZ_FORM_BATCHED || form == BOLTZ_FORM_PLAIN || form == BOLTZ_FORM_SPLIT_BF16 ||
           form == BOLTZ_FORM_CARLEMAN;
}

// The Carleman form exists for gamma = d - 2 only; it is built for every
// shape but the 2D 128^2 grid (whose transforms use 4-lane line groups).
bool carleman_kernel(double gamma, int D) { return std::fabs(gamma - (D - 2)) < 1e-12; }
bool carleman_shape(int N, int D) { return !(D == 2 && N == 128); }

// voxels per chunk of the shifted-field layout (must match Geo<N, D>::VCH)
int voxel_chunk(int N, int D) {
    const int n = D == 3 ? N * N * N : N * N;
    return n < 256 ? n : (N % 3 == 0 ? 288 : 256);
}


// ---------------------------------------------------------------- planning

// Build the chunk/tile/slot structure of a batch.  BATCHED: unordered gain
// slots shared by (j,l) and (l,j), inputs shared by every pair in a chunk.
// PLAIN: every evaluation gets its own two inputs and its own slot.
// elem: bytes per real (4 for the FP32 path, 8 for the FP64 check build, whose
// triangle and full tiles are 8 wide to bound the accumulator registers).
boltz_status build_plan_carleman(const boltz_grid_s* g, const int32_t* pj, const int32_t* pl, int n_pairs,
                                 Plan& plan);

// Direction tree of a 3D rule for the pipelined schedule.  Components are
// compared exactly: the rules are built by permutations and sign changes of
// their generators, so equal components are equal bit for bit.
PencilTree build_pencil_tree(const boltz_grid_s* g) {
    namespace pc = boltz_dev::pencil;
    PencilTree T;
    const int M = g->M;
    const std::vector<double>& sg = g->dir.sigma;
    std::vector<double> v0;                           // distinct sigma_0
    std::vector<std::vector<double>> v1;              // distinct sigma_1 below each sigma_0
    std::vector<int> p0(M), p1(M);
    for (int p = 0; p < M; ++p) {
        const double a = sg[3 * p], b = sg[3 * p + 1];
        int i = (int)(std::find(v0.begin(), v0.end(), a) - v0.begin());
        if (i == (int)v0.size()) {
            v0.push_back(a);
            v1.emplace_back();
        }
        int k = (int)(std::find(v1[i].begin(), v1[i].end(), b) - v1[i].begin());
        if (k == (int)v1[i].size()) v1[i].push_back(b);
        p0[p] = i;
        p1[p] = k;
    }
    const int n0 = (int)v0.size();
    std::vector<int> rep0(n0, -1);
    std::vector<std::vector<int>> rep(n0);
    for (int i = 0; i < n0; ++i) rep[i].assign(v1[i].size(), -1);
    for (int p = 0; p < M; ++p) {
        if (rep0[p0[p]] < 0) rep0[p0[p]] = p;
        if (rep[p0[p]][p1[p]] < 0) rep[p0[p]][p1[p]] = p;
    }
    // tree items: sigma_0 values grouped by longest-first assignment of their
    // (1 + children) transform passes, about 16 passes per group (three groups
    // for the 38-point rule; measured faster than two or four)
    int total = 0, max_rows = 0;
    for (int i = 0; i < n0; ++i) {
        total += 1 + (int)v1[i].size();
        max_rows = std::max(max_rows, 1 + (int)v1[i].size());
    }
    if (max_rows > pc::MAX_ROWS) return T;
    const int ng = std::max(1, std::min(n0, (total + 15) / 16));
    std::vector<int> order(n0);
    for (int i = 0; i < n0; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return v1[a].size() > v1[b].size(); });
    std::vector<int> load(ng, 0);
    std::vector<std::vector<int>> bins(ng);
    for (int i : order) {
        const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        bins[b].push_back(i);
        load[b] += 1 + (int)v1[i].size();
    }
    std::map<std::pair<int, int>, int> s01_index;
    T.grp.push_back(0);
    for (int b = 0; b < ng; ++b) {
        for (int i : bins[b]) {
            T.s0_dir.push_back(rep0[i]);
            T.s0_child.push_back((int)T.s01_dir.size());
            for (int k = 0; k < (int)v1[i].size(); ++k) {
                s01_index[{i, k}] = (int)T.s01_dir.size();
                T.s01_dir.push_back(rep[i][k]);
            }
        }
        T.grp.push_back((int)T.s0_dir.size());
    }
    T.s0_child.push_back((int)T.s01_dir.size());
    T.n_s0 = n0;
    T.n_s01 = (int)T.s01_dir.size();
    T.n_grp = ng;
    std::vector<int> blk_of(M);
    for (int p = 0; p < M; ++p) blk_of[p] = s01_index[{p0[p], p1[p]}];
    // steps: two antipodal pairs each, pairs that read the same two X blocks together
    std::map<std::pair<int, int>, std::vector<int>> buckets;
    for (int p = 0; p < M; ++p) {
        const int pb = g->dir.antipode[p];
        if (p < pb) buckets[{std::min(blk_of[p], blk_of[pb]), std::max(blk_of[p], blk_of[pb])}].push_back(p);
    }
    std::vector<std::vector<int>> steps;
    std::vector<int> singles;
    for (auto& kv : buckets) {
        const std::vector<int>& v = kv.second;
        size_t i = 0;
        for (; i + 1 < v.size(); i += 2) steps.push_back({v[i], v[i + 1]});
        if (i < v.size()) singles.push_back(v[i]);
    }
    for (size_t i = 0; i < singles.size(); i += 2) {
        if (i + 1 < singles.size()) steps.push_back({singles[i], singles[i + 1]});
        else steps.push_back({singles[i]});
    }
    for (const auto& stp : steps) {
        int dirs[4] = {-1, -1, -1, -1}, blk[4] = {-1, -1, -1, -1}, sel[4] = {0, 0, 0, 0};
        float w[2] = {0.f, 0.f};
        for (size_t k = 0; k < stp.size(); ++k) {
            dirs[2 * k] = stp[k];
            dirs[2 * k + 1] = g->dir.antipode[stp[k]];
            w[k] = (float)g->dir.w[stp[k]];
        }
        int nb = 0;
        for (int d = 0; d < 4; ++d) {
            if (dirs[d] < 0) continue;
            const int x = blk_of[dirs[d]];
            int k = 0;
            while (k < nb && blk[k] != x) ++k;
            if (k == nb) blk[nb++] = x;
            sel[d] = k;
        }
        T.step_blk.push_back(make_int4(blk[0], blk[1], blk[2], blk[3]));
        T.step_dir.push_back(make_int4(dirs[0], dirs[1], dirs[2], dirs[3]));
        T.step_sel.push_back(make_int4(sel[0], sel[1], sel[2], sel[3]));
        T.step_w.push_back(make_float2(w[0], w[1]));
    }
    // the kernel keeps these tables in fixed-size shared arrays, and a tree
    // item stages the phase rows of its whole group
    bool rows_fit = true;
    for (int b = 0; b < ng; ++b) rows_fit = rows_fit && load[b] <= pc::MAX_ROWS;
    T.ok = !T.step_dir.empty() && T.n_s0 <= pc::MAX_S && T.n_s01 <= pc::MAX_S &&
           (int)T.step_dir.size() <= pc::MAX_STEP && rows_fit;
    return T;
}

// Chunks of the pipelined schedule: the inputs of every connected component
// of the pair graph (inputs joined by a pair) stay together, and components
// are packed largest first into chunks of at most 16 inputs (first fit), each
// chunk's inputs in ascending order.  False when a component has more than
// 16 inputs.
bool pencil_chunks(const int32_t* pj, const int32_t* pl, int n_pairs, std::vector<std::vector<int>>& chunks) {
    namespace pc = boltz_dev::pencil;
    std::map<int, int> parent;
    std::function<int(int)> find = [&](int a) {
        while (parent[a] != a) a = parent[a] = parent[parent[a]];
        return a;
    };
    for (int e = 0; e < n_pairs; ++e) {
        for (int v : {pj[e], pl[e]})
            if (!parent.count(v)) parent[v] = v;
        const int a = find(pj[e]), b = find(pl[e]);
        if (a != b) parent[std::max(a, b)] = std::min(a, b);
    }
    std::map<int, std::vector<int>> comp;
    for (auto& kv : parent) comp[find(kv.first)].push_back(kv.first);
    std::vector<std::vector<int>> cs;
    for (auto& kv : comp) {
        if ((int)kv.second.size() > pc::NJ) return false;
        cs.push_back(kv.second);
    }
    std::stable_sort(cs.begin(), cs.end(), [](const std::vector<int>& a, const std::vector<int>& b) {
        return a.size() > b.size();
    });
    chunks.clear();
    for (const auto& c : cs) {
        size_t k = 0;
        while (k < chunks.size() && chunks[k].size() + c.size() > (size_t)pc::NJ) ++k;
        if (k == chunks.size()) chunks.emplace_back();
        chunks[k].insert(chunks[k].end(), c.begin(), c.end());
    }
    for (auto& c : chunks) std::sort(c.begin(), c.end());
    return !chunks.empty();
}

// Whether a batch runs on the pipelined schedule: batched FP32 form on a 3D
// 32^3 grid whose tree was built, every connected group of inputs at most 16.
bool pencil_applies(const boltz_grid_s* g, const int32_t* pj, const int32_t* pl, int n_pairs, int form,
                    size_t elem) {
    if (form != BOLTZ_FORM_BATCHED || elem != 4 || g->D != 3 || g->N != 32 || !g->pen_tree.ok ||
        g->schedule != BOLTZ_SCHEDULE_AUTO || g->pen_ctas <= 0)
        return false;
    std::vector<std::vector<int>> chunks;
    return pencil_chunks(pj, pl, n_pairs, chunks);
}

// Chunks of one shape that share a persistent launch, at most this many: the
// launch's f_N, Lambda and Qhat+ grow with its chunks (about 9 MB each).
constexpr int kPenChunksPerLaunch = 64;

// Plan of the pipelined schedule: the inputs in chunks of at most 16, gain
// slot u = TRI16 index of the chunk-local pair, outputs listed per used slot
// (Qhat+ and the output kernel run over the used slots only).  Chunks with
// the same input count and used slots run in one persistent launch (its node
// list runs through the chunks one after another); the launches run in order
// and share the node buffers.  Workspace:
// descriptors | f_N, Lambda | X node buffers | Pt node buffers | Qhat+ | counters.
boltz_status build_plan_pencil(const boltz_grid_s* g, const int32_t* pj, const int32_t* pl, int n_pairs,
                               Plan& plan) {
    namespace pc = boltz_dev::pencil;
    plan = Plan();
    plan.pencil = true;
    std::vector<std::vector<int>> groups;
    if (!pencil_chunks(pj, pl, n_pairs, groups)) return BOLTZ_EINVAL;
    std::map<int, int> chunk_of, loc;
    for (int k = 0; k < (int)groups.size(); ++k)
        for (int i = 0; i < (int)groups[k].size(); ++i) {
            chunk_of[groups[k][i]] = k;
            loc[groups[k][i]] = i;
        }
    std::vector<std::vector<std::vector<int>>> outs_of(groups.size(), std::vector<std::vector<int>>(pc::NSLOT));
    for (int e = 0; e < n_pairs; ++e) {
        const int a = loc[pj[e]], b = loc[pl[e]];
        outs_of[chunk_of[pj[e]]][pc::tri_slot(std::min(a, b), std::max(a, b))].push_back(e);
    }
    // direction tree, then each chunk's slot list, as one blob (16-byte aligned tables)
    const PencilTree& T = g->pen_tree;
    std::vector<char>& blob = plan.pen_blob;
    auto put = [&](const void* src, size_t bytes) {
        const size_t at = align_up(blob.size(), 16);
        blob.resize(at + bytes);
        if (bytes) std::memcpy(blob.data() + at, src, bytes);
        return at;
    };
    plan.pen_off[0] = put(T.grp.data(), T.grp.size() * sizeof(int));
    plan.pen_off[1] = put(T.s0_dir.data(), T.s0_dir.size() * sizeof(int));
    plan.pen_off[2] = put(T.s0_child.data(), T.s0_child.size() * sizeof(int));
    plan.pen_off[3] = put(T.s01_dir.data(), T.s01_dir.size() * sizeof(int));
    plan.pen_off[4] = put(T.step_blk.data(), T.step_blk.size() * sizeof(int4));
    plan.pen_off[5] = put(T.step_dir.data(), T.step_dir.size() * sizeof(int4));
    plan.pen_off[6] = put(T.step_sel.data(), T.step_sel.size() * sizeof(int4));
    plan.pen_off[7] = put(T.step_w.data(), T.step_w.size() * sizeof(float2));
    std::vector<std::vector<int>> slots_of(groups.size());
    std::vector<std::array<unsigned, 5>> mask_of(groups.size());
    for (size_t k = 0; k < groups.size(); ++k) {
        mask_of[k].fill(0u);
        for (int u = 0; u < pc::NSLOT; ++u) {
            if (outs_of[k][u].empty()) continue;
            slots_of[k].push_back(u);
            mask_of[k][u >> 5] |= 1u << (u & 31);
        }
    }
    // launches: chunks of one shape, in the order of their first chunk
    std::vector<std::vector<int>> launches;
    for (int k = 0; k < (int)groups.size(); ++k) {
        int at = -1;
        for (int j = 0; j < (int)launches.size() && at < 0; ++j) {
            const int k0 = launches[j][0];
            if ((int)launches[j].size() < kPenChunksPerLaunch && groups[k0].size() == groups[k].size() &&
                mask_of[k0] == mask_of[k])
                at = j;
        }
        if (at < 0) {
            at = (int)launches.size();
            launches.emplace_back();
        }
        launches[at].push_back(k);
    }
    for (const auto& ln : launches) {
        ChunkPlan c;
        const int nc = (int)groups[ln[0]].size();
        const std::vector<int>& slots = slots_of[ln[0]];
        for (int k : ln) c.inputs.insert(c.inputs.end(), groups[k].begin(), groups[k].end());
        for (int ci = 0; ci < (int)ln.size(); ++ci)
            for (int u : slots) {
                c.out_start.push_back((int)c.outs.size());
                for (int e : outs_of[ln[ci]][u])
                    c.outs.push_back(make_int4(e, ci * nc + loc[pj[e]], ci * nc + loc[pl[e]], 0));
            }
        c.out_start.push_back((int)c.outs.size());
        c.U = (int)(ln.size() * slots.size());
        bool diag = true;
        for (int u : slots) {
            bool on_diagonal = false;
            for (int a = 0; a < pc::NJ; ++a) on_diagonal = on_diagonal || u == pc::tri_slot(a, a);
            diag = diag && on_diagonal;
        }
        plan.pen_nchunk.push_back((int)ln.size());
        plan.pen_diag.push_back(diag);
        plan.pen_slot_off.push_back(put(slots.data(), slots.size() * sizeof(int)));
        plan.pen_mask.push_back(mask_of[ln[0]]);
        plan.max_nc = std::max(plan.max_nc, (int)c.inputs.size());
        plan.max_U = std::max(plan.max_U, c.U);
        plan.chunks.push_back(std::move(c));
    }
    blob.resize(align_up(blob.size(), 16));
    plan.nq = g->n_rho;
    size_t off = 0;
    for (auto& c : plan.chunks) {
        c.off_inputs = off;
        off = align_up(off + c.inputs.size() * sizeof(int), 256);
        for (int k = 0; k < 3; ++k) c.off_tiles[k] = off;
        c.off_start = off;
        off = align_up(off + c.out_start.size() * sizeof(int), 256);
        c.off_outs = off;
        off = align_up(off + c.outs.size() * sizeof(int4), 256);
    }
    plan.off_pen_blob = off;
    off = align_up(off + blob.size(), 256);
    plan.plan_bytes = off;
    const int nc = plan.max_nc;
    const size_t field_bytes = size_t(g->n) * 4;
    size_t w = align_up(off, 256);
    plan.off_plan = 0;
    plan.off_fN = w;                       // f_N [nc][n] then Lambda [nc][n]
    w = align_up(w + size_t(nc) * field_bytes, 256);
    plan.off_lam = w;
    w = align_up(w + size_t(nc) * field_bytes, 256);
    plan.off_X = w;
    w = align_up(w + size_t(pc::NXB) * T.n_s01 * pc::NLB * pc::XBLK * sizeof(float2), 256);
    plan.off_Pt = w;
    w = align_up(w + size_t(pc::NPB) * pc::NSLOT * pc::NKB * pc::PLANE * sizeof(float2), 256);
    plan.off_qhat = w;                     // packed running sums, then the final sums (standard layout)
    w = align_up(w + size_t(plan.max_U) * pc::NKB * pc::QBLK * sizeof(float2), 256);
    plan.off_qstd = w;
    w = align_up(w + size_t(plan.max_U) * pc::HALF * sizeof(float2), 256);
    plan.off_ctr = w;
    int max_nodes = 0;
    for (int n : plan.pen_nchunk) max_nodes = std::max(max_nodes, n * g->n_rho);
    w = align_up(w + size_t(pc::ctr_count(max_nodes, plan.max_U)) * sizeof(int), 256);
    plan.off_A = plan.off_P = plan.off_img = w;
    plan.total = w;
    return BOLTZ_OK;
}

boltz_status build_plan(const boltz_grid_s* g, int n_inputs, const int32_t* pj, const int32_t* pl, int n_pairs,
                        int form, Plan& plan, size_t elem = 4) {
    if (form == BOLTZ_FORM_CARLEMAN) return build_plan_carleman(g, pj, pl, n_pairs, plan);
    if (pencil_applies(g, pj, pl, n_pairs, form, elem)) return build_plan_pencil(g, pj, pl, n_pairs, plan);
    plan = Plan();
    const size_t field_bytes = size_t(g->n) * elem;
    // inputs per chunk: enough for one radial node's shifted fields to fit the L2-sized
    // budget, but never fewer than 16 (a rank-16 basis stays in one chunk, so its
    // shifted fields are computed once) nor more than 64
    int nc_cap = (int)std::max<size_t>(16, g->field_budget / (field_bytes * g->M));
    nc_cap = std::min(nc_cap, 64);
    if (form == BOLTZ_FORM_PLAIN) {
        const int E = std::max(1, nc_cap / 2);
        for (int e0 = 0; e0 < n_pairs; e0 += E) {
            ChunkPlan c;
            const int ne = std::min(E, n_pairs - e0);
            for (int e = 0; e < ne; ++e) {
                c.inputs.push_back(pj[e0 + e]);
                c.inputs.push_back(pl[e0 + e]);
            }
            for (int t0 = 0; t0 < ne; t0 += 16) {
                Tile t;
                std::memset(&t, 0, sizeof(t));
                t.slot0 = t0;
                t.count = std::min(16, ne - t0);
                for (int i = 0; i < 16; ++i) {
                    const int e = t0 + std::min(i, t.count - 1);
                    t.ja[i] = 2 * e;
                    t.lb[i] = 2 * e + 1;
                }
                c.tiles[TILE_LIST].push_back(t);
            }
            c.U = ne;
            c.out_start.resize(ne + 1);
            for (int e = 0; e < ne; ++e) {
                c.out_start[e] = e;
                c.outs.push_back(make_int4(e0 + e, 2 * e, 2 * e + 1, 0));
            }
            c.out_start[ne] = ne;
            plan.chunks.push_back(std::move(c));
        }
    } else {
        // unordered slots in first-appearance order, with their ordered outputs
        std::map<std::pair<int, int>, int> slot_of;
        std::vector<std::pair<int, int>> slots;
        std::vector<std::vector<std::pair<int, int>>> slot_outs;   // (e, which-first)
        for (int e = 0; e < n_pairs; ++e) {
            const int a = std::min(pj[e], pl[e]), b = std::max(pj[e], pl[e]);
            auto it = slot_of.find({a, b});
            int s;
            if (it == slot_of.end()) {
                s = (int)slots.size();
                slot_of[{a, b}] = s;
                slots.push_back({a, b});
                slot_outs.emplace_back();
            } else {
                s = it->second;
            }
            slot_outs[s].push_back({e, 0});
        }
        // greedy chunking by input set
        std::vector<std::vector<int>> chunk_slots;
        std::vector<std::set<int>> chunk_inputs;
        for (int s = 0; s < (int)slots.size(); ++s) {
            const int a = slots[s].first, b = slots[s].second;
            bool placed = false;
            if (!chunk_slots.empty()) {
                std::set<int>& cur = chunk_inputs.back();
                int grow = (cur.count(a) ? 0 : 1) + (a != b && !cur.count(b) ? 1 : 0);
                if ((int)cur.size() + grow <= nc_cap) {
                    cur.insert(a);
                    cur.insert(b);
                    chunk_slots.back().push_back(s);
                    placed = true;
                }
            }
            if (!placed) {
                chunk_slots.push_back({s});
                chunk_inputs.push_back({a, b});
            }
        }
        for (size_t ci = 0; ci < chunk_slots.size(); ++ci) {
            ChunkPlan c;
            c.inputs.assign(chunk_inputs[ci].begin(), chunk_inputs[ci].end());
            std::map<int, int> loc;
            for (int i = 0; i < (int)c.inputs.size(); ++i) loc[c.inputs[i]] = i;
            const int nc = (int)c.inputs.size();
            // local pair set
            std::map<std::pair<int, int>, int> local;   // (ja <= lb) -> global slot id
            for (int s : chunk_slots[ci]) local[{loc[slots[s].first], loc[slots[s].second]}] = s;
            const int T = (nc >= 16 && elem == 4) ? 16 : 8;
            c.tile_T = T;
            std::vector<std::pair<int, int>> order;     // local slot order
            std::set<std::pair<int, int>> covered;
            auto new_tile = [&](int kind, int j0, int l0, int tj, int tl_) {
                Tile t;
                std::memset(&t, 0, sizeof(t));
                t.slot0 = (int)order.size();
                t.j0 = j0;
                t.l0 = l0;
                for (int x = 0; x < tj; ++x)
                    for (int y = (kind == TILE_TRI ? x : 0); y < tl_; ++y) {
                        order.push_back({j0 + x, l0 + y});
                        covered.insert({j0 + x, l0 + y});
                    }
                t.count = (int)order.size() - t.slot0;
                c.tiles[kind].push_back(t);
            };
            if (nc >= 8) {
                const int nb = nc / T;                  // full-width blocks only
                for (int J = 0; J < nb; ++J) {
                    for (int Lb = J; Lb < nb; ++Lb) {
                        bool full = true;
                        for (int x = 0; x < T && full; ++x)
                            for (int y = (J == Lb ? x : 0); y < T && full; ++y)
                                full = local.count({J * T + x, Lb * T + y}) > 0;
                        if (!full) continue;
                        if (J == Lb) {
                            new_tile(TILE_TRI, J * T, J * T, T, T);
                        } else {
                            // off-diagonal block as 8-row strips (8 x T accumulators per thread)
                            for (int x0 = 0; x0 < T; x0 += 8) new_tile(TILE_FULL, J * T + x0, Lb * T, 8, T);
                        }
                    }
                }
            }
            std::vector<std::pair<int, int>> rest;
            for (auto& kv : local)
                if (!covered.count(kv.first)) rest.push_back(kv.first);
            for (size_t t0 = 0; t0 < rest.size(); t0 += 16) {
                Tile t;
                std::memset(&t, 0, sizeof(t));
                t.slot0 = (int)order.size();
                t.count = (int)std::min<size_t>(16, rest.size() - t0);
                for (int i = 0; i < 16; ++i) {
                    const auto& pr = rest[t0 + std::min(i, t.count - 1)];
                    t.ja[i] = pr.first;
                    t.lb[i] = pr.second;
                }
                for (int i = 0; i < t.count; ++i) order.push_back(rest[t0 + i]);
                c.tiles[TILE_LIST].push_back(t);
            }
            c.U = (int)order.size();
            c.out_start.resize(c.U + 1);
            for (int u = 0; u < c.U; ++u) {
                c.out_start[u] = (int)c.outs.size();
                const int s = local[order[u]];
                for (auto& eo : slot_outs[s]) {
                    const int e = eo.first;
                    c.outs.push_back(make_int4(e, loc[pj[e]], loc[pl[e]], 0));
                }
            }
            c.out_start[c.U] = (int)c.outs.size();
            plan.chunks.push_back(std::move(c));
        }
    }
    // sizes
    for (auto& c : plan.chunks) {
        plan.max_nc = std::max(plan.max_nc, (int)c.inputs.size());
        plan.max_U = std::max(plan.max_U, c.U);
    }
    const size_t per_node = size_t(g->M) * plan.max_nc * field_bytes + size_t(plan.max_U) * field_bytes;
    plan.nq = (int)std::max<size_t>(1, std::min<size_t>(g->n_rho, g->field_budget / std::max<size_t>(per_node, 1)));
    // device plan descriptors
    size_t off = 0;
    for (auto& c : plan.chunks) {
        c.off_inputs = off;
        off = align_up(off + c.inputs.size() * sizeof(int), 256);
        for (int k = 0; k < 3; ++k) {
            c.off_tiles[k] = off;
            off = align_up(off + c.tiles[k].size() * sizeof(Tile), 256);
        }
        c.off_start = off;
        off = align_up(off + c.out_start.size() * sizeof(int), 256);
        c.off_outs = off;
        off = align_up(off + c.outs.size() * sizeof(int4), 256);
    }
    plan.plan_bytes = off;
    size_t w = align_up(off, 256);
    plan.off_plan = 0;
    plan.off_A = w;
    w = align_up(w + size_t(plan.nq) * g->M * plan.max_nc * field_bytes, 256);
    plan.off_P = w;       // two buffers: the radial step of one node block overlaps the next block
    w = align_up(w + 2 * size_t(plan.nq) * plan.max_U * field_bytes, 256);
    plan.off_qhat = w;
    w = align_up(w + size_t(plan.max_U) * g->half * 2 * elem, 256);
    plan.off_fN = w;
    w = align_up(w + size_t(plan.max_nc) * field_bytes, 256);
    plan.off_lam = w;
    w = align_up(w + size_t(plan.max_nc) * field_bytes, 256);
    plan.off_img = w;     // pre-split inputs of the split-precision form
    if (form == BOLTZ_FORM_SPLIT_BF16) w = align_up(w + size_t(plan.max_nc) * split_image_bytes(g->N), 256);
    plan.total = w;
    return BOLTZ_OK;
}

// Plan of the Carleman form: every distinct ordered pair (j, l) has its own
// gain slot (the form is not symmetric in g and f); chunks of inputs as in the
// batched form; complete T x T blocks of ordered pairs become FULL strips of
// 8 x T, the rest LIST tiles of 16; one slot group of M fields per input
// (M/2 g-side and M/2 f-side multipliers).
boltz_status build_plan_carleman(const boltz_grid_s* g, const int32_t* pj, const int32_t* pl, int n_pairs,
                                 Plan& plan) {
    plan = Plan();
    const size_t field_bytes = size_t(g->n) * 4;
    int nc_cap = (int)std::max<size_t>(16, g->field_budget / (field_bytes * g->M));
    nc_cap = std::min(nc_cap, 64);
    std::map<std::pair<int, int>, int> slot_of;
    std::vector<std::pair<int, int>> slots;
    std::vector<std::vector<int>> slot_outs;
    for (int e = 0; e < n_pairs; ++e) {
        auto it = slot_of.find({pj[e], pl[e]});
        int s;
        if (it == slot_of.end()) {
            s = (int)slots.size();
            slot_of[{pj[e], pl[e]}] = s;
            slots.push_back({pj[e], pl[e]});
            slot_outs.emplace_back();
        } else {
            s = it->second;
        }
        slot_outs[s].push_back(e);
    }
    std::vector<std::vector<int>> chunk_slots;
    std::vector<std::set<int>> chunk_inputs;
    for (int s = 0; s < (int)slots.size(); ++s) {
        const int a = slots[s].first, b = slots[s].second;
        bool placed = false;
        if (!chunk_slots.empty()) {
            std::set<int>& cur = chunk_inputs.back();
            const int grow = (cur.count(a) ? 0 : 1) + (a != b && !cur.count(b) ? 1 : 0);
            if ((int)cur.size() + grow <= nc_cap) {
                cur.insert(a);
                cur.insert(b);
                chunk_slots.back().push_back(s);
                placed = true;
            }
        }
        if (!placed) {
            chunk_slots.push_back({s});
            chunk_inputs.push_back({a, b});
        }
    }
    for (size_t ci = 0; ci < chunk_slots.size(); ++ci) {
        ChunkPlan c;
        c.inputs.assign(chunk_inputs[ci].begin(), chunk_inputs[ci].end());
        std::map<int, int> loc;
        for (int i = 0; i < (int)c.inputs.size(); ++i) loc[c.inputs[i]] = i;
        const int nc = (int)c.inputs.size();
        std::map<std::pair<int, int>, int> local;       // ordered local pair -> global slot
        for (int s : chunk_slots[ci]) local[{loc[slots[s].first], loc[slots[s].second]}] = s;
        const int T = nc >= 16 ? 16 : 8;
        c.tile_T = T;
        std::vector<std::pair<int, int>> order;
        std::set<std::pair<int, int>> covered;
        if (nc >= 8) {
            const int nb = nc / T;
            for (int J = 0; J < nb; ++J)
                for (int Lb = 0; Lb < nb; ++Lb) {
                    bool full = true;
                    for (int x = 0; x < T && full; ++x)
                        for (int y = 0; y < T && full; ++y) full = local.count({J * T + x, Lb * T + y}) > 0;
                    if (!full) continue;
                    for (int x0 = 0; x0 < T; x0 += 8) {
                        Tile t;
                        std::memset(&t, 0, sizeof(t));
                        t.slot0 = (int)order.size();
                        t.j0 = J * T + x0;
                        t.l0 = Lb * T;
                        for (int x = 0; x < 8; ++x)
                            for (int y = 0; y < T; ++y) {
                                order.push_back({t.j0 + x, t.l0 + y});
                                covered.insert({t.j0 + x, t.l0 + y});
                            }
                        t.count = 8 * T;
                        c.tiles[TILE_FULL].push_back(t);
                    }
                }
        }
        std::vector<std::pair<int, int>> rest;
        for (auto& kv : local)
            if (!covered.count(kv.first)) rest.push_back(kv.first);
        for (size_t t0 = 0; t0 < rest.size(); t0 += 16) {
            Tile t;
            std::memset(&t, 0, sizeof(t));
            t.slot0 = (int)order.size();
            t.count = (int)std::min<size_t>(16, rest.size() - t0);
            for (int i = 0; i < 16; ++i) {
                const auto& pr = rest[t0 + std::min(i, t.count - 1)];
                t.ja[i] = pr.first;
                t.lb[i] = pr.second;
            }
            for (int i = 0; i < t.count; ++i) order.push_back(rest[t0 + i]);
            c.tiles[TILE_LIST].push_back(t);
        }
        c.U = (int)order.size();
        c.out_start.resize(c.U + 1);
        for (int u = 0; u < c.U; ++u) {
            c.out_start[u] = (int)c.outs.size();
            for (int e : slot_outs[local[order[u]]]) c.outs.push_back(make_int4(e, loc[pj[e]], loc[pl[e]], 0));
        }
        c.out_start[c.U] = (int)c.outs.size();
        plan.chunks.push_back(std::move(c));
    }
    // a chunk of few voxel-chunk x tile blocks splits the direction pairs over
    // up to 8 blocks (at least two pairs each) to fill more SMs; the partial
    // sums are added by the output kernel
    size_t max_pu = 0;
    for (auto& c : plan.chunks) {
        plan.max_nc = std::max(plan.max_nc, (int)c.inputs.size());
        plan.max_U = std::max(plan.max_U, c.U);
        const long long blocks =
            (long long)(g->n / voxel_chunk(g->N, g->D)) * (long long)(c.tiles[TILE_FULL].size() + c.tiles[TILE_LIST].size());
        c.split = (int)std::max<long long>(1, std::min<long long>({8, (long long)(g->M / 2) / 2, 152 / std::max(1LL, blocks)}));
        max_pu = std::max(max_pu, (size_t)c.split * c.U);
    }
    plan.nq = 1;
    size_t off = 0;
    for (auto& c : plan.chunks) {
        c.off_inputs = off;
        off = align_up(off + c.inputs.size() * sizeof(int), 256);
        for (int k = 0; k < 3; ++k) {
            c.off_tiles[k] = off;
            off = align_up(off + c.tiles[k].size() * sizeof(Tile), 256);
        }
        c.off_start = off;
        off = align_up(off + c.out_start.size() * sizeof(int), 256);
        c.off_outs = off;
        off = align_up(off + c.outs.size() * sizeof(int4), 256);
    }
    plan.plan_bytes = off;
    size_t w = align_up(off, 256);
    plan.off_plan = 0;
    plan.off_A = w;
    w = align_up(w + size_t(g->M) * plan.max_nc * field_bytes, 256);
    plan.off_P = w;
    w = align_up(w + max_pu * field_bytes, 256);
    plan.off_qhat = w;
    plan.off_fN = w;
    w = align_up(w + size_t(plan.max_nc) * field_bytes, 256);
    plan.off_lam = w;
    w = align_up(w + size_t(plan.max_nc) * field_bytes, 256);
    plan.off_img = w;
    plan.total = w;
    return BOLTZ_OK;
}

// Host-side fault injection for the error paths (environment variable
// BOLTZ_FAULT, read at every call): "alloc" fails every workspace allocation
// with BOLTZ_ENOMEM, "badplan" makes batch planning reject every batch with
// BOLTZ_EINVAL, "nan" marks every queued collision batch as having written a
// non-finite value (boltz_sync_status then reports BOLTZ_ENONFINITE).
// Nothing is injected on the device.
bool fault_injected(const char* what) {
    const char* v = std::getenv("BOLTZ_FAULT");
    return v && std::strcmp(v, what) == 0;
}

boltz_status ensure_workspace(boltz_grid_s* g, size_t bytes, cudaStream_t stream) {
    if (bytes <= g->ws_cap) return BOLTZ_OK;
    if (bytes > g->ws_max || fault_injected("alloc")) return BOLTZ_ENOMEM;
    if (g->d_ws) {
        BZ_CUDA(cudaStreamSynchronize(stream));
        BZ_CUDA(cudaFree(g->d_ws));
        g->d_ws = nullptr;
        g->ws_cap = 0;
    }
    const size_t cap = align_up(bytes + bytes / 8, size_t(1) << 20);
    cudaError_t e = cudaMalloc(&g->d_ws, cap);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        g->d_ws = nullptr;
        return BOLTZ_ENOMEM;
    }
    g->ws_cap = cap;
    g->plan_uploaded = false;
    return BOLTZ_OK;
}

boltz_status upload_plan(boltz_grid_s* g, const Plan& plan, cudaStream_t stream) {
    std::vector<char> host(plan.plan_bytes, 0);
    for (const auto& c : plan.chunks) {
        std::memcpy(host.data() + c.off_inputs, c.inputs.data(), c.inputs.size() * sizeof(int));
        for (int k = 0; k < 3; ++k)
            if (!c.tiles[k].empty())
                std::memcpy(host.data() + c.off_tiles[k], c.tiles[k].data(), c.tiles[k].size() * sizeof(Tile));
        std::memcpy(host.data() + c.off_start, c.out_start.data(), c.out_start.size() * sizeof(int));
        if (!c.outs.empty()) std::memcpy(host.data() + c.off_outs, c.outs.data(), c.outs.size() * sizeof(int4));
    }
    if (plan.pencil && !plan.pen_blob.empty())
        std::memcpy(host.data() + plan.off_pen_blob, plan.pen_blob.data(), plan.pen_blob.size());
    if (plan.plan_bytes) {
        BZ_CUDA(cudaMemcpyAsync(g->d_ws + plan.off_plan, host.data(), plan.plan_bytes, cudaMemcpyHostToDevice, stream));
        BZ_CUDA(cudaStreamSynchronize(stream));   // host staging buffer goes out of scope
    }
    return BOLTZ_OK;
}

// ---------------------------------------------------------------- profiling

cudaEvent_t take_event(boltz_grid_s* g) {
    if (!g->event_pool.empty()) {
        cudaEvent_t e = g->event_pool.back();
        g->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Brackets one kernel launch: counts it and, when profiling is on, records an
// event pair around it on the launching stream.
struct ProfScope {
    boltz_grid_s* g;
    int cls;
    cudaStream_t st;
    cudaEvent_t e0 = nullptr;
    ProfScope(boltz_grid_s* g_, int cls_, cudaStream_t st_) : g(g_), cls(cls_), st(st_) {
        ++g->launches[cls];
        if (g->prof_on && (e0 = take_event(g))) cudaEventRecord(e0, st);
    }
    ~ProfScope() {
        if (!e0) return;
        cudaEvent_t e1 = take_event(g);
        if (!e1) return;
        cudaEventRecord(e1, st);
        g->prof_events.push_back({cls, {e0, e1}});
    }
};

// ---------------------------------------------------------------- launches

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Clusters of more than 8 CTAs (the portable limit) must be allowed per kernel.
template <typename K>
cudaError_t allow_big_cluster(K kernel) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

template <int N, int D>
struct Launch {
    using G = Geo<N, D>;
    // 3D fields of 32^3, 48^3 and 64^3 run on clusters of CL CTAs (2, 8 and 16
    // CTAs per field); the synthesis uses clusters of CLS CTAs (4, 8, 16).  A
    // cluster must fit in one GPC (19 SMs), so a cluster shape wastes the SMs
    // left over after whole clusters: 8-CTA clusters of one 141 KB CTA per SM
    // (the former 64^3 shape) ran only 15 clusters at a time, a sixth of the
    // SMs idle, while 16-CTA clusters of 71 KB CTAs (three per SM) use all but
    // 9 of a GPC's 57 slots and ran the C4 step 29% faster; 48^3 on 8 CTAs of
    // 60 KB (three per SM) is 4% faster on the mixed batch than 4 CTAs of
    // 118 KB.  For 32^3, 4-CTA synthesis clusters (six per SM) overlap the
    // transform phases of more fields and were 5% faster per step than pairs.
    // Smaller fields run FPC to a CTA
    static constexpr int CLS = (D == 3 && N == 32) ? 4 : ((D == 3 && N == 64) ? 16 : ((D == 3 && N == 48) ? 8 : 0));
    static constexpr int CL = (D == 3 && N == 32) ? 2 : ((D == 3 && N == 64) ? 16 : ((D == 3 && N == 48) ? 8 : 0));
    static constexpr int FPC = (D == 3) ? (N == 24 ? 1 : (N == 16 ? 4 : 8))
                                        : (N == 64 ? 4 : ((N == 32 || N == 48) ? 16 : (N == 8 ? 64 : 32)));
    static constexpr int BLOCK = G::TPF * FPC;
    static constexpr size_t SMEM = size_t(G::SMEM_F) * FPC * sizeof(float2);
    // 2D analysis and output kernels: about 64 threads a CTA.  Their launches
    // carry one field per radial slot (U of them, often under a thousand), so
    // the synthesis's many fields per CTA would leave most SMs idle.
    static constexpr int FPC_A = (D == 2) ? (64 / G::TPF > 1 ? 64 / G::TPF : 1) : FPC;
    static constexpr int BLOCK_A = G::TPF * FPC_A;
    static constexpr size_t SMEM_A = size_t(G::SMEM_F) * FPC_A * sizeof(float2);
    // 2D synthesis launches of fewer than two CTAs per SM at FPC fields a CTA
    // (small batches, e.g. the bases of a low-rank step) run FPC_A a CTA
    static constexpr bool SMALL_SYN = (D == 2 && FPC_A < FPC);
    static constexpr int kSmallSynCtas = 2 * 152;

    // 2D N = 128: lines split over 4-lane groups
    static constexpr bool WIDE = (D == 2 && N == 128);

    static cudaError_t prepare() {
        cudaError_t e;
        if constexpr (WIDE) {
            if ((e = set_smem(k_synth_w128<SYN_SHIFT>, kWSMEM)) != cudaSuccess) return e;
            if ((e = set_smem(k_synth_w128<SYN_PREP>, kWSMEM)) != cudaSuccess) return e;
            if ((e = set_smem(k_analysis_w128<ANA_SPECTRUM>, kWSMEM)) != cudaSuccess) return e;
            if ((e = set_smem(k_analysis_w128<ANA_ACCUM>, kWSMEM)) != cudaSuccess) return e;
            return set_smem(k_output_w128, kWSMEM);
        } else if constexpr (CL > 0) {
            using CG = ClusterGeo<N, CL>;
            using CGS = ClusterGeo<N, CLS>;
            if ((e = set_smem(k_synth_cl<N, CLS, SYN_SHIFT>, CGS::SMEM)) != cudaSuccess) return e;
            if ((e = set_smem(k_synth_cl<N, CLS, SYN_PREP>, CGS::SMEM)) != cudaSuccess) return e;
            if ((e = set_smem(k_synth_cl<N, CLS, SYN_MULT>, CGS::SMEM)) != cudaSuccess) return e;
            if constexpr (CLS > 8) {
                if ((e = allow_big_cluster(k_synth_cl<N, CLS, SYN_SHIFT>)) != cudaSuccess) return e;
                if ((e = allow_big_cluster(k_synth_cl<N, CLS, SYN_PREP>)) != cudaSuccess) return e;
                if ((e = allow_big_cluster(k_synth_cl<N, CLS, SYN_MULT>)) != cudaSuccess) return e;
            }
            if ((e = set_smem(k_analysis_cl<N, CL, ANA_SPECTRUM>, CG::SMEM)) != cudaSuccess) return e;
            if ((e = set_smem(k_analysis_cl<N, CL, ANA_ACCUM>, CG::SMEM)) != cudaSuccess) return e;
            if constexpr (CL > 8) {
                if ((e = allow_big_cluster(k_analysis_cl<N, CL, ANA_SPECTRUM>)) != cudaSuccess) return e;
                if ((e = allow_big_cluster(k_analysis_cl<N, CL, ANA_ACCUM>)) != cudaSuccess) return e;
                if ((e = allow_big_cluster(k_output_cl<N, CL>)) != cudaSuccess) return e;
            }
            return set_smem(k_output_cl<N, CL>, CG::SMEM);
        } else {
            if ((e = set_smem(k_synth<N, D, FPC, SYN_SHIFT>, SMEM)) != cudaSuccess) return e;
            if ((e = set_smem(k_synth<N, D, FPC, SYN_PREP>, SMEM)) != cudaSuccess) return e;
            if ((e = set_smem(k_synth<N, D, FPC, SYN_MULT>, SMEM)) != cudaSuccess) return e;
            if constexpr (SMALL_SYN) {
                if ((e = set_smem(k_synth<N, D, FPC_A, SYN_SHIFT>, SMEM_A)) != cudaSuccess) return e;
                if ((e = set_smem(k_synth<N, D, FPC_A, SYN_PREP>, SMEM_A)) != cudaSuccess) return e;
                if ((e = set_smem(k_synth<N, D, FPC_A, SYN_MULT>, SMEM_A)) != cudaSuccess) return e;
            }
            if ((e = set_smem(k_analysis<N, D, FPC_A, ANA_SPECTRUM>, SMEM_A)) != cudaSuccess) return e;
            if ((e = set_smem(k_analysis<N, D, FPC_A, ANA_ACCUM>, SMEM_A)) != cudaSuccess) return e;
            return set_smem(k_output<N, D, FPC_A>, SMEM_A);
        }
    }
    static void synth(const SynParams& p, int mode, cudaStream_t st) {
        if constexpr (WIDE) {
            const int grid = (p.n_fields + kWFPC - 1) / kWFPC;
            if (mode == SYN_SHIFT) k_synth_w128<SYN_SHIFT><<<grid, kWTPF * kWFPC, kWSMEM, st>>>(p);
            else k_synth_w128<SYN_PREP><<<grid, kWTPF * kWFPC, kWSMEM, st>>>(p);
        } else if constexpr (CL > 0) {
            using CG = ClusterGeo<N, CLS>;
            if (mode == SYN_SHIFT)
                k_synth_cl<N, CLS, SYN_SHIFT><<<CLS * p.n_fields, CG::NT, CG::SMEM, st>>>(p);
            else if (mode == SYN_MULT)
                k_synth_cl<N, CLS, SYN_MULT><<<CLS * p.n_fields, CG::NT, CG::SMEM, st>>>(p);
            else
                k_synth_cl<N, CLS, SYN_PREP><<<CLS * p.n_fields, CG::NT, CG::SMEM, st>>>(p);
        } else {
            const int grid = (p.n_fields + FPC - 1) / FPC;
            if constexpr (SMALL_SYN) {
                if (grid < kSmallSynCtas) {
                    const int ga = (p.n_fields + FPC_A - 1) / FPC_A;
                    if (mode == SYN_SHIFT)
                        k_synth<N, D, FPC_A, SYN_SHIFT><<<ga, BLOCK_A, SMEM_A, st>>>(p);
                    else if (mode == SYN_MULT)
                        k_synth<N, D, FPC_A, SYN_MULT><<<ga, BLOCK_A, SMEM_A, st>>>(p);
                    else
                        k_synth<N, D, FPC_A, SYN_PREP><<<ga, BLOCK_A, SMEM_A, st>>>(p);
                    return;
                }
            }
            if (mode == SYN_SHIFT)
                k_synth<N, D, FPC, SYN_SHIFT><<<grid, BLOCK, SMEM, st>>>(p);
            else if (mode == SYN_MULT)
                k_synth<N, D, FPC, SYN_MULT><<<grid, BLOCK, SMEM, st>>>(p);
            else
                k_synth<N, D, FPC, SYN_PREP><<<grid, BLOCK, SMEM, st>>>(p);
        }
    }
    static void analysis(const AnaParams& p, int mode, cudaStream_t st) {
        if constexpr (WIDE) {
            const int grid = (p.n_fields + kWFPC - 1) / kWFPC;
            if (mode == ANA_SPECTRUM) k_analysis_w128<ANA_SPECTRUM><<<grid, kWTPF * kWFPC, kWSMEM, st>>>(p);
            else k_analysis_w128<ANA_ACCUM><<<grid, kWTPF * kWFPC, kWSMEM, st>>>(p);
        } else if constexpr (CL > 0) {
            using CG = ClusterGeo<N, CL>;
            if (mode == ANA_SPECTRUM)
                k_analysis_cl<N, CL, ANA_SPECTRUM><<<CL * p.n_fields, CG::NT, CG::SMEM, st>>>(p);
            else
                k_analysis_cl<N, CL, ANA_ACCUM><<<CL * p.n_fields, CG::NT, CG::SMEM, st>>>(p);
        } else {
            const int grid = (p.n_fields + FPC_A - 1) / FPC_A;
            if (mode == ANA_SPECTRUM)
                k_analysis<N, D, FPC_A, ANA_SPECTRUM><<<grid, BLOCK_A, SMEM_A, st>>>(p);
            else
                k_analysis<N, D, FPC_A, ANA_ACCUM><<<grid, BLOCK_A, SMEM_A, st>>>(p);
        }
    }
    static void output(const OutParams& p, cudaStream_t st) {
        if constexpr (WIDE) {
            k_output_w128<<<(p.U + kWFPC - 1) / kWFPC, kWTPF * kWFPC, kWSMEM, st>>>(p);
        } else if constexpr (CL > 0) {
            using CG = ClusterGeo<N, CL>;
            k_output_cl<N, CL><<<CL * p.U, CG::NT, CG::SMEM, st>>>(p);
        } else {
            const int grid = (p.U + FPC_A - 1) / FPC_A;
            k_output<N, D, FPC_A><<<grid, BLOCK_A, SMEM_A, st>>>(p);
        }
    }
};

template <typename R>
struct DispatchT {
    cudaError_t (*prepare)();
    void (*synth)(const SynParamsT<R>&, int, cudaStream_t);
    void (*analysis)(const AnaParamsT<R>&, int, cudaStream_t);
    void (*output)(const OutParamsT<R>&, cudaStream_t);
};
using Dispatch = DispatchT<float>;

template <int N, int D>
Dispatch make_dispatch() {
    return {&Launch<N, D>::prepare, &Launch<N, D>::synth, &Launch<N, D>::analysis, &Launch<N, D>::output};
}

const Dispatch* dispatch_for(int N, int D) {
    static const Dispatch d3_8 = make_dispatch<8, 3>(), d3_16 = make_dispatch<16, 3>(),
                          d3_24 = make_dispatch<24, 3>(), d3_48 = make_dispatch<48, 3>(),
                          d2_24 = make_dispatch<24, 2>(), d2_48 = make_dispatch<48, 2>(),
                          d2_128 = make_dispatch<128, 2>(),
                          d3_32 = make_dispatch<32, 3>(), d3_64 = make_dispatch<64, 3>(), d2_8 = make_dispatch<8, 2>(),
                          d2_16 = make_dispatch<16, 2>(), d2_32 = make_dispatch<32, 2>(),
                          d2_64 = make_dispatch<64, 2>();
    if (D == 3)
        return N == 8 ? &d3_8 : N == 16 ? &d3_16 : N == 24 ? &d3_24 : N == 32 ? &d3_32 : N == 48 ? &d3_48
             : N == 64 ? &d3_64 : nullptr;
    return N == 8 ? &d2_8 : N == 16 ? &d2_16 : N == 24 ? &d2_24 : N == 32 ? &d2_32 : N == 48 ? &d2_48
         : N == 64 ? &d2_64 : N == 128 ? &d2_128 : nullptr;
}

// FP64 check build: the single-CTA field kernels instantiated on double, with
// half as many fields per CTA as the FP32 path (twice the shared memory per field).
template <int N, int D>
struct Launch64 {
    using G = Geo<N, D>;
    static constexpr int FPC = Launch<N, D>::FPC / 2 > 0 ? Launch<N, D>::FPC / 2 : 1;
    static constexpr int BLOCK = G::TPF * FPC;
    static constexpr size_t SMEM = size_t(G::SMEM_F) * FPC * sizeof(double2);
    static_assert(Launch<N, D>::CL == 0 && !Launch<N, D>::WIDE, "single-CTA shapes only");
    static_assert(SMEM <= (200u << 10), "FP64 field tile fits in shared memory");

    static cudaError_t prepare() {
        cudaError_t e;
        if ((e = set_smem(k_synth<N, D, FPC, SYN_SHIFT, double>, SMEM)) != cudaSuccess) return e;
        if ((e = set_smem(k_synth<N, D, FPC, SYN_PREP, double>, SMEM)) != cudaSuccess) return e;
        if ((e = set_smem(k_analysis<N, D, FPC, ANA_SPECTRUM, double>, SMEM)) != cudaSuccess) return e;
        if ((e = set_smem(k_analysis<N, D, FPC, ANA_ACCUM, double>, SMEM)) != cudaSuccess) return e;
        return set_smem(k_output<N, D, FPC, double>, SMEM);
    }
    static void synth(const SynParamsT<double>& p, int mode, cudaStream_t st) {
        const int grid = (p.n_fields + FPC - 1) / FPC;
        if (mode == SYN_SHIFT) k_synth<N, D, FPC, SYN_SHIFT, double><<<grid, BLOCK, SMEM, st>>>(p);
        else k_synth<N, D, FPC, SYN_PREP, double><<<grid, BLOCK, SMEM, st>>>(p);
    }
    static void analysis(const AnaParamsT<double>& p, int mode, cudaStream_t st) {
        const int grid = (p.n_fields + FPC - 1) / FPC;
        if (mode == ANA_SPECTRUM) k_analysis<N, D, FPC, ANA_SPECTRUM, double><<<grid, BLOCK, SMEM, st>>>(p);
        else k_analysis<N, D, FPC, ANA_ACCUM, double><<<grid, BLOCK, SMEM, st>>>(p);
    }
    static void output(const OutParamsT<double>& p, cudaStream_t st) {
        k_output<N, D, FPC, double><<<(p.U + FPC - 1) / FPC, BLOCK, SMEM, st>>>(p);
    }
};

template <int N, int D>
DispatchT<double> make_dispatch64() {
    return {&Launch64<N, D>::prepare, &Launch64<N, D>::synth, &Launch64<N, D>::analysis, &Launch64<N, D>::output};
}

const DispatchT<double>* dispatch64_for(int N, int D) {
    static const DispatchT<double> d3_8 = make_dispatch64<8, 3>(), d3_16 = make_dispatch64<16, 3>(),
                                   d2_16 = make_dispatch64<16, 2>(), d2_32 = make_dispatch64<32, 2>();
    if (D == 3) return N == 8 ? &d3_8 : N == 16 ? &d3_16 : nullptr;
    return N == 16 ? &d2_16 : N == 32 ? &d2_32 : nullptr;
}

const DispatchT<float>* dispatch_of(int N, int D, float) { return dispatch_for(N, D); }
const DispatchT<double>* dispatch_of(int N, int D, double) { return dispatch64_for(N, D); }

// Pipelined contraction: VC voxels per CTA, ring of STAGES bulk-copy stages
// sized to stay within 192 KB of shared memory.
template <int KIND, int TJ, int TL, int VC>
struct ContractLaunch {
    static constexpr int ROWS = ContractShape<KIND, TJ, TL>::ROWS;
    static constexpr int STAGES = (ROWS * VC * 4 * 4 <= (192 << 10)) ? 4 : 3;
    static constexpr size_t SMEM = size_t(STAGES) * ROWS * VC * sizeof(float);
    static cudaError_t prepare() { return set_smem(k_contract_pipe<KIND, TJ, TL, VC, STAGES>, SMEM); }
    static void launch(const ConParams& cp, int n_tiles, int nq, cudaStream_t st) {
        dim3 grid(cp.n / VC, n_tiles, nq);      // one CTA per voxel chunk of the field layout
        k_contract_pipe<KIND, TJ, TL, VC, STAGES><<<grid, VC, SMEM, st>>>(cp);
    }
};

template <int VC>
cudaError_t prepare_contract_vc() {
    cudaError_t e;
    if ((e = ContractLaunch<TILE_TRI, 16, 16, VC>::prepare()) != cudaSuccess) return e;
    if ((e = ContractLaunch<TILE_TRI, 8, 8, VC>::prepare()) != cudaSuccess) return e;
    if ((e = ContractLaunch<TILE_FULL, 8, 16, VC>::prepare()) != cudaSuccess) return e;
    if ((e = ContractLaunch<TILE_FULL, 8, 8, VC>::prepare()) != cudaSuccess) return e;
    return ContractLaunch<TILE_LIST, 16, 16, VC>::prepare();
}

cudaError_t prepare_contract() {
    cudaError_t e;
    if ((e = prepare_contract_vc<256>()) != cudaSuccess) return e;
    if ((e = prepare_contract_vc<288>()) != cudaSuccess) return e;
    return prepare_contract_vc<64>();
}

template <int VC>
void launch_contract_vc(int kind, int T, const ConParams& cp, int n_tiles, int nq, cudaStream_t st) {
    if (kind == TILE_TRI) {
        if (T == 16) ContractLaunch<TILE_TRI, 16, 16, VC>::launch(cp, n_tiles, nq, st);
        else ContractLaunch<TILE_TRI, 8, 8, VC>::launch(cp, n_tiles, nq, st);
    } else if (kind == TILE_FULL) {
        if (T == 16) ContractLaunch<TILE_FULL, 8, 16, VC>::launch(cp, n_tiles, nq, st);
        else ContractLaunch<TILE_FULL, 8, 8, VC>::launch(cp, n_tiles, nq, st);
    } else {
        ContractLaunch<TILE_LIST, 16, 16, VC>::launch(cp, n_tiles, nq, st);
    }
}

// VC equals the voxel chunk of the shifted-field layout: 64 (the 8^2 grid),
// 256 (other powers of two) or 288 (N = 24, 48)
void launch_contract(int vch, int kind, int T, const ConParams& cp, int n_tiles, int nq, cudaStream_t st) {
    if (vch == 256) launch_contract_vc<256>(kind, T, cp, n_tiles, nq, st);
    else if (vch == 288) launch_contract_vc<288>(kind, T, cp, n_tiles, nq, st);
    else launch_contract_vc<64>(kind, T, cp, n_tiles, nq, st);
}

// FP64 contraction (voxel chunk 256, tiles TRI 8, FULL 8x8, LIST 16): as many
// stages as fit in 200 KB of shared memory, at least one.
template <int KIND, int TJ, int TL>
struct ContractLaunch64 {
    static constexpr int VC = 256;
    static constexpr int ROWS = ContractShape<KIND, TJ, TL>::ROWS;
    static constexpr size_t STAGE = size_t(ROWS) * VC * sizeof(double);
    static constexpr int FIT = (int)((200u << 10) / STAGE);
    static constexpr int STAGES = FIT < 1 ? 1 : (FIT > 4 ? 4 : FIT);
    static constexpr size_t SMEM = STAGES * STAGE;
    static_assert(SMEM <= (227u << 10), "one stage fits in shared memory");
    static cudaError_t prepare() { return set_smem(k_contract_pipe<KIND, TJ, TL, VC, STAGES, double>, SMEM); }
    static void launch(const ConParamsT<double>& cp, int n_tiles, int nq, cudaStream_t st) {
        dim3 grid(cp.n / VC, n_tiles, nq);
        k_contract_pipe<KIND, TJ, TL, VC, STAGES, double><<<grid, VC, SMEM, st>>>(cp);
    }
};

cudaError_t prepare_contract64() {
    cudaError_t e;
    if ((e = ContractLaunch64<TILE_TRI, 8, 8>::prepare()) != cudaSuccess) return e;
    if ((e = ContractLaunch64<TILE_FULL, 8, 8>::prepare()) != cudaSuccess) return e;
    return ContractLaunch64<TILE_LIST, 16, 16>::prepare();
}

void launch_contract_of(int vch, int kind, int T, const ConParamsT<float>& cp, int n_tiles, int nq,
                        cudaStream_t st) {
    launch_contract(vch, kind, T, cp, n_tiles, nq, st);
}

void launch_contract_of(int, int kind, int, const ConParamsT<double>& cp, int n_tiles, int nq, cudaStream_t st) {
    if (kind == TILE_TRI) ContractLaunch64<TILE_TRI, 8, 8>::launch(cp, n_tiles, nq, st);
    else if (kind == TILE_FULL) ContractLaunch64<TILE_FULL, 8, 8>::launch(cp, n_tiles, nq, st);
    else ContractLaunch64<TILE_LIST, 16, 16>::launch(cp, n_tiles, nq, st);
}

// Device tables of one precision.
template <typename R>
struct TablesT {
    const typename Prec<R>::C* phase;
    const R* ctab;
    const R* gm;
    const R* w;
    const R* gmf;            // per-mode loss weight (mass-consistent loss) or null
};
TablesT<float> tables_of(const boltz_grid_s* g, float) { return {g->d_phase, g->d_ctab, g->d_gm, g->d_w, g->d_gmf}; }
TablesT<double> tables_of(const boltz_grid_s* g, double) {
    return {g->d_phase64, g->d_ctab64, g->d_gm64, g->d_w64, g->d_gmf64};
}

// Asymmetric contraction of the Carleman form (FULL 8 x T strips and LIST 16).
template <int KIND, int TJ, int TL, int VC>
struct ContractLaunchA {
    static constexpr int ROWS = ContractShapeA<KIND, TJ, TL>::ROWS;
    static constexpr int STAGES = (ROWS * VC * 4 * 4 <= (192 << 10)) ? 4 : 3;
    static constexpr size_t SMEM = size_t(STAGES) * ROWS * VC * sizeof(float);
    static cudaError_t prepare() { return set_smem(k_contract_pipe<KIND, TJ, TL, VC, STAGES, float, true>, SMEM); }
    static void launch(const ConParams& cp, int n_tiles, cudaStream_t st) {
        dim3 grid(cp.n / VC, n_tiles, cp.n_split > 1 ? cp.n_split : 1);
        k_contract_pipe<KIND, TJ, TL, VC, STAGES, float, true><<<grid, VC, SMEM, st>>>(cp);
    }
};

template <int VC>
cudaError_t prepare_contract_asym_vc() {
    cudaError_t e;
    if ((e = ContractLaunchA<TILE_FULL, 8, 16, VC>::prepare()) != cudaSuccess) return e;
    if ((e = ContractLaunchA<TILE_FULL, 8, 8, VC>::prepare()) != cudaSuccess) return e;
    return ContractLaunchA<TILE_LIST, 16, 16, VC>::prepare();
}

template <int VC>
void launch_contract_asym_vc(int kind, int T, const ConParams& cp, int n_tiles, cudaStream_t st) {
    if (kind == TILE_FULL) {
        if (T == 16) ContractLaunchA<TILE_FULL, 8, 16, VC>::launch(cp, n_tiles, st);
        else ContractLaunchA<TILE_FULL, 8, 8, VC>::launch(cp, n_tiles, st);
    } else {
        ContractLaunchA<TILE_LIST, 16, 16, VC>::launch(cp, n_tiles, st);
    }
}

void launch_contract_asym(int vch, int kind, int T, const ConParams& cp, int n_tiles, cudaStream_t st) {
    if (vch == 256) launch_contract_asym_vc<256>(kind, T, cp, n_tiles, st);
    else if (vch == 288) launch_contract_asym_vc<288>(kind, T, cp, n_tiles, st);
    else launch_contract_asym_vc<64>(kind, T, cp, n_tiles, st);
}

cudaError_t prepare_contract_asym() {
    cudaError_t e;
    if ((e = prepare_contract_asym_vc<256>()) != cudaSuccess) return e;
    if ((e = prepare_contract_asym_vc<288>()) != cudaSuccess) return e;
    return prepare_contract_asym_vc<64>();
}

boltz_status check_pairs(int n_inputs, const int32_t* pj, const int32_t* pl, int n_pairs) {
    if (n_pairs < 0) return BOLTZ_EINVAL;
    if (n_pairs == 0) return BOLTZ_OK;
    if (!pj || !pl || n_inputs <= 0) return BOLTZ_EINVAL;
    for (int e = 0; e < n_pairs; ++e)
        if (pj[e] < 0 || pj[e] >= n_inputs || pl[e] < 0 || pl[e] >= n_inputs) return BOLTZ_EINVAL;
    return BOLTZ_OK;
}

// Makes the grid's cached plan the one for this batch (building, sizing the
// workspace to at least `min_ws` bytes and uploading the descriptors when the
// pair list changed).  Synchronous; never called during stream capture.
boltz_status prepare_plan(boltz_grid_s* g, int n_inputs, const int32_t* pj, const int32_t* pl, int n_pairs, int form,
                          size_t min_ws, cudaStream_t st, size_t elem = 4) {
    if (fault_injected("badplan")) return BOLTZ_EINVAL;
    const bool same = g->plan_uploaded && form == g->last_form && n_inputs == g->last_n_inputs &&
                      elem == g->last_elem &&
                      (int)g->last_j.size() == n_pairs &&
                      std::equal(pj, pj + n_pairs, g->last_j.begin()) &&
                      std::equal(pl, pl + n_pairs, g->last_l.begin());
    boltz_status s;
    if (same) {
        if (g->ws_cap >= min_ws) return BOLTZ_OK;
        // a larger workspace loses the uploaded descriptors: upload them again
        if ((s = ensure_workspace(g, min_ws, st)) != BOLTZ_OK) return s;
        if ((s = upload_plan(g, g->last_plan, st)) != BOLTZ_OK) return s;
        g->plan_uploaded = true;
        return BOLTZ_OK;
    }
    Plan plan;
    if ((s = build_plan(g, n_inputs, pj, pl, n_pairs, form, plan, elem)) != BOLTZ_OK) return s;
    if ((s = ensure_workspace(g, std::max(plan.total, min_ws), st)) != BOLTZ_OK) return s;
    if ((s = upload_plan(g, plan, st)) != BOLTZ_OK) return s;
    g->last_plan = std::move(plan);
    g->last_j.assign(pj, pj + n_pairs);
    g->last_l.assign(pl, pl + n_pairs);
    g->last_form = form;
    g->last_n_inputs = n_inputs;
    g->last_elem = elem;
    g->plan_uploaded = true;
    return BOLTZ_OK;
}

// ---------------------------------------------------------------- split-precision form

// FP32 -> BF16, round to nearest even (finite inputs).
uint16_t bf16_rne(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

float bf16_value(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// Per-node B' operands of the split-precision form: for node (q, p) and axis
// a the shift-interpolation matrix S(s)[i][m] = (1/N) sum_{|k| < N/2}
// exp(i pi k ((i - m) dv - s) / L), s = rho_q sigma_{p,a} / 2 (real: the
// Nyquist mode is excluded), split into BF16 hi/lo and laid out as the
// K-major core-matrix operand described in split.cuh.  Built once per grid
// (synchronous; never during stream capture).
template <int N, int CL>
void fill_split_tables(const boltz_grid_s* g, std::vector<uint16_t>& img) {
    using S = SplitGeo<N, CL>;                    // B' depends on N only
    const int nodes = g->n_rho * g->M;
    img.assign(size_t(nodes) * S::B_BYTES / 2, 0);
    std::vector<double> sv(N);
    for (int node = 0; node < nodes; ++node) {
        for (int a = 0; a < 3; ++a) {
            const double sh = 0.5 * g->rho[node / g->M] * g->dir.sigma[(node % g->M) * 3 + a];
            for (int d = 0; d < N; ++d) {            // d = (i - m) mod N
                double acc = 1.0;
                for (int k = 1; k < N / 2; ++k) acc += 2.0 * std::cos(kPi * k * (2.0 * d / N - sh / g->L));
                sv[d] = acc / N;
            }
            uint16_t hi[N], lo[N];
            for (int d = 0; d < N; ++d) {
                hi[d] = bf16_rne((float)sv[d]);
                lo[d] = bf16_rne((float)(sv[d] - (double)bf16_value(hi[d])));
            }
            uint16_t* B = img.data() + (size_t(node) * S::B_BYTES + size_t(a) * S::B_AXIS_BYTES) / 2;
            for (int n = 0; n < S::NB; ++n) {
                const int i = n % N;
                for (int kp = 0; kp < S::KP; ++kp) {
                    const int d = (i - kp / 2 + N) % N;
                    const uint16_t v = n < N ? hi[d] : ((kp & 1) ? (uint16_t)0 : lo[d]);
                    const size_t off = (size_t(n / 8) * S::KCORES + kp / 8) * 128 + (n % 8) * 16 + (kp % 8) * 2;
                    B[off / 2] = v;
                }
            }
        }
    }
}

// Clusters of the split kernel that fit on the device at once (all resident).
template <int N, int CL>
int resident_split_clusters(int sms) {
    using S = SplitGeo<N, CL>;
    if constexpr (CL == 1) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_shift_split<N, CL>, kSplitThreads, S::SMEM) !=
                cudaSuccess ||
            per_sm < 1) {
            (void)cudaGetLastError();
            return sms;
        }
        return per_sm * sms;
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(CL * 64, 1, 1);
        cfg.blockDim = dim3(kSplitThreads, 1, 1);
        cfg.dynamicSmemBytes = S::SMEM;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_shift_split<N, CL>, &cfg) != cudaSuccess || n < 1) {
            (void)cudaGetLastError();
            return std::max(1, sms / CL);
        }
        return n;
    }
}

// Per-node B' operands of the split-precision form: for node (q, p) and axis
// a the shift-interpolation matrix S(s)[i][m] = (1/N) sum_{|k| < N/2}
// exp(i pi k ((i - m) dv - s) / L), s = rho_q sigma_{p,a} / 2 (real: the
// Nyquist mode is excluded), split into BF16 hi/lo and laid out as the
// K-major core-matrix operand described in split.cuh.  Built once per grid
// (synchronous; never during stream capture).
boltz_status ensure_split_tables(boltz_grid_s* g) {
    if (g->d_smat) return BOLTZ_OK;
    std::vector<uint16_t> img;
    cudaError_t e;
    if (g->N == 64) {
        fill_split_tables<64, kSplitCL64>(g, img);
        e = set_smem(k_shift_split<64, kSplitCL64>, SplitGeo<64, kSplitCL64>::SMEM);
        if (e == cudaSuccess) g->split_clusters = resident_split_clusters<64, kSplitCL64>(g->sms);
    } else {
        fill_split_tables<32, kSplitCL32>(g, img);
        e = set_smem(k_shift_split<32, kSplitCL32>, SplitGeo<32, kSplitCL32>::SMEM);
        if (e == cudaSuccess) g->split_clusters = resident_split_clusters<32, kSplitCL32>(g->sms);
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return BOLTZ_ECUDA;
    }
    uint8_t* d = nullptr;
    if (cudaMalloc(&d, img.size() * 2) != cudaSuccess) {
        (void)cudaGetLastError();
        return BOLTZ_ENOMEM;
    }
    if (cudaMemcpy(d, img.data(), img.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return BOLTZ_ECUDA;
    }
    g->d_smat = d;
    return BOLTZ_OK;
}

void launch_split_input(int N, const float* fN, uint8_t* img, int nc, cudaStream_t st) {
    const size_t total = size_t(nc) * N * N * N;
    const int grid = (int)std::min<size_t>((total + 255) / 256, 4096);
    if (N == 64) k_split_input<64, kSplitCL64><<<grid, 256, 0, st>>>(fN, img, nc);
    else k_split_input<32, kSplitCL32><<<grid, 256, 0, st>>>(fN, img, nc);
}

// Persistent launch: every resident cluster takes a contiguous range of fields.
void launch_shift_split(int N, const SplitParams& p, int clusters, cudaStream_t st) {
    const int ncl = std::max(1, std::min(p.n_fields, clusters));
    if (N == 64)
        k_shift_split<64, kSplitCL64><<<ncl * kSplitCL64, kSplitThreads, SplitGeo<64, kSplitCL64>::SMEM, st>>>(p);
    else
        k_shift_split<32, kSplitCL32><<<ncl * kSplitCL32, kSplitThreads, SplitGeo<32, kSplitCL32>::SMEM, st>>>(p);
}

// ---------------------------------------------------------------- Carleman form

// int_{-R}^{R} |rho|^{d-2} exp(i rho s) drho (real, even in s)
double carleman_phi(int d, double R, double s) {
    if (std::fabs(s) < 1e-6) return d == 2 ? 2.0 * R - R * R * R * s * s / 3.0 : R * R - R * R * R * R * s * s / 4.0;
    if (d == 2) return 2.0 * std::sin(R * s) / s;
    return 2.0 * (R * std::sin(R * s) / s + (std::cos(R * s) - 1.0) / (s * s));
}

// integral of exp(i y.t) over the (d-1)-ball of radius R perpendicular to e, t = |t|
double carleman_psi(int d, double R, double t) {
    t = std::fabs(t);
    if (t < 1e-6) return d == 2 ? 2.0 * R - R * R * R * t * t / 3.0 : kPi * R * R * (1.0 - R * R * t * t / 8.0);
    if (d == 2) return 2.0 * std::sin(R * t) / t;
    return 2.0 * kPi * R * std::cyl_bessel_j(1.0, R * t) / t;
}

// Tables of the Carleman form (built once per grid, synchronously):
//   mult[p][k]      = (-1)^k psi(pi |k - (k.e_p) e_p| / L)   g side, p < M/2
//   mult[M/2+p][k]  = (-1)^k phi(pi k.e_p / L)                f side
//   (zero at the Nyquist indices), gm[k] = Bt sum_p w_p phi psi (the loss
//   uses the same discrete beta at m = l), w = Bt w_p, Bt = 2^{d-1} b, over one
//   direction e_p of every antipodal pair of the grid's rule.
boltz_status ensure_carleman_tables(boltz_grid_s* g) {
    if (g->d_cm_mult) return BOLTZ_OK;
    const int N = g->N, D = g->D, H = N / 2, NH = H + 1;
    std::vector<int> dirs;
    for (int p = 0; p < g->M; ++p)
        if (g->dir.antipode[p] > p) dirs.push_back(p);
    const int M2 = (int)dirs.size();
    const double Bt = std::pow(2.0, D - 1) * g->b;
    const size_t half = g->half;
    std::vector<float> mult(size_t(2) * M2 * half), gm(half), w(M2);
    std::vector<int2> dp(M2);
    for (size_t idx = 0; idx < half; ++idx) {
        int k0, k1 = 0, k2;
        if (D == 3) {
            k0 = (int)(idx / (size_t(N) * NH));
            k1 = (int)((idx / NH) % N);
            k2 = (int)(idx % NH);
        } else {
            k0 = (int)(idx / NH);
            k2 = (int)(idx % NH);
        }
        const bool nyq = k0 == H || k2 == H || (D == 3 && k1 == H);
        const double sg = ((k0 + k1 + k2) & 1) ? -1.0 : 1.0;
        double kv[3] = {(double)(k0 < H ? k0 : k0 - N), 0.0, 0.0};
        if (D == 3) {
            kv[1] = k1 < H ? k1 : k1 - N;
            kv[2] = k2;
        } else {
            kv[1] = k2;
        }
        double k2sum = 0.0;
        for (int a = 0; a < D; ++a) k2sum += kv[a] * kv[a];
        double loss = 0.0;
        for (int q = 0; q < M2; ++q) {
            const double* e = &g->dir.sigma[size_t(dirs[q]) * D];
            double ke = 0.0;
            for (int a = 0; a < D; ++a) ke += kv[a] * e[a];
            const double perp = std::sqrt(std::max(0.0, k2sum - ke * ke));
            const double ph = carleman_phi(D, g->R, kPi * ke / g->L);
            const double ps = carleman_psi(D, g->R, kPi * perp / g->L);
            mult[size_t(q) * half + idx] = nyq ? 0.f : (float)(sg * ps);
            mult[size_t(M2 + q) * half + idx] = nyq ? 0.f : (float)(sg * ph);
            loss += g->dir.w[dirs[q]] * ph * ps;
        }
        gm[idx] = (float)(Bt * loss);
    }
    for (int q = 0; q < M2; ++q) {
        w[q] = (float)(Bt * g->dir.w[dirs[q]]);
        dp[q] = make_int2(q, M2 + q);
    }
    auto fail = [&](boltz_status st) {
        cudaFree(g->d_cm_mult);
        cudaFree(g->d_cm_gm);
        cudaFree(g->d_cm_w);
        cudaFree(g->d_cm_dpair);
        g->d_cm_mult = nullptr;
        g->d_cm_gm = nullptr;
        g->d_cm_w = nullptr;
        g->d_cm_dpair = nullptr;
        (void)cudaGetLastError();
        return st;
    };
    if (cudaMalloc(&g->d_cm_mult, mult.size() * 4) != cudaSuccess || cudaMalloc(&g->d_cm_gm, gm.size() * 4) != cudaSuccess ||
        cudaMalloc(&g->d_cm_w, w.size() * 4) != cudaSuccess || cudaMalloc(&g->d_cm_dpair, dp.size() * sizeof(int2)) != cudaSuccess)
        return fail(BOLTZ_ENOMEM);
    if (cudaMemcpy(g->d_cm_mult, mult.data(), mult.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->d_cm_gm, gm.data(), gm.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->d_cm_w, w.data(), w.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->d_cm_dpair, dp.data(), dp.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess ||
        prepare_contract_asym() != cudaSuccess)
        return fail(BOLTZ_ECUDA);
    return BOLTZ_OK;
}

// One evaluation batch in the Carleman form: per chunk f_N and Lambda (per-mode
// loss table), the M multiplier fields of every input in one launch, the
// asymmetric contraction into one slot per ordered pair, and the output
// Q = P - f_N Lambda (no forward transform).
boltz_status run_carleman(boltz_grid_s* g, const float2* spectra, int n_inputs, const int32_t* pj,
                          const int32_t* pl, int n_pairs, float* Q_out, cudaStream_t st) {
    if (!carleman_kernel(g->gamma, g->D)) return BOLTZ_EINVAL;
    if (!carleman_shape(g->N, g->D)) return BOLTZ_EUNSUPPORTED;
    boltz_status s0 = ensure_carleman_tables(g);
    if (s0 != BOLTZ_OK) return s0;
    s0 = prepare_plan(g, n_inputs, pj, pl, n_pairs, BOLTZ_FORM_CARLEMAN, 0, st, 4);
    if (s0 != BOLTZ_OK) return s0;
    const Plan& plan = g->last_plan;
    const Dispatch* dp = dispatch_for(g->N, g->D);
    char* ws = g->d_ws;
    float* A = reinterpret_cast<float*>(ws + plan.off_A);
    float* Pbuf = reinterpret_cast<float*>(ws + plan.off_P);
    float* fN = reinterpret_cast<float*>(ws + plan.off_fN);
    for (const auto& c : plan.chunks) {
        const int nc = (int)c.inputs.size();
        SynParams sp{};
        sp.spectra = spectra;
        sp.inputs = reinterpret_cast<const int*>(ws + plan.off_plan + c.off_inputs);
        sp.phase = g->d_phase;
        sp.gm = g->d_gm;
        sp.gm_full = g->d_cm_gm;
        sp.n_c = nc;
        sp.M = g->M;
        sp.id_node = g->n_rho * g->M;
        sp.out = fN;
        sp.n_fields = 2 * nc;
        {
            ProfScope ps(g, BOLTZ_KCLASS_PREP, st);
            dp->synth(sp, SYN_PREP, st);
        }
        SynParams sm = sp;
        sm.gm_full = nullptr;
        sm.mult = g->d_cm_mult;
        sm.out = A;
        sm.n_fields = g->M * nc;
        {
            ProfScope ps(g, BOLTZ_KCLASS_SHIFT, st);
            dp->synth(sm, SYN_MULT, st);
        }
        ConParams cp{};
        cp.A = A;
        cp.P = Pbuf;
        cp.w = g->d_cm_w;
        cp.dpair = g->d_cm_dpair;
        cp.err = g->d_err;
        cp.n_dpair = g->M / 2;
        cp.M = g->M;
        cp.n_c = nc;
        cp.U = c.U;
        cp.n = g->n;
        cp.n_split = c.split;
        for (int k : {TILE_FULL, TILE_LIST}) {
            if (c.tiles[k].empty()) continue;
            cp.tiles = reinterpret_cast<const Tile*>(ws + plan.off_plan + c.off_tiles[k]);
            ProfScope ps(g, BOLTZ_KCLASS_CONTRACT, st);
            launch_contract_asym(voxel_chunk(g->N, g->D), k, k == TILE_LIST ? 16 : c.tile_T, cp,
                                 (int)c.tiles[k].size(), st);
        }
        ProfScope ps(g, BOLTZ_KCLASS_OUTPUT, st);
        const dim3 grid((g->n / 4 + 255) / 256, c.U);
        k_carleman_output<<<grid, 256, 0, st>>>(Pbuf, fN, fN + size_t(nc) * g->n,
                                                 reinterpret_cast<const int*>(ws + plan.off_plan + c.off_start),
                                                 reinterpret_cast<const int4*>(ws + plan.off_plan + c.off_outs), Q_out,
                                                 g->n, g->d_err, c.split, c.U);
    }
    BZ_CUDA(cudaGetLastError());
    return BOLTZ_OK;
}

// One batched evaluation on the pipelined schedule (plan.pencil), launch by
// launch (one chunk, or several of one shape): f_N and Lambda of the
// launch's inputs, the persistent kernel of pencil.cuh (shifted fields,
// sigma-contraction and radial step of every node of every chunk), then the
// output kernel over the launch's used gain slots.
boltz_status run_pencil(boltz_grid_s* g, const float2* spectra, float* Q_out, cudaStream_t st) {
    namespace pc = boltz_dev::pencil;
    const Plan& plan = g->last_plan;
    const Dispatch* dp = dispatch_for(g->N, g->D);
    char* ws = g->d_ws;
    const char* blob = ws + plan.off_plan + plan.off_pen_blob;
    const PencilTree& T = g->pen_tree;
    float* fN = reinterpret_cast<float*>(ws + plan.off_fN);
    for (size_t k = 0; k < plan.chunks.size(); ++k) {
        const ChunkPlan& c = plan.chunks[k];
        const int nc = (int)c.inputs.size();          // inputs of the launch (all its chunks)
        const int n_chunk = plan.pen_nchunk[k];
        const int* d_inputs = reinterpret_cast<const int*>(ws + plan.off_plan + c.off_inputs);
        SynParams sp{};
        sp.spectra = spectra;
        sp.inputs = d_inputs;
        sp.phase = g->d_phase;
        sp.gm = g->d_gm;
        sp.gm_full = g->d_gmf;
        sp.n_c = nc;
        sp.M = g->M;
        sp.id_node = g->n_rho * g->M;
        sp.out = fN;                                 // f < nc: f_N, f >= nc: Lambda
        sp.n_fields = 2 * nc;
        {
            ProfScope ps(g, BOLTZ_KCLASS_PREP, st);
            dp->synth(sp, SYN_PREP, st);
        }
        pc::Params P{};
        P.spectra = spectra;
        P.inputs = d_inputs;
        P.phase = g->d_phase;
        P.ctab = g->d_ctab;
        P.X = reinterpret_cast<float2*>(ws + plan.off_X);
        P.Pt = reinterpret_cast<float2*>(ws + plan.off_Pt);
        P.qhat = reinterpret_cast<float2*>(ws + plan.off_qhat);
        P.qstd = reinterpret_cast<float2*>(ws + plan.off_qstd);
        P.slots = reinterpret_cast<const int*>(blob + plan.pen_slot_off[k]);
        for (int w = 0; w < 5; ++w) P.used[w] = plan.pen_mask[k][w];
        P.ctr = reinterpret_cast<int*>(ws + plan.off_ctr);
        P.err = g->d_err;
        P.tr.n_s0 = T.n_s0;
        P.tr.n_s01 = T.n_s01;
        P.tr.n_grp = T.n_grp;
        P.tr.n_step = (int)T.step_dir.size();
        P.tr.grp = reinterpret_cast<const int*>(blob + plan.pen_off[0]);
        P.tr.s0_dir = reinterpret_cast<const int*>(blob + plan.pen_off[1]);
        P.tr.s0_child = reinterpret_cast<const int*>(blob + plan.pen_off[2]);
        P.tr.s01_dir = reinterpret_cast<const int*>(blob + plan.pen_off[3]);
        P.tr.step_blk = reinterpret_cast<const int4*>(blob + plan.pen_off[4]);
        P.tr.step_dir = reinterpret_cast<const int4*>(blob + plan.pen_off[5]);
        P.tr.step_sel = reinterpret_cast<const int4*>(blob + plan.pen_off[6]);
        P.tr.step_w = reinterpret_cast<const float2*>(blob + plan.pen_off[7]);
        P.n_c = nc / n_chunk;
        P.M = g->M;
        P.n_rho = g->n_rho;
        P.n_used = c.U / n_chunk;
        P.n_node = n_chunk * g->n_rho;
        BZ_CUDA(cudaMemsetAsync(P.ctr, 0, size_t(pc::ctr_count(P.n_node, c.U)) * sizeof(int), st));
        const long long items =
            (long long)P.n_node * (pc::NLB + pc::tree_items(P.n_c, T.n_grp) + (long long)P.n_used);
        const bool diag = plan.pen_diag[k];
        const int grid = (int)std::min<long long>(diag ? g->pen_ctas_diag : g->pen_ctas, items);
        {
            ProfScope ps(g, BOLTZ_KCLASS_PIPELINE, st);
            if (diag) pc::k_pencil<true><<<grid, pc::NT, pc::SM_TOTAL, st>>>(P);
            else pc::k_pencil<false><<<grid, pc::NT, pc::SM_TOTAL, st>>>(P);
        }
        OutParams op{};
        op.qhat = P.qstd;
        op.fN = fN;
        op.lam = fN + size_t(nc) * g->n;
        op.out_start = reinterpret_cast<const int*>(ws + plan.off_plan + c.off_start);
        op.outs = reinterpret_cast<const int4*>(ws + plan.off_plan + c.off_outs);
        op.Q = Q_out;
        op.err = g->d_err;
        op.U = c.U;
        {
            ProfScope ps(g, BOLTZ_KCLASS_OUTPUT, st);
            dp->output(op, st);
        }
    }
    BZ_CUDA(cudaGetLastError());
    return BOLTZ_OK;
}

// One batched evaluation in precision R (float: the product path; double:
// the FP64 check build, same kernels and schedule).
template <typename R>
boltz_status run_batched(boltz_grid_s* g, const typename Prec<R>::C* spectra, int n_inputs, const int32_t* pj,
                         const int32_t* pl, int n_pairs, R* Q_out, int form, cudaStream_t st) {
    using C = typename Prec<R>::C;
    if (form == BOLTZ_FORM_CARLEMAN) {
        if constexpr (sizeof(R) == 4) return run_carleman(g, spectra, n_inputs, pj, pl, n_pairs, Q_out, st);
        else return BOLTZ_EUNSUPPORTED;
    }
    const bool split = form == BOLTZ_FORM_SPLIT_BF16;
    if (split && (sizeof(R) != 4 || !split_shape(g->N, g->D))) return BOLTZ_EUNSUPPORTED;
    boltz_status s0;
    if (split && (s0 = ensure_split_tables(g)) != BOLTZ_OK) return s0;
    s0 = prepare_plan(g, n_inputs, pj, pl, n_pairs, form, 0, st, sizeof(R));
    if (s0 != BOLTZ_OK) return s0;
    const Plan& plan = g->last_plan;
    if constexpr (sizeof(R) == 4) {
        if (plan.pencil) return run_pencil(g, spectra, Q_out, st);
    }
    const DispatchT<R>* dp = dispatch_of(g->N, g->D, R(0));
    const TablesT<R> tb = tables_of(g, R(0));
    char* ws = g->d_ws;
    R* A = reinterpret_cast<R*>(ws + plan.off_A);
    R* Pbuf = reinterpret_cast<R*>(ws + plan.off_P);
    C* qhat = reinterpret_cast<C*>(ws + plan.off_qhat);
    R* fN = reinterpret_cast<R*>(ws + plan.off_fN);
    R* lam = reinterpret_cast<R*>(ws + plan.off_lam);
    for (const auto& c : plan.chunks) {
        const int nc = (int)c.inputs.size();
        const int* d_inputs = reinterpret_cast<const int*>(ws + plan.off_plan + c.off_inputs);
        // f_N and Lambda_g of the chunk's inputs (fN and lam are contiguous: [2][nc_max][n])
        SynParamsT<R> sp{};
        sp.spectra = spectra;
        sp.inputs = d_inputs;
        sp.phase = tb.phase;
        sp.gm = tb.gm;
        sp.gm_full = tb.gmf;
        sp.n_c = nc;
        sp.M = g->M;
        sp.id_node = g->n_rho * g->M;
        // PREP writes field f at out + f*n: f < nc -> f_N, f >= nc -> Lambda
        sp.out = fN;
        sp.n_fields = 2 * nc;
        {
            ProfScope ps(g, BOLTZ_KCLASS_PREP, st);
            dp->synth(sp, SYN_PREP, st);
        }
        const R* lam_c = fN + size_t(nc) * g->n;
        uint8_t* img = reinterpret_cast<uint8_t*>(ws + plan.off_img);
        (void)img;
        if constexpr (sizeof(R) == 4) {
            if (split) {
                ProfScope ps(g, BOLTZ_KCLASS_PREP, st);
                launch_split_input(g->N, fN, img, nc, st);
            }
        }
        BZ_CUDA(cudaMemsetAsync(qhat, 0, size_t(c.U) * g->half * sizeof(C), st));
        // Node blocks run synth -> contract on the caller's stream and the radial
        // step on the side stream, with P double-buffered: the radial step of
        // block i overlaps synth/contract of block i+1.
        BZ_CUDA(cudaEventRecord(g->ev_fork, st));
        BZ_CUDA(cudaStreamWaitEvent(g->side, g->ev_fork, 0));
        const size_t pbuf_elems = size_t(plan.nq) * plan.max_U * g->n;
        int blk = 0;
        for (int q0 = 0; q0 < g->n_rho; q0 += plan.nq, ++blk) {
            const int nq = std::min(plan.nq, g->n_rho - q0);
            const int b = blk & 1;
            R* Pb = Pbuf + b * pbuf_elems;
            SynParamsT<R> ss = sp;
            ss.out = A;
            ss.q0 = q0;
            ss.n_fields = nq * g->M * nc;
            {
                ProfScope ps(g, BOLTZ_KCLASS_SHIFT, st);
                if constexpr (sizeof(R) == 4) {
                    if (split) {
                        SplitParams spp{img, g->d_smat, A, g->d_err, nc, g->M, q0, ss.n_fields};
                        launch_shift_split(g->N, spp, g->split_clusters, st);
                    } else {
                        dp->synth(ss, SYN_SHIFT, st);
                    }
                } else {
                    dp->synth(ss, SYN_SHIFT, st);
                }
            }
            if (blk >= 2) BZ_CUDA(cudaStreamWaitEvent(st, g->ev_free[b], 0));
            ConParamsT<R> cp{};
            cp.A = A;
            cp.P = Pb;
            cp.w = tb.w;
            cp.dpair = g->d_dpair;
            cp.err = g->d_err;
            cp.n_dpair = g->M / 2;
            cp.M = g->M;
            cp.n_c = nc;
            cp.U = c.U;
            cp.n = g->n;
            for (int k = 0; k < 3; ++k) {
                if (c.tiles[k].empty()) continue;
                cp.tiles = reinterpret_cast<const Tile*>(ws + plan.off_plan + c.off_tiles[k]);
                ProfScope ps(g, BOLTZ_KCLASS_CONTRACT, st);
                launch_contract_of(voxel_chunk(g->N, g->D), k, k == TILE_LIST ? 16 : c.tile_T, cp,
                                   (int)c.tiles[k].size(), nq, st);
            }
            BZ_CUDA(cudaEventRecord(g->ev_ready[b], st));
            BZ_CUDA(cudaStreamWaitEvent(g->side, g->ev_ready[b], 0));
            AnaParamsT<R> ap{};
            ap.in = Pb;
            ap.out = qhat;
            ap.ctab = tb.ctab;
            ap.n_fields = c.U;
            ap.nq = nq;
            ap.q0 = q0;
            ap.U = c.U;
            {
                ProfScope ps(g, BOLTZ_KCLASS_RADIAL, g->side);
                dp->analysis(ap, ANA_ACCUM, g->side);
            }
            BZ_CUDA(cudaEventRecord(g->ev_free[b], g->side));
        }
        BZ_CUDA(cudaEventRecord(g->ev_join, g->side));
        BZ_CUDA(cudaStreamWaitEvent(st, g->ev_join, 0));
        OutParamsT<R> op{};
        op.qhat = qhat;
        op.fN = fN;
        op.lam = lam_c;
        op.out_start = reinterpret_cast<const int*>(ws + plan.off_plan + c.off_start);
        op.outs = reinterpret_cast<const int4*>(ws + plan.off_plan + c.off_outs);
        op.Q = Q_out;
        op.err = g->d_err;
        op.U = c.U;
        ProfScope ps(g, BOLTZ_KCLASS_OUTPUT, st);
        dp->output(op, st);
    }
    (void)lam;
    BZ_CUDA(cudaGetLastError());
    return BOLTZ_OK;
}

// Projection on the tensor cores (3xTF32 split, FP32-accurate) when the grid
// has at least 512 voxels; a CUDA-core kernel for the tiny 2D grids.
template <int NP>
void launch_project_tc(const float* V, const float* Q, float* partial, int r, int n, int kpc, int* err,
                       cudaStream_t st) {
    const dim3 grid(n / kpc, (r * r + 127) / 128);
    k_project_tc<NP><<<grid, kProjThreads, ProjTcShape<NP>::SMEM, st>>>(V, Q, partial, r, n, kpc, err);
}

cudaError_t prepare_project_tc() {
    cudaError_t e;
    if ((e = set_smem(k_project_tc<16>, ProjTcShape<16>::SMEM)) != cudaSuccess) return e;
    if ((e = set_smem(k_project_tc<32>, ProjTcShape<32>::SMEM)) != cudaSuccess) return e;
    if ((e = set_smem(k_project_tc<48>, ProjTcShape<48>::SMEM)) != cudaSuccess) return e;
    return set_smem(k_project_tc<64>, ProjTcShape<64>::SMEM);
}

// Room for the projection's partial sums: at most 64 voxel slices of r^3.
long long project_partial_floats(int r) { return 64LL * r * r * r; }

// CUDA-core projection (tiny grids, and the allocation-free entry point):
// partial sums of voxel slices, then their reduction in a fixed order with the
// midpoint-rule weight dv^d.  The slice count is bounded by the room in
// `partial` (max_partial floats, at least r^3).  Every partial entry the
// reduction reads is written by k_project of the same call first, so nothing
// an earlier call left in `partial` is ever read.
boltz_status run_project_cuda_cores(boltz_grid_s* g, const float* V, int r, const float* Q, float* T, float* partial,
                                    long long max_partial, cudaStream_t st) {
    constexpr int PB = 8, RT = 16;
    const int r2 = r * r;
    const long long r3 = (long long)r * r2;
    const int bx = (r2 + PB - 1) / PB, bz = (r + RT - 1) / RT;
    int slices = std::max(1, std::min(64, (2 * 152) / std::max(1, bx * bz)));
    slices = std::min(slices, std::max(1, g->n / 256));
    slices = (int)std::max<long long>(1, std::min<long long>(slices, max_partial / r3));
    {
        ProfScope ps(g, BOLTZ_KCLASS_PROJECT, st);
        k_project<PB, RT><<<dim3(bx, slices, bz), 256, 0, st>>>(V, Q, partial, r, g->n, slices);
    }
    const float scale = (float)std::pow(2.0 * g->L / g->N, g->D);
    ProfScope ps(g, BOLTZ_KCLASS_PROJECT, st);
    k_project_reduce<<<(int)((r3 + 255) / 256), 256, 0, st>>>(partial, T, (int)r3, slices, scale);
    BZ_CUDA(cudaGetLastError());
    return BOLTZ_OK;
}

boltz_status run_project(boltz_grid_s* g, const float* V, int r, const float* Q, float* T, float* partial,
                         cudaStream_t st) {
    const int r2 = r * r;
    const int count = r * r2;
    const float scale = (float)std::pow(2.0 * g->L / g->N, g->D);
    int slices;
    if (g->n >= 512 && r > 8) {                             // small r: the CUDA-core kernels fill more SMs
        const int kpc = std::max(512, g->n / 64);           // n is a power of two: kpc divides it
        slices = g->n / kpc;
        ProfScope ps(g, BOLTZ_KCLASS_PROJECT, st);
        if (r <= 16) launch_project_tc<16>(V, Q, partial, r, g->n, kpc, g->d_err, st);
        else if (r <= 32) launch_project_tc<32>(V, Q, partial, r, g->n, kpc, g->d_err, st);
        else if (r <= 48) launch_project_tc<48>(V, Q, partial, r, g->n, kpc, g->d_err, st);
        else launch_project_tc<64>(V, Q, partial, r, g->n, kpc, g->d_err, st);
    } else {
        return run_project_cuda_cores(g, V, r, Q, T, partial, project_partial_floats(r), st);
    }
    ProfScope ps(g, BOLTZ_KCLASS_PROJECT, st);
    k_project_reduce<<<(count + 255) / 256, 256, 0, st>>>(partial, T, count, slices, scale);
    BZ_CUDA(cudaGetLastError());
    return BOLTZ_OK;
}

size_t project_partial_bytes(int r) { return size_t(project_partial_floats(r)) * sizeof(float); }

// FP64 projection of the check build: CUDA-core partial sums over voxel
// slices, reduced in a fixed order (the same kernels as the FP32 fallback for
// tiny grids, on double).
boltz_status run_project64(boltz_grid_s* g, const double* V, int r, const double* Q, double* T, double* partial,
                           cudaStream_t st) {
    constexpr int PB = 4, RT = 8;
    const int r2 = r * r;
    const int count = r * r2;
    const int bx = (r2 + PB - 1) / PB, bz = (r + RT - 1) / RT;
    int slices = std::max(1, std::min(32, (2 * 152) / std::max(1, bx * bz)));
    slices = std::min(slices, std::max(1, g->n / 256));
    {
        ProfScope ps(g, BOLTZ_KCLASS_PROJECT, st);
        k_project<PB, RT, double><<<dim3(bx, slices, bz), 256, 0, st>>>(V, Q, partial, r, g->n, slices);
    }
    ProfScope ps(g, BOLTZ_KCLASS_PROJECT, st);
    k_project_reduce<double><<<(count + 255) / 256, 256, 0, st>>>(partial, T, count, slices,
                                                                 std::pow(2.0 * g->L / g->N, g->D));
    BZ_CUDA(cudaGetLastError());
    return BOLTZ_OK;
}

size_t project64_partial_bytes(int r) { return size_t(32) * r * r * r * sizeof(double); }

// ---------------------------------------------------------------- allocation-free projection
// Partial sums of boltz_project_noalloc: a fixed 2 MiB array that every device
// which loads the library holds until the process exits.  In host code the
// symbol is only a host-side stand-in; kernels get the device address that
// cudaGetSymbolAddress returns for the current device.
constexpr int kNoAllocProjectFloats = 1 << 19;
static __device__ __align__(256) float g_noalloc_project_partial[kNoAllocProjectFloats];

// The array's device address on the current device.  It is resolved with
// cudaGetSymbolAddress on every call made outside stream capture (so that a
// device reset, which reloads the module, cannot leave a stale address), and
// cached per device for calls made while `st` is capturing, which must not
// make that runtime call; the first call on a device must therefore come
// before any capture.
boltz_status noalloc_project_partial(float** out, cudaStream_t st) {
    static std::mutex mu;
    static std::map<int, float*> addr;
    int dev = 0;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        (void)cudaGetLastError();
        return BOLTZ_ECUDA;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_project_partial) != cudaSuccess || p == nullptr) {
            (void)cudaGetLastError();
            return BOLTZ_ECUDA;
        }
        addr[dev] = static_cast<float*>(p);
    }
    auto it = addr.find(dev);
    if (it == addr.end()) return BOLTZ_ECUDA;       // first call on this device made during capture
    *out = it->second;
    return BOLTZ_OK;
}

// The twiddle tables (FP32 and FP64) live in constant memory, once per device.
boltz_status ensure_twiddles(int device) {
    static std::mutex mu;
    static std::set<int> done;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count(device)) return BOLTZ_OK;
    float2 tw[128];
    for (int t = 0; t < 128; ++t)
        tw[t] = make_float2((float)std::cos(-2.0 * kPi * t / 128), (float)std::sin(-2.0 * kPi * t / 128));
    if (cudaMemcpyToSymbol(c_twiddle, tw, sizeof(tw)) != cudaSuccess) return BOLTZ_ECUDA;
    float2 tw48[48];
    for (int t = 0; t < 48; ++t)
        tw48[t] = make_float2((float)std::cos(-2.0 * kPi * t / 48), (float)std::sin(-2.0 * kPi * t / 48));
    if (cudaMemcpyToSymbol(c_twiddle48, tw48, sizeof(tw48)) != cudaSuccess) return BOLTZ_ECUDA;
    double2 twd[128], tw48d[48];
    for (int t = 0; t < 128; ++t) twd[t] = make_double2(std::cos(-2.0 * kPi * t / 128), std::sin(-2.0 * kPi * t / 128));
    for (int t = 0; t < 48; ++t) tw48d[t] = make_double2(std::cos(-2.0 * kPi * t / 48), std::sin(-2.0 * kPi * t / 48));
    if (cudaMemcpyToSymbol(c_twiddle_d, twd, sizeof(twd)) != cudaSuccess) return BOLTZ_ECUDA;
    if (cudaMemcpyToSymbol(c_twiddle48_d, tw48d, sizeof(tw48d)) != cudaSuccess) return BOLTZ_ECUDA;
    done.insert(device);
    return BOLTZ_OK;
}

}  // namespace

// ==================================================================== autotuning

namespace {

// Candidate budgets (MB) for the shifted fields of one radial block: they set
// how many inputs share a chunk and how many radial nodes a launch covers.
const int kBudgetCandidatesMB[] = {48, 96, 192, 384, 768};

// Minimal persistent cache: one JSON object {"key": value, ...} of integers.
std::map<std::string, long> read_cache(const char* path) {
    std::map<std::string, long> m;
    FILE* f = path ? std::fopen(path, "r") : nullptr;
    if (!f) return m;
    std::string text;
    char buf[4096];
    size_t k;
    while ((k = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, k);
    std::fclose(f);
    size_t pos = 0;
    while ((pos = text.find('"', pos)) != std::string::npos) {
        const size_t end = text.find('"', pos + 1);
        if (end == std::string::npos) break;
        const std::string key = text.substr(pos + 1, end - pos - 1);
        const size_t colon = text.find(':', end);
        if (colon == std::string::npos) break;
        m[key] = std::strtol(text.c_str() + colon + 1, nullptr, 10);
        pos = text.find_first_of(",}", colon);
        if (pos == std::string::npos) break;
    }
    return m;
}

bool write_cache(const char* path, const std::map<std::string, long>& m) {
    if (!path) return false;
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return false;
    std::fprintf(f, "{");
    bool first = true;
    for (auto& kv : m) {
        std::fprintf(f, "%s\n  \"%s\": %ld", first ? "" : ",", kv.first.c_str(), kv.second);
        first = false;
    }
    std::fprintf(f, "\n}\n");
    std::fclose(f);
    return std::rename(tmp.c_str(), path) == 0;
}

std::string tune_key(const boltz_grid_s* g, int n_inputs, int n_pairs, int form, int sms) {
    char k[256];
    std::snprintf(k, sizeof(k), "N%d_d%d_M%d_nrho%d_in%d_pairs%d_form%d_sm%d", g->N, g->D, g->M, g->n_rho,
                  n_inputs, n_pairs, form, sms);
    return k;
}

}  // namespace

// ==================================================================== batches

struct boltz_batch_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t origin = nullptr;
    std::vector<cudaStream_t> branch;
    std::vector<cudaEvent_t> events;
    int n_kernels = 0;
};

namespace {

void destroy_batch(boltz_batch_s* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto s : b->branch) cudaStreamDestroy(s);
    for (auto e : b->events) cudaEventDestroy(e);
    if (b->origin) cudaStreamDestroy(b->origin);
    delete b;
}

}  // namespace

// ==================================================================== low-rank step consumers

namespace {

// The FP64 r x r kernels use more than 48 KB of dynamic shared memory: set once per device.
boltz_status ensure_lowrank_attrs() {
    static std::mutex mu;
    static std::set<int> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return BOLTZ_ECUDA;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (done.count(dev)) return BOLTZ_OK;
    if (set_smem(k_chol_f64, kCholSmem) != cudaSuccess || set_smem(k_svd_jacobi_f64, kSvdSmem) != cudaSuccess ||
        set_smem(k_lstep_collision<64>, lstep_smem<64>()) != cudaSuccess ||
        set_smem(k_lr_coupling, kCouplingSmem) != cudaSuccess) {
        (void)cudaGetLastError();
        return BOLTZ_ECUDA;
    }
    done.insert(dev);
    return BOLTZ_OK;
}

int qr_slices(int n) { return std::max(1, std::min(512, n / 128)); }

size_t qr_workspace_bytes(int r, int n) {
    return std::max(align_up(size_t(qr_slices(n) + 2) * r * r * sizeof(double), 256),
                    align_up(qr_spread_bytes(), 256));
}

template <int RMAX>
void launch_qr(const double* W, int r, int n, double w, double* Y, double* R, char* ws, int* info, cudaStream_t st) {
    const int ns = qr_slices(n);
    double* part = reinterpret_cast<double*>(ws);
    double* Rinv = part + size_t(ns) * r * r;
    double* R1 = Rinv + size_t(r) * r;
    const int grid = (n + kLrThreads - 1) / kLrThreads;
    k_gram_f64<<<ns, kLrThreads, 0, st>>>(W, r, n, ns, part);
    k_chol_f64<<<1, kCholThreads, kCholSmem, st>>>(part, ns, r, w, nullptr, R1, Rinv, info);
    k_apply_rinv_f64<RMAX><<<grid, kLrThreads, 0, st>>>(W, Rinv, r, n, Y);
    k_gram_f64<<<ns, kLrThreads, 0, st>>>(Y, r, n, ns, part);
    k_chol_f64<<<1, kCholThreads, kCholSmem, st>>>(part, ns, r, w, R1, R, Rinv, info);
    k_apply_rinv_f64<RMAX><<<grid, kLrThreads, 0, st>>>(Y, Rinv, r, n, Y);
}

// Cholesky-QR2 of boltz_qr_f64.  tickets: two counters of the spread kernels
// that are zero and that nothing else writes (every call leaves them at zero);
// null puts them at the end of the spread layout in ws and clears them first
// (a workspace of unknown contents, which the multi-kernel path also writes).
boltz_status qr_f64_launch(const double* W, int r, int n, double w, double* Y, double* R, char* ws, int* info,
                           cudaStream_t st, unsigned* tickets) {
    boltz_status s = ensure_lowrank_attrs();
    if (s != BOLTZ_OK) return s;
    BZ_CUDA(cudaMemsetAsync(info, 0, sizeof(int), st));
    if (r <= kQrSpreadR && n <= kQrSpreadMaxN) {      // Gram sums and applications over up to 152 CTAs
        const int rows = qr_spread_rows(n), grid = (n + rows - 1) / rows;
        double* wsd = reinterpret_cast<double*>(ws);
        if (!tickets) {
            tickets = reinterpret_cast<unsigned*>(ws + qr_spread_ticket_offset());
            BZ_CUDA(cudaMemsetAsync(tickets, 0, 2 * sizeof(unsigned), st));
        }
        k_qr_spread_f64<0><<<grid, kQrSpreadThreads, 0, st>>>(W, r, n, w, rows, Y, R, wsd, tickets, info);
        k_qr_spread_f64<1><<<grid, kQrSpreadThreads, 0, st>>>(W, r, n, w, rows, Y, R, wsd, tickets, info);
        k_qr_spread_apply<<<(n + kQrSpreadThreads - 1) / kQrSpreadThreads, kQrSpreadThreads, 0, st>>>(Y, r, n, wsd);
    } else if (r <= 16) {
        launch_qr<16>(W, r, n, w, Y, R, ws, info, st);
    } else if (r <= 32) {
        launch_qr<32>(W, r, n, w, Y, R, ws, info, st);
    } else {
        launch_qr<64>(W, r, n, w, Y, R, ws, info, st);
    }
    BZ_CUDA(cudaGetLastError());
    return BOLTZ_OK;
}

}  // namespace

// ==================================================================== C ABI

extern "C" {

int boltz_abi_version(void) { return BOLTZ_ABI_VERSION; }

const char* boltz_status_string(boltz_status s) {
    switch (s) {
        case BOLTZ_OK: return "ok";
        case BOLTZ_EINVAL: return "invalid argument";
        case BOLTZ_ENOMEM: return "out of memory";
        case BOLTZ_ECUDA: return "CUDA error";
        case BOLTZ_ETIMEOUT: return "device wait timed out";
        case BOLTZ_EUNSUPPORTED: return "unsupported configuration";
        case BOLTZ_ENONFINITE: return "non-finite value";
    }
    return "unknown status";
}

boltz_status boltz_host_quadrature(int d_v, int N_rho, int M, double R, double* rho, double* w_rho, double* sigma,
                                   double* w_sigma) {
    if ((d_v != 2 && d_v != 3) || N_rho < 1 || N_rho > 128 || !(R > 0) || !rho || !w_rho || !sigma || !w_sigma)
        return BOLTZ_EINVAL;
    std::vector<double> x, w;
    if (!boltz::gauss_legendre(N_rho, x, w)) return BOLTZ_EINVAL;
    boltz::DirectionRule dr;
    if (!boltz::direction_rule(d_v, M, dr)) return BOLTZ_EINVAL;
    for (int q = 0; q < N_rho; ++q) {
        rho[q] = 0.5 * R * (x[q] + 1.0);
        w_rho[q] = 0.5 * R * w[q];
    }
    for (int p = 0; p < M; ++p) {
        w_sigma[p] = dr.w[p];
        for (int a = 0; a < d_v; ++a) sigma[p * d_v + a] = dr.sigma[p * d_v + a];
    }
    return BOLTZ_OK;
}

boltz_status boltz_grid_init(boltz_grid* out, int N, int d_v, double L, double R, double gamma, int N_rho, int M,
                             const boltz_options* opt) {
    if (!out) return BOLTZ_EINVAL;
    if ((d_v != 2 && d_v != 3) || N < 4 || N % 2 || N > 256 || !(L > 0) || !(R > 0) || !(gamma > -d_v) ||
        !std::isfinite(L) || !std::isfinite(R) || !std::isfinite(gamma) || N_rho < 1 || N_rho > 128)
        return BOLTZ_EINVAL;
    if (d_v == 2 && (M < 2 || M % 2 || M > 256)) return BOLTZ_EINVAL;
    if (d_v == 3 && !(M == 6 || M == 14 || M == 26 || M == 38 || M == 50 || M == 86)) return BOLTZ_EINVAL;
    if (!supported_shape(N, d_v)) return BOLTZ_EUNSUPPORTED;

    boltz_grid_s* g = new (std::nothrow) boltz_grid_s();
    if (!g) return BOLTZ_ENOMEM;
    g->N = N;
    g->D = d_v;
    g->L = L;
    g->R = R;
    g->gamma = gamma;
    g->n_rho = N_rho;
    g->M = M;
    const double area = d_v == 2 ? 2.0 * kPi : 4.0 * kPi;
    g->b = (opt && opt->b > 0) ? opt->b : 1.0 / area;
    if (opt && opt->workspace_max) g->ws_max = opt->workspace_max;
    if (opt && opt->field_budget_mb < 0) {
        delete g;
        return BOLTZ_EINVAL;
    }
    if (opt && opt->field_budget_mb > 0) g->field_budget = size_t(opt->field_budget_mb) << 20;
    if (opt && opt->schedule != BOLTZ_SCHEDULE_AUTO && opt->schedule != BOLTZ_SCHEDULE_NODE_BLOCKS) {
        delete g;
        return BOLTZ_EINVAL;
    }
    if (opt) g->schedule = opt->schedule;
    if (opt && opt->loss != BOLTZ_LOSS_EXACT && opt->loss != BOLTZ_LOSS_MASS_CONSISTENT) {
        delete g;
        return BOLTZ_EINVAL;
    }
    if (opt) g->loss = opt->loss;
    g->n = d_v == 3 ? N * N * N : N * N;
    g->half = d_v == 3 ? N * N * (N / 2 + 1) : N * (N / 2 + 1);
    g->smax = d_v * (N / 2) * (N / 2);
    std::vector<double> x, w;
    boltz::gauss_legendre(N_rho, x, w);
    g->rho.resize(N_rho);
    g->w_rho.resize(N_rho);
    for (int q = 0; q < N_rho; ++q) {
        g->rho[q] = 0.5 * R * (x[q] + 1.0);
        g->w_rho[q] = 0.5 * R * w[q];
    }
    if (!boltz::direction_rule(d_v, M, g->dir)) {
        delete g;
        return BOLTZ_EINVAL;
    }
    // ---- tables in FP64, rounded once to FP32
    const int H = N / 2;
    const int nodes = N_rho * M + 1;
    std::vector<double2> phase64(size_t(nodes) * d_v * N);
    for (int node = 0; node < nodes; ++node) {
        for (int a = 0; a < d_v; ++a) {
            const double s = node < N_rho * M ? 0.5 * g->rho[node / M] * g->dir.sigma[(node % M) * d_v + a] : 0.0;
            for (int i = 0; i < N; ++i) {
                const int k = i < H ? i : i - N;
                double2 v = make_double2(0.0, 0.0);
                if (i != H) {
                    const double ang = -kPi * k * s / L;
                    const double sg = (i & 1) ? -1.0 : 1.0;
                    v = make_double2(sg * std::cos(ang), sg * std::sin(ang));
                }
                phase64[(size_t(node) * d_v + a) * N + i] = v;
            }
        }
    }
    const double kp = gamma + d_v - 1;
    std::vector<double> ctab64(size_t(N_rho) * (g->smax + 1)), gm64(g->smax + 1);
    for (int sq = 0; sq <= g->smax; ++sq) {
        const double km = std::sqrt((double)sq);
        double acc = 0;
        for (int q = 0; q < N_rho; ++q) {
            const double base = g->w_rho[q] * std::pow(g->rho[q], kp);
            ctab64[size_t(q) * (g->smax + 1) + sq] =
                g->b * base * boltz::omega_average(d_v, kPi * g->rho[q] * km / (2.0 * L)) / g->n;
            acc += base * boltz::omega_average(d_v, kPi * g->rho[q] * km / L);
        }
        gm64[sq] = g->b * area * acc;
    }
    // mass-consistent loss: G-(l) = G_sep(l, -l) = b F_d(0) sum_q w_q rho_q^kp
    // sum_p w_p cos(pi rho_q l.sigma_p / L) per half-spectrum mode, the direction
    // sum formed as the real part of a product of per-axis phases
    std::vector<double> gmf64;
    if (g->loss == BOLTZ_LOSS_MASS_CONSISTENT) {
        const int NHh = N / 2 + 1;
        gmf64.assign(g->half, 0.0);
        std::vector<double> er(size_t(d_v) * N), ei(size_t(d_v) * N);
        for (int q = 0; q < N_rho; ++q) {
            const double cq = g->b * area * g->w_rho[q] * std::pow(g->rho[q], kp);   // F_d(0) = |S^{d-1}|
            for (int p = 0; p < M; ++p) {
                const double wq = cq * g->dir.w[p];
                for (int a = 0; a < d_v; ++a)
                    for (int i = 0; i < N; ++i) {
                        const int k = i < H ? i : i - N;
                        const double ang = -kPi * g->rho[q] * k * g->dir.sigma[p * d_v + a] / L;
                        er[size_t(a) * N + i] = std::cos(ang);
                        ei[size_t(a) * N + i] = std::sin(ang);
                    }
                if (d_v == 3) {
                    for (int i0 = 0; i0 < N; ++i0)
                        for (int i1 = 0; i1 < N; ++i1) {
                            const double zr = er[i0] * er[N + i1] - ei[i0] * ei[N + i1];
                            const double zi = er[i0] * ei[N + i1] + ei[i0] * er[N + i1];
                            double* row = &gmf64[(size_t(i0) * N + i1) * NHh];
                            for (int i2 = 0; i2 < NHh; ++i2)
                                row[i2] += wq * (zr * er[2 * N + (i2 % N)] - zi * ei[2 * N + (i2 % N)]);
                        }
                } else {
                    for (int i0 = 0; i0 < N; ++i0)
                        for (int i1 = 0; i1 < NHh; ++i1)
                            gmf64[size_t(i0) * NHh + i1] += wq * (er[i0] * er[N + (i1 % N)] - ei[i0] * ei[N + (i1 % N)]);
                }
            }
        }
    }
    std::vector<float2> phase(phase64.size());
    for (size_t i = 0; i < phase.size(); ++i) phase[i] = make_float2((float)phase64[i].x, (float)phase64[i].y);
    std::vector<float> ctab(ctab64.begin(), ctab64.end()), gm(gm64.begin(), gm64.end());
    // antipodal direction pairs (p, p'), p < p'; the rules are centrally symmetric with w_p = w_p'
    std::vector<float> wdir;
    std::vector<double> wdir64;
    std::vector<int2> dpair;
    for (int p = 0; p < M; ++p) {
        const int pb = g->dir.antipode[p];
        if (pb == p || std::fabs(g->dir.w[p] - g->dir.w[pb]) > 1e-12 * g->dir.w[p]) {
            delete g;
            return BOLTZ_EINVAL;
        }
        if (p < pb) {
            dpair.push_back(make_int2(p, pb));
            wdir.push_back((float)g->dir.w[p]);
            wdir64.push_back(g->dir.w[p]);
        }
    }
    const int n_dp = (int)dpair.size();

    auto fail = [&](boltz_status s) {
        boltz_grid_destroy(g);
        return s;
    };
    if (cudaGetDevice(&g->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess) {
        (void)cudaGetLastError();
        delete g;
        return BOLTZ_ECUDA;
    }
    if (ensure_twiddles(g->device) != BOLTZ_OK) return fail(BOLTZ_ECUDA);
    if (cudaMalloc(&g->d_phase, phase.size() * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&g->d_ctab, ctab.size() * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&g->d_gm, gm.size() * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&g->d_w, n_dp * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&g->d_dpair, n_dp * sizeof(int2)) != cudaSuccess ||
        cudaMalloc(&g->d_err, sizeof(int)) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(BOLTZ_ENOMEM);
    }
    if (cudaMemcpy(g->d_phase, phase.data(), phase.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->d_ctab, ctab.data(), ctab.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->d_gm, gm.data(), gm.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->d_w, wdir.data(), n_dp * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->d_dpair, dpair.data(), n_dp * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(g->d_err, 0, sizeof(int)) != cudaSuccess)
        return fail(BOLTZ_ECUDA);
    if (!gmf64.empty()) {
        std::vector<float> gmf(gmf64.begin(), gmf64.end());
        if (cudaMalloc(&g->d_gmf, gmf.size() * sizeof(float)) != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(BOLTZ_ENOMEM);
        }
        if (cudaMemcpy(g->d_gmf, gmf.data(), gmf.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(BOLTZ_ECUDA);
        if (fp64_shape(N, d_v)) {
            if (cudaMalloc(&g->d_gmf64, gmf64.size() * sizeof(double)) != cudaSuccess) {
                (void)cudaGetLastError();
                return fail(BOLTZ_ENOMEM);
            }
            if (cudaMemcpy(g->d_gmf64, gmf64.data(), gmf64.size() * sizeof(double), cudaMemcpyHostToDevice) !=
                cudaSuccess)
                return fail(BOLTZ_ECUDA);
        }
    }
    if (fp64_shape(N, d_v)) {
        if (cudaMalloc(&g->d_phase64, phase64.size() * sizeof(double2)) != cudaSuccess ||
            cudaMalloc(&g->d_ctab64, ctab64.size() * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&g->d_gm64, gm64.size() * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&g->d_w64, n_dp * sizeof(double)) != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(BOLTZ_ENOMEM);
        }
        if (cudaMemcpy(g->d_phase64, phase64.data(), phase64.size() * sizeof(double2), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemcpy(g->d_ctab64, ctab64.data(), ctab64.size() * sizeof(double), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemcpy(g->d_gm64, gm64.data(), gm64.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(g->d_w64, wdir64.data(), n_dp * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(BOLTZ_ECUDA);
        if (dispatch64_for(N, d_v)->prepare() != cudaSuccess || prepare_contract64() != cudaSuccess)
            return fail(BOLTZ_ECUDA);
    }
    if (dispatch_for(N, d_v)->prepare() != cudaSuccess || prepare_contract() != cudaSuccess ||
        prepare_project_tc() != cudaSuccess)
        return fail(BOLTZ_ECUDA);
    if (d_v == 3 && N == 32) {
        namespace pc = boltz_dev::pencil;
        g->pen_tree = build_pencil_tree(g);
        // Resident CTAs per SM of the pipelined kernel, from its registers,
        // shared memory and tensor-memory columns.  (The runtime's occupancy
        // query reports one CTA per SM for any kernel that allocates tensor
        // memory; three of these CTAs hold 384 of the SM's 512 columns.)
        int regs_sm = 0, smem_sm = 0, resv = 0;
        if (cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, g->device) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, g->device) != cudaSuccess ||
            cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, g->device) != cudaSuccess)
            return fail(BOLTZ_ECUDA);
        auto resident = [&](auto kernel, bool uses_tmem, int& ctas) {
            cudaFuncAttributes fa;
            if (set_smem(kernel, pc::SM_TOTAL) != cudaSuccess || cudaFuncGetAttributes(&fa, kernel) != cudaSuccess)
                return false;
            const int regs_cta = ((fa.numRegs + 7) / 8 * 8) * pc::NT;
            const int smem_cta = (int)fa.sharedSizeBytes + pc::SM_TOTAL + resv;
            int per_sm = std::min(regs_sm / std::max(regs_cta, 1), smem_sm / std::max(smem_cta, 1));
            per_sm = std::min(per_sm, pc::CTAS_PER_SM);
            if (uses_tmem) per_sm = std::min(per_sm, 512 / (int)pc::TMEM_COLS);
            ctas = std::max(per_sm, 0) * g->sms;
            return true;
        };
        if (!resident(pc::k_pencil<false>, true, g->pen_ctas) ||
            !resident(pc::k_pencil<true>, false, g->pen_ctas_diag))
            return fail(BOLTZ_ECUDA);
    }
    if (cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking) != cudaSuccess) return fail(BOLTZ_ECUDA);
    for (int b = 0; b < 2; ++b)
        if (cudaEventCreateWithFlags(&g->ev_ready[b], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&g->ev_free[b], cudaEventDisableTiming) != cudaSuccess)
            return fail(BOLTZ_ECUDA);
    if (cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming) != cudaSuccess)
        return fail(BOLTZ_ECUDA);
    *out = g;
    return BOLTZ_OK;
}

boltz_status boltz_grid_destroy(boltz_grid g) {
    if (!g) return BOLTZ_OK;
    if (g->d_phase || g->d_ws) cudaDeviceSynchronize();
    for (auto& pe : g->prof_events) {
        cudaEventDestroy(pe.second.first);
        cudaEventDestroy(pe.second.second);
    }
    for (auto e : g->event_pool) cudaEventDestroy(e);
    for (int b = 0; b < 2; ++b) {
        if (g->ev_ready[b]) cudaEventDestroy(g->ev_ready[b]);
        if (g->ev_free[b]) cudaEventDestroy(g->ev_free[b]);
    }
    if (g->ev_join) cudaEventDestroy(g->ev_join);
    if (g->ev_fork) cudaEventDestroy(g->ev_fork);
    if (g->side) cudaStreamDestroy(g->side);
    cudaFree(g->d_phase);
    cudaFree(g->d_ctab);
    cudaFree(g->d_gm);
    cudaFree(g->d_gmf);
    cudaFree(g->d_gmf64);
    cudaFree(g->d_w);
    cudaFree(g->d_dpair);
    cudaFree(g->d_err);
    cudaFree(g->d_phase64);
    cudaFree(g->d_ctab64);
    cudaFree(g->d_gm64);
    cudaFree(g->d_w64);
    cudaFree(g->d_smat);
    cudaFree(g->d_scalar);
    cudaFree(g->d_cm_mult);
    cudaFree(g->d_cm_gm);
    cudaFree(g->d_cm_w);
    cudaFree(g->d_cm_dpair);
    cudaFree(g->d_ws);
    delete g;
    return BOLTZ_OK;
}

boltz_status boltz_spectrum(boltz_grid g, const float* f, int n_inputs, void* spectra_out, void* stream) {
    if (!g || n_inputs < 0) return BOLTZ_EINVAL;
    if (n_inputs == 0) return BOLTZ_OK;
    if (!f || !spectra_out) return BOLTZ_EINVAL;
    AnaParams ap{};
    ap.in = f;
    ap.out = reinterpret_cast<float2*>(spectra_out);
    ap.ctab = g->d_ctab;
    ap.n_fields = n_inputs;
    ap.nq = 1;
    ap.inv_n = 1.0f / (float)g->n;
    {
        ProfScope ps(g, BOLTZ_KCLASS_SPECTRUM, reinterpret_cast<cudaStream_t>(stream));
        dispatch_for(g->N, g->D)->analysis(ap, ANA_SPECTRUM, reinterpret_cast<cudaStream_t>(stream));
    }
    BZ_CUDA(cudaGetLastError());
    return BOLTZ_OK;
}

boltz_status boltz_workspace_size(boltz_grid g, int n_inputs, const int32_t* pair_j, const int32_t* pair_l,
                                  int n_pairs, int form, size_t* bytes) {
    if (!g || !bytes || !valid_form(form)) return BOLTZ_EINVAL;
    if (form == BOLTZ_FORM_SPLIT_BF16 && !split_shape(g->N, g->D)) return BOLTZ_EUNSUPPORTED;
    if (form == BOLTZ_FORM_CARLEMAN && !carleman_kernel(g->gamma, g->D)) return BOLTZ_EINVAL;
    if (form == BOLTZ_FORM_CARLEMAN && !carleman_shape(g->N, g->D)) return BOLTZ_EUNSUPPORTED;
    boltz_status s = check_pairs(n_inputs, pair_j, pair_l, n_pairs);
    if (s != BOLTZ_OK) return s;
    if (n_pairs == 0) {
        *bytes = 0;
        return BOLTZ_OK;
    }
    Plan plan;
    if ((s = build_plan(g, n_inputs, pair_j, pair_l, n_pairs, form, plan)) != BOLTZ_OK) return s;
    *bytes = plan.total;
    return BOLTZ_OK;
}

boltz_status boltz_collide_batched(boltz_grid g, const void* spectra, int n_inputs, const int32_t* pair_j,
                                   const int32_t* pair_l, int n_pairs, float* Q_out, int form, void* stream) {
    if (!g || !valid_form(form)) return BOLTZ_EINVAL;
    boltz_status s = check_pairs(n_inputs, pair_j, pair_l, n_pairs);
    if (s != BOLTZ_OK) return s;
    if (n_pairs == 0) return BOLTZ_OK;
    if (!spectra || !Q_out) return BOLTZ_EINVAL;
    s = run_batched(g, reinterpret_cast<const float2*>(spectra), n_inputs, pair_j, pair_l, n_pairs, Q_out, form,
                    reinterpret_cast<cudaStream_t>(stream));
    if (s == BOLTZ_OK && fault_injected("nan")) {
        static const int bit = kErrNonFinite;
        BZ_CUDA(cudaMemcpyAsync(g->d_err, &bit, sizeof(int), cudaMemcpyHostToDevice,
                                reinterpret_cast<cudaStream_t>(stream)));
    }
    return s;
}

boltz_status boltz_project(boltz_grid g, const float* V, int r, const float* Q, float* T_out, void* stream) {
    if (!g || !V || !Q || !T_out || r < 1 || r > 64) return BOLTZ_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // the partial sums go right after the cached plan descriptors (the field
    // buffers behind them are free once earlier work on the stream is done)
    const size_t off = g->plan_uploaded ? align_up(g->last_plan.plan_bytes, 256) : 0;
    boltz_status s = ensure_workspace(g, off + project_partial_bytes(r), st);
    if (s != BOLTZ_OK) return s;
    const size_t off2 = g->plan_uploaded ? align_up(g->last_plan.plan_bytes, 256) : 0;
    return run_project(g, V, r, Q, T_out, reinterpret_cast<float*>(g->d_ws + off2), st);
}

boltz_status boltz_project_noalloc(boltz_grid g, const float* V, int r, const float* Q, float* T_out,
                                   void* stream) {
    if (!g || !V || !Q || !T_out || r < 1 || r > 64) return BOLTZ_EINVAL;
    const long long r3 = (long long)r * r * r;
    if (r3 > kNoAllocProjectFloats) return BOLTZ_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    float* partial = nullptr;
    boltz_status s = noalloc_project_partial(&partial, st);
    if (s != BOLTZ_OK) return s;
    return run_project_cuda_cores(g, V, r, Q, T_out, partial, kNoAllocProjectFloats, st);
}

boltz_status boltz_spectrum_f64(boltz_grid g, const double* f, int n_inputs, void* spectra_out, void* stream) {
    if (!g || n_inputs < 0) return BOLTZ_EINVAL;
    if (!fp64_shape(g->N, g->D)) return BOLTZ_EUNSUPPORTED;
    if (n_inputs == 0) return BOLTZ_OK;
    if (!f || !spectra_out) return BOLTZ_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    AnaParamsT<double> ap{};
    ap.in = f;
    ap.out = reinterpret_cast<double2*>(spectra_out);
    ap.ctab = g->d_ctab64;
    ap.n_fields = n_inputs;
    ap.nq = 1;
    ap.inv_n = 1.0 / (double)g->n;
    {
        ProfScope ps(g, BOLTZ_KCLASS_SPECTRUM, st);
        dispatch64_for(g->N, g->D)->analysis(ap, ANA_SPECTRUM, st);
    }
    BZ_CUDA(cudaGetLastError());
    return BOLTZ_OK;
}

boltz_status boltz_collide_batched_f64(boltz_grid g, const void* spectra, int n_inputs, const int32_t* pair_j,
                                       const int32_t* pair_l, int n_pairs, double* Q_out, int form, void* stream) {
    if (!g || !valid_form(form)) return BOLTZ_EINVAL;
    if (!fp64_shape(g->N, g->D)) return BOLTZ_EUNSUPPORTED;
    boltz_status s = check_pairs(n_inputs, pair_j, pair_l, n_pairs);
    if (s != BOLTZ_OK) return s;
    if (n_pairs == 0) return BOLTZ_OK;
    if (!spectra || !Q_out) return BOLTZ_EINVAL;
    return run_batched<double>(g, reinterpret_cast<const double2*>(spectra), n_inputs, pair_j, pair_l, n_pairs, Q_out,
                               form, reinterpret_cast<cudaStream_t>(stream));
}

boltz_status boltz_project_f64(boltz_grid g, const double* V, int r, const double* Q, double* T_out, void* stream) {
    if (!g || !V || !Q || !T_out || r < 1 || r > 64) return BOLTZ_EINVAL;
    if (!fp64_shape(g->N, g->D)) return BOLTZ_EUNSUPPORTED;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t off = g->plan_uploaded ? align_up(g->last_plan.plan_bytes, 256) : 0;
    boltz_status s = ensure_workspace(g, off + project64_partial_bytes(r), st);
    if (s != BOLTZ_OK) return s;
    const size_t off2 = g->plan_uploaded ? align_up(g->last_plan.plan_bytes, 256) : 0;
    return run_project64(g, V, r, Q, T_out, reinterpret_cast<double*>(g->d_ws + off2), st);
}

boltz_status boltz_lowrank_step_host(boltz_grid g, const float* V_host, int r, float* Q_host, float* T_host,
                                     void* stream) {
    if (!g || !V_host || !T_host || r < 1 || r > 64) return BOLTZ_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int r2 = r * r;
    std::vector<int32_t> pj(r2), pl(r2);
    for (int j = 0; j < r; ++j)
        for (int l = 0; l < r; ++l) {
            pj[j * r + l] = j;
            pl[j * r + l] = l;
        }
    // the grid's cached plan of the all-pairs batch (built on the host only when r changes;
    // run_batched uploads it again if the workspace below has to grow)
    boltz_status s = prepare_plan(g, r, pj.data(), pl.data(), r2, BOLTZ_FORM_BATCHED, 0, st);
    if (s != BOLTZ_OK) return s;
    const size_t plan_total = g->last_plan.total;
    // staging after the batched workspace: V, spectra, Q, T, partial sums
    const size_t nb = size_t(g->n) * 4;
    size_t off_V = align_up(plan_total, 256);
    size_t off_S = align_up(off_V + size_t(r) * nb, 256);
    size_t off_Q = align_up(off_S + size_t(r) * g->half * 8, 256);
    size_t off_T = align_up(off_Q + size_t(r2) * nb, 256);
    size_t off_part = align_up(off_T + size_t(r) * r2 * 4, 256);
    size_t total = align_up(off_part + project_partial_bytes(r), 256);
    if ((s = ensure_workspace(g, total, st)) != BOLTZ_OK) return s;
    float* dV = reinterpret_cast<float*>(g->d_ws + off_V);
    float2* dS = reinterpret_cast<float2*>(g->d_ws + off_S);
    float* dQ = reinterpret_cast<float*>(g->d_ws + off_Q);
    float* dT = reinterpret_cast<float*>(g->d_ws + off_T);
    float* dP = reinterpret_cast<float*>(g->d_ws + off_part);
    BZ_CUDA(cudaMemcpyAsync(dV, V_host, size_t(r) * nb, cudaMemcpyHostToDevice, st));
    if ((s = boltz_spectrum(g, dV, r, dS, stream)) != BOLTZ_OK) return s;
    if ((s = run_batched(g, dS, r, pj.data(), pl.data(), r2, dQ, BOLTZ_FORM_BATCHED, st)) != BOLTZ_OK) return s;
    // Q goes back to the host on the side stream while the projection (which
    // only reads Q) runs on the caller's stream
    if (Q_host) {
        BZ_CUDA(cudaEventRecord(g->ev_fork, st));
        BZ_CUDA(cudaStreamWaitEvent(g->side, g->ev_fork, 0));
        BZ_CUDA(cudaMemcpyAsync(Q_host, dQ, size_t(r2) * nb, cudaMemcpyDeviceToHost, g->side));
        BZ_CUDA(cudaEventRecord(g->ev_join, g->side));
    }
    if ((s = run_project(g, dV, r, dQ, dT, dP, st)) != BOLTZ_OK) return s;
    BZ_CUDA(cudaMemcpyAsync(T_host, dT, size_t(r) * r2 * 4, cudaMemcpyDeviceToHost, st));
    if (Q_host) BZ_CUDA(cudaStreamWaitEvent(st, g->ev_join, 0));
    BZ_CUDA(cudaStreamSynchronize(st));
    return BOLTZ_OK;
}

boltz_status boltz_mott_smith(boltz_grid g, const void* spectra, double rho_L, double u_L, double T_L, double T_R,
                              double R_gas, float* Q_scratch, double* alpha, double* beta, void* stream) {
    if (!g || !spectra || !Q_scratch || !alpha || !beta) return BOLTZ_EINVAL;
    const double denom = (g->D - 1) * rho_L * u_L * R_gas * (T_L - T_R);
    if (!std::isfinite(denom) || denom == 0.0) return BOLTZ_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!g->d_scalar) {
        if (cudaMalloc(&g->d_scalar, 8 * sizeof(double)) != cudaSuccess) {
            (void)cudaGetLastError();
            g->d_scalar = nullptr;
            return BOLTZ_ENOMEM;
        }
    }
    const int32_t pj[2] = {0, 1}, pl[2] = {1, 0};     // Q(f_L, f_R), Q(f_R, f_L)
    boltz_status s = run_batched(g, reinterpret_cast<const float2*>(spectra), 2, pj, pl, 2, Q_scratch,
                                 BOLTZ_FORM_BATCHED, st);
    if (s != BOLTZ_OK) return s;
    const double dv = 2.0 * g->L / g->N;
    if (g->D == 3) k_axis0_second_moment<3><<<1, 256, 0, st>>>(Q_scratch, 2, g->N, g->L, dv, g->d_scalar);
    else k_axis0_second_moment<2><<<1, 256, 0, st>>>(Q_scratch, 2, g->N, g->L, dv, g->d_scalar);
    BZ_CUDA(cudaGetLastError());
    double a = 0.0;
    BZ_CUDA(cudaMemcpyAsync(&a, g->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, st));
    BZ_CUDA(cudaStreamSynchronize(st));
    *alpha = a;
    *beta = a / denom;
    return BOLTZ_OK;
}

boltz_status boltz_moments(boltz_grid g, const float* Q, int n_fields, double* out, void* stream) {
    if (!g || n_fields < 0) return BOLTZ_EINVAL;
    if (n_fields == 0) return BOLTZ_OK;
    if (!Q || !out) return BOLTZ_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const double dv = 2.0 * g->L / g->N;
    if (g->D == 3) k_moments<3><<<n_fields, 256, 0, st>>>(Q, out, g->N, g->L, dv);
    else k_moments<2><<<n_fields, 256, 0, st>>>(Q, out, g->N, g->L, dv);
    BZ_CUDA(cudaGetLastError());
    return BOLTZ_OK;
}

boltz_status boltz_batch_plan(boltz_batch* out, const boltz_work* items, int n_items, int form) {
    if (!out || !items || n_items <= 0 || !valid_form(form))
        return BOLTZ_EINVAL;
    for (int i = 0; i < n_items; ++i) {
        const boltz_work& w = items[i];
        if (!w.grid || !w.spectra || !w.Q_out || w.n_pairs <= 0) return BOLTZ_EINVAL;
        boltz_status s = check_pairs(w.n_inputs, w.pair_j, w.pair_l, w.n_pairs);
        if (s != BOLTZ_OK) return s;
        if (w.V && (!w.T_out || w.r < 1 || w.r > 64 || w.r * w.r != w.n_pairs)) return BOLTZ_EINVAL;
        for (int k = 0; k < i; ++k)
            if (items[k].grid == w.grid) return BOLTZ_EINVAL;      // one item per grid
        if (form == BOLTZ_FORM_SPLIT_BF16) {
            if (!split_shape(w.grid->N, w.grid->D)) return BOLTZ_EUNSUPPORTED;
            if ((s = ensure_split_tables(w.grid)) != BOLTZ_OK) return s;
        }
        if (form == BOLTZ_FORM_CARLEMAN) {
            if (!carleman_kernel(w.grid->gamma, w.grid->D)) return BOLTZ_EINVAL;
            if (!carleman_shape(w.grid->N, w.grid->D)) return BOLTZ_EUNSUPPORTED;
            if ((s = ensure_carleman_tables(w.grid)) != BOLTZ_OK) return s;
        }
    }
    boltz_batch_s* b = new (std::nothrow) boltz_batch_s();
    if (!b) return BOLTZ_ENOMEM;
    auto fail = [&](boltz_status st) {
        destroy_batch(b);
        return st;
    };
    if (cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess) return fail(BOLTZ_ECUDA);
    // plans and workspaces first: nothing may allocate or synchronise during capture
    for (int i = 0; i < n_items; ++i) {
        const boltz_work& w = items[i];
        const size_t proj = w.V ? align_up(0, 256) + project_partial_bytes(w.r) : 0;
        boltz_status s = prepare_plan(w.grid, w.n_inputs, w.pair_j, w.pair_l, w.n_pairs, form, 0, b->origin);
        if (s != BOLTZ_OK) return fail(s);
        const size_t need = align_up(w.grid->last_plan.plan_bytes, 256) + proj;
        if (w.grid->ws_cap < need) {
            if ((s = prepare_plan(w.grid, w.n_inputs, w.pair_j, w.pair_l, w.n_pairs, form, need, b->origin)) !=
                BOLTZ_OK)
                return fail(s);
        }
        cudaStream_t br;
        cudaEvent_t ev;
        if (cudaStreamCreateWithFlags(&br, cudaStreamNonBlocking) != cudaSuccess) return fail(BOLTZ_ECUDA);
        b->branch.push_back(br);
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return fail(BOLTZ_ECUDA);
        b->events.push_back(ev);
    }
    cudaEvent_t fork;
    if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) return fail(BOLTZ_ECUDA);
    b->events.push_back(fork);
    if (cudaStreamSynchronize(b->origin) != cudaSuccess) return fail(BOLTZ_ECUDA);
    // capture: one branch per item, forked from and joined to the origin stream
    if (cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return fail(BOLTZ_ECUDA);
    boltz_status cs = BOLTZ_OK;
    if (cudaEventRecord(fork, b->origin) != cudaSuccess) cs = BOLTZ_ECUDA;
    for (int i = 0; i < n_items && cs == BOLTZ_OK; ++i) {
        const boltz_work& w = items[i];
        boltz_grid_s* g = w.grid;
        const bool prof = g->prof_on;
        long long saved[BOLTZ_KCLASS_COUNT];
        std::memcpy(saved, g->launches, sizeof(saved));
        g->prof_on = false;
        cudaStream_t br = b->branch[i];
        if (cudaStreamWaitEvent(br, fork, 0) != cudaSuccess) cs = BOLTZ_ECUDA;
        if (cs == BOLTZ_OK && w.fields) cs = boltz_spectrum(g, w.fields, w.n_inputs, const_cast<void*>(w.spectra), br);
        if (cs == BOLTZ_OK)
            cs = run_batched(g, reinterpret_cast<const float2*>(w.spectra), w.n_inputs, w.pair_j, w.pair_l,
                             w.n_pairs, w.Q_out, form, br);
        if (cs == BOLTZ_OK && w.V) {
            float* partial = reinterpret_cast<float*>(g->d_ws + align_up(g->last_plan.plan_bytes, 256));
            cs = run_project(g, w.V, w.r, w.Q_out, w.T_out, partial, br);
        }
        if (cs == BOLTZ_OK && (cudaEventRecord(b->events[i], br) != cudaSuccess ||
                               cudaStreamWaitEvent(b->origin, b->events[i], 0) != cudaSuccess))
            cs = BOLTZ_ECUDA;
        g->prof_on = prof;
        std::memcpy(g->launches, saved, sizeof(saved));
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->origin, &graph);
    b->graph = graph;
    if (cs != BOLTZ_OK || ec != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(cs != BOLTZ_OK ? cs : BOLTZ_ECUDA);
    }
    if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) return fail(BOLTZ_ECUDA);
    size_t nn = 0;
    if (cudaGraphGetNodes(b->graph, nullptr, &nn) != cudaSuccess) return fail(BOLTZ_ECUDA);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn && cudaGraphGetNodes(b->graph, nodes.data(), &nn) != cudaSuccess) return fail(BOLTZ_ECUDA);
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++b->n_kernels;
    }
    *out = b;
    return BOLTZ_OK;
}

boltz_status boltz_batch_run(boltz_batch b, void* stream) {
    if (!b || !b->exec) return BOLTZ_EINVAL;
    BZ_CUDA(cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(stream)));
    return BOLTZ_OK;
}

boltz_status boltz_batch_kernel_count(boltz_batch b, int* n_kernels) {
    if (!b || !n_kernels) return BOLTZ_EINVAL;
    *n_kernels = b->n_kernels;
    return BOLTZ_OK;
}

boltz_status boltz_batch_destroy(boltz_batch b) {
    if (!b) return BOLTZ_OK;
    cudaDeviceSynchronize();
    destroy_batch(b);
    return BOLTZ_OK;
}

boltz_status boltz_autotune(boltz_grid g, const void* spectra, int n_inputs, const int32_t* pair_j,
                            const int32_t* pair_l, int n_pairs, float* Q_scratch, int form, const char* cache_path,
                            void* stream, int* chosen_mb) {
    if (!g || !valid_form(form)) return BOLTZ_EINVAL;
    boltz_status s = check_pairs(n_inputs, pair_j, pair_l, n_pairs);
    if (s != BOLTZ_OK) return s;
    if (n_pairs == 0 || !spectra || !Q_scratch) return BOLTZ_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess) return BOLTZ_ECUDA;
    const std::string key = tune_key(g, n_inputs, n_pairs, form, sms);
    auto cache = read_cache(cache_path);
    auto it = cache.find(key);
    long best_mb = -1;
    if (it != cache.end() && it->second > 0) {
        best_mb = it->second;
    } else {
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return BOLTZ_ECUDA;
        float best_ms = 1e30f;
        for (int mb : kBudgetCandidatesMB) {
            g->field_budget = size_t(mb) << 20;
            g->plan_uploaded = false;
            float ms_sum = 0.f;
            boltz_status rs = BOLTZ_OK;
            for (int rep = 0; rep < 3 && rs == BOLTZ_OK; ++rep) {         // rep 0 warms up
                cudaEventRecord(e0, st);
                rs = run_batched(g, reinterpret_cast<const float2*>(spectra), n_inputs, pair_j, pair_l, n_pairs,
                                 Q_scratch, form, st);
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) rs = BOLTZ_ECUDA;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) ms_sum += ms;
            }
            if (rs == BOLTZ_ENOMEM) continue;                               // candidate too large
            if (rs != BOLTZ_OK) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return rs;
            }
            if (ms_sum < best_ms) {
                best_ms = ms_sum;
                best_mb = mb;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (best_mb < 0) return BOLTZ_ENOMEM;
        if (cache_path) {
            cache[key] = best_mb;
            write_cache(cache_path, cache);
        }
    }
    g->field_budget = size_t(best_mb) << 20;
    g->plan_uploaded = false;
    if (chosen_mb) *chosen_mb = (int)best_mb;
    return BOLTZ_OK;
}

boltz_status boltz_sync_status(boltz_grid g, void* stream) {
    if (!g) return BOLTZ_EINVAL;
    BZ_CUDA(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
    int err = 0;
    BZ_CUDA(cudaMemcpy(&err, g->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        BZ_CUDA(cudaMemset(g->d_err, 0, sizeof(int)));
        if (err & kErrTimeout) return BOLTZ_ETIMEOUT;
        return (err & kErrNonFinite) ? BOLTZ_ENONFINITE : BOLTZ_ECUDA;
    }
    return BOLTZ_OK;
}

boltz_status boltz_selftest(boltz_grid g, int which, void* stream) {
    if (!g || which != 0) return BOLTZ_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    k_selftest_wait_timeout<<<1, 32, 0, st>>>(g->d_err);
    BZ_CUDA(cudaGetLastError());
    return boltz_sync_status(g, stream);
}

boltz_status boltz_profile_enable(boltz_grid g, int enable) {
    if (!g) return BOLTZ_EINVAL;
    g->prof_on = enable != 0;
    return BOLTZ_OK;
}

boltz_status boltz_profile_read(boltz_grid g, int reset, long long* launches, double* ms) {
    if (!g || !launches || !ms) return BOLTZ_EINVAL;
    for (int c = 0; c < BOLTZ_KCLASS_COUNT; ++c) {
        launches[c] = g->launches[c];
        ms[c] = 0.0;
    }
    for (auto& pe : g->prof_events) {
        float t = 0.f;
        if (cudaEventSynchronize(pe.second.second) != cudaSuccess ||
            cudaEventElapsedTime(&t, pe.second.first, pe.second.second) != cudaSuccess)
            return BOLTZ_ECUDA;
        ms[pe.first] += t;
    }
    if (reset) {
        for (auto& pe : g->prof_events) {
            g->event_pool.push_back(pe.second.first);
            g->event_pool.push_back(pe.second.second);
        }
        g->prof_events.clear();
        for (int c = 0; c < BOLTZ_KCLASS_COUNT; ++c) g->launches[c] = 0;
    }
    return BOLTZ_OK;
}

boltz_status boltz_kstep_collision(const float* T, int r, const float* K, int n_x, float* C_out, void* stream) {
    if (r < 1 || r > 64 || n_x < 0) return BOLTZ_EINVAL;
    if (n_x == 0) return BOLTZ_OK;
    if (!T || !K || !C_out) return BOLTZ_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // j-chunks of at most 48 KB of T; enough block rows to give every SM work
    const int gx = (n_x + kLrThreads - 1) / kLrThreads;
    const int jmax = std::max(1, std::min(r, 12288 / (r * r)));
    const int jt = std::max(1, std::min(jmax, (r * gx + 303) / 304));
    const dim3 grid(gx, (r + jt - 1) / jt);
    const size_t smem = size_t(jt) * r * r * sizeof(float);
    if (r <= 16) k_kstep_collision<16><<<grid, kLrThreads, smem, st>>>(T, K, C_out, r, n_x, jt);
    else if (r <= 32) k_kstep_collision<32><<<grid, kLrThreads, smem, st>>>(T, K, C_out, r, n_x, jt);
    else k_kstep_collision<64><<<grid, kLrThreads, smem, st>>>(T, K, C_out, r, n_x, jt);
    BZ_CUDA(cudaGetLastError());
    return BOLTZ_OK;
}

boltz_status boltz_lstep_collision(const float* Q, int r, const float* C, int n_v, float* G_out, void* stream) {
    if (r < 1 || r > 64 || n_v < 0) return BOLTZ_EINVAL;
    if (n_v == 0) return BOLTZ_OK;
    if (!Q || !C || !G_out) return BOLTZ_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    boltz_status s = ensure_lowrank_attrs();
    if (s != BOLTZ_OK) return s;
    const int grid = (n_v + kLstepVB - 1) / kLstepVB;
    if (r <= 16) k_lstep_collision<16><<<grid, kLrThreads, lstep_smem<16>(), st>>>(Q, C, G_out, r, n_v);
    else if (r <= 32) k_lstep_collision<32><<<grid, kLrThreads, lstep_smem<32>(), st>>>(Q, C, G_out, r, n_v);
    else k_lstep_collision<64><<<grid, kLrThreads, lstep_smem<64>(), st>>>(Q, C, G_out, r, n_v);
    BZ_CUDA(cudaGetLastError());
    return BOLTZ_OK;
}

boltz_status boltz_lowrank_coupling(const float* E, const float* S, int r, const float* T, float* C_out,
                                    float* D_out, void* stream) {
    if (r < 1 || r > 64 || !E || !S || !C_out || (T && !D_out)) return BOLTZ_EINVAL;
    boltz_status s = ensure_lowrank_attrs();
    if (s != BOLTZ_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    k_lr_coupling<<<r, kLrThreads, kCouplingSmem, st>>>(E, S, T, r, C_out, D_out);
    BZ_CUDA(cudaGetLastError());
    return BOLTZ_OK;
}

boltz_status boltz_qr_f64_workspace(int r, int n, size_t* bytes) {
    if (r < 1 || r > 64 || n < r || !bytes) return BOLTZ_EINVAL;
    *bytes = qr_workspace_bytes(r, n);
    return BOLTZ_OK;
}

boltz_status boltz_qr_f64(const double* W, int r, int n, double w, double* Y, double* R, void* workspace,
                          int* info, void* stream) {
    if (r < 1 || r > 64 || n < r || !(w > 0) || !std::isfinite(w) || !W || !Y || !R || !workspace || !info)
        return BOLTZ_EINVAL;
    return qr_f64_launch(W, r, n, w, Y, R, static_cast<char*>(workspace), info,
                         reinterpret_cast<cudaStream_t>(stream), nullptr);
}

boltz_status boltz_svd_truncate_f64(const double* S, int r, double drop_tol, double* U, double* sigma, double* Q,
                                    int* r_keep, int* info, void* stream) {
    if (r < 1 || r > 64 || !(drop_tol >= 0) || !std::isfinite(drop_tol) || !S || !U || !sigma || !Q || !r_keep ||
        !info)
        return BOLTZ_EINVAL;
    boltz_status s = ensure_lowrank_attrs();
    if (s != BOLTZ_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (r <= kSvdSmallR) k_svd_small_f64<<<1, 32, 0, st>>>(S, r, drop_tol, U, sigma, Q, r_keep, info);
    else k_svd_jacobi_f64<<<1, 1024, kSvdSmem, st>>>(S, r, drop_tol, U, sigma, Q, r_keep, info);
    BZ_CUDA(cudaGetLastError());
    return BOLTZ_OK;
}

boltz_status boltz_basis_rotate_f64(const double* X, int r, int n, const double* U, int r_new, double* X_out,
                                    void* stream) {
    if (r < 1 || r > 64 || n < 0 || r_new < 0 || r_new > r) return BOLTZ_EINVAL;
    if (n == 0 || r_new == 0) return BOLTZ_OK;
    if (!X || !U || !X_out || X_out == X) return BOLTZ_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int grid = (n + kLrThreads - 1) / kLrThreads;
    if (r <= 8) k_rotate_f64<8><<<grid, kLrThreads, 0, st>>>(X, U, r, r_new, n, X_out);
    else if (r <= 16) k_rotate_f64<16><<<grid, kLrThreads, 0, st>>>(X, U, r, r_new, n, X_out);
    else if (r <= 32) k_rotate_f64<32><<<grid, kLrThreads, 0, st>>>(X, U, r, r_new, n, X_out);
    else k_rotate_f64<64><<<grid, kLrThreads, 0, st>>>(X, U, r, r_new, n, X_out);
    BZ_CUDA(cudaGetLastError());
    return BOLTZ_OK;
}

}  // extern "C"

// ==================================================================== 1D normal shock

struct boltz_shock_s {
    boltz_grid g = nullptr;
    int n_x = 0, n_v = 0, r_max = 0, rb = 0, form = 0;
    double dx = 0, wv = 0;
    char* mem = nullptr;
    double *fL = nullptr, *fR = nullptr, *v1 = nullptr;
    // full tensor
    double* f_next = nullptr;
    float *fx32 = nullptr, *Qx = nullptr;
    void* spec_x = nullptr;
    std::vector<int32_t> pair_x;
    // low rank
    double *Vh = nullptr, *K = nullptr, *K1 = nullptr, *X1 = nullptr, *S1 = nullptr, *S2 = nullptr, *L = nullptr,
           *L1 = nullptr, *Kt = nullptr, *Vn = nullptr, *R = nullptr, *Sn = nullptr, *U = nullptr, *Qm = nullptr,
           *sig = nullptr, *Ap = nullptr, *Am = nullptr, *Pl = nullptr, *Pr = nullptr, *bl = nullptr,
           *br = nullptr, *Bp = nullptr, *Bm = nullptr, *cvec = nullptr,
           *nrm = nullptr, *Pk = nullptr, *Gv = nullptr, *nk = nullptr, *nl = nullptr, *errd = nullptr;
    float *V32 = nullptr, *Q32 = nullptr, *T32 = nullptr, *K32 = nullptr, *C32 = nullptr, *E32 = nullptr,
          *S32 = nullptr, *D32 = nullptr, *Cs32 = nullptr, *G32 = nullptr;
    void* spec_v = nullptr;
    void* qr_ws = nullptr;
    int* d_int = nullptr;                 // [0] QR info (K), [1] QR info (L), [2] r_keep, [3] SVD info,
                                          // [4] skip bits of a replayed step (1: a boundary vector not
                                          // kept, 2: a QR or the rank failed), [8] k_sh_change's ticket,
                                          // [10..11] the spread QR's tickets
    double* d_tol = nullptr;              // drop_tol of a replayed step
    boltz_dev::AugState* aug = nullptr;   // scratch of the basis augmentation
    // replayed steps: one CUDA graph per (rank, X, S, V, dt) seen twice, both boundary
    // vectors kept; h_pin: [0] drop_tol, [1..2] d_int[0..4] read back, [3] the step's err
    double* h_pin = nullptr;
    cudaStream_t cap_stream = nullptr;
    struct GraphKey {
        int r;
        const double *X, *S, *V;
        double dt;
        bool operator<(const GraphKey& o) const {
            return std::tie(r, X, S, V, dt) < std::tie(o.r, o.X, o.S, o.V, o.dt);
        }
    };
    struct StepGraph {
        cudaGraphExec_t exec = nullptr;
        char* ws = nullptr;               // the grid workspace the graph's kernels read
    };
    std::map<GraphKey, StepGraph> graphs;
    std::set<GraphKey> seen, direct_only;    // keys seen once; keys whose replay found a vector not kept
};

namespace {

int sh_grid(size_t n) { return (int)std::min<size_t>((n + boltz_dev::kShT - 1) / boltz_dev::kShT, 4096); }

}  // namespace

extern "C" {

boltz_status boltz_shock_create(boltz_grid g, int n_x, double L_x, const double* f_L, const double* f_R, int r_max,
                                int form, boltz_shock* out) {
    if (!g || !out || !f_L || !f_R || n_x < 2 || !(L_x > 0) || !std::isfinite(L_x) || r_max < 3 || r_max > 64 ||
        !valid_form(form))
        return BOLTZ_EINVAL;
    boltz_shock s = new (std::nothrow) boltz_shock_s;
    if (!s) return BOLTZ_ENOMEM;
    s->g = g;
    s->n_x = n_x;
    s->n_v = g->n;
    s->r_max = r_max;
    s->form = form;
    s->dx = 2.0 * L_x / n_x;
    s->wv = std::pow(2.0 * g->L / g->N, g->D);
    const size_t nv = s->n_v, nx = n_x, rm = r_max, half = g->half;
    size_t qr_bytes = 0;
    boltz_qr_f64_workspace(r_max, (int)std::max<size_t>(std::max(nx, nv), rm), &qr_bytes);
    // one allocation, 256-byte aligned pieces
    std::vector<std::pair<void**, size_t>> parts = {
        {(void**)&s->fL, nv * 8}, {(void**)&s->fR, nv * 8}, {(void**)&s->v1, nv * 8},
        {(void**)&s->f_next, nx * nv * 8}, {(void**)&s->fx32, nx * nv * 4}, {(void**)&s->Qx, nx * nv * 4},
        {(void**)&s->spec_x, nx * half * 8},
        {(void**)&s->Vh, rm * nv * 8}, {(void**)&s->K, rm * nx * 8}, {(void**)&s->K1, rm * nx * 8},
        {(void**)&s->X1, rm * nx * 8}, {(void**)&s->S1, rm * rm * 8}, {(void**)&s->S2, rm * rm * 8},
        {(void**)&s->L, rm * nv * 8}, {(void**)&s->L1, rm * nv * 8}, {(void**)&s->Kt, rm * nx * 8},
        {(void**)&s->Vn, rm * nv * 8}, {(void**)&s->R, rm * rm * 8}, {(void**)&s->Sn, rm * rm * 8},
        {(void**)&s->U, rm * rm * 8}, {(void**)&s->Qm, rm * rm * 8}, {(void**)&s->sig, rm * 8},
        {(void**)&s->Ap, rm * rm * 8}, {(void**)&s->Am, rm * rm * 8},
        {(void**)&s->Pl, rm * rm * 8}, {(void**)&s->Pr, rm * rm * 8}, {(void**)&s->bl, rm * 8},
        {(void**)&s->br, rm * 8},
        {(void**)&s->Bp, rm * rm * 8}, {(void**)&s->Bm, rm * rm * 8}, {(void**)&s->cvec, rm * 8},
        {(void**)&s->nrm, 4 * 8}, {(void**)&s->Pk, rm * rm * 8}, {(void**)&s->Gv, rm * rm * 8},
        {(void**)&s->nk, rm * 8}, {(void**)&s->nl, rm * 8}, {(void**)&s->errd, 8},
        {(void**)&s->V32, rm * nv * 4}, {(void**)&s->Q32, rm * rm * nv * 4}, {(void**)&s->T32, rm * rm * rm * 4},
        {(void**)&s->K32, rm * nx * 4}, {(void**)&s->C32, rm * nx * 4}, {(void**)&s->E32, rm * rm * rm * 4},
        {(void**)&s->S32, rm * rm * 4}, {(void**)&s->D32, rm * rm * 4}, {(void**)&s->Cs32, rm * rm * rm * 4},
        {(void**)&s->G32, rm * nv * 4}, {(void**)&s->spec_v, rm * half * 8}, {&s->qr_ws, qr_bytes},
        {(void**)&s->d_int, 64}, {(void**)&s->d_tol, 8}, {(void**)&s->aug, sizeof(boltz_dev::AugState)}};
    size_t total = 0;
    for (auto& pt : parts) total = align_up(total + pt.second, 256);
    if (cudaMalloc(&s->mem, total) != cudaSuccess) {
        (void)cudaGetLastError();
        delete s;
        return BOLTZ_ENOMEM;
    }
    size_t off = 0;
    for (auto& pt : parts) {
        *pt.first = s->mem + off;
        off = align_up(off + pt.second, 256);
    }
    // the tickets of the spread QR, k_sh_change and the augmentation start at zero (each launch
    // leaves them so)
    if (cudaMemset(s->d_int, 0, 64) != cudaSuccess ||
        cudaMemset(s->aug, 0, sizeof(boltz_dev::AugState)) != cudaSuccess) {
        boltz_shock_destroy(s);
        return BOLTZ_ECUDA;
    }
    // inflow Maxwellians and the v_1 coordinate of every grid point (axis 0 is v_1)
    std::vector<double> v1(nv);
    const double dv = 2.0 * g->L / g->N;
    const size_t inner = nv / g->N;
    for (size_t k = 0; k < nv; ++k) v1[k] = -g->L + (double)(k / inner) * dv;
    if (cudaMemcpy(s->fL, f_L, nv * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(s->fR, f_R, nv * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(s->v1, v1.data(), nv * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
        boltz_shock_destroy(s);
        return BOLTZ_ECUDA;
    }
    // rank of the boundary data F_b = [f_L; f_R] (Sec. 3.1: singular values >= 1e-10 kept),
    // from its 2 x 2 Gram matrix on the device
    boltz_dev::k_sh_rowdots<<<1, boltz_dev::kShT>>>(s->fL, (int)nv, s->fL, 1.0, s->cvec);
    boltz_dev::k_sh_rowdots<<<1, boltz_dev::kShT>>>(s->fL, (int)nv, s->fR, 1.0, s->cvec + 1);
    boltz_dev::k_sh_rowdots<<<1, boltz_dev::kShT>>>(s->fR, (int)nv, s->fR, 1.0, s->cvec + 2);
    double gm[3];
    if (cudaMemcpy(gm, s->cvec, 3 * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
        boltz_shock_destroy(s);
        return BOLTZ_ECUDA;
    }
    const double a = gm[0], b = gm[1], d = gm[2];
    const double mid = 0.5 * (a + d), rad = std::sqrt(0.25 * (a - d) * (a - d) + b * b);
    s->rb = (std::sqrt(std::max(mid + rad, 0.0)) >= 1e-10) + (std::sqrt(std::max(mid - rad, 0.0)) >= 1e-10);
    s->pair_x.resize(n_x);
    for (int p = 0; p < n_x; ++p) s->pair_x[p] = p;
    if (cudaMallocHost(&s->h_pin, 64) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        boltz_shock_destroy(s);
        return BOLTZ_ENOMEM;
    }
    *out = s;
    return BOLTZ_OK;
}

boltz_status boltz_shock_destroy(boltz_shock s) {
    if (!s) return BOLTZ_OK;
    cudaDeviceSynchronize();
    for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second.exec);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    cudaFreeHost(s->h_pin);
    cudaFree(s->mem);
    delete s;
    return BOLTZ_OK;
}

boltz_status boltz_shock_full_step(boltz_shock s, double* f, int n_steps, double dt, void* stream) {
    if (!s || !f || n_steps < 0 || !(dt > 0) || !std::isfinite(dt)) return BOLTZ_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t n = (size_t)s->n_x * s->n_v;
    for (int k = 0; k < n_steps; ++k) {
        boltz_dev::k_sh_to_f32<<<sh_grid(n), boltz_dev::kShT, 0, st>>>(f, s->fx32, n);
        boltz_status rs = boltz_spectrum(s->g, s->fx32, s->n_x, s->spec_x, stream);
        if (rs != BOLTZ_OK) return rs;
        rs = boltz_collide_batched(s->g, s->spec_x, s->n_x, s->pair_x.data(), s->pair_x.data(), s->n_x, s->Qx,
                                   s->form, stream);
        if (rs != BOLTZ_OK) return rs;
        boltz_dev::k_sh_full<<<sh_grid(n), boltz_dev::kShT, 0, st>>>(f, s->Qx, s->fL, s->fR, s->v1, s->n_x, s->n_v,
                                                                     dt, s->dx, s->f_next);
        BZ_CUDA(cudaMemcpyAsync(f, s->f_next, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    BZ_CUDA(cudaGetLastError());
    return BOLTZ_OK;
}

}  // extern "C"

namespace {

// The collision batch and steps 1-4 of a low-rank step on the augmented basis
// Vh of rh rows (filled by the caller): the collision batch of all ordered
// pairs of Vh and its projection, the K-, S- and L-steps (Sec. 2.4), the
// change of f over the step (Sec. 5.1) and the SVD of the new S with the drop
// tolerance (Sec. 3.2).  drop_tol_dev, when not null, replaces drop_tol.
boltz_status lr_core(boltz_shock s, const double* X, const double* S, int r, int rh, double dt, double drop_tol,
                     const double* drop_tol_dev, cudaStream_t st) {
    using namespace boltz_dev;
    const int T = kShT, nx = s->n_x, nv = s->n_v;
    void* stream = reinterpret_cast<void*>(st);
    boltz_status rs;
    // K = X^T S on the old rows, zero on the added ones (the added directions carry no weight)
    k_sh_comb<false><<<sh_grid((size_t)r * nx), T, 0, st>>>(X, r, nx, S, r, r, s->K);
    if (rh > r) BZ_CUDA(cudaMemsetAsync(s->K + (size_t)r * nx, 0, (size_t)(rh - r) * nx * 8, st));
    // velocity Grams of V_hat, boundary projections
    k_sh_vgram<<<dim3(rh, rh + 1), T, 0, st>>>(s->Vh, rh, nv, s->v1, s->fL, s->fR, s->wv, s->Ap, s->Am, s->Pl, s->Pr,
                                              s->bl, s->br);
    // collision batch of all ordered pairs of V_hat and its projection T_jmn
    k_sh_to_f32<<<sh_grid((size_t)rh * nv), T, 0, st>>>(s->Vh, s->V32, (size_t)rh * nv);
    if ((rs = boltz_spectrum(s->g, s->V32, rh, s->spec_v, stream)) != BOLTZ_OK) return rs;
    std::vector<int32_t> pm(rh * rh), pn(rh * rh);
    for (int k = 0; k < rh * rh; ++k) {
        pm[k] = k / rh;
        pn[k] = k % rh;
    }
    if ((rs = boltz_collide_batched(s->g, s->spec_v, rh, pm.data(), pn.data(), rh * rh, s->Q32, s->form, stream)) !=
        BOLTZ_OK)
        return rs;
    if ((rs = boltz_project(s->g, s->V32, rh, s->Q32, s->T32, stream)) != BOLTZ_OK) return rs;
    // 1. K-step (Sec. 2.4 K-step): Euler with the upwind transport and the collision term, then QR
    k_sh_to_f32<<<sh_grid((size_t)rh * nx), T, 0, st>>>(s->K, s->K32, (size_t)rh * nx);
    if ((rs = boltz_kstep_collision(s->T32, rh, s->K32, nx, s->C32, stream)) != BOLTZ_OK) return rs;
    k_sh_kupdate<<<sh_grid((size_t)rh * nx), T, 0, st>>>(s->K, s->C32, s->Ap, s->Am, s->Pl, s->Pr, s->bl, s->br, rh, nx,
                                                         dt, s->dx,
                                                         s->K1);
    if ((rs = qr_f64_launch(s->K1, rh, nx, s->dx, s->X1, s->S1, static_cast<char*>(s->qr_ws), s->d_int, st,
                            reinterpret_cast<unsigned*>(s->d_int + 10))) != BOLTZ_OK)
        return rs;
    // 2. S-step (Sec. 2.4 S-step): transport through the updated K, collision term with S1
    k_sh_xgram<<<dim3(rh, rh), T, 0, st>>>(s->X1, s->K1, s->Pl, s->Pr, s->bl, s->br, rh, nx, s->Bp, s->Bm);
    k_sh_triple<<<dim3(rh, rh), T, 0, st>>>(s->X1, rh, nx, s->dx, s->E32);
    k_sh_to_f32<<<1, T, 0, st>>>(s->S1, s->S32, (size_t)rh * rh);
    if ((rs = boltz_lowrank_coupling(s->E32, s->S32, rh, s->T32, s->Cs32, s->D32, stream)) != BOLTZ_OK) return rs;
    k_sh_supdate<<<1, 1024, 0, st>>>(s->S1, s->Ap, s->Am, s->Bp, s->Bm, s->D32, rh, dt, s->S2);
    // 3. L-step (Sec. 2.4 L-step): L = S2 V, transport through K~ = X'^T S2, collision term, then QR
    k_sh_comb<true><<<sh_grid((size_t)rh * nv), T, 0, st>>>(s->Vh, rh, nv, s->S2, rh, rh, s->L);
    k_sh_comb<false><<<sh_grid((size_t)rh * nx), T, 0, st>>>(s->X1, rh, nx, s->S2, rh, rh, s->Kt);
    k_sh_xgram<<<dim3(rh, rh), T, 0, st>>>(s->X1, s->Kt, s->Pl, s->Pr, s->bl, s->br, rh, nx, s->Bp, s->Bm);
    k_sh_to_f32<<<1, T, 0, st>>>(s->S2, s->S32, (size_t)rh * rh);
    if ((rs = boltz_lowrank_coupling(s->E32, s->S32, rh, nullptr, s->Cs32, nullptr, stream)) != BOLTZ_OK) return rs;
    if ((rs = boltz_lstep_collision(s->Q32, rh, s->Cs32, nv, s->G32, stream)) != BOLTZ_OK) return rs;
    k_sh_lupdate<<<sh_grid((size_t)rh * nv), T, 0, st>>>(s->L, s->Vh, s->v1, s->Bp, s->Bm, s->G32, rh, nv, dt, s->L1);
    if ((rs = qr_f64_launch(s->L1, rh, nv, s->wv, s->Vn, s->R, static_cast<char*>(s->qr_ws), s->d_int + 1, st,
                            reinterpret_cast<unsigned*>(s->d_int + 10))) != BOLTZ_OK)
        return rs;
    k_sh_transpose<<<1, T, 0, st>>>(s->R, rh, rh, s->Sn);          // L_i = sum_j R_ji V'_j
    // change of f over the step from the increments (Sec. 5.1), before the drop
    k_sh_change<<<2 * rh + 2 * rh * rh, T, 0, st>>>(s->K1, s->K, s->X1, s->L1, s->L, s->Vh, rh, nx, nv, s->dx, s->wv,
                                                   s->S1, s->S2, s->nk, s->nl, s->Pk, s->Gv,
                                                   reinterpret_cast<unsigned*>(s->d_int + 8), s->errd);
    // 4. drop (Sec. 3.2): SVD of S, keep sigma >= drop_tol
    if ((rs = ensure_lowrank_attrs()) != BOLTZ_OK) return rs;
    if (rh <= kSvdSmallR)
        k_svd_small_f64<<<1, 32, 0, st>>>(s->Sn, rh, drop_tol, s->U, s->sig, s->Qm, s->d_int + 2, s->d_int + 3,
                                          drop_tol_dev);
    else
        k_svd_jacobi_f64<<<1, 1024, kSvdSmem, st>>>(s->Sn, rh, drop_tol, s->U, s->sig, s->Qm, s->d_int + 2, s->d_int + 3,
                                                drop_tol_dev);
    BZ_CUDA(cudaGetLastError());
    return BOLTZ_OK;
}

// Rotation of the bases by the kept singular vectors: X <- X1 U, V <- Vn Qm,
// S <- diag(sigma); r_dev / skip as in k_rotate_f64 (null: the host's rk).
void lr_rotate(boltz_shock s, double* X, double* S, double* V, int rh, int rk, const int* r_dev, const int* skip,
               cudaStream_t st) {
    using namespace boltz_dev;
    const int gx = (s->n_x + kLrThreads - 1) / kLrThreads, gv = (s->n_v + kLrThreads - 1) / kLrThreads;
    // the smallest bound >= rh: unused slots of the unrolled sums still cost FP64 issue
    if (rh <= 8) {
        k_rotate_f64<8><<<gx, kLrThreads, 0, st>>>(s->X1, s->U, rh, rk, s->n_x, X, r_dev, skip);
        k_rotate_f64<8><<<gv, kLrThreads, 0, st>>>(s->Vn, s->Qm, rh, rk, s->n_v, V, r_dev, skip);
    } else if (rh <= 16) {
        k_rotate_f64<16><<<gx, kLrThreads, 0, st>>>(s->X1, s->U, rh, rk, s->n_x, X, r_dev, skip);
        k_rotate_f64<16><<<gv, kLrThreads, 0, st>>>(s->Vn, s->Qm, rh, rk, s->n_v, V, r_dev, skip);
    } else if (rh <= 32) {
        k_rotate_f64<32><<<gx, kLrThreads, 0, st>>>(s->X1, s->U, rh, rk, s->n_x, X, r_dev, skip);
        k_rotate_f64<32><<<gv, kLrThreads, 0, st>>>(s->Vn, s->Qm, rh, rk, s->n_v, V, r_dev, skip);
    } else {
        k_rotate_f64<64><<<gx, kLrThreads, 0, st>>>(s->X1, s->U, rh, rk, s->n_x, X, r_dev, skip);
        k_rotate_f64<64><<<gv, kLrThreads, 0, st>>>(s->Vn, s->Qm, rh, rk, s->n_v, V, r_dev, skip);
    }
    k_sh_diag<<<1, kShT, 0, st>>>(s->sig, rk, S, r_dev, skip);
}

// Step 0, adding the boundary basis (Sec. 3.1): V_hat = [V; f_L, f_R
// orthonormalised against V by Gram-Schmidt, twice].  KEEP_ALL (a replayed
// step): both are appended and the device records whether that was right;
// otherwise a vector keeping less than 1e-10 of its norm lies in span(V)
// already and is not appended (it would carry no weight and make the K-step
// QR singular), a decision read back on the host.  Up to 31 basis columns
// the augmentation runs on the k_aug_* kernels (inner products spread over
// up to 128 CTAs, 3 launches per vector), beyond that as a chain of dot,
// subtract and normalise kernels.  Returns rh.
template <bool KEEP_ALL>
boltz_status lr_append(boltz_shock s, const double* V, int r, int* rh_out, cudaStream_t st) {
    using namespace boltz_dev;
    const int T = kShT, nv = s->n_v;
    BZ_CUDA(cudaMemcpyAsync(s->Vh, V, (size_t)r * nv * 8, cudaMemcpyDeviceToDevice, st));
    int rh = r;
    if (r + s->rb <= kAugR && s->rb <= 2) {
        const int G = (int)std::min<size_t>(std::max<size_t>((nv + kAugT - 1) / kAugT, 1), kAugCtas);
        // RM: the smallest instantiated bound >= the columns (unused slots still cost FP64 issue)
        auto with_rm = [](int rc, auto&& f) {
            if (rc <= 2) f(std::integral_constant<int, 2>{});
            else if (rc <= 4) f(std::integral_constant<int, 4>{});
            else if (rc <= 6) f(std::integral_constant<int, 6>{});
            else if (rc <= 8) f(std::integral_constant<int, 8>{});
            else if (rc <= 16) f(std::integral_constant<int, 16>{});
            else f(std::integral_constant<int, 32>{});
        };
        auto start = [&](int rc, const double* src, int scale_prev, int k) {
            with_rm(rc, [&](auto RMc) {
                k_aug_start<decltype(RMc)::value>
                    <<<G, kAugT, 0, st>>>(s->Vh, rc, nv, s->wv, src, scale_prev, s->nrm, k, s->aug);
            });
        };
        auto update = [&](int rc, int k, int* skip) {
            with_rm(rc, [&](auto RMc) {
                constexpr int RM = decltype(RMc)::value;
                k_aug_update<RM, 0><<<G, kAugT, 0, st>>>(s->Vh, rc, nv, s->wv, s->nrm, k, skip, s->aug);
                k_aug_update<RM, 1><<<G, kAugT, 0, st>>>(s->Vh, rc, nv, s->wv, s->nrm, k, skip, s->aug);
            });
        };
        if constexpr (KEEP_ALL) {
            // both vectors, the first scaled at the start of the second
            for (int k = 0; k < s->rb; ++k) {
                start(r + k, k == 0 ? s->fL : s->fR, k > 0, k);
                update(r + k, k, s->d_int + 4);
            }
            k_aug_scale<<<G, kAugT, 0, st>>>(s->Vh, r + s->rb - 1, nv, s->aug);
            *rh_out = r + s->rb;
            return BOLTZ_OK;
        }
        for (int k = 0; k < s->rb; ++k) {
            start(rh, k == 0 ? s->fL : s->fR, 0, 0);
            update(rh, 0, nullptr);
            double hn[2];
            BZ_CUDA(cudaMemcpyAsync(hn, s->nrm, sizeof(hn), cudaMemcpyDeviceToHost, st));
            BZ_CUDA(cudaStreamSynchronize(st));
            if (hn[1] > 1e-20 * hn[0]) {
                k_aug_scale<<<G, kAugT, 0, st>>>(s->Vh, rh, nv, s->aug);
                ++rh;
            }
        }
        *rh_out = rh;
        return BOLTZ_OK;
    }
    for (int k = 0; k < s->rb; ++k) {
        double* b = s->Vh + (size_t)rh * nv;
        const double* src = k == 0 ? s->fL : s->fR;
        BZ_CUDA(cudaMemcpyAsync(b, src, (size_t)nv * 8, cudaMemcpyDeviceToDevice, st));
        k_sh_rowdots<<<1, T, 0, st>>>(src, nv, src, 1.0, s->nrm);
        for (int pass = 0; pass < 2; ++pass) {
            k_sh_rowdots<<<rh, T, 0, st>>>(s->Vh, nv, b, s->wv, s->cvec);
            k_sh_subtract<<<sh_grid(nv), T, 0, st>>>(b, s->Vh, s->cvec, rh, nv);
        }
        k_sh_rowdots<<<1, T, 0, st>>>(b, nv, b, 1.0, s->nrm + 1);
        if constexpr (KEEP_ALL) {
            k_sh_keep_check<<<1, 32, 0, st>>>(s->nrm, s->d_int + 4);
        } else {
            double hn[2];
            BZ_CUDA(cudaMemcpyAsync(hn, s->nrm, sizeof(hn), cudaMemcpyDeviceToHost, st));
            BZ_CUDA(cudaStreamSynchronize(st));
            if (!(hn[1] > 1e-20 * hn[0])) continue;
        }
        k_sh_normalize<<<1, T, 0, st>>>(b, nv, s->wv);
        ++rh;
    }
    *rh_out = rh;
    return BOLTZ_OK;
}

// One low-rank step with every decision made on the host (the reference path).
boltz_status lr_step_direct(boltz_shock s, double* X, double* S, double* V, int* r_io, double dt, double drop_tol,
                            double* err_out, cudaStream_t st) {
    const int r = *r_io;
    int rh = r;
    boltz_status rs;
    if ((rs = lr_append<false>(s, V, r, &rh, st)) != BOLTZ_OK) return rs;
    if ((rs = lr_core(s, X, S, r, rh, dt, drop_tol, nullptr, st)) != BOLTZ_OK) return rs;
    int hinfo[4] = {0, 0, 0, 0};
    double herr = 0.0;
    BZ_CUDA(cudaMemcpyAsync(hinfo, s->d_int, sizeof(hinfo), cudaMemcpyDeviceToHost, st));
    BZ_CUDA(cudaMemcpyAsync(&herr, s->errd, sizeof(double), cudaMemcpyDeviceToHost, st));
    BZ_CUDA(cudaStreamSynchronize(st));
    if (err_out) *err_out = herr;
    if (hinfo[0] != 0 || hinfo[1] != 0) return BOLTZ_ENONFINITE;       // a QR met linearly dependent rows
    const int rk = hinfo[2];
    if (rk < 1) return BOLTZ_ENONFINITE;
    lr_rotate(s, X, S, V, rh, rk, nullptr, nullptr, st);
    BZ_CUDA(cudaGetLastError());
    *r_io = rk;
    return BOLTZ_OK;
}

// The launches of a replayed step (captured once): both boundary vectors
// appended, drop_tol from s->d_tol (copied from the pinned h_pin[0] by the
// graph's first node), the rank-dependent tail driven by the device's r_keep
// and skip bits, and the values the host needs copied back to h_pin.
boltz_status lr_step_graph_body(boltz_shock s, double* X, double* S, double* V, int r, double dt, cudaStream_t st) {
    using namespace boltz_dev;
    boltz_status rs;
    BZ_CUDA(cudaMemcpyAsync(s->d_tol, s->h_pin, sizeof(double), cudaMemcpyHostToDevice, st));
    BZ_CUDA(cudaMemsetAsync(s->d_int + 4, 0, sizeof(int), st));
    int rh = r;
    if ((rs = lr_append<true>(s, V, r, &rh, st)) != BOLTZ_OK) return rs;
    if ((rs = lr_core(s, X, S, r, rh, dt, 0.0, s->d_tol, st)) != BOLTZ_OK) return rs;
    k_sh_step_check<<<1, 32, 0, st>>>(s->d_int, s->d_int + 4);
    lr_rotate(s, X, S, V, rh, rh, s->d_int + 2, s->d_int + 4, st);
    BZ_CUDA(cudaMemcpyAsync(s->h_pin + 1, s->d_int, 5 * sizeof(int), cudaMemcpyDeviceToHost, st));
    BZ_CUDA(cudaMemcpyAsync(s->h_pin + 4, s->errd, sizeof(double), cudaMemcpyDeviceToHost, st));
    BZ_CUDA(cudaGetLastError());
    return BOLTZ_OK;
}

// Whether the grid's cached plan is the all-pairs batch of n inputs in `form`.
bool plan_is_all_pairs(const boltz_grid_s* g, int n, int form) {
    if (!g->plan_uploaded || g->last_form != form || g->last_n_inputs != n || g->last_elem != 4 ||
        (int)g->last_j.size() != n * n)
        return false;
    for (int k = 0; k < n * n; ++k)
        if (g->last_j[k] != k / n || g->last_l[k] != k % n) return false;
    return true;
}

}  // namespace

extern "C" {

boltz_status boltz_shock_lowrank_step(boltz_shock s, double* X, double* S, double* V, int* r_io, double dt,
                                      double drop_tol, double* err_out, void* stream) {
    if (!s || !X || !S || !V || !r_io || !(dt > 0) || !std::isfinite(dt) || !(drop_tol >= 0) ||
        !std::isfinite(drop_tol))
        return BOLTZ_EINVAL;
    const int r = *r_io, nx = s->n_x;
    if (r < 1 || r + s->rb > s->r_max || r + s->rb > nx) return BOLTZ_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    boltz_grid_s* g = s->g;
    // Replayed steps: a step with the same (rank, X, S, V, dt) as an earlier one, both
    // boundary vectors kept, runs as one CUDA graph, with one host synchronisation
    // instead of three and no per-kernel launch cost.  The first such step runs
    // directly (it also leaves the grid's all-pairs plan cached for the graph); the
    // graph is captured at the second and replayed while the grid's workspace and
    // cached plan stay those it was captured with.  A replay that finds a boundary
    // vector in span(V) writes nothing, and the step runs directly.
    const boltz_shock_s::GraphKey key{r, X, S, V, dt};
    const int rh = r + s->rb;
    const char* env = std::getenv("BOLTZ_SHOCK_GRAPH");
    const bool eligible = s->rb == 2 && !g->prof_on && !fault_injected("badplan") && !fault_injected("alloc") &&
                          !(env && std::strcmp(env, "0") == 0) && !s->direct_only.count(key);
    if (eligible && s->seen.count(key) && plan_is_all_pairs(g, rh, s->form)) {
        auto it = s->graphs.find(key);
        if (it != s->graphs.end() && it->second.ws != g->d_ws) {
            cudaGraphExecDestroy(it->second.exec);
            s->graphs.erase(it);
            it = s->graphs.end();
        }
        if (it == s->graphs.end()) {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            bool ok = cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                const boltz_status rs = lr_step_graph_body(s, X, S, V, r, dt, s->cap_stream);
                ok = cudaStreamEndCapture(s->cap_stream, &graph) == cudaSuccess && rs == BOLTZ_OK;
                ok = ok && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
                if (graph) cudaGraphDestroy(graph);
            }
            (void)cudaGetLastError();
            if (ok) it = s->graphs.emplace(key, boltz_shock_s::StepGraph{exec, g->d_ws}).first;
            else if (exec) cudaGraphExecDestroy(exec);
        }
        if (it != s->graphs.end()) {
            s->h_pin[0] = drop_tol;
            BZ_CUDA(cudaGraphLaunch(it->second.exec, st));
            BZ_CUDA(cudaStreamSynchronize(st));
            int hinfo[5];
            std::memcpy(hinfo, s->h_pin + 1, sizeof(hinfo));
            if (!(hinfo[4] & 1)) {
                if (err_out) *err_out = s->h_pin[4];
                if (hinfo[0] != 0 || hinfo[1] != 0 || hinfo[2] < 1) return BOLTZ_ENONFINITE;
                *r_io = hinfo[2];
                return BOLTZ_OK;
            }
            s->direct_only.insert(key);            // this basis keeps dropping a boundary vector
            cudaGraphExecDestroy(it->second.exec);
            s->graphs.erase(it);
        }
    }
    if (eligible) s->seen.insert(key);
    return lr_step_direct(s, X, S, V, r_io, dt, drop_tol, err_out, st);
}

boltz_status boltz_shock_reconstruct(boltz_shock s, const double* X, const double* S, const double* V, int r,
                                     double* f, void* stream) {
    if (!s || !X || !S || !V || !f || r < 1 || r > s->r_max) return BOLTZ_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int T = boltz_dev::kShT, nx = s->n_x, nv = s->n_v;
    boltz_dev::k_sh_comb<true><<<sh_grid((size_t)r * nv), T, 0, st>>>(V, r, nv, S, r, r, s->L);
    boltz_dev::k_sh_outer<<<sh_grid((size_t)nx * nv), T, 0, st>>>(X, s->L, r, nx, nv, f);
    BZ_CUDA(cudaGetLastError());
    return BOLTZ_OK;
}

}  // extern "C"
