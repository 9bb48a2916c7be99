// ff_api.cu -- C-ABI of libff: contexts, feature pyramids, match plans (merged launches over many pairs, CUDA-graph
// capture and replay), profiling.  The operations follow FlowFields++ (arXiv 1805.03517), Sec. 3.1.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "ff.h"
#include "ff_internal.h"

using namespace ff;

namespace {

constexpr int kMaxDim = 8192;
// The initial matching compares every pixel of the coarsest level with every other one (work and CTA counts grow
// with the square of its pixel count), so the coarsest level is limited to 2^20 pixels.
constexpr int kMaxCoarsePixels = 1 << 20;
constexpr size_t kAlign = 256;

size_t align_up(size_t v, size_t a = kAlign) { return (v + a - 1) / a * a; }
int round_up(int v, int a) { return (v + a - 1) / a * a; }

void level_dims(int w, int h, int L, int* ws, int* hs) {
    ws[0] = w;
    hs[0] = h;
    for (int s = 1; s < L; s++) {
        ws[s] = std::max(1, ws[s - 1] / 2);
        hs[s] = std::max(1, hs[s - 1] / 2);
    }
}

// A device allocation owned by a context.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct ff_pyr {
    int w = 0, h = 0, L = 0;
    int ws[kMaxLevels] = {}, hs[kMaxLevels] = {};
    uint8_t* img[kMaxLevels] = {};   // levels 1..L-1 (level 0 is the caller's image, read only by ff_features)
    int16_t* feat[kMaxLevels] = {};
    uint32_t* cen[kMaxLevels] = {};  // Census patterns [h][w][8] (contexts with the Census cost only)
    int8_t* seed_desc = nullptr;     // [n_pad][64]
    int32_t* seed_norm = nullptr;    // [n_coarse]
    int n_coarse = 0, n_pad = 0;
    void* desc16 = nullptr;          // f16 [n_pad128][64] for the tensor-core seed
    void* tmap = nullptr;            // device copy of its TMA tensor map (128 B)
    int n_pad128 = 0;
    DevBuf mem;
    bool in_use = false;
};

namespace {

enum class Kind { Memset, Seed, SeedTc, Handover, Propagate, Consistency, ConsistencyTab };

struct Launch {
    Kind kind;
    int phase;
    int level = -1;
    int desc_level = -1;     // the finest pyramid level whose descriptors the launch reads (-1: none)
    // seed / handover / propagate: problem arrays in the plan's device table
    const void* probs = nullptr;
    int n_probs = 0;
    int total = 0;           // row tiles (seed) / queue length (propagate)
    int64_t total_pix = 0;   // handover
    const int2* queue = nullptr;
    int* counter = nullptr;
    int grid = 0;
    PropLaunch prop{};
    // consistency
    const uint32_t* fwd = nullptr;
    const uint32_t* bwd = nullptr;
    const uint32_t* bwd2 = nullptr;
    int w = 0, h = 0, eps = 0;
    uint8_t* mask = nullptr;
    // memset
    void* set_ptr = nullptr;
    size_t set_bytes = 0;
    int set_value = 0;
    // hand-over
    int cost = 0;
    // tensor-core seed
    uint32_t wait_limit = 0;
    int withhold = 0;
    int* err = nullptr;
};

// One direction of one pair.
struct DirJob {
    const ff_pyr* a;
    const ff_pyr* b;
    int dir;            // 0 forward, 1 inverse, 2 second inverse (its own random stream)
    uint32_t* flow_out;
    int32_t* cost_out;  // may be null
    int rs_radius;
};
struct ConsJob {
    int dj_fwd, dj_bwd;  // indices into the plan's DirJobs
    uint8_t* mask;
    int dj_bwd2;         // second inverse field, or -1
};

struct Plan {
    std::vector<uintptr_t> key;
    std::vector<Launch> launches;
    std::vector<DevBuf> bufs;
    cudaGraphExec_t exec = nullptr;
    int graph_nodes = 0;
    int cluster_nodes = 0;  // of graph_nodes: propagation launches of the cluster form
    // ff_match_frames: the same launches in one graph with the fine levels' descriptor launch on a branch from
    // launch split_at[0] to launch split_at[1], for the descriptor table split_tab (split_n entries, split_tiles CTAs)
    cudaGraphExec_t split_exec = nullptr;
    size_t split_at[2] = {0, 0};
    const void* split_tab = nullptr;
    int split_n = 0, split_tiles = 0;
    int split_nodes = 0, split_clusters = 0;
};

// The descriptor launch of the fine pyramid levels that ff_match_frames runs beside the coarse levels' matching.
struct FineWht {
    const WhtLevel* tab = nullptr;  // device table of the fine levels (in the context's feature table)
    int n = 0;                      // entries
    int tiles = 0;                  // CTAs
};

struct TileCfg {
    int tw, th, k, threads, spec;  // tile interior, iterations fused per launch, CTA size, speculative random
    int cluster = 0;               // > 0: the cluster form with this many CTAs per problem (tw, th unused)
    int dataflow = 0;              // 1: the dataflow form (every iteration in one launch; k unused), 2: affine
};

// Candidate propagation configurations (tile shape, fused iterations, CTA size) the autotuner times per level.
const TileCfg kCands[] = {
    {64, 32, 1, 256, 0}, {32, 32, 1, 256, 0}, {32, 16, 1, 256, 0}, {16, 16, 1, 256, 0}, {32, 16, 2, 256, 0},
    {16, 16, 2, 256, 0}, {16, 8, 2, 256, 0},  {16, 8, 3, 256, 0},  {8, 8, 3, 256, 0},   {8, 8, 6, 256, 0},
    {32, 16, 1, 128, 0}, {16, 16, 1, 128, 0}, {16, 8, 2, 128, 0},  {8, 8, 3, 128, 0},   {32, 32, 1, 512, 0},
    {32, 16, 2, 512, 0}, {16, 16, 2, 512, 0}, {24, 24, 1, 512, 0}, {32, 16, 1, 128, 1}, {16, 16, 1, 128, 1},
    {16, 8, 2, 128, 1},  {8, 8, 3, 128, 1},   {32, 16, 1, 256, 1}, {16, 16, 1, 256, 1}, {16, 8, 2, 256, 1},
    {8, 8, 3, 256, 1},   {32, 32, 1, 512, 1}, {16, 16, 2, 512, 1}, {24, 24, 1, 512, 1},
    // coarse levels: one pixel per thread per half-sweep (fewer dependent loads in a row)
    {8, 8, 3, 512, 0},   {8, 8, 2, 512, 0},   {16, 8, 2, 512, 0},   {16, 16, 1, 512, 0}, {8, 8, 3, 512, 1},
    {16, 8, 2, 512, 1},  {16, 16, 1, 512, 1}, {8, 8, 6, 512, 0},   {8, 8, 6, 512, 1},
    // fine levels: larger tiles recompute a smaller share of halo pixels
    {64, 32, 1, 128, 0}, {48, 32, 1, 128, 0}, {48, 32, 1, 256, 0}, {64, 16, 1, 128, 0}, {40, 24, 1, 128, 0},
    {48, 24, 1, 128, 0}, {64, 24, 1, 256, 0}, {64, 24, 1, 128, 0}, {96, 24, 1, 256, 0}, {80, 24, 1, 256, 0},
    {128, 16, 1, 256, 0}, {96, 32, 1, 256, 0}, {64, 24, 1, 512, 0}, {64, 20, 1, 256, 0}, {48, 24, 1, 256, 0},
    {64, 16, 1, 256, 0}, {96, 16, 1, 256, 0}, {128, 24, 1, 512, 0}, {96, 24, 1, 128, 0}, {80, 24, 1, 128, 0},
    {96, 32, 1, 128, 0}, {80, 32, 1, 128, 0}, {64, 28, 1, 128, 0}, {56, 24, 1, 128, 0}, {72, 24, 1, 128, 0},
    {64, 20, 1, 128, 0}, {24, 16, 1, 512, 0}, {32, 16, 1, 512, 0}, {20, 16, 1, 512, 0}, {26, 16, 1, 512, 0},
    // the cluster form (every iteration in one launch, no halo): small levels of a few problems
    {0, 0, 255, 256, 0, 16}, {0, 0, 255, 512, 0, 16}, {0, 0, 255, 256, 0, 8}, {0, 0, 255, 512, 0, 8},
    // the dataflow form (every iteration in one launch, tiles start as their neighbours finish): without a last
    // wave to fill, the fine levels can take larger tiles (a smaller share of halo pixels)
    {50, 32, 1, 256, 0, 0, 1},  {64, 32, 1, 256, 0, 0, 1},  {80, 32, 1, 256, 0, 0, 1},  {96, 32, 1, 256, 0, 0, 1},
    {128, 32, 1, 256, 0, 0, 1}, {64, 40, 1, 256, 0, 0, 1},  {64, 48, 1, 256, 0, 0, 1},  {96, 24, 1, 256, 0, 0, 1},
    {128, 24, 1, 256, 0, 0, 1}, {48, 32, 1, 256, 0, 0, 1},  {64, 24, 1, 256, 0, 0, 1},  {32, 32, 1, 256, 0, 0, 1},
    {32, 16, 1, 256, 0, 0, 1},  {16, 16, 1, 256, 0, 0, 1},  {8, 8, 1, 256, 0, 0, 1},    {48, 24, 1, 128, 0, 0, 1},
    {64, 24, 1, 128, 0, 0, 1},  {32, 32, 1, 128, 0, 0, 1},  {32, 16, 1, 128, 0, 0, 1},  {64, 32, 1, 512, 0, 0, 1},
    {96, 32, 1, 512, 0, 0, 1},  {128, 32, 1, 512, 0, 0, 1}, {64, 64, 1, 512, 0, 0, 1},  {64, 27, 1, 512, 0, 0, 1},
    {32, 32, 1, 512, 0, 0, 1},  {26, 16, 1, 512, 0, 0, 1},  {16, 16, 1, 512, 0, 0, 1},  {16, 8, 1, 512, 0, 0, 1},
    {8, 8, 1, 512, 0, 0, 1},
    // its affine variant (fixed tiles per CTA, warm L1 across iterations): coarse levels, few tiles per CTA
    {26, 16, 1, 512, 0, 0, 2},  {32, 16, 1, 512, 0, 0, 2},  {16, 16, 1, 512, 0, 0, 2},  {16, 8, 1, 512, 0, 0, 2},
    {8, 8, 1, 512, 0, 0, 2},    {16, 8, 1, 256, 0, 0, 2},   {8, 8, 1, 256, 0, 0, 2},    {32, 16, 1, 256, 0, 0, 2},
    {32, 32, 1, 256, 0, 0, 2},  {64, 32, 1, 256, 0, 0, 2},  {64, 24, 1, 512, 0, 0, 2}};
constexpr int kNCands = sizeof(kCands) / sizeof(kCands[0]);

// Tuning key: pass index, grid size of the first job, number of directions in the launch, iterations.  A pass is
// a level (index s) or one of its sub-scale grids of stride 2^k (index s + 8k).
using TuneKey = std::tuple<int, int, int, int, int>;
constexpr int kMaxPasses = 3 * kMaxLevels;
static_assert(kMaxPasses == FF_N_PASSES, "pass indices of the profile readout");
int pass_index(int s, int k) { return s + kMaxLevels * k; }
int grid_dim(int v, int k) { return (v + (1 << k) - 1) >> k; }
// sub-scale grids of level s (the coarsest level has none)
int grids_of(const ff_params& p, int s) { return s == p.n_scales - 1 ? 0 : p.sub_scales; }

}  // namespace

struct ff_ctx {
    int device = 0;
    int n_sms = 0;
    cudaStream_t stream = nullptr;
    ff_params prm{};
    std::vector<std::unique_ptr<ff_pyr>> pyrs;
    std::map<std::vector<uintptr_t>, std::unique_ptr<Plan>> plans;
    std::map<TuneKey, TileCfg> tuned;
    std::map<TuneKey, TileCfg> tuned_queue;  // the best of the tile and dataflow forms (server, no-alloc path)
    TileCfg forced[kMaxPasses] = {};  // per-pass override (threads == 0: none)
    int seed_kernel = FF_SEED_TCGEN05;
    uint32_t wait_limit = 1u << 22;    // polls before a device-side wait gives up (~1 s)
    int withhold = 0;                  // test of the bounded waits: the tensor-core seed issues no copies
    int* d_err = nullptr;              // device error word of bounded waits
    void* noalloc_scratch = nullptr;   // device address of ff_match_pair_noalloc's fixed scratch array
    int64_t fail_allocs = 0;           // test of the out-of-memory paths: device allocations still to fail
    DevBuf feat_tab;                   // device table of ff_features_batch (frames' pyramid and WHT launch entries)
    int overlap = 2;                   // ff_match_frames: where the fine levels' descriptors fork off (FF_OPT_OVERLAP)
    cudaStream_t side = nullptr;       // ff_match_frames: carries the descriptor branch while a graph is captured
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::string err;
    int64_t launches = 0, replays = 0, plans_built = 0, bytes = 0;
    int64_t cluster_launches = 0;      // of `launches`: propagation launches of the cluster form
    bool profiling = false;
    struct Ev {
        int phase, level;
        cudaEvent_t a, b;
        int n;
    };
    std::vector<Ev> events;
    std::vector<cudaEvent_t> event_pool;
};

namespace {

ff_status fail(ff_ctx* c, ff_status s, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
ff_status fail(ff_ctx* c, ff_status s, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

#define FF_CUDA(ctx, call)                                                                             \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return fail((ctx), FF_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));           \
    } while (0)

ff_status dev_alloc(ff_ctx* c, DevBuf& b, size_t bytes) {
    b.bytes = bytes;
    if (bytes == 0) {
        b.p = nullptr;
        return FF_OK;
    }
    cudaError_t e = ctx_malloc(c, &b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(c, e == cudaErrorMemoryAllocation ? FF_ERR_OOM : FF_ERR_CUDA, "cudaMalloc(%zu) failed: %s",
                    bytes, cudaGetErrorString(e));
    }
    c->bytes += (int64_t)bytes;
    return FF_OK;
}

void dev_free(ff_ctx* c, DevBuf& b) {
    if (b.p) {
        cudaFree(b.p);
        c->bytes -= (int64_t)b.bytes;
    }
    b.p = nullptr;
    b.bytes = 0;
}

ff_status check_params(const ff_params* p, ff_ctx* c) {
    if (!p) return fail(c, FF_ERR_ARG, "params is NULL");
    if (p->n_scales < 1 || p->n_scales > kMaxLevels) return fail(c, FF_ERR_ARG, "n_scales must be 1..%d", kMaxLevels);
    if (p->iters < 1 || p->iters > 255) return fail(c, FF_ERR_ARG, "iters must be 1..255");
    if (p->patch != 8) return fail(c, FF_ERR_ARG, "patch must be 8");
    if (p->n_coef != 16) return fail(c, FF_ERR_ARG, "n_coef must be 16");
    if (p->rs_radius < 0 || p->rs_radius > 16) return fail(c, FF_ERR_ARG, "rs_radius must be 0..16");
    if (p->eps < 0 || p->eps > 32767) return fail(c, FF_ERR_ARG, "eps must be 0..32767");
    if (p->rs_radius2 < 0 || p->rs_radius2 > 16) return fail(c, FF_ERR_ARG, "rs_radius2 must be 0..16");
    if (p->cost != FF_COST_WHT_SAD && p->cost != FF_COST_CENSUS)
        return fail(c, FF_ERR_ARG, "cost must be FF_COST_WHT_SAD or FF_COST_CENSUS");
    if (p->sub_scales < 0 || p->sub_scales > 2) return fail(c, FF_ERR_ARG, "sub_scales must be 0, 1 or 2");
    return FF_OK;
}

// Whether a tile-form configuration's tile and halo fit in shared memory (a cluster-form configuration is
// checked per pass by cluster_fits).
bool cfg_fits(const TileCfg& t) {
    return t.cluster > 0 || prop_smem_bytes(t.tw, t.th, t.dataflow ? 1 : t.k) <= kMaxPropSmem;
}

// Whether the cluster form of `t` can run pass (s, k) of these jobs: a partition of every problem, its shared
// memory within the limit, and clusters of that shape launchable on this device.  *smem: the largest CTA's bytes.
bool cluster_fits(const ff_ctx* c, const std::vector<DirJob>& jobs, int s, int k, const TileCfg& t, size_t* smem) {
    size_t most = 0;
    for (const DirJob& j : jobs) {
        const int w = grid_dim(j.a->ws[s], k), h = grid_dim(j.a->hs[s], k);
        int bx = 0, by = 0;
        if (!cluster_partition(w, h, t.cluster, bx, by)) return false;
        most = std::max(most, cluster_smem_bytes(w, h, bx, by));
    }
    if (most > kMaxPropSmem || prop_cluster_capacity(t.cluster, t.threads, c->prm.cost, k > 0, most) < 1)
        return false;
    *smem = most;
    return true;
}

// Default propagation configuration of a level when it has not been tuned: large tiles with one iteration per
// launch when the level fills the GPU, otherwise small tiles with fused iterations (idle SMs absorb the halo).
TileCfg default_cfg(const ff_ctx* c, int64_t level_pix_all, int T) {
    const int64_t slots = (int64_t)c->n_sms * 2;
    if (level_pix_all / (32 * 32) >= 2 * slots) return {32, 32, 1, 256, 0};
    if (level_pix_all / (32 * 16) >= 2 * slots) return {32, 16, 1, 256, 0};
    if (level_pix_all / (16 * 16) >= slots) return {16, 16, std::min(2, T), 256, 1};
    return {8, 8, std::min(3, T), 256, 1};
}

ff_status enqueue_launch(ff_ctx* c, const Launch& L) {
    cudaStream_t st = c->stream;
    switch (L.kind) {
        case Kind::Memset:
            FF_CUDA(c, cudaMemsetAsync(L.set_ptr, L.set_value, L.set_bytes, st));
            return FF_OK;
        case Kind::SeedTc:
            launch_seed_tc(static_cast<const SeedTcProblem*>(L.probs), L.n_probs, L.total, L.total_pix, L.wait_limit,
                           L.withhold, L.err, st);
            break;
        case Kind::Seed:
            launch_seed(static_cast<const SeedProblem*>(L.probs), L.n_probs, L.total, st);
            break;
        case Kind::Handover:
            launch_handover(static_cast<const HandoverProblem*>(L.probs), L.n_probs, L.total_pix, L.cost, st);
            break;
        case Kind::Propagate:
            launch_propagate(static_cast<const PropProblem*>(L.probs), L.queue, L.total, L.counter, L.grid, L.prop,
                             st);
            break;
        case Kind::Consistency:
            launch_consistency(L.fwd, L.bwd, L.bwd2, L.w, L.h, L.eps, L.mask, st);
            break;
        case Kind::ConsistencyTab:
            launch_consistency_tab(static_cast<const ConsProblem*>(L.probs), L.n_probs, L.total_pix, L.eps, st);
            break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, FF_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    return FF_OK;
}

int kernels_of(const Launch& l) { return l.kind == Kind::Memset ? 0 : l.kind == Kind::SeedTc ? 2 : 1; }
int clusters_of(const Launch& l) { return l.kind == Kind::Propagate && l.prop.cluster > 0 ? 1 : 0; }

ff_status ensure_err_word(ff_ctx* c) {
    if (c->d_err) return FF_OK;
    if (ctx_malloc(c, reinterpret_cast<void**>(&c->d_err), 256) != cudaSuccess) {
        cudaGetLastError();
        c->d_err = nullptr;
        return fail(c, FF_ERR_OOM, "error word allocation failed");
    }
    FF_CUDA(c, cudaMemset(c->d_err, 0, 256));
    return FF_OK;
}

cudaEvent_t get_event(ff_ctx* c) {
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Enqueue a sequence of launches; with `timed`, each run of consecutive launches of the same phase (and, for
// propagation, the same level) is bracketed by events recorded into c->events.
ff_status run_launches(ff_ctx* c, const std::vector<Launch>& ls, bool timed) {
    size_t i = 0;
    while (i < ls.size()) {
        size_t j = i;
        while (j < ls.size() && ls[j].phase == ls[i].phase && ls[j].level == ls[i].level) j++;
        cudaEvent_t ea = nullptr, eb = nullptr;
        if (timed) {
            ea = get_event(c);
            eb = get_event(c);
            FF_CUDA(c, cudaEventRecord(ea, c->stream));
        }
        int nk = 0;
        for (size_t k = i; k < j; k++) {
            ff_status s = enqueue_launch(c, ls[k]);
            if (s != FF_OK) return s;
            nk += kernels_of(ls[k]);
            c->cluster_launches += clusters_of(ls[k]);
        }
        c->launches += nk;
        if (timed) {
            FF_CUDA(c, cudaEventRecord(eb, c->stream));
            c->events.push_back({ls[i].phase, ls[i].level, ea, eb, nk});
        }
        i = j;
    }
    return FF_OK;
}

// The descriptors a level is matched with: the WHT features, or the Census patterns under the Census cost.
const void* cost_desc(const ff_pyr* p, int level, int cost) {
    return cost == FF_COST_CENSUS ? static_cast<const void*>(p->cen[level]) : static_cast<const void*>(p->feat[level]);
}

// Build the launch sequence of a set of matching directions (+ consistency checks).  `force` (optional, one entry
// per pass index) imposes the propagation configuration of every level and grid (used by the autotuner).
ff_status build_plan(ff_ctx* c, const std::vector<DirJob>& jobs, const std::vector<ConsJob>& cons, Plan& P,
                     const TileCfg* force) {
    const int L = c->prm.n_scales, T = c->prm.iters, cost = c->prm.cost;
    const int nj = (int)jobs.size();
    // per job and level: two flow and two cost buffers (ping-pong) + seed distances
    // per job, level and grid (k = 0: the level; k = 1, 2: its sub-scale grids of stride 2^k)
    struct LevelBufs {
        uint32_t* flow[2];
        int32_t* cost[2];
    };
    auto gdim = grid_dim;
    auto k_first = [&](int s) { return grids_of(c->prm, s); };
    std::vector<std::vector<std::array<LevelBufs, 3>>> lb(nj, std::vector<std::array<LevelBufs, 3>>(L));
    std::vector<int32_t*> seed_dist(nj);
    std::vector<unsigned long long*> seed_keys(nj);
    const bool tc = c->seed_kernel == FF_SEED_TCGEN05;
    {  // the error word of the bounded waits (tensor-core seed, cluster-form propagation)
        ff_status se = ensure_err_word(c);
        if (se != FF_OK) return se;
    }
    size_t scratch = 0, keys_bytes = 0;
    for (int j = 0; j < nj; j++) {
        for (int s = 0; s < L; s++)
            for (int k = 0; k <= k_first(s); k++)
                scratch += 4 * align_up((size_t)gdim(jobs[j].a->ws[s], k) * gdim(jobs[j].a->hs[s], k) * 4);
        scratch += align_up((size_t)jobs[j].a->n_coarse * 4);
        if (tc) keys_bytes += (size_t)jobs[j].a->n_coarse * 8;
    }
    scratch += align_up(keys_bytes);
    P.bufs.emplace_back();
    ff_status st = dev_alloc(c, P.bufs.back(), scratch);
    if (st != FF_OK) return st;
    char* base = static_cast<char*>(P.bufs.back().p);
    size_t off = 0;
    for (int j = 0; j < nj; j++) {
        for (int s = 0; s < L; s++)
            for (int k = 0; k <= k_first(s); k++) {
                size_t n = (size_t)gdim(jobs[j].a->ws[s], k) * gdim(jobs[j].a->hs[s], k);
                for (int b = 0; b < 2; b++) {
                    lb[j][s][k].flow[b] = reinterpret_cast<uint32_t*>(base + off);
                    off += align_up(n * 4);
                    lb[j][s][k].cost[b] = reinterpret_cast<int32_t*>(base + off);
                    off += align_up(n * 4);
                }
            }
        seed_dist[j] = reinterpret_cast<int32_t*>(base + off);
        off += align_up((size_t)jobs[j].a->n_coarse * 4);
    }
    char* keys_base = base + off;
    for (int j = 0, ko = 0; j < nj && tc; j++) {
        seed_keys[j] = reinterpret_cast<unsigned long long*>(keys_base) + ko;
        ko += jobs[j].a->n_coarse;
    }
    // queue order: the two directions of a pair interleaved tile by tile (they read the same two frames), pairs
    // one after another; directions without a partner follow
    std::vector<std::vector<int>> groups;
    std::vector<bool> grouped(nj, false);
    for (const ConsJob& cj : cons) {
        if (cj.dj_bwd2 >= 0) {
            groups.push_back({cj.dj_fwd, cj.dj_bwd, cj.dj_bwd2});
            grouped[cj.dj_bwd2] = true;
        } else {
            groups.push_back({cj.dj_fwd, cj.dj_bwd});
        }
        grouped[cj.dj_fwd] = grouped[cj.dj_bwd] = true;
    }
    for (int j = 0; j < nj; j++)
        if (!grouped[j]) groups.push_back({j});

    std::vector<SeedProblem> seeds;
    std::vector<SeedTcProblem> tcseeds;
    std::vector<HandoverProblem> hos;
    std::vector<PropProblem> props;
    std::vector<int2> queue;
    int n_counters = 0;
    std::vector<std::pair<size_t, int>> progress;  // dataflow problems: (index in props, first progress counter)
    struct Pending {
        Launch l;
        size_t off_probs, off_queue;
        int counter;
    };
    std::vector<Pending> pend;
    pend.push_back({Launch{Kind::Memset, FF_PHASE_SEED}, 0, 0, -1});  // queue counters <- 0
    if (tc) {  // seed keys <- all ones (the neutral element of the atomicMin merge)
        Launch l{};
        l.kind = Kind::Memset;
        l.phase = FF_PHASE_SEED;
        l.set_ptr = keys_base;
        l.set_bytes = keys_bytes;
        l.set_value = 0xFF;
        pend.push_back({l, 0, 0, -1});
    }

    // 1. exact initial matches at the coarsest level
    if (tc) {
        Launch l{};
        l.kind = Kind::SeedTc;
        l.phase = FF_PHASE_SEED;
        l.desc_level = L - 1;
        int ctas = 0;
        int64_t pix = 0;
        for (int j = 0; j < nj; j++) {
            const ff_pyr* A = jobs[j].a;
            const ff_pyr* B = jobs[j].b;
            SeedTcProblem sp{};
            sp.map_a = A->tmap;
            sp.map_b = B->tmap;
            sp.normA = A->seed_norm;
            sp.normB = B->seed_norm;
            sp.n = A->n_coarse;
            sp.w = A->ws[L - 1];
            sp.row_tiles = (sp.n + kSeedTcRows - 1) / kSeedTcRows;
            sp.col_tiles = (sp.n + kSeedTcCols - 1) / kSeedTcCols;
            sp.cta_base = ctas;
            ctas += sp.row_tiles * sp.col_tiles;
            sp.keys = seed_keys[j];
            sp.flow = lb[j][L - 1][0].flow[0];
            sp.dist = seed_dist[j];
            sp.pix_base = pix;
            pix += sp.n;
            tcseeds.push_back(sp);
        }
        l.n_probs = nj;
        l.total = ctas;
        l.total_pix = pix;
        l.wait_limit = c->wait_limit;
        l.withhold = c->withhold;
        l.err = c->d_err;
        pend.push_back({l, 0, 0, -1});
    } else {
        Launch l{};
        l.kind = Kind::Seed;
        l.phase = FF_PHASE_SEED;
        l.desc_level = L - 1;
        int tiles = 0;
        size_t o = seeds.size();
        for (int j = 0; j < nj; j++) {
            const ff_pyr* A = jobs[j].a;
            const ff_pyr* B = jobs[j].b;
            SeedProblem sp{};
            sp.A = A->seed_desc;
            sp.B = B->seed_desc;
            sp.normA = A->seed_norm;
            sp.normB = B->seed_norm;
            sp.n = A->n_coarse;
            sp.w = A->ws[L - 1];
            sp.flow = lb[j][L - 1][0].flow[0];
            sp.dist = seed_dist[j];
            sp.warp_base = tiles;
            tiles += (sp.n + 15) / 16;
            seeds.push_back(sp);
        }
        l.n_probs = nj;
        l.total = tiles;
        pend.push_back({l, o, 0, -1});
    }
    // 2. per level, and before it per sub-scale grid (sparsest first): hand-over (the cost of the seed at the
    //    coarsest level), then the propagation launches
    std::vector<int> cur_buf(nj, 0);
    for (int s = L - 1; s >= 0; s--) {
      for (int k = k_first(s); k >= 0; k--) {
        {
            Launch l{};
            l.kind = Kind::Handover;
            l.phase = s == L - 1 ? FF_PHASE_SEED : FF_PHASE_HANDOVER;
            l.desc_level = s;
            size_t o = hos.size();
            int64_t pix = 0;
            for (int j = 0; j < nj; j++) {
                const ff_pyr* A = jobs[j].a;
                HandoverProblem hp{};
                hp.fa = cost_desc(A, s, cost);
                hp.fb = cost_desc(jobs[j].b, s, cost);
                hp.w = gdim(A->ws[s], k);
                hp.h = gdim(A->hs[s], k);
                hp.g = 1 << k;
                hp.lw = A->ws[s];
                hp.lh = A->hs[s];
                if (s == L - 1) {
                    hp.parent = nullptr;
                    hp.flow_in = lb[j][s][0].flow[0];
                } else if (k == k_first(s)) {  // from the level above
                    hp.parent = lb[j][s + 1][0].flow[cur_buf[j]];
                    hp.pw = A->ws[s + 1];
                    hp.ph = A->hs[s + 1];
                } else {  // from the sparser grid of this level
                    hp.parent = lb[j][s][k + 1].flow[cur_buf[j]];
                    hp.pw = gdim(A->ws[s], k + 1);
                    hp.ph = gdim(A->hs[s], k + 1);
                    hp.same_level = 1;
                }
                hp.flow_out = lb[j][s][k].flow[0];
                hp.cost_out = lb[j][s][k].cost[0];
                hp.pix_base = pix;
                pix += (int64_t)hp.w * hp.h;
                hos.push_back(hp);
                cur_buf[j] = 0;
            }
            l.n_probs = nj;
            l.total_pix = pix;
            l.cost = cost;
            pend.push_back({l, o, 0, -1});
        }
        int64_t level_pix = 0;
        for (int j = 0; j < nj; j++) level_pix += (int64_t)gdim(jobs[j].a->ws[s], k) * gdim(jobs[j].a->hs[s], k);
        const int pass = pass_index(s, k);
        TileCfg tc;
        if (force) {
            tc = force[pass];
            tc.k = std::min(tc.k, T);
        } else if (c->forced[pass].threads > 0) {
            tc = c->forced[pass];
            tc.k = std::min(tc.k, T);
        } else {
            auto it = c->tuned.find(TuneKey{pass, gdim(jobs[0].a->ws[s], k), gdim(jobs[0].a->hs[s], k), nj, T});
            tc = it != c->tuned.end() ? it->second : default_cfg(c, level_pix, T);
        }
        size_t cl_smem = 0;
        if (tc.cluster > 0 && !cluster_fits(c, jobs, s, k, tc, &cl_smem)) tc = default_cfg(c, level_pix, T);
        const bool cl = tc.cluster > 0, df = tc.dataflow > 0;
        if (df) tc.k = T;  // one launch, one iteration per tile task
        const size_t smem = cl ? 0 : prop_smem_bytes(tc.tw, tc.th, df ? 1 : tc.k);
        const int blocks = cl ? 0 : prop_blocks_per_sm(smem, tc.threads, tc.spec != 0, cost, k > 0, df) * c->n_sms;
        for (int t0 = 0; t0 < T; t0 += tc.k) {
            int n_iter = std::min(tc.k, T - t0);
            bool last = t0 + n_iter == T;
            Launch l{};
            l.kind = Kind::Propagate;
            l.phase = FF_PHASE_PROPAGATE;
            l.level = pass;
            l.desc_level = s;
            l.prop.tw = tc.tw;
            l.prop.th = tc.th;
            l.prop.max_iter = df ? 1 : n_iter;
            l.prop.dataflow = df ? T : 0;
            l.prop.affine = tc.dataflow == 2;
            l.prop.threads = tc.threads;
            l.prop.spec = tc.spec;
            l.prop.cost = cost;
            l.prop.grid = k > 0;
            l.prop.cluster = tc.cluster;
            l.prop.cl_smem = (int)cl_smem;
            l.prop.wait_limit = c->wait_limit;
            l.prop.withhold = c->withhold;
            l.prop.err = c->d_err;
            size_t oq = queue.size();
            std::vector<int> pidx(nj), ntiles(nj);
            for (int j = 0; j < nj; j++) {
                const ff_pyr* A = jobs[j].a;
                PropProblem pp{};
                pp.fa = cost_desc(A, s, cost);
                pp.fb = cost_desc(jobs[j].b, s, cost);
                pp.w = gdim(A->ws[s], k);
                pp.h = gdim(A->hs[s], k);
                pp.g = 1 << k;
                pp.lw = A->ws[s];
                pp.lh = A->hs[s];
                int in = cur_buf[j], out = in ^ 1;
                const LevelBufs& B = lb[j][s][k];
                pp.flow_in = B.flow[in];
                pp.cost_in = B.cost[in];
                if (df) {  // iterations alternate: even ones write buffer `out` (flow_alt), odd ones `in`
                    pp.flow_alt = B.flow[out];
                    pp.cost_alt = B.cost[out];
                    out = (T - 1) % 2 == 0 ? out : in;  // where the last iteration lands, apart from its source
                }
                if (last && s == 0 && k == 0) {  // the final launch writes the caller's buffers (cost to scratch if NULL)
                    pp.flow_out = jobs[j].flow_out;
                    pp.cost_out = jobs[j].cost_out ? jobs[j].cost_out : B.cost[out];
                } else {
                    pp.flow_out = B.flow[out];
                    pp.cost_out = B.cost[out];
                }
                cur_buf[j] = out;
                pp.tiles_x = cl ? 1 : (pp.w + tc.tw - 1) / tc.tw;
                ntiles[j] = cl ? 0 : pp.tiles_x * ((pp.h + tc.th - 1) / tc.th);
                pp.t0 = t0;
                pp.n_iter = df ? 1 : n_iter;
                pp.level = s + 8 * k;  // the hash stream of this level or grid
                pp.dir = jobs[j].dir;
                pp.seed = c->prm.seed;
                pp.rs_radius = jobs[j].rs_radius;
                pidx[j] = (int)props.size();
                props.push_back(pp);
            }
            if (cl) {  // cluster i of the launch runs problem pidx[0] + i
                l.n_probs = nj;
                l.grid = nj * tc.cluster;
                pend.push_back({l, (size_t)pidx[0], 0, -1});
                continue;
            }
            for (const std::vector<int>& g : groups) {
                int most = 0;
                for (int j : g) most = std::max(most, ntiles[j]);
                for (int q = 0; q < most; q++)
                    for (int j : g)
                        if (q < ntiles[j]) queue.push_back(make_int2(pidx[j], q));
            }
            l.n_probs = nj;
            l.total = (int)(queue.size() - oq);
            l.grid = (int)std::min<int64_t>((int64_t)l.total * (df && tc.dataflow != 2 ? T : 1), blocks);
            pend.push_back({l, 0, oq, n_counters++});
            if (df)  // the tiles' progress counters follow the launch's queue counter in the zeroed block
                for (int j = 0; j < nj; j++) {
                    progress.push_back({(size_t)pidx[j], n_counters});
                    n_counters += ntiles[j];
                }
        }
      }
    }
    // 3. consistency of each pair: the forward flow and the inverse flow, both at level 0
    //    (one launch for a single pair; the pairs of a batch share one launch over a table)
    std::vector<ConsProblem> cps;
    if (cons.size() == 1) {
        const ConsJob& cj = cons[0];
        Launch l{};
        l.kind = Kind::Consistency;
        l.phase = FF_PHASE_CONSISTENCY;
        l.fwd = jobs[cj.dj_fwd].flow_out;
        l.bwd = jobs[cj.dj_bwd].flow_out;
        l.bwd2 = cj.dj_bwd2 >= 0 ? jobs[cj.dj_bwd2].flow_out : nullptr;
        l.w = jobs[cj.dj_fwd].a->w;
        l.h = jobs[cj.dj_fwd].a->h;
        l.eps = c->prm.eps;
        l.mask = cj.mask;
        pend.push_back({l, 0, 0, -1});
    } else if (cons.size() > 1) {
        Launch l{};
        l.kind = Kind::ConsistencyTab;
        l.phase = FF_PHASE_CONSISTENCY;
        int64_t pix = 0;
        for (const ConsJob& cj : cons) {
            ConsProblem cp{};
            cp.fwd = jobs[cj.dj_fwd].flow_out;
            cp.bwd = jobs[cj.dj_bwd].flow_out;
            cp.bwd2 = cj.dj_bwd2 >= 0 ? jobs[cj.dj_bwd2].flow_out : nullptr;
            cp.w = jobs[cj.dj_fwd].a->w;
            cp.h = jobs[cj.dj_fwd].a->h;
            cp.mask = cj.mask;
            cp.pix_base = pix;
            pix += (int64_t)cp.w * cp.h;
            cps.push_back(cp);
        }
        l.n_probs = (int)cps.size();
        l.total_pix = pix;
        l.eps = c->prm.eps;
        pend.push_back({l, 0, 0, -1});
    }

    // upload the problem tables, queues and counters in one block
    size_t o_seed = 0, o_tc = align_up(seeds.size() * sizeof(SeedProblem));
    size_t o_ho = o_tc + align_up(tcseeds.size() * sizeof(SeedTcProblem));
    size_t o_prop = o_ho + align_up(hos.size() * sizeof(HandoverProblem));
    size_t o_q = o_prop + align_up(props.size() * sizeof(PropProblem));
    size_t o_cnt = o_q + align_up(queue.size() * sizeof(int2));
    size_t o_cons = o_cnt + align_up((size_t)std::max(n_counters, 1) * sizeof(int));
    size_t tbytes = o_cons + align_up(cps.size() * sizeof(ConsProblem));
    P.bufs.emplace_back();
    st = dev_alloc(c, P.bufs.back(), tbytes);
    if (st != FF_OK) return st;
    char* tb = static_cast<char*>(P.bufs.back().p);
    for (auto [pi, first] : progress) props[pi].progress = reinterpret_cast<int*>(tb + o_cnt) + first;
    std::vector<char> host(tbytes, 0);
    memcpy(host.data() + o_seed, seeds.data(), seeds.size() * sizeof(SeedProblem));
    memcpy(host.data() + o_tc, tcseeds.data(), tcseeds.size() * sizeof(SeedTcProblem));
    memcpy(host.data() + o_ho, hos.data(), hos.size() * sizeof(HandoverProblem));
    memcpy(host.data() + o_prop, props.data(), props.size() * sizeof(PropProblem));
    memcpy(host.data() + o_q, queue.data(), queue.size() * sizeof(int2));
    memcpy(host.data() + o_cons, cps.data(), cps.size() * sizeof(ConsProblem));
    FF_CUDA(c, cudaMemcpy(tb, host.data(), tbytes, cudaMemcpyHostToDevice));
    for (Pending& pd : pend) {
        Launch l = pd.l;
        switch (l.kind) {
            case Kind::Memset:
                if (!l.set_ptr) {  // the queue counters of this plan
                    l.set_ptr = tb + o_cnt;
                    l.set_bytes = (size_t)std::max(n_counters, 1) * sizeof(int);
                }
                break;
            case Kind::SeedTc:
                l.probs = tb + o_tc;
                break;
            case Kind::Seed:
                l.probs = tb + o_seed + pd.off_probs * sizeof(SeedProblem);
                break;
            case Kind::Handover:
                l.probs = tb + o_ho + pd.off_probs * sizeof(HandoverProblem);
                break;
            case Kind::Propagate:  // queue entries hold absolute indices into the problem table
                if (l.prop.cluster > 0) {  // the launch's problems are consecutive
                    l.probs = tb + o_prop + pd.off_probs * sizeof(PropProblem);
                    break;
                }
                l.probs = tb + o_prop;
                l.queue = reinterpret_cast<const int2*>(tb + o_q) + pd.off_queue;
                l.counter = reinterpret_cast<int*>(tb + o_cnt) + pd.counter;
                break;
            case Kind::Consistency:
                break;
            case Kind::ConsistencyTab:
                l.probs = tb + o_cons;
                break;
        }
        P.launches.push_back(l);
    }
    return FF_OK;
}

void free_plan(ff_ctx* c, Plan& P) {
    if (P.exec) cudaGraphExecDestroy(P.exec);
    P.exec = nullptr;
    if (P.split_exec) cudaGraphExecDestroy(P.split_exec);
    P.split_exec = nullptr;
    for (DevBuf& b : P.bufs) dev_free(c, b);
}

// Record launches [i0, i1) of the plan into one executable graph (none when the range is empty).
ff_status capture_range(ff_ctx* c, const Plan& P, size_t i0, size_t i1, cudaGraphExec_t* out, int* nk, int* nc) {
    *out = nullptr;
    *nk = *nc = 0;
    if (i0 >= i1) return FF_OK;
    cudaGraph_t g = nullptr;
    FF_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    ff_status s = FF_OK;
    for (size_t i = i0; i < i1; i++) {
        s = enqueue_launch(c, P.launches[i]);
        if (s != FF_OK) break;
        *nk += kernels_of(P.launches[i]);
        *nc += clusters_of(P.launches[i]);
    }
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (s != FF_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return fail(c, FF_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        return fail(c, FF_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    }
    return FF_OK;
}

ff_status execute_plan(ff_ctx* c, Plan& P) {
    // graphs need a capturable (non-legacy) stream; profiling brackets phases with events instead
    bool use_graph = !c->profiling && c->stream != nullptr;
    if (!use_graph) return run_launches(c, P.launches, c->profiling);
    if (!P.exec) {
        ff_status s = capture_range(c, P, 0, P.launches.size(), &P.exec, &P.graph_nodes, &P.cluster_nodes);
        if (s != FF_OK) return s;
    }
    FF_CUDA(c, cudaGraphLaunch(P.exec, c->stream));
    c->replays += 1;
    c->launches += P.graph_nodes;
    c->cluster_launches += P.cluster_nodes;
    return FF_OK;
}

// The side stream and the two events of ff_match_frames, created on first use.
ff_status ensure_side(ff_ctx* c) {
    if (!c->side) FF_CUDA(c, cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    if (!c->ev_fork) FF_CUDA(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    if (!c->ev_join) FF_CUDA(c, cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    return FF_OK;
}

// Record the plan's launches into one graph with the fine levels' descriptor launch on a branch: it starts after
// launch `fork` - 1 and joins before launch `join`, the first that reads a level below the split.  The side stream
// only carries the branch during the capture.  Every kernel node but the descriptor launch gets the highest
// priority, so that the block scheduler serves the latency-bound coarse levels' launches first and the descriptor
// launch takes the SMs they leave idle.
ff_status capture_split(ff_ctx* c, Plan& P, size_t fork, size_t join, const FineWht& fine) {
    int least = 0, greatest = 0;
    FF_CUDA(c, cudaDeviceGetStreamPriorityRange(&least, &greatest));
    cudaGraph_t g = nullptr;
    FF_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    ff_status s = FF_OK;
    cudaError_t e = cudaSuccess;
    bool forked = false;
    int nk = 1, nc = 0;  // the descriptor launch, then the plan's
    for (size_t i = 0; i < P.launches.size() && s == FF_OK && e == cudaSuccess; i++) {
        if (i == fork) {
            e = cudaEventRecord(c->ev_fork, c->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->ev_fork, 0);
            if (e != cudaSuccess) break;
            forked = true;
            launch_wht_tab(fine.tab, fine.n, fine.tiles, c->side, false);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, c->side);
            if (e != cudaSuccess) break;
        }
        if (i == join) {
            e = cudaStreamWaitEvent(c->stream, c->ev_join, 0);
            forked = false;
            if (e != cudaSuccess) break;
        }
        s = enqueue_launch(c, P.launches[i]);
        nk += kernels_of(P.launches[i]);
        nc += clusters_of(P.launches[i]);
    }
    if (forked) {  // the branch rejoins the capture in every case
        cudaError_t ej = cudaStreamWaitEvent(c->stream, c->ev_join, 0);
        if (e == cudaSuccess) e = ej;
    }
    cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
    if (s != FF_OK || e != cudaSuccess || ee != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (s != FF_OK) return s;
        return fail(c, FF_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : ee));
    }
    size_t nn = 0;
    e = cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (e == cudaSuccess && nn) e = cudaGraphGetNodes(g, nodes.data(), &nn);
    for (size_t i = 0; i < nn && e == cudaSuccess; i++) {
        cudaGraphNodeType t;
        e = cudaGraphNodeGetType(nodes[i], &t);
        if (e != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp{};
        e = cudaGraphKernelNodeGetParams(nodes[i], &kp);
        if (e != cudaSuccess || kp.func == wht_tab_kernel()) continue;
        cudaLaunchAttributeValue v{};
        v.priority = greatest;
        e = cudaGraphKernelNodeSetAttribute(nodes[i], cudaLaunchAttributePriority, &v);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiateWithFlags(&P.split_exec, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        P.split_exec = nullptr;
        return fail(c, FF_ERR_CUDA, "split graph failed: %s", cudaGetErrorString(e));
    }
    P.split_at[0] = fork;
    P.split_at[1] = join;
    P.split_tab = fine.tab;
    P.split_n = fine.n;
    P.split_tiles = fine.tiles;
    P.split_nodes = nk;
    P.split_clusters = nc;
    return FF_OK;
}

// Run the plan with the fine levels' descriptor launch beside the coarse levels' matching (ff_match_frames).
// Fork point: FF_OPT_OVERLAP 1, the start of the matching; 2, the first propagation launch (the coarsest level's,
// once its initial matches and their costs are done).  Join: the first launch that reads a level below
// `fine_below`.
ff_status execute_plan_split(ff_ctx* c, Plan& P, const FineWht& fine, int fine_below) {
    const size_t n = P.launches.size();
    size_t join = n, fork = 0;
    for (size_t i = 0; i < n; i++)
        if (P.launches[i].desc_level >= 0 && P.launches[i].desc_level < fine_below) {
            join = i;
            break;
        }
    if (c->overlap == 2)
        for (size_t i = 0; i < join; i++)
            if (P.launches[i].kind == Kind::Propagate) {
                fork = i;
                break;
            }
    if (!P.split_exec || P.split_at[0] != fork || P.split_at[1] != join || P.split_tab != fine.tab ||
        P.split_n != fine.n || P.split_tiles != fine.tiles) {
        if (P.split_exec) cudaGraphExecDestroy(P.split_exec);
        P.split_exec = nullptr;
        ff_status s = capture_split(c, P, fork, join, fine);
        if (s != FF_OK) return s;
    }
    FF_CUDA(c, cudaGraphLaunch(P.split_exec, c->stream));
    c->replays += 1;
    c->launches += P.split_nodes;
    c->cluster_launches += P.split_clusters;
    return FF_OK;
}

std::vector<uintptr_t> plan_key(const std::vector<DirJob>& jobs, const std::vector<ConsJob>& cons) {
    std::vector<uintptr_t> key;
    key.reserve(jobs.size() * 5 + cons.size() * 3 + 1);
    for (const DirJob& j : jobs) {
        key.push_back((uintptr_t)j.a);
        key.push_back((uintptr_t)j.b);
        key.push_back((uintptr_t)j.dir);
        key.push_back((uintptr_t)j.flow_out);
        key.push_back((uintptr_t)j.cost_out);
        key.push_back((uintptr_t)j.rs_radius);
    }
    key.push_back(~(uintptr_t)0);
    for (const ConsJob& cj : cons) {
        key.push_back((uintptr_t)cj.dj_fwd);
        key.push_back((uintptr_t)cj.dj_bwd);
        key.push_back((uintptr_t)cj.mask);
        key.push_back((uintptr_t)(intptr_t)cj.dj_bwd2);
    }
    return key;
}

ff_status drop_plans(ff_ctx* c) {
    FF_CUDA(c, cudaStreamSynchronize(c->stream));
    for (auto& kv : c->plans) free_plan(c, *kv.second);
    c->plans.clear();
    return FF_OK;
}

// The cached plan of these jobs, built on first use.
ff_status find_plan(ff_ctx* c, const std::vector<DirJob>& jobs, const std::vector<ConsJob>& cons, Plan** out) {
    std::vector<uintptr_t> key = plan_key(jobs, cons);
    auto it = c->plans.find(key);
    if (it == c->plans.end()) {
        if (c->plans.size() >= 64) {  // bound the cache: drop everything (plans are cheap to rebuild)
            ff_status s = drop_plans(c);
            if (s != FF_OK) return s;
        }
        auto P = std::make_unique<Plan>();
        P->key = key;
        ff_status s = build_plan(c, jobs, cons, *P, nullptr);
        if (s != FF_OK) {
            free_plan(c, *P);
            return s;
        }
        c->plans_built += 1;
        it = c->plans.emplace(key, std::move(P)).first;
    }
    *out = it->second.get();
    return FF_OK;
}

ff_status run_jobs(ff_ctx* c, const std::vector<DirJob>& jobs, const std::vector<ConsJob>& cons) {
    Plan* P = nullptr;
    ff_status s = find_plan(c, jobs, cons, &P);
    if (s != FF_OK) return s;
    return execute_plan(c, *P);
}

// Time every candidate configuration on the given jobs and keep, per level, the fastest.  Runs the real
// matching (outputs are overwritten by every trial; all configurations give identical results).
// Tiles a launch of this configuration processes in pass (s, k) (all jobs) and the CTAs resident at once.
void wave_shape(const ff_ctx* c, const std::vector<DirJob>& jobs, int s, int k, const TileCfg& t, int64_t* tiles,
                int64_t* slots) {
    int64_t n = 0;
    for (const DirJob& j : jobs)
        n += (int64_t)((grid_dim(j.a->ws[s], k) + t.tw - 1) / t.tw) * ((grid_dim(j.a->hs[s], k) + t.th - 1) / t.th);
    *tiles = n;
    *slots = (int64_t)prop_blocks_per_sm(prop_smem_bytes(t.tw, t.th, t.k), t.threads, t.spec != 0, c->prm.cost,
                                         k > 0) *
             c->n_sms;
}

// A launch whose last wave is a small remainder of tiles runs at about the speed of one more full wave.  The
// wave-fitted variant of a configuration grows the tile (height first, then width, by at most a quarter) just
// enough that the tiles fill one wave fewer; it returns the configuration unchanged when none does.
TileCfg wave_fitted(const ff_ctx* c, const std::vector<DirJob>& jobs, int s, int k, TileCfg t) {
    if (t.cluster > 0 || t.dataflow > 0) return t;  // no launch boundary per iteration, no last wave to fill
    int64_t tiles, slots;
    wave_shape(c, jobs, s, k, t, &tiles, &slots);
    if (slots < 1 || tiles <= slots) return t;
    const int64_t waves = (tiles + slots - 1) / slots;
    if (tiles - (waves - 1) * slots > slots / 2) return t;  // the last wave is at least half full
    for (int grow = 1; grow <= std::max(1, t.th / 4) + std::max(1, t.tw / 4); grow++)
        for (int dim = 0; dim < 2; dim++) {
            TileCfg u = t;
            if (dim == 0) {
                if (grow > std::max(1, t.th / 4)) continue;
                u.th += grow;
            } else {
                if (grow > std::max(1, t.tw / 4)) continue;
                u.tw += grow;
            }
            if (!cfg_fits(u)) continue;
            int64_t tu, su;
            wave_shape(c, jobs, s, k, u, &tu, &su);
            if (su > 0 && tu <= (waves - 1) * su) return u;
        }
    return t;
}

ff_status autotune(ff_ctx* c, const std::vector<DirJob>& jobs, const std::vector<ConsJob>& cons, int reps) {
    const int L = c->prm.n_scales, T = c->prm.iters, nj = (int)jobs.size();
    // the passes of a plan: every level and, with sub-scales, its grids
    std::vector<std::pair<int, int>> passes;
    for (int s = 0; s < L; s++)
        for (int k = 0; k <= grids_of(c->prm, s); k++) passes.push_back({s, k});
    // per pass, the best time and configuration seen; each candidate is timed as given and, where it leaves a
    // short last wave in some pass, once more with its wave-fitted variant in those passes
    std::vector<double> best_ms(kMaxPasses, 1e30), best_queue_ms(kMaxPasses, 1e30);
    std::vector<TileCfg> best_cfg(kMaxPasses), best_queue_cfg(kMaxPasses);
    ff_status s = drop_plans(c);
    if (s != FF_OK) return s;
    bool was_profiling = c->profiling;
    auto time_plan = [&](const std::vector<TileCfg>& per_pass) -> ff_status {
        Plan P;
        ff_status st = build_plan(c, jobs, cons, P, per_pass.data());
        if (st != FF_OK) {
            free_plan(c, P);
            return st;
        }
        std::vector<double> pass_best(kMaxPasses, 1e30);
        for (int r = 0; r < reps + 1; r++) {
            c->events.clear();
            st = run_launches(c, P.launches, true);
            if (st == FF_OK) st = [&]() -> ff_status {
                FF_CUDA(c, cudaStreamSynchronize(c->stream));
                return FF_OK;
            }();
            if (st != FF_OK) {
                free_plan(c, P);
                return st;
            }
            std::vector<double> lv(kMaxPasses, 0.0);
            for (auto& e : c->events) {
                float t = 0.f;
                cudaEventElapsedTime(&t, e.a, e.b);
                if (e.phase == FF_PHASE_PROPAGATE && e.level >= 0 && e.level < kMaxPasses) lv[e.level] += t;
                c->event_pool.push_back(e.a);
                c->event_pool.push_back(e.b);
            }
            c->events.clear();
            if (r > 0)  // the first run warms caches and clocks
                for (auto [ps, pk] : passes) {
                    const int p = pass_index(ps, pk);
                    pass_best[p] = std::min(pass_best[p], lv[p]);
                }
        }
        free_plan(c, P);
        for (auto [ps, pk] : passes) {
            const int p = pass_index(ps, pk);
            size_t sm = 0;  // a cluster-form candidate that cannot run this pass was replaced by the default there
            if (per_pass[p].cluster > 0 && !cluster_fits(c, jobs, ps, pk, per_pass[p], &sm)) continue;
            if (pass_best[p] < best_ms[p]) {
                best_ms[p] = pass_best[p];
                best_cfg[p] = per_pass[p];
            }
            if (per_pass[p].cluster == 0 && pass_best[p] < best_queue_ms[p]) {
                best_queue_ms[p] = pass_best[p];
                best_queue_cfg[p] = per_pass[p];
            }
        }
        return FF_OK;
    };
    for (int ci = 0; ci < kNCands; ci++) {
        TileCfg cfg = kCands[ci];
        cfg.k = std::min(cfg.k, T);
        if (!cfg_fits(cfg)) continue;
        std::vector<TileCfg> per_pass(kMaxPasses, cfg), fitted(kMaxPasses, cfg);
        bool any = false;
        for (auto [ps, pk] : passes) {
            const int p = pass_index(ps, pk);
            fitted[p] = wave_fitted(c, jobs, ps, pk, cfg);
            any = any || fitted[p].tw != cfg.tw || fitted[p].th != cfg.th;
        }
        s = time_plan(per_pass);
        if (s == FF_OK && any) s = time_plan(fitted);
        if (s != FF_OK) return s;
    }
    c->profiling = was_profiling;
    for (auto [ps, pk] : passes) {
        const int p = pass_index(ps, pk);
        const TuneKey key{p, grid_dim(jobs[0].a->ws[ps], pk), grid_dim(jobs[0].a->hs[ps], pk), nj, T};
        if (best_ms[p] < 1e29) c->tuned[key] = best_cfg[p];
        if (best_queue_ms[p] < 1e29) c->tuned_queue[key] = best_queue_cfg[p];
    }
    return FF_OK;
}

}  // namespace

namespace ff {

bool ctx_view(const ff_ctx* c, CtxView* out) {
    if (!c || !out) return false;
    out->device = c->device;
    out->n_sms = c->n_sms;
    out->stream = c->stream;
    out->n_scales = c->prm.n_scales;
    out->iters = c->prm.iters;
    out->rs_radius = c->prm.rs_radius;
    out->eps = c->prm.eps;
    out->seed = c->prm.seed;
    out->cost = c->prm.cost;
    out->noalloc_scratch = c->noalloc_scratch;
    out->sub_scales = c->prm.sub_scales;
    out->wait_limit = c->wait_limit;
    out->withhold = c->withhold;
    out->err_word = c->d_err;
    return true;
}

bool ctx_owns_live_pyr(const ff_ctx* c, const ff_pyr* p) {
    if (!c || !p) return false;
    for (auto& q : c->pyrs)
        if (q.get() == p) return p->in_use;
    return false;
}

bool pyr_view(const ff_pyr* p, PyrView* out) {
    if (!p || !out) return false;
    out->w = p->w;
    out->h = p->h;
    out->L = p->L;
    for (int s = 0; s < kMaxLevels; s++) {
        out->ws[s] = p->ws[s];
        out->hs[s] = p->hs[s];
        out->feat[s] = p->feat[s];
        out->cen[s] = p->cen[s];
    }
    out->seed_desc = p->seed_desc;
    out->seed_norm = p->seed_norm;
    out->n_coarse = p->n_coarse;
    return true;
}

// The configuration for pass `level` (a level s or a sub-scale grid s + 8k) of size w x h, in the tile or (if
// dataflow_ok) the dataflow form: the override if it is of one of these forms, else the best of them the
// autotuner timed for this size with the nearest number of directions per launch, else the default.  A dataflow
// configuration where it is not wanted becomes its tiles with one iteration per launch.
TileChoice ctx_level_choice(const ff_ctx* c, int level, int w, int h, int n_dirs, int64_t level_pix_all,
                            bool dataflow_ok) {
    const int T = c->prm.iters;
    TileCfg tc;
    if (level >= 0 && level < kMaxPasses && c->forced[level].threads > 0 && c->forced[level].cluster == 0) {
        tc = c->forced[level];
    } else {
        const TileCfg* best = nullptr;
        int best_d = 0;
        for (const auto& kv : c->tuned_queue) {
            if (std::get<0>(kv.first) != level || std::get<1>(kv.first) != w || std::get<2>(kv.first) != h ||
                std::get<4>(kv.first) != T)
                continue;
            const int d = std::abs(std::get<3>(kv.first) - n_dirs);
            if (!best || d < best_d) {
                best = &kv.second;
                best_d = d;
            }
        }
        tc = best ? *best : default_cfg(c, level_pix_all, T);
    }
    if (tc.dataflow > 0 && !dataflow_ok) tc = TileCfg{tc.tw, tc.th, 1, tc.threads, 0};
    if (tc.dataflow > 0) return {tc.tw, tc.th, T, tc.threads, 0, tc.dataflow};
    return {tc.tw, tc.th, std::min(tc.k, T), tc.threads, tc.spec, 0};
}

int* ctx_err_word(ff_ctx* c) {
    if (ensure_err_word(c) != FF_OK) return nullptr;
    return c->d_err;
}

int ctx_set_error(ff_ctx* c, int status, const char* msg) {
    return (int)fail(c, (ff_status)status, "%s", msg);
}

cudaError_t ctx_malloc(ff_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (c->fail_allocs > 0) {  // FF_OPT_TEST_FAIL_ALLOCS: behave as an exhausted device, allocate nothing
        c->fail_allocs--;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

}  // namespace ff

namespace {

bool aligned4(const void* p) { return ((uintptr_t)p & 3) == 0; }

ff_status check_pyr(ff_ctx* c, const ff_pyr* p, const char* what) {
    if (!p) return fail(c, FF_ERR_ARG, "%s is NULL", what);
    bool found = false;
    for (auto& q : c->pyrs)
        if (q.get() == p) found = true;
    if (!found) return fail(c, FF_ERR_ARG, "%s does not belong to this context", what);
    if (!p->in_use) return fail(c, FF_ERR_ARG, "%s has been released", what);
    return FF_OK;
}

// A frame's pyramid from the context's pool (allocated if no free one of its size exists), after validating the
// frame.  Launches nothing except, for a new pyramid, the zeroing of its seed rows' padding.
ff_status acquire_pyr(ff_ctx* c, const uint8_t* rgb_dev, int w, int h, int pitch_bytes, ff_pyr** out) {
    if (!rgb_dev) return fail(c, FF_ERR_ARG, "rgb_dev is NULL");
    if (w < 1 || h < 1 || w > kMaxDim || h > kMaxDim) return fail(c, FF_ERR_ARG, "size %dx%d outside 1..%d", w, h, kMaxDim);
    if (pitch_bytes < 3 * w) return fail(c, FF_ERR_ARG, "pitch %d < 3*w", pitch_bytes);
    const int L = c->prm.n_scales;
    {
        int ws[kMaxLevels], hs[kMaxLevels];
        level_dims(w, h, L, ws, hs);
        if ((int64_t)ws[L - 1] * hs[L - 1] > kMaxCoarsePixels)
            return fail(c, FF_ERR_ARG,
                        "coarsest level %dx%d has more than %d pixels for the exhaustive initial matching: use more "
                        "scales for a %dx%d frame", ws[L - 1], hs[L - 1], kMaxCoarsePixels, w, h);
    }
    FF_CUDA(c, cudaSetDevice(c->device));
    const bool census = c->prm.cost == FF_COST_CENSUS;
    ff_pyr* P = nullptr;
    for (auto& q : c->pyrs)
        if (!q->in_use && q->w == w && q->h == h && q->L == L) {
            P = q.get();
            break;
        }
    if (!P) {
        auto np = std::make_unique<ff_pyr>();
        np->w = w;
        np->h = h;
        np->L = L;
        level_dims(w, h, L, np->ws, np->hs);
        np->n_coarse = np->ws[L - 1] * np->hs[L - 1];
        np->n_pad = round_up(np->n_coarse, 16);
        np->n_pad128 = round_up(np->n_coarse, kSeedTcRows);
        size_t bytes = 0;
        for (int s = 1; s < L; s++) bytes += align_up((size_t)np->ws[s] * np->hs[s] * 3);
        for (int s = 0; s < L; s++) bytes += align_up((size_t)np->ws[s] * np->hs[s] * kDescBytes);
        if (census)
            for (int s = 0; s < L; s++) bytes += align_up((size_t)np->ws[s] * np->hs[s] * kCensusBytes);
        bytes += align_up((size_t)np->n_pad * kSeedK) + align_up((size_t)np->n_coarse * 4);
        bytes += align_up((size_t)np->n_pad128 * 128) + align_up(128);
        ff_status s = dev_alloc(c, np->mem, bytes);
        if (s != FF_OK) return s;
        char* b = static_cast<char*>(np->mem.p);
        size_t o = 0;
        for (int l = 1; l < L; l++) {
            np->img[l] = reinterpret_cast<uint8_t*>(b + o);
            o += align_up((size_t)np->ws[l] * np->hs[l] * 3);
        }
        for (int l = 0; l < L; l++) {
            np->feat[l] = reinterpret_cast<int16_t*>(b + o);
            o += align_up((size_t)np->ws[l] * np->hs[l] * kDescBytes);
        }
        if (census)
            for (int l = 0; l < L; l++) {
                np->cen[l] = reinterpret_cast<uint32_t*>(b + o);
                o += align_up((size_t)np->ws[l] * np->hs[l] * kCensusBytes);
            }
        np->seed_desc = reinterpret_cast<int8_t*>(b + o);
        o += align_up((size_t)np->n_pad * kSeedK);
        np->seed_norm = reinterpret_cast<int32_t*>(b + o);
        o += align_up((size_t)np->n_coarse * 4);
        np->desc16 = b + o;
        o += align_up((size_t)np->n_pad128 * 128);
        np->tmap = b + o;
        alignas(64) unsigned char map[128];
        if (!seed_tc_encode_map(map, np->desc16, np->n_pad128)) {
            dev_free(c, np->mem);
            return fail(c, FF_ERR_CUDA, "TMA tensor map encoding failed");
        }
        FF_CUDA(c, cudaMemcpy(np->tmap, map, sizeof map, cudaMemcpyHostToDevice));
        // padding rows of the seed descriptors are never written: zero them once
        FF_CUDA(c, cudaMemsetAsync(np->seed_desc, 0, (size_t)np->n_pad * kSeedK, c->stream));
        FF_CUDA(c, cudaMemsetAsync(np->desc16, 0, (size_t)np->n_pad128 * 128, c->stream));
        P = np.get();
        c->pyrs.push_back(std::move(np));
    }
    P->in_use = true;
    *out = P;
    return FF_OK;
}

// Arguments of the fused pyramid launch of a frame (levels 1..min(L-1, 6)).
PyrArgs pyramid_args(const ff_pyr* P, const uint8_t* rgb_dev, int pitch_bytes) {
    PyrArgs pa{};
    pa.src = rgb_dev;
    pa.spitch = pitch_bytes;
    for (int s = 0; s < P->L; s++) {
        pa.dst[s] = P->img[s];
        pa.w[s] = P->ws[s];
        pa.h[s] = P->hs[s];
    }
    pa.top = std::min(P->L - 1, kPyrFusedTop);
    return pa;
}

// Levels past the fused pyramid launch (L = 8 only): one launch each; returns the number of launches.
int deep_levels(const ff_pyr* P, cudaStream_t st) {
    int nl = 0;
    for (int s = kPyrFusedTop + 1; s < P->L; s++) {
        launch_downsample(P->img[s - 1], P->ws[s - 1], P->hs[s - 1], P->ws[s - 1] * 3, P->img[s], P->ws[s], P->hs[s],
                          st);
        nl++;
    }
    return nl;
}

// WHT launch entry of level s of a frame; *tiles is the first CTA of the entry and is advanced past it.
WhtLevel wht_level(const ff_pyr* P, int s, const uint8_t* rgb_dev, int pitch_bytes, int* tiles) {
    WhtLevel lv{};
    lv.img = s == 0 ? rgb_dev : P->img[s];
    lv.pitch = s == 0 ? pitch_bytes : P->ws[s] * 3;
    lv.w = P->ws[s];
    lv.h = P->hs[s];
    lv.feat = P->feat[s];
    lv.census = P->cen[s];
    if (s == P->L - 1) {  // the coarsest level also writes the initial-matching descriptors
        lv.seed_desc = P->seed_desc;
        lv.seed_norm = P->seed_norm;
        lv.desc16 = P->desc16;
    }
    lv.tiles_x = wht_tiles_x(P->ws[s]);
    lv.tile_base = *tiles;
    *tiles += wht_tiles(P->ws[s], P->hs[s]);
    return lv;
}

}  // namespace

extern "C" {

void ff_default_params(ff_params* p) {
    if (!p) return;
    p->n_scales = 5;
    p->iters = 6;
    p->patch = 8;
    p->n_coef = 16;
    p->rs_radius = 2;
    p->eps = 1;
    p->seed = 0x20180503u;
    p->rs_radius2 = 4;
    p->cost = FF_COST_WHT_SAD;
    p->sub_scales = 0;
}

ff_status ff_create(ff_ctx** out, const ff_params* p, int device, void* cuda_stream) {
    if (!out) return FF_ERR_ARG;
    *out = nullptr;
    ff_status s = check_params(p, nullptr);
    if (s != FF_OK) return s;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return FF_ERR_ARG;
    }
    ff_ctx* c = new (std::nothrow) ff_ctx();
    if (!c) return FF_ERR_OOM;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->prm = *p;
    // with the device current: kernel attributes, and the set-up of ff_match_pair_noalloc (its scratch array and
    // kernels are loaded here, so that its calls never load code or reserve memory)
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = init_kernel_attributes();
    if (e == cudaSuccess) e = seed_tc_init_attributes();
    if (e == cudaSuccess) e = noalloc_prepare(&c->noalloc_scratch);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return e == cudaErrorMemoryAllocation ? FF_ERR_OOM : FF_ERR_CUDA;
    }
    *out = c;
    return FF_OK;
}

ff_status ff_features(ff_ctx* c, const uint8_t* rgb_dev, int w, int h, int pitch_bytes, ff_pyr** out) {
    if (!c) return FF_ERR_ARG;
    if (!out) return fail(c, FF_ERR_ARG, "out is NULL");
    *out = nullptr;
    ff_pyr* P = nullptr;
    ff_status s = acquire_pyr(c, rgb_dev, w, h, pitch_bytes, &P);
    if (s != FF_OK) return s;
    const int L = P->L;

    cudaEvent_t ea = nullptr, eb = nullptr;
    if (c->profiling) {
        ea = get_event(c);
        eb = get_event(c);
        FF_CUDA(c, cudaEventRecord(ea, c->stream));
    }
    int nl = 0;
    if (L > 1) {  // levels 1..min(L-1, 6) in one launch, deeper levels one launch each
        PyrArgs pa = pyramid_args(P, rgb_dev, pitch_bytes);
        launch_pyramid(pa, c->stream);
        nl++;
        nl += deep_levels(P, c->stream);
    }
    WhtArgs wa{};
    wa.n = L;
    int tiles = 0;
    for (int s = L - 1; s >= 0; s--) wa.lv[L - 1 - s] = wht_level(P, s, rgb_dev, pitch_bytes, &tiles);
    launch_wht(wa, tiles, c->stream);
    nl++;
    c->launches += nl;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        P->in_use = false;
        return fail(c, FF_ERR_CUDA, "feature launch failed: %s", cudaGetErrorString(e));
    }
    if (c->profiling) {
        FF_CUDA(c, cudaEventRecord(eb, c->stream));
        c->events.push_back({FF_PHASE_FEATURES, -1, ea, eb, nl});
    }
    *out = P;
    return FF_OK;
}

// ff_features_batch; with fine_below > 0 the levels below it are left out of the launches and their table entries
// returned in *fine, for the caller to launch.
static ff_status features_batch_impl(ff_ctx* c, int n, const ff_frame* frames, ff_pyr** out, int fine_below,
                                     FineWht* fine) {
    if (!c) return FF_ERR_ARG;
    if (n < 0 || (n > 0 && (!frames || !out))) return fail(c, FF_ERR_ARG, "bad frame list");
    if (fine) *fine = FineWht{};
    for (int i = 0; i < n; i++) out[i] = nullptr;
    if (n == 0) return FF_OK;
    for (int i = 0; i < n; i++) {
        ff_status s = acquire_pyr(c, frames[i].rgb_dev, frames[i].w, frames[i].h, frames[i].pitch_bytes, &out[i]);
        if (s != FF_OK) {  // give back what this call took; nothing was launched
            for (int j = 0; j < i; j++) {
                out[j]->in_use = false;
                out[j] = nullptr;
            }
            return s;
        }
    }
    // tables: one pyramid entry per frame with more than one level; the WHT levels of all frames, coarsest levels
    // first (their CTAs also write the seed rows, the longest tiles)
    std::vector<PyrArgs> pyr_tab;
    std::vector<WhtLevel> wht_tab, wht_fine;
    int ctas = 0, tiles = 0, fine_tiles = 0, max_L = 0;
    for (int i = 0; i < n; i++) {
        max_L = std::max(max_L, out[i]->L);
        if (out[i]->L > 1) {
            PyrArgs pa = pyramid_args(out[i], frames[i].rgb_dev, frames[i].pitch_bytes);
            pa.cta_base = ctas;
            pa.bx = pyramid_blocks_x(out[i]->ws[1]);
            ctas += pyramid_blocks(out[i]->ws[1], out[i]->hs[1]);
            pyr_tab.push_back(pa);
        }
    }
    for (int up = 0; up < max_L; up++)  // up = levels above the finest: 0 is each frame's coarsest level
        for (int i = 0; i < n; i++) {
            const int L = out[i]->L;
            if (up >= L) continue;
            if (L - 1 - up < fine_below)
                wht_fine.push_back(wht_level(out[i], L - 1 - up, frames[i].rgb_dev, frames[i].pitch_bytes, &fine_tiles));
            else
                wht_tab.push_back(wht_level(out[i], L - 1 - up, frames[i].rgb_dev, frames[i].pitch_bytes, &tiles));
        }
    const size_t o_wht = align_up(pyr_tab.size() * sizeof(PyrArgs));
    const size_t o_fine = o_wht + align_up(wht_tab.size() * sizeof(WhtLevel));
    const size_t bytes = wht_fine.empty() ? o_wht + wht_tab.size() * sizeof(WhtLevel)
                                          : o_fine + wht_fine.size() * sizeof(WhtLevel);
    auto give_back = [&]() {
        for (int i = 0; i < n; i++) {
            out[i]->in_use = false;
            out[i] = nullptr;
        }
    };
    if (c->feat_tab.bytes < bytes) {  // grow the context's table buffer (after the work that still reads it)
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            give_back();
            return fail(c, FF_ERR_CUDA, "cudaStreamSynchronize failed: %s", cudaGetErrorString(e));
        }
        dev_free(c, c->feat_tab);
        ff_status s = dev_alloc(c, c->feat_tab, std::max(bytes, (size_t)64 << 10));
        if (s != FF_OK) {
            give_back();
            return s;
        }
    }
    std::vector<char> host(bytes);
    memcpy(host.data(), pyr_tab.data(), pyr_tab.size() * sizeof(PyrArgs));
    memcpy(host.data() + o_wht, wht_tab.data(), wht_tab.size() * sizeof(WhtLevel));
    if (!wht_fine.empty()) memcpy(host.data() + o_fine, wht_fine.data(), wht_fine.size() * sizeof(WhtLevel));
    char* dev = static_cast<char*>(c->feat_tab.p);

    cudaEvent_t ea = nullptr, eb = nullptr;
    if (c->profiling) {
        ea = get_event(c);
        eb = get_event(c);
        FF_CUDA(c, cudaEventRecord(ea, c->stream));
    }
    // from pageable memory: the copy is staged before the call returns, so the host table can go at once; it runs
    // after the work already on the stream (which may still read the previous table)
    cudaError_t e = cudaMemcpyAsync(dev, host.data(), bytes, cudaMemcpyHostToDevice, c->stream);
    int nl = 0;
    if (e == cudaSuccess && !pyr_tab.empty()) {
        launch_pyramid_tab(reinterpret_cast<const PyrArgs*>(dev), (int)pyr_tab.size(), ctas, c->stream);
        nl++;
        for (int i = 0; i < n; i++) nl += deep_levels(out[i], c->stream);
    }
    if (e == cudaSuccess && !wht_tab.empty()) {
        launch_wht_tab(reinterpret_cast<const WhtLevel*>(dev + o_wht), (int)wht_tab.size(), tiles, c->stream);
        nl++;
        e = cudaGetLastError();
    }
    c->launches += nl;
    if (e != cudaSuccess) {
        give_back();
        return fail(c, FF_ERR_CUDA, "feature launch failed: %s", cudaGetErrorString(e));
    }
    if (c->profiling) {
        FF_CUDA(c, cudaEventRecord(eb, c->stream));
        c->events.push_back({FF_PHASE_FEATURES, -1, ea, eb, nl});
    }
    if (fine && !wht_fine.empty()) {
        fine->tab = reinterpret_cast<const WhtLevel*>(dev + o_fine);
        fine->n = (int)wht_fine.size();
        fine->tiles = fine_tiles;
    }
    return FF_OK;
}

ff_status ff_features_batch(ff_ctx* c, int n, const ff_frame* frames, ff_pyr** out) {
    return features_batch_impl(c, n, frames, out, 0, nullptr);
}

ff_status ff_match_pair(ff_ctx* c, const ff_pyr* a, const ff_pyr* b, int dir, int16_t* flow_dev, int32_t* cost_dev) {
    if (!c) return FF_ERR_ARG;
    ff_status s;
    if ((s = check_pyr(c, a, "a")) != FF_OK) return s;
    if ((s = check_pyr(c, b, "b")) != FF_OK) return s;
    if (a->w != b->w || a->h != b->h) return fail(c, FF_ERR_ARG, "pyramids differ in size");
    if (dir != 0 && dir != 1) return fail(c, FF_ERR_ARG, "dir must be 0 or 1");
    if (!flow_dev || !aligned4(flow_dev)) return fail(c, FF_ERR_ARG, "flow_dev must be a 4-byte aligned device pointer");
    if (cost_dev && !aligned4(cost_dev)) return fail(c, FF_ERR_ARG, "cost_dev must be 4-byte aligned");
    FF_CUDA(c, cudaSetDevice(c->device));
    std::vector<DirJob> jobs{{a, b, dir, reinterpret_cast<uint32_t*>(flow_dev), cost_dev, c->prm.rs_radius}};
    return run_jobs(c, jobs, {});
}

static ff_status collect_batch(ff_ctx* c, int n, const ff_pair_job* jobs, std::vector<DirJob>& dj,
                               std::vector<ConsJob>& cj) {
    for (int i = 0; i < n; i++) {
        const ff_pair_job& J = jobs[i];
        ff_status s;
        if ((s = check_pyr(c, J.a, "job.a")) != FF_OK) return s;
        if ((s = check_pyr(c, J.b, "job.b")) != FF_OK) return s;
        if (J.a->w != J.b->w || J.a->h != J.b->h) return fail(c, FF_ERR_ARG, "job %d: pyramids differ in size", i);
        if (!J.flow_fwd || !J.flow_bwd || !J.mask) return fail(c, FF_ERR_ARG, "job %d: NULL output", i);
        if (!aligned4(J.flow_fwd) || !aligned4(J.flow_bwd) || (J.cost_fwd && !aligned4(J.cost_fwd)) ||
            (J.cost_bwd && !aligned4(J.cost_bwd)))
            return fail(c, FF_ERR_ARG, "job %d: outputs must be 4-byte aligned", i);
        if (J.flow_bwd2 && !aligned4(J.flow_bwd2)) return fail(c, FF_ERR_ARG, "job %d: flow_bwd2 misaligned", i);
        const int f0 = (int)dj.size();
        dj.push_back({J.a, J.b, 0, reinterpret_cast<uint32_t*>(J.flow_fwd), J.cost_fwd, c->prm.rs_radius});
        dj.push_back({J.b, J.a, 1, reinterpret_cast<uint32_t*>(J.flow_bwd), J.cost_bwd, c->prm.rs_radius});
        int b2 = -1;
        if (J.flow_bwd2) {
            b2 = (int)dj.size();
            dj.push_back({J.b, J.a, 2, reinterpret_cast<uint32_t*>(J.flow_bwd2), nullptr, c->prm.rs_radius2});
        }
        cj.push_back({f0, f0 + 1, J.mask, b2});
    }
    return FF_OK;
}

ff_status ff_match_batch(ff_ctx* c, int n, const ff_pair_job* jobs) {
    if (!c) return FF_ERR_ARG;
    if (n < 0 || (n > 0 && !jobs)) return fail(c, FF_ERR_ARG, "bad job list");
    if (n == 0) return FF_OK;
    std::vector<DirJob> dj;
    std::vector<ConsJob> cj;
    ff_status s = collect_batch(c, n, jobs, dj, cj);
    if (s != FF_OK) return s;
    FF_CUDA(c, cudaSetDevice(c->device));
    return run_jobs(c, dj, cj);
}

ff_status ff_match_frames(ff_ctx* c, int n_frames, const ff_frame* frames, int n_jobs, const ff_frame_job* jobs,
                          ff_pyr** out) {
    if (!c) return FF_ERR_ARG;
    if (n_frames < 1 || !frames || n_jobs < 1 || !jobs) return fail(c, FF_ERR_ARG, "bad frame or job list");
    if (out)
        for (int i = 0; i < n_frames; i++) out[i] = nullptr;
    for (int i = 0; i < n_jobs; i++) {  // everything the jobs can get wrong, before anything is launched
        const ff_frame_job& J = jobs[i];
        if (J.a < 0 || J.a >= n_frames || J.b < 0 || J.b >= n_frames)
            return fail(c, FF_ERR_ARG, "job %d: frame index outside 0..%d", i, n_frames - 1);
        if (frames[J.a].w != frames[J.b].w || frames[J.a].h != frames[J.b].h)
            return fail(c, FF_ERR_ARG, "job %d: frames differ in size", i);
        if (!J.flow_fwd || !J.flow_bwd || !J.mask) return fail(c, FF_ERR_ARG, "job %d: NULL output", i);
        if (!aligned4(J.flow_fwd) || !aligned4(J.flow_bwd) || (J.cost_fwd && !aligned4(J.cost_fwd)) ||
            (J.cost_bwd && !aligned4(J.cost_bwd)) || (J.flow_bwd2 && !aligned4(J.flow_bwd2)))
            return fail(c, FF_ERR_ARG, "job %d: outputs must be 4-byte aligned", i);
    }
    FF_CUDA(c, cudaSetDevice(c->device));
    // the fine levels' descriptors go beside the coarse levels' matching when the matching runs as graphs on a
    // stream of its own and the coarsest level is above them
    const int fine_below = 2;
    const bool overlap = c->overlap > 0 && !c->profiling && c->stream != nullptr && c->prm.n_scales > fine_below;
    if (overlap) {
        ff_status s = ensure_side(c);
        if (s != FF_OK) return s;
    }
    std::vector<ff_pyr*> pyrs(n_frames, nullptr);
    FineWht fine;
    ff_status s = features_batch_impl(c, n_frames, frames, pyrs.data(), overlap ? fine_below : 0, &fine);
    if (s != FF_OK) return s;
    std::vector<ff_pair_job> pj(n_jobs);
    for (int i = 0; i < n_jobs; i++) {
        const ff_frame_job& J = jobs[i];
        pj[i] = ff_pair_job{pyrs[J.a], pyrs[J.b], J.flow_fwd, J.flow_bwd, J.cost_fwd, J.cost_bwd, J.mask, J.flow_bwd2};
    }
    std::vector<DirJob> dj;
    std::vector<ConsJob> cj;
    s = collect_batch(c, n_jobs, pj.data(), dj, cj);
    Plan* P = nullptr;
    if (s == FF_OK) s = find_plan(c, dj, cj, &P);
    if (s == FF_OK) s = fine.n > 0 ? execute_plan_split(c, *P, fine, fine_below) : execute_plan(c, *P);
    if (s != FF_OK && fine.n > 0) {  // no (or a failed) matching: the pyramids are still completed on the stream
        launch_wht_tab(fine.tab, fine.n, fine.tiles, c->stream);
        c->launches += 1;
    }
    for (int i = 0; i < n_frames; i++) {
        if (out && s == FF_OK)
            out[i] = pyrs[i];
        else
            pyrs[i]->in_use = false;  // recycled by later calls, after this call's work on the stream
    }
    return s;
}

ff_status ff_autotune(ff_ctx* c, int n, const ff_pair_job* jobs, int reps) {
    if (!c) return FF_ERR_ARG;
    if (n < 1 || !jobs || reps < 1 || reps > 100) return fail(c, FF_ERR_ARG, "bad autotune arguments");
    std::vector<DirJob> dj;
    std::vector<ConsJob> cj;
    ff_status s = collect_batch(c, n, jobs, dj, cj);
    if (s != FF_OK) return s;
    FF_CUDA(c, cudaSetDevice(c->device));
    return autotune(c, dj, cj, reps);
}

ff_status ff_set_tuning(ff_ctx* c, int level, const ff_tuning* t) {
    if (!c) return FF_ERR_ARG;
    if (level < 0 || level >= kMaxPasses)
        return fail(c, FF_ERR_ARG, "pass %d outside 0..%d", level, kMaxPasses - 1);
    TileCfg cfg{0, 0, 0, 0, 0, 0, 0};
    if (t) {
        cfg = TileCfg{t->tile_w, t->tile_h, t->iters_per_launch, t->threads, t->speculate, t->cluster, t->dataflow};
        bool ok = t->iters_per_launch >= 1 && t->iters_per_launch <= 255 && (t->speculate == 0 || t->speculate == 1) &&
                  t->dataflow >= 0 && t->dataflow <= 2;
        if (t->dataflow > 0)  // one iteration per task, its 4-pixel halo within the 3x3 tiles around it
            ok = ok && t->cluster == 0 && t->iters_per_launch == 1 && t->speculate == 0 && t->tile_w >= 4 &&
                 t->tile_h >= 4;
        if (t->cluster == 0)
            ok = ok && t->tile_w >= 1 && t->tile_h >= 1 && t->tile_w <= 1024 && t->tile_h <= 1024 &&
                 prop_threads_ok(t->threads) && cfg_fits(cfg);
        else  // the cluster form: the tile fields are unused, no speculation; whether a level can take it is
              // decided per plan
            ok = ok && t->cluster >= 1 && t->cluster <= kMaxCluster && (t->threads == 256 || t->threads == 512) &&
                 t->tile_w == 0 && t->tile_h == 0 && t->speculate == 0;
        if (!ok)
            return fail(c, FF_ERR_ARG,
                        "configuration %dx%d, %d iterations, %d threads, speculate %d, cluster %d, dataflow %d is not "
                        "valid",
                        t->tile_w, t->tile_h, t->iters_per_launch, t->threads, t->speculate, t->cluster, t->dataflow);
    }
    FF_CUDA(c, cudaSetDevice(c->device));
    ff_status s = drop_plans(c);
    if (s != FF_OK) return s;
    c->forced[level] = cfg;
    return FF_OK;
}

ff_status ff_get_tuning(ff_ctx* c, int level, ff_tuning* out) {
    if (!c || !out || level < 0 || level >= kMaxPasses) return FF_ERR_ARG;
    const TileCfg* f = nullptr;
    if (c->forced[level].threads > 0) {
        f = &c->forced[level];
    } else {
        for (auto& kv : c->tuned)
            if (std::get<0>(kv.first) == level) {
                f = &kv.second;
                break;
            }
    }
    if (!f) return fail(c, FF_ERR_ARG, "level %d has not been tuned", level);
    *out = ff_tuning{f->tw, f->th, f->k, f->threads, f->spec, f->cluster, f->dataflow};
    return FF_OK;
}

ff_status ff_consistency(ff_ctx* c, const int16_t* fwd, const int16_t* bwd, int w, int h, int eps, uint8_t* mask_dev) {
    if (!c) return FF_ERR_ARG;
    if (!fwd || !bwd || !mask_dev || !aligned4(fwd) || !aligned4(bwd)) return fail(c, FF_ERR_ARG, "bad pointer");
    if (w < 1 || h < 1 || w > kMaxDim || h > kMaxDim) return fail(c, FF_ERR_ARG, "size %dx%d outside 1..%d", w, h, kMaxDim);
    if (eps < 0 || eps > 32767) return fail(c, FF_ERR_ARG, "eps must be 0..32767");
    FF_CUDA(c, cudaSetDevice(c->device));
    Launch l{};
    l.kind = Kind::Consistency;
    l.phase = FF_PHASE_CONSISTENCY;
    l.fwd = reinterpret_cast<const uint32_t*>(fwd);
    l.bwd = reinterpret_cast<const uint32_t*>(bwd);
    l.w = w;
    l.h = h;
    l.eps = eps;
    l.mask = mask_dev;
    return run_launches(c, {l}, c->profiling);
}

ff_status ff_sparsify(ff_ctx* c, const int16_t* fwd, const int16_t* bwd, const uint8_t* keep_dev, int w, int h,
                      int eps, int min_matches, uint8_t* sparse_dev) {
    if (!c) return FF_ERR_ARG;
    if (!fwd || !bwd || !sparse_dev || !aligned4(fwd) || !aligned4(bwd)) return fail(c, FF_ERR_ARG, "bad pointer");
    if (w < 1 || h < 1 || w > kMaxDim || h > kMaxDim) return fail(c, FF_ERR_ARG, "size %dx%d outside 1..%d", w, h, kMaxDim);
    if (eps < 0 || eps > 32767) return fail(c, FF_ERR_ARG, "eps must be 0..32767");
    if (min_matches < 1 || min_matches > 9) return fail(c, FF_ERR_ARG, "min_matches must be 1..9");
    FF_CUDA(c, cudaSetDevice(c->device));
    launch_sparsify(reinterpret_cast<const uint32_t*>(fwd), reinterpret_cast<const uint32_t*>(bwd), keep_dev, w, h,
                    eps, min_matches, sparse_dev, c->stream);
    FF_CUDA(c, cudaGetLastError());
    c->launches += 1;
    return FF_OK;
}

ff_status ff_pyr_release(ff_ctx* c, ff_pyr* p) {
    if (!c) return FF_ERR_ARG;
    ff_status s = check_pyr(c, p, "pyr");
    if (s != FF_OK) return s;
    p->in_use = false;
    return FF_OK;
}

ff_status ff_pyr_level_dims(const ff_pyr* p, int level, int* w, int* h) {
    if (!p || level < 0 || level >= p->L) return FF_ERR_ARG;
    if (w) *w = p->ws[level];
    if (h) *h = p->hs[level];
    return FF_OK;
}

const int16_t* ff_pyr_features(const ff_pyr* p, int level) {
    if (!p || level < 0 || level >= p->L) return nullptr;
    return p->feat[level];
}

const uint32_t* ff_pyr_census(const ff_pyr* p, int level) {
    if (!p || level < 0 || level >= p->L) return nullptr;
    return p->cen[level];
}

const char* ff_last_error(ff_ctx* c) { return c ? c->err.c_str() : "null context"; }

ff_status ff_sync(ff_ctx* c) {
    if (!c) return FF_ERR_ARG;
    FF_CUDA(c, cudaSetDevice(c->device));
    FF_CUDA(c, cudaStreamSynchronize(c->stream));
    FF_CUDA(c, cudaGetLastError());
#if FF_DEBUG_BOUNDS
    {  // a debug-bounds build: an index check failed since the last check
        int rec[3];
        for (int tu = 0; tu < 3; tu++) {
            FF_CUDA(c, tu == 0 ? bounds_take_propagate(rec) : tu == 1 ? bounds_take_filter(rec) : bounds_take_features(rec));
            if (rec[0] != 0)
                return fail(c, FF_ERR_CUDA, "bounds check %d failed: index %d outside 0..%d (access skipped)", rec[0],
                            rec[1], rec[2] - 1);
        }
    }
#endif
    if (c->d_err) {  // a bounded device-side wait gave up since the last check
        int e = 0;
        FF_CUDA(c, cudaMemcpy(&e, c->d_err, sizeof e, cudaMemcpyDeviceToHost));
        if (e != 0) {
            FF_CUDA(c, cudaMemset(c->d_err, 0, sizeof e));
            return fail(c, FF_ERR_TIMEOUT, "a device-side wait expired (code %d: %s)", e,
                        e == kErrClusterEdges ? "block edges of the cluster-form propagation"
                        : e == kErrDataflow   ? "tile progress of the dataflow-form propagation"
                                              : "copies or products of the tensor-core seed");
        }
    }
    return FF_OK;
}

ff_status ff_set_option(ff_ctx* c, int option, int64_t value) {
    if (!c) return FF_ERR_ARG;
    switch (option) {
        case FF_OPT_SEED_KERNEL:
            if (value != FF_SEED_MMA_SYNC && value != FF_SEED_TCGEN05) return fail(c, FF_ERR_ARG, "bad seed kernel");
            break;
        case FF_OPT_WAIT_LIMIT:
            if (value < 1 || value > (1ll << 30)) return fail(c, FF_ERR_ARG, "wait limit must be 1..2^30 polls");
            break;
        case FF_OPT_TEST_WITHHOLD_COPIES:
            if (value != 0 && value != 1) return fail(c, FF_ERR_ARG, "withhold must be 0 or 1");
            break;
        case FF_OPT_TEST_FAIL_ALLOCS:
            if (value < 0 || value > (1ll << 30)) return fail(c, FF_ERR_ARG, "allocation failures must be 0..2^30");
            c->fail_allocs = value;  // takes effect at once and keeps the cached plans
            return FF_OK;
        case FF_OPT_OVERLAP:
            if (value < 0 || value > 2) return fail(c, FF_ERR_ARG, "overlap must be 0, 1 or 2");
            c->overlap = (int)value;  // the plans' split graphs are recaptured when the fork point moves
            return FF_OK;
        default:
            return fail(c, FF_ERR_ARG, "unknown option %d", option);
    }
    FF_CUDA(c, cudaSetDevice(c->device));
    ff_status s = drop_plans(c);  // plans bake the options in
    if (s != FF_OK) return s;
    if (option == FF_OPT_SEED_KERNEL) c->seed_kernel = (int)value;
    if (option == FF_OPT_WAIT_LIMIT) c->wait_limit = (uint32_t)value;
    if (option == FF_OPT_TEST_WITHHOLD_COPIES) c->withhold = (int)value;
    return FF_OK;
}

ff_status ff_get_stats(ff_ctx* c, ff_stats* out) {
    if (!c || !out) return FF_ERR_ARG;
    out->kernel_launches = c->launches;
    out->graph_replays = c->replays;
    out->plans_built = c->plans_built;
    out->scratch_bytes = c->bytes;
    out->cluster_launches = c->cluster_launches;
    return FF_OK;
}

ff_status ff_profile_enable(ff_ctx* c, int on) {
    if (!c) return FF_ERR_ARG;
    c->profiling = on != 0;
    return FF_OK;
}

ff_status ff_profile_read(ff_ctx* c, double* ms, int64_t* launches) {
    if (!c) return FF_ERR_ARG;
    FF_CUDA(c, cudaStreamSynchronize(c->stream));
    double acc[FF_N_PHASES] = {0};
    int64_t cnt[FF_N_PHASES] = {0};
    for (auto& e : c->events) {
        float t = 0.f;
        FF_CUDA(c, cudaEventElapsedTime(&t, e.a, e.b));
        acc[e.phase] += t;
        cnt[e.phase] += e.n;
        c->event_pool.push_back(e.a);
        c->event_pool.push_back(e.b);
    }
    c->events.clear();
    for (int i = 0; i < FF_N_PHASES; i++) {
        if (ms) ms[i] = acc[i];
        if (launches) launches[i] = cnt[i];
    }
    return FF_OK;
}

ff_status ff_profile_read_passes(ff_ctx* c, double* ms, int64_t* launches) {
    if (!c) return FF_ERR_ARG;
    FF_CUDA(c, cudaStreamSynchronize(c->stream));
    double acc[FF_N_PASSES] = {0};
    int64_t cnt[FF_N_PASSES] = {0};
    for (auto& e : c->events) {
        float t = 0.f;
        FF_CUDA(c, cudaEventElapsedTime(&t, e.a, e.b));
        if (e.phase == FF_PHASE_PROPAGATE && e.level >= 0 && e.level < FF_N_PASSES) {
            acc[e.level] += t;
            cnt[e.level] += e.n;
        }
        c->event_pool.push_back(e.a);
        c->event_pool.push_back(e.b);
    }
    c->events.clear();
    for (int i = 0; i < FF_N_PASSES; i++) {
        if (ms) ms[i] = acc[i];
        if (launches) launches[i] = cnt[i];
    }
    return FF_OK;
}

ff_status ff_work_counts(ff_ctx* c, int w, int h, int64_t* pixel_iters, int64_t* pixels) {
    if (!c || w < 1 || h < 1 || w > kMaxDim || h > kMaxDim) return FF_ERR_ARG;
    int ws[kMaxLevels], hs[kMaxLevels];
    level_dims(w, h, c->prm.n_scales, ws, hs);
    int64_t pi = 0;
    for (int s = 0; s < c->prm.n_scales; s++)
        for (int k = 0; k <= (s == c->prm.n_scales - 1 ? 0 : c->prm.sub_scales); k++) {
            const int g = 1 << k;
            pi += (int64_t)((ws[s] + g - 1) / g) * ((hs[s] + g - 1) / g) * c->prm.iters;
        }
    if (pixel_iters) *pixel_iters = pi;
    if (pixels) *pixels = (int64_t)w * h;
    return FF_OK;
}

ff_status ff_destroy(ff_ctx* c) {
    if (!c) return FF_ERR_ARG;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->side) cudaStreamSynchronize(c->side);
    for (auto& kv : c->plans) free_plan(c, *kv.second);
    for (auto& p : c->pyrs) dev_free(c, p->mem);
    dev_free(c, c->feat_tab);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->d_err) cudaFree(c->d_err);
    for (auto& e : c->events) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
    delete c;
    return FF_OK;
}

}  // extern "C"
