// ff_internal.h -- internal types and launch wrappers of libff (GB300 / sm_103a).
//
// Device data layout (all row-major, pixel (x, y) at y*w + x):
//   image     uint8 [h][w][3]
//   features  int16 [h][w][48]  96 B per pixel: three 32-B sectors (R, G, B), coefficient u*4+v in each,
//                               stored in offset binary (C ^ 0x8000, read back with feature_coef);
//                               colour-split rows: within row y the descriptors of even x come first, then odd x
//                               (feat_index), so the pixels of one red-black half-sweep are contiguous
//   census    uint32 [h][w][8]  32 B per pixel (FF_COST_CENSUS only): words 2c, 2c+1 = channel c's 48-bit 7x7
//                               Census pattern, words 6, 7 zero; same colour-split order as the features
//   seed desc int8  [N16][64]   coarsest level, C >> 7, zero-padded from 48 to 64 and to a multiple of 16 rows
//   seed norm int32 [N]         squared norm of the 8-bit descriptor
//   flow      uint32 [h][w]     packed (dx & 0xffff) | (dy << 16): the int16 [h][w][2] layout of the C-ABI
//   cost      int32 [h][w]
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ff.h"

namespace ff {

constexpr int kNF = 48;           // int16 coefficients per pixel
constexpr int kDescBytes = 96;    // bytes per pixel descriptor
constexpr int kCensusBytes = 32;  // bytes per pixel Census pattern
constexpr int kSeedK = 64;        // padded 8-bit seed descriptor length
constexpr int kMaxLevels = 8;
constexpr int kHaloPerIter = 4;   // halo growth per fused propagation iteration (one per half-sweep quadrant side)

// ---------------------------------------------------------------------------------------------------------
// features

struct WhtLevel {
    const uint8_t* img;  // level image
    int pitch;           // bytes between rows
    int w, h;
    int16_t* feat;       // [h][w][48]
    uint32_t* census;    // [h][w][8], or null: no Census patterns
    int8_t* seed_desc;   // coarsest level only (else null): int8 [n_pad][64] rows y*w + x, padding rows zero
    int32_t* seed_norm;  //   [w*h] squared norms
    void* desc16;        //   f16 [n_pad128][64] rows y*w + x, padding rows zero
    int tiles_x;
    int tile_base;       // first CTA of this level in the fused launch
};
struct WhtArgs {
    WhtLevel lv[kMaxLevels];
    int n;
};

void launch_downsample(const uint8_t* src, int sw, int sh, int spitch, uint8_t* dst, int dw, int dh,
                       cudaStream_t st);
constexpr int kPyrBlock = 32;       // level-1 pixels per CTA side of the fused pyramid kernel
constexpr int kPyrFusedTop = 6;     // deepest level it derives (32 >> 5 = 1 pixel per CTA)
struct PyrArgs {
    const uint8_t* src;             // level 0, rows spitch bytes apart
    int spitch;
    uint8_t* dst[kMaxLevels];       // level s >= 1, compact rows (3 * w[s] bytes)
    int w[kMaxLevels], h[kMaxLevels];
    int top;                        // last level computed (1..kPyrFusedTop)
    int cta_base, bx;               // table launches: first CTA of this frame, level-1 blocks per row
};
void launch_pyramid(const PyrArgs& a, cudaStream_t st);
// many frames in one launch (tab_dev: n entries in device memory, cta_base ascending)
void launch_pyramid_tab(const PyrArgs* tab_dev, int n, int total_ctas, cudaStream_t st);
int pyramid_blocks_x(int w1);        // level-1 blocks per row / in all of a frame with level 1 of size w1 x h1
int pyramid_blocks(int w1, int h1);
// kernels ff_features launches for an L-level pyramid: the fused pyramid (+ one per level past kPyrFusedTop), WHT
inline int features_launches(int L) {
    return (L > 1 ? 1 + (L - 1 > kPyrFusedTop ? L - 1 - kPyrFusedTop : 0) : 0) + 1;
}
int wht_tiles_x(int w);
int wht_tiles(int w, int h);
void launch_wht(const WhtArgs& a, int total_tiles, cudaStream_t st);
// the levels of many frames in one launch (tab_dev: n entries in device memory, tile_base ascending)
void launch_wht_tab(const WhtLevel* tab_dev, int n, int total_tiles, cudaStream_t st, bool after_kernel = true);
const void* wht_tab_kernel();  // the kernel of launch_wht_tab (to find its node in a captured graph)

// ---------------------------------------------------------------------------------------------------------
// initial matches (exact nearest neighbour at the coarsest level)

struct SeedProblem {
    const int8_t* A;       // source descriptors [N16][64]
    const int8_t* B;       // target descriptors [N16][64]
    const int32_t* normA;  // [N]
    const int32_t* normB;  // [N]
    int n, w;              // pixels and level width (both frames have the same level size)
    uint32_t* flow;        // [N] packed
    int32_t* dist;         // [N] squared distance of the winner (may be null)
    int warp_base;         // first 16-row tile of this problem in the launch
};
void launch_seed(const SeedProblem* probs_dev, int n_probs, int total_row_tiles, cudaStream_t st);

// Tensor-core (tcgen05) version: descriptors as f16 [n_pad][64] behind a TMA tensor map (128 x 64 boxes).
constexpr int kSeedTcRows = 128, kSeedTcCols = 256;
struct SeedTcProblem {
    const void* map_a;             // device address of the source frame's CUtensorMap
    const void* map_b;             // target frame's
    const int32_t* normA;
    const int32_t* normB;
    int n, w;
    int row_tiles, col_tiles;      // ceil(n / 128), ceil(n / 256)
    int cta_base;                  // first CTA of this problem in the launch
    unsigned long long* keys;      // [n] (score + 2^31) << 32 | q, must start at all ones
    uint32_t* flow;                // [n] packed q - p
    int32_t* dist;                 // [n] or null
    int64_t pix_base;              // first pixel of this problem in the launch
};
cudaError_t seed_tc_init_attributes();
bool seed_tc_encode_map(void* map_host_128b, const void* desc16_dev, int n_pad);
// wait_limit: polls before a wait gives up (then *err_dev is set); withhold: issue no copies (test of the waits)
void launch_seed_tc(const SeedTcProblem* probs_dev, int n_probs, int total_ctas, int64_t total_pix,
                    uint32_t wait_limit, int withhold, int* err_dev, cudaStream_t st);

// ---------------------------------------------------------------------------------------------------------
// hand-over (coarse-to-fine initialisation) and cost initialisation

// A flow field lives on a grid of source pixels of its level: every pixel (g = 1), or every g-th pixel in both
// directions (g = 2, 4: the sub-scale grids).  Grid pixel (u, v) is level pixel (g*u, g*v); flows are in level
// pixels and may point to any pixel of the target level (lw x lh).
struct HandoverProblem {
    const void* fa;          // cost descriptors of the source frame (WHT features or Census patterns)
    const void* fb;          // and of the target frame
    int w, h;                // the grid this hand-over fills
    int g, lw, lh;           // its stride and level size (g <= 1: every pixel, lw x lh = w x h)
    const uint32_t* parent;  // flow of the level above or of the grid of stride 2g (pw x ph), or null: flow_in
    int pw, ph;
    int same_level;          // 1: parent is the grid of stride 2g of this level (flow copied, target clamped);
                             // 0: parent is the level above (flow doubled)
    const uint32_t* flow_in;
    uint32_t* flow_out;
    int32_t* cost_out;
    int64_t pix_base;        // first pixel of this problem in the launch
};
// cost: FF_COST_WHT_SAD or FF_COST_CENSUS (selects the descriptor type of fa/fb)
void launch_handover(const HandoverProblem* probs_dev, int n_probs, int64_t total_pix, int cost, cudaStream_t st);

// ---------------------------------------------------------------------------------------------------------
// propagation + random search, `n_iter` iterations of one level per launch, temporally blocked tiles

struct PropProblem {  // one (pair, direction, level) of a propagation launch
    const void* fa;  // cost descriptors of the source frame (WHT features or Census patterns)
    const void* fb;  // and of the target frame
    uint32_t* flow_in;  // (written too by the odd iterations of the dataflow form)
    int32_t* cost_in;
    uint32_t* flow_out;
    int32_t* cost_out;
    int w, h;        // the grid propagated (the level itself unless g > 1)
    int g, lw, lh;   // grid stride and level size (used by the grid kernels only, g > 1)
    int tiles_x;
    int t0;          // first iteration index (for the random-search hash)
    int n_iter;      // iterations fused into this launch
    int level;       // stream id of the random-search hash: the level, + 8 * log2(g) on a sub-scale grid
    int dir;
    uint32_t seed;
    int rs_radius;
    // dataflow form only: the state buffers iterations alternate with (iteration t writes flow_alt for even t,
    // flow_in for odd t, flow_out for the last) and the tiles' progress counters (zero at the launch's start)
    uint32_t* flow_alt;
    int32_t* cost_alt;
    int* progress;   // [tiles_x * tiles_y]: iterations each tile has finished
};
struct PropLaunch {
    int tw, th;      // tile interior
    int max_iter;    // largest n_iter of the launch (sizes the shared-memory halo)
    int threads;     // CTA size: 128, 256 or 512
    int spec;        // 1: load the random candidate together with the neighbour candidates
    int cost;        // FF_COST_WHT_SAD or FF_COST_CENSUS
    int grid;        // 1: the problems are sub-scale grids (g > 1)
    int cluster;     // 0: tiles from a queue; n = 1..16: cluster form, one cluster of n CTAs per problem
    int dataflow;    // > 0: dataflow form, this many iterations (of one each per tile task) in the launch
    int affine;      // dataflow form: 1 = each CTA keeps fixed tiles (no queue counter), 0 = tiles from the queue
    int cl_smem;     // cluster form: dynamic shared memory per CTA (the largest over the launch's problems)
    uint32_t wait_limit;  // cluster and dataflow forms: polls before a wait gives up
    int withhold;    // test of the bounded waits: the cluster form sends no block edges, the dataflow form
                     // publishes no tile progress
    int* err;        // device error word (kErrClusterEdges / kErrDataflow when a wait gave up)
};
constexpr int kErrClusterEdges = 3;  // error-word codes of expired waits (1, 2: tensor-core seed)
constexpr int kErrDataflow = 4;
constexpr size_t kMaxPropSmem = 200 * 1024;
constexpr int kMaxCluster = 16;
size_t prop_smem_bytes(int tw, int th, int n_iter);

// Cluster form of a propagation launch: the n CTAs of a cluster split a w x h problem into bx x by blocks
// (bx * by = n), CTA r owning block (r % bx, r / bx) with columns [i*w/bx, (i+1)*w/bx) and rows
// [j*h/by, (j+1)*h/by).  The divisor pair with the smallest total block perimeter (w*by + h*bx) is taken, among
// those that leave every block at least one pixel wide and high; false if there is none.
__host__ __device__ inline bool cluster_partition(int w, int h, int n, int& bx, int& by) {
    bool found = false;
    long long best = 0;
    for (int a = 1; a <= n; a++) {
        if (n % a != 0) continue;
        const int b = n / a;
        if (a > w || b > h) continue;
        const long long score = (long long)w * b + (long long)h * a;
        if (!found || score < best) {
            found = true;
            best = score;
            bx = a;
            by = b;
        }
    }
    return found;
}
// Shared memory of a CTA of the cluster form (the same layout in every CTA of a cluster): two mbarriers; the
// rings of neighbouring edge flows (left and right columns of mh, upper and lower rows of mw entries); the flows
// and costs of the block (mw x mh each), where mw x mh = ceil(w / bx) x ceil(h / by) bounds every block.
__host__ __device__ inline size_t cluster_smem_bytes(int w, int h, int bx, int by) {
    const size_t mw = (size_t)(w + bx - 1) / bx, mh = (size_t)(h + by - 1) / by;
    return 16 + 4 * (2 * mw + 2 * mh) + 8 * mw * mh;
}
cudaError_t init_kernel_attributes();  // once per device, before the first launch (also loads k_handover)
cudaError_t seed_load_kernel();        // loads k_seed onto the current device (lazy module loading)
// Set-up of ff_match_pair_noalloc on the current device, run by ff_create: loads its module (which reserves the
// fixed scratch array) and the kernels it launches, and returns the array's device address.
cudaError_t noalloc_prepare(void** scratch);
bool prop_threads_ok(int threads);
// resident CTAs per SM of the tile form (dataflow: of its dataflow kernel)
int prop_blocks_per_sm(size_t smem, int threads, bool spec, int cost, bool grid = false, bool dataflow = false);
// Tile form (L.cluster == 0): queue_dev[i] = (problem index, tile index); counter_dev must be zero when the launch
// starts; `grid` CTAs.  Dataflow form (L.dataflow = T): the same queue, taken T times (iteration-major).  Cluster form: problem i is probs_dev[i], `grid` = number of problems x L.cluster CTAs;
// queue_dev and counter_dev are unused.
void launch_propagate(const PropProblem* probs_dev, const int2* queue_dev, int n_tiles, int* counter_dev, int grid,
                      const PropLaunch& L, cudaStream_t st);
// Clusters of the cluster form that can be resident at once (0: this shape cannot be launched).
int prop_cluster_capacity(int cluster, int threads, int cost, bool grid, size_t smem);

// ---------------------------------------------------------------------------------------------------------
// consistency

void launch_consistency(const uint32_t* fwd, const uint32_t* bwd, const uint32_t* bwd2, int w, int h, int eps,
                        uint8_t* mask, cudaStream_t st);  // bwd2 may be null
// The consistency checks of many pairs in one launch (a batch): one entry per pair, pix_base ascending.
struct ConsProblem {
    const uint32_t* fwd;
    const uint32_t* bwd;
    const uint32_t* bwd2;  // or null
    int w, h;
    uint8_t* mask;
    int64_t pix_base;      // first pixel of this pair in the launch
};
void launch_consistency_tab(const ConsProblem* probs_dev, int n, int64_t total_pix, int eps, cudaStream_t st);
void launch_sparsify(const uint32_t* fwd, const uint32_t* bwd, const uint8_t* keep, int w, int h, int eps, int s,
                     uint8_t* out, cudaStream_t st);

// ---------------------------------------------------------------------------------------------------------
// read-only views of context and pyramid internals for other translation units of the library

struct PyrView {
    int w, h, L;
    int ws[kMaxLevels], hs[kMaxLevels];
    const int16_t* feat[kMaxLevels];
    const uint32_t* cen[kMaxLevels];  // null unless the context matches with the Census cost
    const int8_t* seed_desc;
    const int32_t* seed_norm;
    int n_coarse;
};
struct CtxView {
    int device, n_sms;
    cudaStream_t stream;
    int n_scales, iters, rs_radius, eps;
    uint32_t seed;
    int cost;
    void* noalloc_scratch;  // device address of ff_match_pair_noalloc's scratch array on this device
    int sub_scales;
    uint32_t wait_limit;    // FF_OPT_WAIT_LIMIT
    int withhold;           // FF_OPT_TEST_WITHHOLD_COPIES
    int* err_word;          // device error word of the bounded waits (null until ctx_err_word)
};
struct TileChoice {
    int tw, th, k, threads, spec;
    int dataflow;  // 1: the dataflow form (k = iters: one launch per pass), 2: its affine variant; 0: tile form
};

// ---------------------------------------------------------------------------------------------------------
// shared device helpers (library only)

// Coefficient value of a stored feature (the maps hold offset binary: C ^ 0x8000).
__host__ __device__ __forceinline__ int feature_coef(int16_t stored) {
    return (int)(int16_t)((uint16_t)stored ^ 0x8000u);
}

// Position of pixel (x, y) in a colour-split feature map of width w.
__host__ __device__ __forceinline__ int feat_index(int x, int y, int w) {
    return y * w + ((x & 1) ? ((w + 1) >> 1) + (x >> 1) : (x >> 1));
}

__host__ __device__ __forceinline__ uint32_t mix32(uint32_t x) {
    // lowbias32 integer finaliser (C. Wellons, hash-prospector)
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// ---------------------------------------------------------------------------------------------------------
// mbarrier helpers (shared memory of the executing CTA; waits are CTA-scope acquires)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: true when the phase completed, false after `limit` polls; after the first `spin` polls each
// further poll is preceded by a 256 ns sleep (so the default limit of 2^22 polls is about a second).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit, uint32_t spin = 64) {
    for (uint32_t i = 0; i < limit; i++) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > spin) __nanosleep(256);
    }
    return false;
}

// ---------------------------------------------------------------------------------------------------------
// Programmatic dependent launch: every kernel of the library is launched with programmatic stream serialization,
// so the next kernel's CTAs are launched while the last CTAs of the previous one finish, and starts with
// grid_dependency_sync(), which waits until the previous grid has completed and its memory is visible (hence
// also every grid before it) before anything it produced is read; it then lets its own dependent launch.
#ifndef FF_PDL
#define FF_PDL 1
#endif

__device__ __forceinline__ void grid_dependency_sync() {
#if FF_PDL
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

// Debug-bounds build (compiled with -DFF_DEBUG_BOUNDS=1; a stand-in for a memory checker): the feature,
// propagation, hand-over and filter kernels check their gather, store and shared-memory indices before the access;
// the first violation (code, index, limit) is recorded in its translation unit's record, the access is skipped
// (a load reads zeros) and nothing traps.  ff_sync reports a recorded violation as FF_ERR_CUDA and clears it.
// Release builds compile every check away.
#ifndef FF_DEBUG_BOUNDS
#define FF_DEBUG_BOUNDS 0
#endif

__device__ __forceinline__ bool idx_ok(int* rec, int code, long long idx, long long lim) {
#if FF_DEBUG_BOUNDS
    if (idx >= 0 && idx < lim) return true;
    if (atomicCAS(rec, 0, code) == 0) {
        rec[1] = (int)idx;
        rec[2] = (int)lim;
    }
    return false;
#else
    (void)rec, (void)code, (void)idx, (void)lim;
    return true;
#endif
}

// Bytes of dynamic shared memory the running launch was given (read only by debug-bounds checks).
__device__ __forceinline__ unsigned dyn_smem_bytes() {
    unsigned n;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(n));
    return n;
}

// Take (read and clear) the bounds record of propagate.cu / filter.cu; rec[0] == 0: no violation.
cudaError_t bounds_take_propagate(int rec[3]);
cudaError_t bounds_take_filter(int rec[3]);
cudaError_t bounds_take_features(int rec[3]);

template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = FF_PDL;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace ff

// Accessors implemented in ff_api.cu (ff_ctx and ff_pyr are opaque outside it).
struct ff_ctx;
struct ff_pyr;
namespace ff {
bool ctx_view(const ff_ctx* c, CtxView* out);
bool ctx_owns_live_pyr(const ff_ctx* c, const ff_pyr* p);
bool pyr_view(const ff_pyr* p, PyrView* out);
// the launch configuration of a pass (level s, or its sub-scale grid s + 8k) of size w x h for the server and the
// no-allocation entry point, which launch the tile form and (dataflow_ok) the dataflow form, never the cluster form
TileChoice ctx_level_choice(const ff_ctx* c, int level, int w, int h, int n_dirs, int64_t level_pix_all,
                            bool dataflow_ok);
// the context's error word of the bounded device waits, allocated on first use (null if that fails)
int* ctx_err_word(ff_ctx* c);
// cudaMalloc on behalf of a context; fails as out of memory while the context's FF_OPT_TEST_FAIL_ALLOCS count lasts
cudaError_t ctx_malloc(ff_ctx* c, void** p, size_t bytes);
int ctx_set_error(ff_ctx* c, int status, const char* msg);
}  // namespace ff
