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
};
void launch_pyramid(const PyrArgs& a, cudaStream_t st);
// kernels ff_features launches for an L-level pyramid: the fused pyramid (+ one per level past kPyrFusedTop), WHT
inline int features_launches(int L) {
    return (L > 1 ? 1 + (L - 1 > kPyrFusedTop ? L - 1 - kPyrFusedTop : 0) : 0) + 1;
}
int wht_tiles_x(int w);
int wht_tiles(int w, int h);
void launch_wht(const WhtArgs& a, int total_tiles, cudaStream_t st);

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

struct HandoverProblem {
    const void* fa;          // cost descriptors of the source frame (WHT features or Census patterns)
    const void* fb;          // and of the target frame
    int w, h;
    const uint32_t* parent;  // flow of the level above (pw x ph), or null: take flow_in as is
    int pw, ph;
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
    const uint32_t* flow_in;
    const int32_t* cost_in;
    uint32_t* flow_out;
    int32_t* cost_out;
    int w, h;
    int tiles_x;
    int t0;          // first iteration index (for the random-search hash)
    int n_iter;      // iterations fused into this launch
    int level;
    int dir;
    uint32_t seed;
    int rs_radius;
};
struct PropLaunch {
    int tw, th;      // tile interior
    int max_iter;    // largest n_iter of the launch (sizes the shared-memory halo)
    int threads;     // CTA size: 128, 256 or 512
    int spec;        // 1: load the random candidate together with the neighbour candidates
    int cost;        // FF_COST_WHT_SAD or FF_COST_CENSUS
};
constexpr size_t kMaxPropSmem = 200 * 1024;
size_t prop_smem_bytes(int tw, int th, int n_iter);
cudaError_t init_kernel_attributes();  // once per device, before the first launch (also loads k_handover)
cudaError_t seed_load_kernel();        // loads k_seed onto the current device (lazy module loading)
// Set-up of ff_match_pair_noalloc on the current device, run by ff_create: loads its module (which reserves the
// fixed scratch array) and the kernels it launches, and returns the array's device address.
cudaError_t noalloc_prepare(void** scratch);
bool prop_threads_ok(int threads);
int prop_blocks_per_sm(size_t smem, int threads, bool spec, int cost);  // resident CTAs per SM of the kernel
// queue_dev[i] = (problem index, tile index); counter_dev must be zero when the launch starts
void launch_propagate(const PropProblem* probs_dev, const int2* queue_dev, int n_tiles, int* counter_dev, int grid,
                      const PropLaunch& L, cudaStream_t st);

// ---------------------------------------------------------------------------------------------------------
// consistency

void launch_consistency(const uint32_t* fwd, const uint32_t* bwd, const uint32_t* bwd2, int w, int h, int eps,
                        uint8_t* mask, cudaStream_t st);  // bwd2 may be null
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
};
struct TileChoice {
    int tw, th, k, threads, spec;
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
TileChoice ctx_level_choice(const ff_ctx* c, int level, int w, int h, int n_dirs, int64_t level_pix_all);
int ctx_set_error(ff_ctx* c, int status, const char* msg);
}  // namespace ff
