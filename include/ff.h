/*
 * ff.h -- C-ABI of the GB300 (sm_103a) Flow Fields dense-matching library (libff.so).
 *
 * The library computes the matching stage of FlowFields++ (Schuster, Bailer, Wasenmueller, Stricker,
 * arXiv 1805.03517), Sec. 3.1 "Matches": for a pair of RGB frames it builds an image pyramid and per-level
 * Walsh-Hadamard patch descriptors, finds initial matches at the coarsest level, refines them level by level
 * with propagation towards the four quadrants plus random search, computes the inverse flow field and rejects
 * matches whose forward/backward consistency error exceeds eps (Table 3 gives eps).  Interpolation (Sec. 3.2)
 * and variational refinement (Sec. 3.3) are not part of this library.
 *
 * Conventions shared by every call:
 *   - All arithmetic is integer and the result of every call is deterministic, independent of batching,
 *     tiling and launch order.
 *   - Image     uint8 [h][w][3] (RGB), rows `pitch_bytes` apart (pitch_bytes >= 3*w).
 *   - Flow      int16 [h][w][2] row-major, (dx, dy) in whole pixels; pixel (x, y) of the source frame
 *               matches pixel (x+dx, y+dy) of the target frame.  4-byte aligned.
 *   - Cost      int32 [h][w]: the matching cost of the match (ff_params.cost): by default the sum of absolute
 *               differences of the 48 int16 descriptor coefficients.
 *   - Mask      uint8 [h][w]: 1 = the match passed the consistency check, 0 = rejected.
 *   - Pointers marked "device" must point to memory of the context's device; the caller owns them.
 *     Calls only enqueue work on the context's stream and return; a device buffer handed in must stay
 *     valid until that work has run (ff_sync waits for it).
 *   - Sizes: 1 <= w, h <= 8192; n_scales 1..8 (every level is at least 1x1); the coarsest level has at most
 *     2^20 pixels (the initial matching is exhaustive, its work grows with the square of that count).  A
 *     violation returns FF_ERR_ARG and launches nothing.
 *   - Errors: every call returns an ff_status; ff_last_error() gives a message for the last failure.  A
 *     CUDA failure (including one from earlier asynchronous work) returns FF_ERR_CUDA.
 *   - A context is not thread-safe: use one context per host thread (or serialise calls).
 */
#ifndef FF_H
#define FF_H

#include <stdint.h>

#if defined(__GNUC__)
#define FF_API __attribute__((visibility("default")))
#else
#define FF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ff_ctx ff_ctx; /* matching context: device, stream, parameters, scratch and plan caches */
typedef struct ff_pyr ff_pyr; /* one frame's feature pyramid, owned by the context that made it */

typedef enum {
    FF_OK = 0,
    FF_ERR_ARG = 1,     /* invalid argument (nothing was launched) */
    FF_ERR_OOM = 2,     /* device or host allocation failed */
    FF_ERR_CUDA = 3,    /* a CUDA call failed, or earlier asynchronous work failed */
    FF_ERR_TIMEOUT = 4, /* a bounded device-side wait gave up */
    FF_ERR_BUSY = 5     /* resource in use (e.g. a pyramid released while a plan still refers to it) */
} ff_status;

/* Matching parameters (Sec. 3.1; eps from Table 3).
 *   n_scales  pyramid levels L (1..8); level 0 is full resolution, each level halves the previous one.
 *   iters     propagation iterations per level (1..255); the paper uses 12.
 *   patch     patch size; must be 8.
 *   n_coef    Walsh-Hadamard coefficients per channel; must be 16 (the 4x4 lowest sequencies).
 *   rs_radius random-search radius R (0..16): each random candidate moves both flow components by an
 *             integer in [-R, R].
 *   eps       consistency threshold in pixels (>= 0); a match is kept iff |f(p) + b(p + f(p))| <= eps.
 *   seed      seed of the counter-based random-search hash. */
typedef struct {
    int n_scales;
    int iters;
    int patch;
    int n_coef;
    int rs_radius;
    int eps;
    uint32_t seed;
    int rs_radius2;  /* random-search radius (0..16) of the second inverse field of the two-check mode (Sec. 3.1
                        computes the two inverse fields with differing matching settings); it also runs on its own
                        random stream */
    int cost;        /* matching cost of propagation and random search: FF_COST_WHT_SAD (default) or
                        FF_COST_CENSUS (see below); the coarsest-level initial matches use the WHT descriptors
                        either way */
    int sub_scales;  /* 0 (default), 1 or 2.  Sec. 3.1 matches on "sub-scales and sub-sub-scales" as in Flow
                        Fields+, which it does not restate; this library's reading: every level below the
                        coarsest is first matched on the grid of every 2^n-th pixel of the level (n = sub_scales),
                        then of every 2^(n-1)-th, ..., then on every pixel.  A grid pixel (u, v) is level pixel
                        (g*u, g*v) with the level's own descriptors; flows are in level pixels and may point to
                        any level pixel; each grid runs the level's whole propagation schedule (neighbours one grid
                        step apart) on its own random stream.  The first grid takes the usual hand-over from the
                        level above; each later grid takes its parent grid pixel's flow with the target clamped
                        into the level.  Supported by ff_match_pair, ff_match_batch, ff_autotune and the server;
                        ff_match_pair_noalloc rejects it (FF_ERR_ARG). */
} ff_params;

/* Matching costs (Sec. 3.1 matches with a Census cost or SIFT descriptors; Sec. 4.1 takes Census for Sintel).
 *   FF_COST_WHT_SAD  sum of absolute differences of the 48 int16 WHT coefficients (cost range 0..3*16*2*2040).
 *   FF_COST_CENSUS   Hamming distance of the 7x7 Census patterns of the three colour channels (0..144): bit k
 *                    of channel c is 1 iff the k-th neighbour of the 7x7 window -- row-major over rows y-3..y+3
 *                    and columns x-3..x+3, centre skipped, edge pixels repeated -- is strictly darker than the
 *                    centre.  RGB stands in for CIELab (integer and exact). */
enum { FF_COST_WHT_SAD = 0, FF_COST_CENSUS = 1 };

/* Default parameters: L=5, iters=6, patch=8, n_coef=16, rs_radius=2, eps=1, seed=0x20180503, rs_radius2=4,
 * cost=FF_COST_WHT_SAD, sub_scales=0. */
FF_API void ff_default_params(ff_params* p);

/* Create a context on CUDA device `device` that enqueues all work on `cuda_stream` (a cudaStream_t; NULL
 * means the legacy default stream).  The parameters are copied.  *out receives the context.  The first context
 * on a device also reserves there the fixed scratch array of ff_match_pair_noalloc (FF_NOALLOC_SCRATCH_BYTES,
 * held until the process exits) and loads the kernels that entry point launches; FF_ERR_OOM if that fails. */
FF_API ff_status ff_create(ff_ctx** out, const ff_params* p, int device, void* cuda_stream);

/* Build the feature pyramid of one frame (Sec. 3 and 3.1): L pyramid levels (2x2 box average, rounded half
 * up, sizes halved rounding down, at least 1), the 48 int16 Walsh-Hadamard coefficients of the 8x8 patch
 * around every pixel of every level (edge pixels repeated), and the packed 8-bit descriptors of the coarsest
 * level used by the initial matching; with FF_COST_CENSUS also the Census patterns of every level.  `rgb_dev`
 * is a device image [h][w][3] with rows pitch_bytes apart.
 * *out receives a pyramid owned by the context; it stays valid until ff_pyr_release or ff_destroy.
 * Released pyramids of the same size are recycled, so steady-state calls allocate nothing. */
FF_API ff_status ff_features(ff_ctx* ctx, const uint8_t* rgb_dev, int w, int h, int pitch_bytes, ff_pyr** out);

/* One frame of ff_features_batch: device image uint8 [h][w][3], rows pitch_bytes apart. */
typedef struct {
    const uint8_t* rgb_dev;
    int w, h, pitch_bytes;
} ff_frame;

/* ff_features for n frames of any sizes in one launch per kernel (Sec. 3 and 3.1, as ff_features): the pyramid
 * levels 1..6 of every frame in one launch and the Walsh-Hadamard descriptors, Census patterns and seed rows of
 * every level of every frame in another (frames with 8 levels add one launch per frame for the last level).
 * out[i] (n entries) receives frame i's pyramid, identical to ff_features on that frame alone.  The launches read
 * a table of the frames that the call copies to a context-owned device buffer on the context's stream (grown,
 * after waiting for the stream, when a larger batch needs it).  The copy is from pageable host memory, so this
 * call cannot be recorded into a CUDA graph (ff_features can).  On an error no pyramid is taken and out[] is
 * all NULL. */
FF_API ff_status ff_features_batch(ff_ctx* ctx, int n, const ff_frame* frames, ff_pyr** out);

/* Match one direction (Sec. 3.1): dir 0 matches frame a to frame b, dir 1 computes the inverse field (the
 * caller passes the pyramids swapped; dir only selects the random-search stream).  Exact nearest-neighbour
 * initial matches at the coarsest level, then per level, coarse to fine: hand-over of twice the parent
 * pixel's flow, `iters` iterations of propagation with random search.  Writes the level-0 flow to flow_dev
 * (device, int16 [h][w][2]) and, if cost_dev is not NULL, the level-0 cost to cost_dev (device, int32
 * [h][w]).  Both pyramids must have the same size. */
FF_API ff_status ff_match_pair(ff_ctx* ctx, const ff_pyr* a, const ff_pyr* b, int dir, int16_t* flow_dev,
                        int32_t* cost_dev);

/* One frame pair of a batch: forward field a -> b, inverse field b -> a and the consistency mask of the
 * forward field.  All outputs are device buffers of the pair's level-0 size; cost_fwd/cost_bwd may be NULL.
 * If flow_bwd2 is not NULL, a second inverse field is computed with the second parameter set (rs_radius2 and its
 * own random stream) into flow_bwd2, and mask keeps a match only if it passes both consistency checks (the two
 * checks of Sec. 3.1). */
typedef struct {
    const ff_pyr* a;
    const ff_pyr* b;
    int16_t* flow_fwd;
    int16_t* flow_bwd;
    int32_t* cost_fwd;
    int32_t* cost_bwd;
    uint8_t* mask;
    int16_t* flow_bwd2;
} ff_pair_job;

/* Match n pairs of possibly different sizes in merged launches: for every job, the forward field, the
 * inverse field and the consistency mask (Sec. 3.1).  Each job's results are identical to matching it alone.
 * The launch sequence of a batch is recorded once into a CUDA graph and replayed when the same jobs (same
 * pyramids and output buffers) are matched again. */
FF_API ff_status ff_match_batch(ff_ctx* ctx, int n, const ff_pair_job* jobs);

/* One frame pair of ff_match_frames: a and b index its frame list; the outputs are those of ff_pair_job. */
typedef struct {
    int a, b;
    int16_t* flow_fwd;
    int16_t* flow_bwd;
    int32_t* cost_fwd;
    int32_t* cost_bwd;
    uint8_t* mask;
    int16_t* flow_bwd2;
} ff_frame_job;

/* ff_features_batch on n_frames frames followed by ff_match_batch on n_jobs pairs of them (Sec. 3 and 3.1), in
 * one call, with results identical to those two calls.  The descriptors of pyramid levels 0 and 1 are needed
 * only once the matching reaches level 1.  So when the context has a stream of its own, is not profiling and
 * matches more than two levels, their launch runs on a branch of the matching's CUDA graph, beside the coarse
 * levels' matching, whose kernels have the higher priority (FF_OPT_OVERLAP); level 1 waits for it.  All work is
 * ordered on the context's stream when the call returns.  If out is not NULL it receives the n_frames
 * pyramids (released by the caller); otherwise they are released at the end of the call and their memory is
 * recycled by later calls.  Argument errors are found before anything is launched; on any error out[] is all
 * NULL and the call keeps no pyramid. */
FF_API ff_status ff_match_frames(ff_ctx* ctx, int n_frames, const ff_frame* frames, int n_jobs,
                                 const ff_frame_job* jobs, ff_pyr** out);

/* Choose, per pyramid level, the propagation tile shape, CTA size and the number of iterations fused into one launch for
 * batches shaped like `jobs` (same level sizes and number of pairs): every candidate configuration is run
 * `reps` (1..100) times on these jobs and the fastest is kept for each level.  Results never depend on the
 * configuration; the jobs' outputs are overwritten.  Cached plans are dropped so later calls use the choice.
 * This is a property of the GB300 implementation (the paper has no counterpart). */
FF_API ff_status ff_autotune(ff_ctx* ctx, int n, const ff_pair_job* jobs, int reps);

/* Propagation launch configuration of one level: tile interior (pixels), iterations fused per launch, threads
 * per CTA (128, 256 or 512), and whether the random candidate is fetched together with the neighbour candidates
 * (speculate = 1; refetched when a neighbour was taken).  With cluster = dataflow = 0 this is the tile form, one
 * launch per iters_per_launch iterations.
 * dataflow = 1 (cluster 0, iters_per_launch 1, speculate 0, tiles at least 4x4): every iteration of the level in
 * one persistent launch of one-iteration tile tasks, a tile starting iteration t as soon as the 3x3 tiles around
 * it have finished t - 1 (no launch boundary, hence no idle tail, between iterations); dataflow = 2 is its affine
 * variant, each CTA keeping the same tiles for every iteration (no shared queue; their descriptors stay in that
 * SM's L1).
 * cluster = n (1..16) selects the cluster form: one thread-block cluster of n CTAs per direction of each pair
 * covers the whole level without a halo, CTAs exchanging their block edges through distributed shared memory
 * (threads 256 or 512, tile_w = tile_h = 0, speculate = 0); a plan falls back to the default tile form for a
 * level the cluster form cannot take (a level narrower or lower than the partition, blocks beyond shared memory,
 * or clusters this device cannot schedule).
 * The server (ff_server_*) and ff_match_pair_noalloc launch the tile form only (a dataflow configuration's tiles,
 * one iteration per launch).  None of these changes any result. */
typedef struct {
    int tile_w, tile_h, iters_per_launch, threads, speculate, cluster, dataflow;
} ff_tuning;

/* Impose the configuration of one pass on every later plan of this context, overriding the autotuner; NULL
 * removes the override.  `level` is a pass index: 0..7 a pyramid level, s + 8k (k = 1, 2) the sub-scale grid of
 * stride 2^k of level s (FF_N_PASSES in all).  FF_ERR_ARG if the tile with its halo does not fit in shared
 * memory or a field is out of range.  Cached plans are dropped. */
FF_API ff_status ff_set_tuning(ff_ctx* ctx, int level, const ff_tuning* cfg);

/* The configuration in force for pass `level`: the override if set, else the autotuner's choice; FF_ERR_ARG if
 * neither exists. */
FF_API ff_status ff_get_tuning(ff_ctx* ctx, int level, ff_tuning* out);

/* Forward/backward consistency check (Sec. 3.1, eps as in Table 3): mask[p] = 1 iff q = p + fwd(p) lies in
 * the image and (fwd_x(p) + bwd_x(q))^2 + (fwd_y(p) + bwd_y(q))^2 <= eps^2.  All pointers are device
 * buffers of size w x h. */
FF_API ff_status ff_consistency(ff_ctx* ctx, const int16_t* fwd, const int16_t* bwd, int w, int h, int eps,
                         uint8_t* mask_dev);

/* Sparsification of the consistent matches (Sec. 3.1; s in Table 3: 7 for KITTI, 4 for Sintel): the image is
 * tiled by 3x3 blocks from (0, 0) (blocks at the right and bottom edges may be smaller); in every block with at
 * least `min_matches` (1..9) matches that pass the consistency check with `eps` -- and, when `keep_dev` is not
 * NULL, are set in that mask (the paper sparsifies what both consistency checks left: pass the `mask` of an
 * ff_pair_job matched with a second inverse field) -- only the match with the lowest squared consistency error
 * against `bwd` is kept (the first in row-major order on ties).  sparse_dev[p] = 1 for kept matches, 0
 * elsewhere.  fwd/bwd: device int16 [h][w][2] flows (4-byte aligned); keep_dev: device uint8 [h][w] or NULL;
 * sparse_dev: device uint8 [h][w], written.  Asynchronous on the context's stream; FF_ERR_ARG (nothing
 * launched) for null or misaligned flow pointers, sizes outside 1..8192, eps outside 0..32767 or min_matches
 * outside 1..9. */
FF_API ff_status ff_sparsify(ff_ctx* ctx, const int16_t* fwd, const int16_t* bwd, const uint8_t* keep_dev, int w,
                             int h, int eps, int min_matches, uint8_t* sparse_dev);

/* Return a pyramid to the context's pool (its memory is reused by a later ff_features of the same size). */
FF_API ff_status ff_pyr_release(ff_ctx* ctx, ff_pyr* pyr);

/* Sizes of level `level` of a pyramid; FF_ERR_ARG if the level does not exist. */
FF_API ff_status ff_pyr_level_dims(const ff_pyr* pyr, int level, int* w, int* h);

/* Device pointer to the 48 features per pixel of `level` (read-only view owned by the pyramid), 16 bits each in
 * offset binary: the stored uint16 is the coefficient + 32768 (the int16 coefficient XOR 0x8000).  Rows are
 * stored colour-split: row y holds the descriptors of x = 0, 2, 4, ... followed by those of x = 1, 3, 5, ...,
 * i.e. pixel (x, y) is descriptor y*w + (x even ? x/2 : (w+1)/2 + x/2). */
FF_API const int16_t* ff_pyr_features(const ff_pyr* pyr, int level);

/* Device pointer to the Census patterns of `level` (read-only view owned by the pyramid), or NULL when the
 * pyramid's context does not match with FF_COST_CENSUS.  32 bytes per pixel, as 8 uint32 words: words 2c and
 * 2c+1 are the low and high halves of channel c's 48-bit pattern (bit k as for FF_COST_CENSUS), words 6 and 7
 * are zero.  Same colour-split pixel order as ff_pyr_features. */
FF_API const uint32_t* ff_pyr_census(const ff_pyr* pyr, int level);

/* Message of the last failure on this context ("" if none).  Valid until the next call on the context. */
FF_API const char* ff_last_error(ff_ctx* ctx);

/* Wait for all work enqueued by this context; reports failures of asynchronous work as FF_ERR_CUDA. */
FF_API ff_status ff_sync(ff_ctx* ctx);

/* Counters of the most recent ff_match_pair / ff_match_batch / ff_features calls. */
typedef struct {
    int64_t kernel_launches;   /* kernels enqueued by this context since creation (graph nodes counted) */
    int64_t graph_replays;     /* CUDA-graph launches since creation */
    int64_t plans_built;       /* distinct match plans built (each may be captured into a graph) */
    int64_t scratch_bytes;     /* device bytes currently held for plans, pyramids and staging */
    int64_t cluster_launches;  /* of kernel_launches: propagation launches of the cluster form (ff_tuning) */
} ff_stats;
FF_API ff_status ff_get_stats(ff_ctx* ctx, ff_stats* out);

/* Per-phase device time.  When enabled, the context brackets each phase of the matching calls with CUDA
 * events (and does not use graphs); ff_profile_read waits for the work and returns, per phase, the summed
 * duration in milliseconds and the number of kernel launches since the last read.  Phases: */
enum { FF_PHASE_FEATURES = 0, FF_PHASE_SEED = 1, FF_PHASE_HANDOVER = 2, FF_PHASE_PROPAGATE = 3,
       FF_PHASE_CONSISTENCY = 4, FF_N_PHASES = 5 };
FF_API ff_status ff_profile_enable(ff_ctx* ctx, int on);
FF_API ff_status ff_profile_read(ff_ctx* ctx, double* ms /* [FF_N_PHASES] */, int64_t* launches /* [FF_N_PHASES] */);
/* The propagation phase split by pass (the same events, read and cleared the same way; use instead of
 * ff_profile_read): entry s is level s, entry s + 8k its sub-scale grid of stride 2^k (k = 1, 2).  ms and launches
 * have FF_N_PASSES entries. */
#define FF_N_PASSES 24
FF_API ff_status ff_profile_read_passes(ff_ctx* ctx, double* ms /* [FF_N_PASSES] */, int64_t* launches /* [FF_N_PASSES] */);

/* Algorithmic work of a plan for pyramids of size w x h with the context's parameters: per direction, the
 * number of (pixel, iteration) updates summed over all levels and sub-scale grids, and the number of level-0
 * pixels. */
FF_API ff_status ff_work_counts(ff_ctx* ctx, int w, int h, int64_t* pixel_iters, int64_t* pixels);

/* ---- continuous-batching server ------------------------------------------------------------------------
 * One request = one frame pair (Sec. 3.1): forward field, inverse field, consistency mask.  Requests are
 * admitted first come first served while at most `max_active` are in flight and the device bytes of the
 * admitted requests (two feature pyramids + flow/cost scratch each) stay within `mem_budget_bytes`.  Each
 * ff_server_step enqueues one tick on the context's stream: every active request advances by one propagation
 * launch of its current level (by all of the level's launches while at most 8 requests are in flight), with the
 * work of all active requests merged into one launch per kernel kind and launch configuration;
 * requests that arrive while others are on the GPU join at the next tick.  A request's results are identical
 * to matching it alone (ff_match_batch), whatever else is in flight.  Not thread-safe per server. */
typedef struct ff_server ff_server;

/* Inputs and outputs of one request; all device buffers owned by the caller and valid until the request has
 * been reported by ff_server_poll.  Frames uint8 [h][w][3] (rows pitch_bytes apart); flows int16 [h][w][2];
 * mask uint8 [h][w]; cost_fwd/cost_bwd int32 [h][w] or NULL. */
typedef struct {
    const uint8_t* rgb_a;
    const uint8_t* rgb_b;
    int w, h, pitch_bytes;
    int16_t* flow_fwd;
    int16_t* flow_bwd;
    int32_t* cost_fwd;
    int32_t* cost_bwd;
    uint8_t* mask;
} ff_request;

FF_API ff_status ff_server_create(ff_ctx* ctx, int64_t mem_budget_bytes, int max_active, ff_server** out);
/* Queue a request under the caller's id; FF_ERR_ARG if it could never fit the memory budget. */
FF_API ff_status ff_server_submit(ff_server* srv, uint64_t id, const ff_request* req);
/* Admit what fits and enqueue one tick; reports the requests in flight and still queued. */
FF_API ff_status ff_server_step(ff_server* srv, int* n_active, int* n_queued);
/* Ids (up to max_ids) of requests whose outputs are complete; with wait != 0 blocks until at least one is. */
FF_API ff_status ff_server_poll(ff_server* srv, int wait, uint64_t* ids, int max_ids, int* n_done);
/* Withdraw a request that is still queued (not yet admitted): FF_OK, and its id is never reported by
 * ff_server_poll; nothing of it was on the device, so its buffers are the caller's again at once.  FF_ERR_BUSY if
 * the request has been admitted (it completes normally and is reported by poll); FF_ERR_ARG for an unknown id. */
FF_API ff_status ff_server_cancel(ff_server* srv, uint64_t id);
/* Ticks enqueued, kernel launches enqueued, and device bytes of the admitted requests. */
FF_API ff_status ff_server_stats(ff_server* srv, int64_t* ticks, int64_t* launches, int64_t* bytes_in_use);
/* Wait for the stream, release every resource of the server (not the context). */
FF_API ff_status ff_server_destroy(ff_server* srv);

/* Size of the fixed device scratch array used by ff_match_pair_noalloc (32 MiB): enough for frames of up to
 * about 1.5 million pixels at level 0. */
#define FF_NOALLOC_SCRATCH_BYTES (32u << 20)

/* ff_match_pair without any memory allocation.  The paper has no counterpart: this serves callers that must
 * not allocate device memory while they run -- a real-time frame loop (cudaMalloc/cudaFree may synchronise the
 * device and stall other streams), code whose device memory belongs to another framework's fixed pool, or a
 * hot path that must not hit out-of-memory half way.  Same arguments and results as ff_match_pair (the caller
 * still passes the pyramids, built beforehand by ff_features, and the outputs).  All scratch lives in one
 * file-scope device array of FF_NOALLOC_SCRATCH_BYTES; pyramids needing more than that return FF_ERR_ARG.
 * The array is reserved on a device, and its address looked up, when the first context is created there
 * (ff_create loads this entry point's module and kernels, which lazy module loading would otherwise do on its
 * first call); it stays reserved until the process exits.  So a call allocates nothing and loads no code.  A
 * context, and these calls, must not outlive a reset of its device.  Every call reuses the same array, which
 * keeps the last call's contents (the call clears what must start at zero); calls whose work overlaps on the
 * GPU -- on different streams or contexts of the same device -- race on the array and must be serialised by
 * the caller.  The initial matches always come from the mma.sync kernel (FF_OPT_SEED_KERNEL is not consulted;
 * both kernels give identical results). */
FF_API ff_status ff_match_pair_noalloc(ff_ctx* ctx, const ff_pyr* a, const ff_pyr* b, int dir, int16_t* flow_dev,
                                       int32_t* cost_dev);

/* Context options (ff_set_option).  Changing one drops the cached plans.
 *   FF_OPT_SEED_KERNEL           which kernel computes the initial matches: FF_SEED_TCGEN05 (default; tcgen05
 *                                tensor cores, TMA-fed) or FF_SEED_MMA_SYNC (warp-level mma.sync); identical
 *                                results.
 *   FF_OPT_WAIT_LIMIT            polls (1..2^30, default 2^22, about a second) before a device-side wait gives
 *                                up; the kernel then records the failure, cleans up and returns, and the next
 *                                ff_sync reports FF_ERR_TIMEOUT with the context still usable.
 *   FF_OPT_TEST_WITHHOLD_COPIES  1: the tensor-core seed issues no copies and the cluster form of the propagation
 *                                sends no block edges, so their waits can only expire (a test of the bounded
 *                                waits); 0 (default) normal operation.
 *   FF_OPT_TEST_FAIL_ALLOCS      n >= 0: the next n device allocations made for this context (pyramids, plans, the
 *                                server's scratch and tables) fail as on an exhausted device, without calling the
 *                                allocator, so the calls that need them return FF_ERR_OOM and launch nothing (a test
 *                                of the out-of-memory paths); 0 (default) normal operation.  Unlike the other
 *                                options it keeps the cached plans.
 *   FF_OPT_OVERLAP               where the branch of ff_match_frames that writes the fine levels' descriptors
 *                                starts: 0, nowhere (they are written before the matching, on the context's
 *                                stream); 1, at the start of the matching; 2 (default), at the coarsest level's
 *                                first propagation launch.  Results never depend on it; it keeps the cached
 *                                plans. */
enum {
    FF_OPT_SEED_KERNEL = 1,
    FF_OPT_WAIT_LIMIT = 2,
    FF_OPT_TEST_WITHHOLD_COPIES = 3,
    FF_OPT_TEST_FAIL_ALLOCS = 4,
    FF_OPT_OVERLAP = 5
};
enum { FF_SEED_MMA_SYNC = 0, FF_SEED_TCGEN05 = 1 };
FF_API ff_status ff_set_option(ff_ctx* ctx, int option, int64_t value);

/* Release every resource of the context (pyramids, plans, graphs); ctx must not be used afterwards. */
FF_API ff_status ff_destroy(ff_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* FF_H */
