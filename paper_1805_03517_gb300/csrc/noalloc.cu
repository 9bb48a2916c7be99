// noalloc.cu -- ff_match_pair_noalloc: one matching direction, like ff_match_pair, without allocating memory.
//
// Some callers must not allocate device memory while they run: code inside a real-time frame loop (cudaMalloc
// and cudaFree can synchronise the whole device and stall other streams), code whose device memory is owned by
// a fixed-size pool of another framework, and code on a hot path that must not fail with out-of-memory part way
// through.  For them this entry point keeps every piece of scratch the matching needs (per-level flow and cost
// ping-pong buffers, seed distances, problem tables, tile queues and their counters) in one file-scope device
// array of fixed size.  The array is part of this library's code on each device that loads it and stays
// resident until the process exits.
#include <cuda_runtime.h>

#include <algorithm>

#include "ff.h"
#include "ff_internal.h"

using namespace ff;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FF_NOALLOC_SCRATCH_BYTES];

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// The descriptors a level is matched with (WHT features, or Census patterns under the Census cost).
const void* cost_desc(const PyrView& v, int level, int cost) {
    return cost == FF_COST_CENSUS ? static_cast<const void*>(v.cen[level]) : static_cast<const void*>(v.feat[level]);
}

// Everything the device-side set-up writes into the scratch array, passed by value.
struct SetupArgs {
    int L, T;
    SeedProblem seed;
    SeedProblem* seed_dst;
    HandoverProblem ho[kMaxLevels];
    HandoverProblem* ho_dst;
    PropProblem base[kMaxLevels];  // per level: all fields except buffers, t0 and n_iter
    int k[kMaxLevels];             // iterations per launch
    int n_launch[kMaxLevels];
    int first_launch[kMaxLevels];
    uint32_t* flow[kMaxLevels][2];
    int32_t* cost[kMaxLevels][2];
    uint32_t* out_flow;
    int32_t* out_cost;
    PropProblem* props;
    int total_launches;
    int2* queue[kMaxLevels];
    int ntiles[kMaxLevels];
};

__global__ void k_noalloc_setup(SetupArgs a) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    if (tid == 0) *a.seed_dst = a.seed;
    for (int s = tid; s < a.L; s += nth) a.ho_dst[s] = a.ho[s];
    for (int i = tid; i < a.total_launches; i += nth) {
        int s = 0;
        while (!(i >= a.first_launch[s] && i < a.first_launch[s] + a.n_launch[s])) s++;
        const int j = i - a.first_launch[s];
        PropProblem p = a.base[s];
        p.t0 = j * a.k[s];
        p.n_iter = min(a.k[s], a.T - p.t0);
        const int in = j & 1, out = in ^ 1;  // the hand-over fills buffer 0
        p.flow_in = a.flow[s][in];
        p.cost_in = a.cost[s][in];
        if (s == 0 && j == a.n_launch[s] - 1) {
            p.flow_out = a.out_flow;
            p.cost_out = a.out_cost ? a.out_cost : a.cost[s][out];
        } else {
            p.flow_out = a.flow[s][out];
            p.cost_out = a.cost[s][out];
        }
        a.props[i] = p;
    }
    for (int s = 0; s < a.L; s++)
        for (int q = tid; q < a.ntiles[s]; q += nth) a.queue[s][q] = make_int2(0, q);
}

}  // namespace

namespace ff {

// Set-up on the current device, run once per context by ff_create.  With lazy module loading (the default) this
// file's module -- and with it the scratch array -- is loaded on a device only when something of it is first
// used there, and each kernel's code on its first use; doing both here keeps ff_match_pair_noalloc from loading
// code or reserving memory.  In host code the array's name is only a host-side stand-in: kernels are given the
// device address cudaGetSymbolAddress returns.
cudaError_t noalloc_prepare(void** scratch) {
    *scratch = nullptr;
    cudaError_t e = cudaGetSymbolAddress(scratch, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, k_noalloc_setup);
    if (e != cudaSuccess) return e;
    return seed_load_kernel();  // k_handover and k_propagate are loaded by init_kernel_attributes
}

}  // namespace ff

extern "C" ff_status ff_match_pair_noalloc(ff_ctx* c, const ff_pyr* a, const ff_pyr* b, int dir, int16_t* flow_dev,
                                           int32_t* cost_dev) {
    CtxView cv;
    if (!ctx_view(c, &cv)) return FF_ERR_ARG;
    auto err = [&](ff_status s, const char* m) { return (ff_status)ctx_set_error(c, s, m); };
    if (!ctx_owns_live_pyr(c, a) || !ctx_owns_live_pyr(c, b))
        return err(FF_ERR_ARG, "pyramids must be live pyramids of this context");
    PyrView A, B;
    pyr_view(a, &A);
    pyr_view(b, &B);
    if (A.w != B.w || A.h != B.h) return err(FF_ERR_ARG, "pyramids differ in size");
    if (dir != 0 && dir != 1) return err(FF_ERR_ARG, "dir must be 0 or 1");
    if (!flow_dev || ((uintptr_t)flow_dev & 3) || ((uintptr_t)cost_dev & 3))
        return err(FF_ERR_ARG, "flow_dev / cost_dev must be 4-byte aligned device pointers");
    if (cv.sub_scales != 0) return err(FF_ERR_ARG, "ff_match_pair_noalloc does not run sub-scale grids");
    if (cudaSetDevice(cv.device) != cudaSuccess) return err(FF_ERR_CUDA, "cudaSetDevice failed");
    void* base = cv.noalloc_scratch;  // looked up by ff_create on this device
    if (!base) return err(FF_ERR_CUDA, "the scratch array of ff_match_pair_noalloc was not set up");

    const int L = A.L, T = cv.iters;
    SetupArgs sa{};
    sa.L = L;
    sa.T = T;
    TileChoice tc[kMaxLevels];
    int grid[kMaxLevels];
    int total_launches = 0;
    for (int s = L - 1; s >= 0; s--) {
        tc[s] = ctx_level_choice(c, s, A.ws[s], A.hs[s], 1, (int64_t)A.ws[s] * A.hs[s], false);
        sa.k[s] = tc[s].k;
        sa.n_launch[s] = (T + tc[s].k - 1) / tc[s].k;
        sa.first_launch[s] = total_launches;
        total_launches += sa.n_launch[s];
        int tiles_x = (A.ws[s] + tc[s].tw - 1) / tc[s].tw;
        sa.ntiles[s] = tiles_x * ((A.hs[s] + tc[s].th - 1) / tc[s].th);
        size_t smem = prop_smem_bytes(tc[s].tw, tc[s].th, tc[s].k);
        grid[s] = std::min(sa.ntiles[s], prop_blocks_per_sm(smem, tc[s].threads, tc[s].spec != 0, cv.cost) * cv.n_sms);
        PropProblem& p = sa.base[s];
        p.fa = cost_desc(A, s, cv.cost);
        p.fb = cost_desc(B, s, cv.cost);
        p.w = A.ws[s];
        p.h = A.hs[s];
        p.tiles_x = tiles_x;
        p.level = s;
        p.dir = dir;
        p.seed = cv.seed;
        p.rs_radius = cv.rs_radius;
    }
    sa.total_launches = total_launches;

    // carve the scratch array; reject what does not fit
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return static_cast<char*>(base) + o;
    };
    sa.seed_dst = reinterpret_cast<SeedProblem*>(take(sizeof(SeedProblem)));
    sa.ho_dst = reinterpret_cast<HandoverProblem*>(take(sizeof(HandoverProblem) * L));
    sa.props = reinterpret_cast<PropProblem*>(take(sizeof(PropProblem) * total_launches));
    int* counters = reinterpret_cast<int*>(take(sizeof(int) * total_launches));
    for (int s = 0; s < L; s++) sa.queue[s] = reinterpret_cast<int2*>(take(sizeof(int2) * sa.ntiles[s]));
    int32_t* dist = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * A.n_coarse));
    for (int s = 0; s < L; s++) {
        size_t n = (size_t)A.ws[s] * A.hs[s];
        for (int k = 0; k < 2; k++) {
            sa.flow[s][k] = reinterpret_cast<uint32_t*>(take(n * 4));
            sa.cost[s][k] = reinterpret_cast<int32_t*>(take(n * 4));
        }
    }
    if (off > (size_t)FF_NOALLOC_SCRATCH_BYTES)
        return err(FF_ERR_ARG, "pyramids too large for the fixed scratch of ff_match_pair_noalloc");

    SeedProblem& sp = sa.seed;
    sp.A = A.seed_desc;
    sp.B = B.seed_desc;
    sp.normA = A.seed_norm;
    sp.normB = B.seed_norm;
    sp.n = A.n_coarse;
    sp.w = A.ws[L - 1];
    sp.flow = sa.flow[L - 1][0];
    sp.dist = dist;
    sp.warp_base = 0;
    for (int s = L - 1; s >= 0; s--) {
        HandoverProblem& hp = sa.ho[s];
        hp.fa = cost_desc(A, s, cv.cost);
        hp.fb = cost_desc(B, s, cv.cost);
        hp.w = A.ws[s];
        hp.h = A.hs[s];
        if (s == L - 1) {
            hp.parent = nullptr;
            hp.flow_in = sa.flow[s][0];
        } else {
            hp.parent = sa.flow[s + 1][sa.n_launch[s + 1] & 1];  // where level s+1's last launch wrote
            hp.pw = A.ws[s + 1];
            hp.ph = A.hs[s + 1];
        }
        hp.flow_out = sa.flow[s][0];
        hp.cost_out = sa.cost[s][0];
        hp.pix_base = 0;
    }
    sa.out_flow = reinterpret_cast<uint32_t*>(flow_dev);
    sa.out_cost = cost_dev;

    // every call shares the array: clear the queue counters, then rewrite tables and queues
    cudaStream_t st = cv.stream;
    if (cudaMemsetAsync(counters, 0, sizeof(int) * total_launches, st) != cudaSuccess)
        return err(FF_ERR_CUDA, "cudaMemsetAsync failed");
    k_noalloc_setup<<<64, 256, 0, st>>>(sa);
    launch_seed(sa.seed_dst, 1, (A.n_coarse + 15) / 16, st);
    for (int s = L - 1; s >= 0; s--) {
        launch_handover(sa.ho_dst + s, 1, (int64_t)A.ws[s] * A.hs[s], cv.cost, st);
        for (int j = 0; j < sa.n_launch[s]; j++) {
            const int li = sa.first_launch[s] + j;
            PropLaunch pl{tc[s].tw, tc[s].th, std::min(tc[s].k, T - j * tc[s].k), tc[s].threads, tc[s].spec, cv.cost};
            launch_propagate(sa.props + li, sa.queue[s], sa.ntiles[s], counters + li, grid[s], pl, st);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return err(FF_ERR_CUDA, cudaGetErrorString(e));
    return FF_OK;
}
