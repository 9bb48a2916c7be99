// server.cu -- continuous-batching server for the Flow Fields matching stage (FlowFields++, arXiv 1805.03517,
// Sec. 3.1, one request = one frame pair: forward field, inverse field, consistency mask).
//
// Requests are queued by ff_server_submit and admitted, first come first served, while the number of active
// requests stays below max_active and the device bytes of admitted requests (their two feature pyramids and
// their flow/cost scratch) stay within the memory budget.  Every ff_server_step enqueues one tick: each active
// request advances by one propagation launch-chunk of its current level (by all remaining chunks of the level
// while at most 8 requests are in flight, which cuts the ticks, and their overhead, on a request's latency at
// light load); a request's first tick also builds its pyramids, finds its initial matches and does the first
// hand-over, the first chunk of every level carries that level's hand-over, and the last chunk of level 0 is
// followed by the consistency check.  Work of all active requests of a tick is merged into one launch per
// kernel kind (propagation: one per launch configuration and chunk position, the configurations running
// concurrently on side streams), so requests that arrive while others are on the GPU join the next tick.  A pass
// whose configuration is of the dataflow form is one chunk (all its iterations in one launch); the cluster form
// is not used here.  A bounded wait of a dataflow launch that expires is reported by the context's next ff_sync.
// Results depend only on the request (the random-search hash is keyed by pixel, level, iteration and
// direction), never on the mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <tuple>
#include <vector>

#include "ff.h"
#include "ff_internal.h"

using namespace ff;

namespace {

constexpr int kRing = 4;         // ticks in flight before the host waits
constexpr int kSideStreams = 3;  // extra streams for the concurrent propagation launches of a tick
constexpr int kWholeLevelMaxActive = 8;  // up to this many requests in flight, a tick runs a whole level
constexpr int kLoadedDirs = 64;          // directions per launch the configurations under load are looked up for

size_t a256(size_t v) { return (v + 255) / 256 * 256; }

struct Req {
    uint64_t id = 0;
    ff_request io{};
    ff_pyr* pa = nullptr;
    ff_pyr* pb = nullptr;
    PyrView A{}, B{};
    int L = 0, T = 0;
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    int64_t footprint = 0;
    // per direction, level and grid (k = 0: the level; k = 1, 2: its sub-scale grids of stride 2^k), ping-pong
    uint32_t* flow[2][kMaxLevels][3][2] = {};
    int32_t* cost[2][kMaxLevels][3][2] = {};
    int32_t* dist[2] = {};
    TileChoice cfg[kMaxLevels][3] = {};
    int n_chunks[kMaxLevels][3] = {};
    int level = 0, grid = 0, chunk = 0, cur[2] = {0, 0};  // the pass in progress: (level, grid), its next chunk
    bool started = false;
    int64_t done_tick = -1;
    bool counted = false;  // footprint added to the server's bytes in use
};

struct RingSlot {
    char* host = nullptr;   // pinned
    char* dev = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
    int64_t tick = -1;
};

int64_t pyr_bytes(int w, int h, int L, bool census) {
    int64_t b = 0;
    int ws = w, hs = h;
    for (int s = 0; s < L; s++) {
        if (s > 0) b += (int64_t)ws * hs * 3;
        b += (int64_t)ws * hs * (kDescBytes + (census ? kCensusBytes : 0));
        if (s + 1 < L) {
            ws = std::max(1, ws / 2);
            hs = std::max(1, hs / 2);
        }
    }
    return b + (int64_t)ws * hs * (kSeedK + 4) + 4096;
}

// The descriptors a level is matched with (WHT features, or Census patterns under the Census cost).
const void* cost_desc(const PyrView& v, int level, int cost) {
    return cost == FF_COST_CENSUS ? static_cast<const void*>(v.cen[level]) : static_cast<const void*>(v.feat[level]);
}

int grid_dim(int v, int k) { return (v + (1 << k) - 1) >> k; }
// sub-scale grids of level s of an L-level pyramid (the coarsest level has none)
int grids_of(int s, int L, int sub_scales) { return s == L - 1 ? 0 : sub_scales; }

size_t scratch_need(int w, int h, int L, int sub_scales) {
    size_t b = 0;
    int ws = w, hs = h;
    for (int s = 0; s < L; s++) {
        for (int k = 0; k <= grids_of(s, L, sub_scales); k++)
            b += 2 * 4 * a256((size_t)grid_dim(ws, k) * grid_dim(hs, k) * 4);
        if (s + 1 < L) {
            ws = std::max(1, ws / 2);
            hs = std::max(1, hs / 2);
        }
    }
    return b + 2 * a256((size_t)ws * hs * 4);
}

}  // namespace

struct ff_server {
    ff_ctx* ctx = nullptr;
    CtxView cv{};
    int64_t budget = 0, in_use = 0;
    int max_active = 0;
    std::deque<std::unique_ptr<Req>> queued;
    std::vector<std::unique_ptr<Req>> active;
    std::vector<std::unique_ptr<Req>> finishing;  // all launches enqueued, waiting for their tick
    std::multimap<size_t, void*> free_scratch;    // recycled scratch blocks by size
    RingSlot ring[kRing];
    int64_t tick = 0;
    int64_t launches = 0;
    // side streams on which the propagation launches of one tick run concurrently (fork/join with events)
    cudaStream_t side[kSideStreams] = {};
    cudaEvent_t fork = nullptr, join[kSideStreams] = {};
};

namespace {

ff_status srv_fail(ff_server* s, ff_status st, const char* msg) { return (ff_status)ctx_set_error(s->ctx, st, msg); }

ff_status ensure_side_streams(ff_server* s) {
    if (s->fork) return FF_OK;
    for (int k = 0; k < kSideStreams; k++)
        if (cudaStreamCreateWithFlags(&s->side[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s->join[k], cudaEventDisableTiming) != cudaSuccess)
            return srv_fail(s, FF_ERR_CUDA, "side stream creation failed");
    if (cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming) != cudaSuccess)
        return srv_fail(s, FF_ERR_CUDA, "event creation failed");
    return FF_OK;
}

ff_status ring_reserve(ff_server* s, RingSlot& r, size_t bytes) {
    if (r.done) {
        if (cudaEventSynchronize(r.done) != cudaSuccess) return srv_fail(s, FF_ERR_CUDA, "tick event failed");
    }
    if (bytes <= r.cap) return FF_OK;
    if (r.host) cudaFreeHost(r.host);
    if (r.dev) cudaFree(r.dev);
    r.host = nullptr;
    r.dev = nullptr;
    size_t cap = std::max(bytes, (size_t)1 << 20) * 2;
    if (cudaMallocHost(&r.host, cap) != cudaSuccess ||
        ctx_malloc(s->ctx, reinterpret_cast<void**>(&r.dev), cap) != cudaSuccess) {
        cudaGetLastError();
        return srv_fail(s, FF_ERR_OOM, "tick table allocation failed");
    }
    r.cap = cap;
    return FF_OK;
}

// Scratch of a request: per direction and level two flow and two cost buffers, plus seed distances.
ff_status take_scratch(ff_server* s, Req& q) {
    size_t need = scratch_need(q.A.w, q.A.h, q.L, s->cv.sub_scales);
    auto it = s->free_scratch.find(need);
    void* p = nullptr;
    if (it != s->free_scratch.end()) {
        p = it->second;
        s->free_scratch.erase(it);
    } else if (ctx_malloc(s->ctx, &p, need) != cudaSuccess) {
        cudaGetLastError();
        return srv_fail(s, FF_ERR_OOM, "scratch allocation failed");
    }
    q.scratch = p;
    q.scratch_bytes = need;
    char* b = static_cast<char*>(p);
    size_t off = 0;
    for (int d = 0; d < 2; d++)
        for (int l = 0; l < q.L; l++)
            for (int g = 0; g <= grids_of(l, q.L, s->cv.sub_scales); g++) {
                size_t n = (size_t)grid_dim(q.A.ws[l], g) * grid_dim(q.A.hs[l], g);
                for (int k = 0; k < 2; k++) {
                    q.flow[d][l][g][k] = reinterpret_cast<uint32_t*>(b + off);
                    off += a256(n * 4);
                    q.cost[d][l][g][k] = reinterpret_cast<int32_t*>(b + off);
                    off += a256(n * 4);
                }
            }
    for (int d = 0; d < 2; d++) {
        q.dist[d] = reinterpret_cast<int32_t*>(b + off);
        off += a256((size_t)q.A.n_coarse * 4);
    }
    return FF_OK;
}

void release_req(ff_server* s, Req& q) {
    if (q.pa) ff_pyr_release(s->ctx, q.pa);
    if (q.pb) ff_pyr_release(s->ctx, q.pb);
    q.pa = q.pb = nullptr;
    if (q.scratch) s->free_scratch.emplace(q.scratch_bytes, q.scratch);
    q.scratch = nullptr;
    if (q.counted) s->in_use -= q.footprint;
    q.counted = false;
}

// Admission: the queued requests that fit (first come first served, while slots and the memory budget allow) have
// the features of all their frames built in one ff_features_batch call, then their scratch and launch
// configurations set up in order.  If the features fail nothing is taken and the requests stay queued; if a later
// step fails, that request and the ones after it stay queued (their pyramids are given back).
ff_status admit(ff_server* s) {
    size_t n_new = 0;
    int64_t in_use = s->in_use;
    bool idle = s->active.empty() && s->finishing.empty();
    for (auto& qp : s->queued) {
        if ((int)(s->active.size() + n_new) >= s->max_active) break;
        if (in_use + qp->footprint > s->budget && !idle) break;  // wait for memory
        in_use += qp->footprint;
        idle = false;
        n_new++;
    }
    if (n_new == 0) return FF_OK;
    std::vector<ff_frame> frames;
    for (size_t i = 0; i < n_new; i++) {
        const ff_request& io = s->queued[i]->io;
        frames.push_back({io.rgb_a, io.w, io.h, io.pitch_bytes});
        frames.push_back({io.rgb_b, io.w, io.h, io.pitch_bytes});
    }
    std::vector<ff_pyr*> pyrs(frames.size(), nullptr);
    ff_status st = ff_features_batch(s->ctx, (int)frames.size(), frames.data(), pyrs.data());
    if (st != FF_OK) return st;
    const int L = s->cv.n_scales;
    const int deep = L - 1 > kPyrFusedTop ? L - 1 - kPyrFusedTop : 0;
    s->launches += (L > 1 ? 1 : 0) + 1 + (int64_t)frames.size() * deep;  // the feature launches just enqueued
    for (size_t i = 0; i < n_new; i++) {
        s->queued[i]->pa = pyrs[2 * i];
        s->queued[i]->pb = pyrs[2 * i + 1];
    }
    size_t admitted = 0;
    for (; admitted < n_new && st == FF_OK; admitted++) {
        Req& q = *s->queued[admitted];
        pyr_view(q.pa, &q.A);
        pyr_view(q.pb, &q.B);
        q.L = q.A.L;
        q.T = s->cv.iters;
        st = take_scratch(s, q);
        if (st != FF_OK) break;
        s->in_use += q.footprint;
        q.counted = true;
        // launch configurations tuned for one pair at light load, for launches shared by many pairs under load
        const int n_dirs = (int)(s->active.size() + admitted) + 1 > kWholeLevelMaxActive ? kLoadedDirs : 2;
        for (int l = 0; l < q.L && st == FF_OK; l++)
            for (int g = 0; g <= grids_of(l, q.L, s->cv.sub_scales); g++) {  // tuning entries: pass l + 8g
                const int gw = grid_dim(q.A.ws[l], g), gh = grid_dim(q.A.hs[l], g);
                q.cfg[l][g] =
                    ctx_level_choice(s->ctx, l + kMaxLevels * g, gw, gh, n_dirs, (int64_t)n_dirs * gw * gh, true);
                const TileChoice& t = q.cfg[l][g];
                if (t.k < 1 || t.tw < 1 || t.th < 1 || !prop_threads_ok(t.threads) ||
                    prop_smem_bytes(t.tw, t.th, t.dataflow ? 1 : t.k) > kMaxPropSmem ||
                    (t.dataflow && (t.tw < 4 || t.th < 4 || t.spec))) {
                    st = srv_fail(s, FF_ERR_CUDA, "invalid launch configuration");
                    break;
                }
                q.n_chunks[l][g] = t.dataflow ? 1 : (q.T + t.k - 1) / t.k;  // dataflow: the pass in one launch
            }
        if (st != FF_OK) break;
        q.level = q.L - 1;
        q.grid = 0;
        q.chunk = 0;
    }
    for (size_t i = admitted; i < n_new; i++) release_req(s, *s->queued[i]);  // stays queued, holds nothing
    for (size_t i = 0; i < admitted; i++) {
        s->active.push_back(std::move(s->queued.front()));
        s->queued.pop_front();
    }
    return st;
}

// Propagation launches of a tick are grouped by phase (the position of a chunk among the chunks one request
// runs in this tick: a request's chunk i + 1 reads what its chunk i wrote) and by launch configuration.
struct PropGroupKey {
    int phase, tw, th, n_iter, threads, spec, grid, dataflow;
    bool operator<(const PropGroupKey& o) const {
        return std::tie(phase, tw, th, n_iter, threads, spec, grid, dataflow) <
               std::tie(o.phase, o.tw, o.th, o.n_iter, o.threads, o.spec, o.grid, o.dataflow);
    }
};

// Build and enqueue one tick for every active request.
ff_status tick(ff_server* s) {
    if (s->active.empty()) return FF_OK;
    const int T = s->cv.iters;
    std::vector<SeedProblem> seeds;
    std::vector<HandoverProblem> hos;
    std::map<PropGroupKey, std::vector<std::pair<PropProblem, int>>> groups;  // (problem, tiles)
    struct Cons {
        const uint32_t* f;
        const uint32_t* b;
        int w, h;
        uint8_t* mask;
    };
    std::vector<Cons> cons;
    int seed_tiles = 0;
    int64_t ho_pix = 0;
    std::vector<size_t> finished;
    // With few requests in flight a tick runs every remaining chunk of each request's level (fewer ticks, so
    // less per-tick overhead on a request's latency); under load one chunk, so that arrivals join sooner.
    const bool whole_level = (int)s->active.size() <= kWholeLevelMaxActive;
    for (size_t ri = 0; ri < s->active.size(); ri++) {
        Req& q = *s->active[ri];
        const int sl = q.level, L = q.L;
        if (!q.started) {  // exact initial matches of both directions at the coarsest level
            for (int d = 0; d < 2; d++) {
                const PyrView& X = d == 0 ? q.A : q.B;
                const PyrView& Y = d == 0 ? q.B : q.A;
                SeedProblem sp{};
                sp.A = X.seed_desc;
                sp.B = Y.seed_desc;
                sp.normA = X.seed_norm;
                sp.normB = Y.seed_norm;
                sp.n = X.n_coarse;
                sp.w = X.ws[L - 1];
                sp.flow = q.flow[d][L - 1][0][0];
                sp.dist = q.dist[d];
                sp.warp_base = seed_tiles;
                seed_tiles += (sp.n + 15) / 16;
                seeds.push_back(sp);
            }
            q.started = true;
        }
        const int gk = q.grid, k_first = grids_of(sl, L, s->cv.sub_scales);
        if (q.chunk == 0) {  // hand-over into this level or grid (the seed's cost at the coarsest level)
            for (int d = 0; d < 2; d++) {
                const PyrView& X = d == 0 ? q.A : q.B;
                const PyrView& Y = d == 0 ? q.B : q.A;
                HandoverProblem hp{};
                hp.fa = cost_desc(X, sl, s->cv.cost);
                hp.fb = cost_desc(Y, sl, s->cv.cost);
                hp.w = grid_dim(X.ws[sl], gk);
                hp.h = grid_dim(X.hs[sl], gk);
                hp.g = 1 << gk;
                hp.lw = X.ws[sl];
                hp.lh = X.hs[sl];
                if (sl == L - 1) {
                    hp.parent = nullptr;
                    hp.flow_in = q.flow[d][sl][0][0];
                } else if (gk == k_first) {  // from the level above
                    hp.parent = q.flow[d][sl + 1][0][q.cur[d]];
                    hp.pw = X.ws[sl + 1];
                    hp.ph = X.hs[sl + 1];
                } else {  // from the sparser grid of this level
                    hp.parent = q.flow[d][sl][gk + 1][q.cur[d]];
                    hp.pw = grid_dim(X.ws[sl], gk + 1);
                    hp.ph = grid_dim(X.hs[sl], gk + 1);
                    hp.same_level = 1;
                }
                hp.flow_out = q.flow[d][sl][gk][0];
                hp.cost_out = q.cost[d][sl][gk][0];
                hp.pix_base = ho_pix;
                ho_pix += (int64_t)hp.w * hp.h;
                hos.push_back(hp);
                q.cur[d] = 0;
            }
        }
        const TileChoice c = q.cfg[sl][gk];
        const int n_run = whole_level ? q.n_chunks[sl][gk] - q.chunk : 1;
        for (int phase = 0; phase < n_run; phase++) {
            const int chunk = q.chunk + phase;
            const int t0 = chunk * c.k, n_iter = std::min(c.k, T - t0);
            const bool last = sl == 0 && gk == 0 && chunk == q.n_chunks[sl][gk] - 1;
            auto& grp = groups[PropGroupKey{phase, c.tw, c.th, n_iter, c.threads, c.spec, gk > 0 ? 1 : 0, c.dataflow}];
            for (int d = 0; d < 2; d++) {
                const PyrView& X = d == 0 ? q.A : q.B;
                const PyrView& Y = d == 0 ? q.B : q.A;
                PropProblem pp{};
                pp.fa = cost_desc(X, sl, s->cv.cost);
                pp.fb = cost_desc(Y, sl, s->cv.cost);
                pp.w = grid_dim(X.ws[sl], gk);
                pp.h = grid_dim(X.hs[sl], gk);
                pp.g = 1 << gk;
                pp.lw = X.ws[sl];
                pp.lh = X.hs[sl];
                int in = q.cur[d], out = in ^ 1;
                pp.flow_in = q.flow[d][sl][gk][in];
                pp.cost_in = q.cost[d][sl][gk][in];
                if (c.dataflow) {  // iterations alternate: even ones write buffer `out`, odd ones `in`
                    pp.flow_alt = q.flow[d][sl][gk][out];
                    pp.cost_alt = q.cost[d][sl][gk][out];
                    out = (T - 1) % 2 == 0 ? out : in;  // where the last iteration lands, apart from its source
                }
                int32_t* user_cost = d == 0 ? q.io.cost_fwd : q.io.cost_bwd;
                if (last) {
                    pp.flow_out = reinterpret_cast<uint32_t*>(d == 0 ? q.io.flow_fwd : q.io.flow_bwd);
                    pp.cost_out = user_cost ? user_cost : q.cost[d][sl][gk][out];
                } else {
                    pp.flow_out = q.flow[d][sl][gk][out];
                    pp.cost_out = q.cost[d][sl][gk][out];
                }
                q.cur[d] = out;
                pp.tiles_x = (pp.w + c.tw - 1) / c.tw;
                pp.t0 = t0;
                pp.n_iter = c.dataflow ? 1 : n_iter;
                pp.level = sl + kMaxLevels * gk;  // the hash stream of this level or grid
                pp.dir = d;
                pp.seed = s->cv.seed;
                pp.rs_radius = s->cv.rs_radius;
                grp.push_back({pp, pp.tiles_x * ((pp.h + c.th - 1) / c.th)});
            }
        }
        q.chunk += n_run;
        if (q.chunk == q.n_chunks[sl][gk] && gk > 0) {  // on to the next finer grid of this level
            q.grid--;
            q.chunk = 0;
        } else if (q.chunk == q.n_chunks[sl][gk]) {
            if (sl == 0) {
                cons.push_back({reinterpret_cast<const uint32_t*>(q.io.flow_fwd),
                                reinterpret_cast<const uint32_t*>(q.io.flow_bwd), q.A.w, q.A.h, q.io.mask});
                finished.push_back(ri);
            } else {
                q.level--;
                q.grid = grids_of(q.level, L, s->cv.sub_scales);
                q.chunk = 0;
            }
        }
    }

    // tables of this tick: seeds | handovers | propagation problems | queues | counters
    size_t n_props = 0, n_queue = 0;
    for (auto& kv : groups) {
        n_props += kv.second.size();
        for (auto& pr : kv.second) n_queue += pr.second;
    }
    const size_t o_seed = 0, o_ho = a256(seeds.size() * sizeof(SeedProblem));
    const size_t o_prop = o_ho + a256(hos.size() * sizeof(HandoverProblem));
    const size_t o_q = o_prop + a256(n_props * sizeof(PropProblem));
    // counters: one queue counter per launch, then the tiles' progress counters of the dataflow launches
    size_t n_progress = 0;
    for (auto& kv : groups)
        if (kv.first.dataflow)
            for (auto& pr : kv.second) n_progress += pr.second;
    const size_t o_cnt = o_q + a256(n_queue * sizeof(int2));
    const size_t bytes = o_cnt + a256((groups.size() + n_progress) * sizeof(int) + 4);
    RingSlot& r = s->ring[s->tick % kRing];
    ff_status st = ring_reserve(s, r, bytes);
    if (st != FF_OK) return st;
    std::memset(r.host, 0, bytes);
    memcpy(r.host + o_seed, seeds.data(), seeds.size() * sizeof(SeedProblem));
    memcpy(r.host + o_ho, hos.data(), hos.size() * sizeof(HandoverProblem));
    PropProblem* hp = reinterpret_cast<PropProblem*>(r.host + o_prop);
    int2* hq = reinterpret_cast<int2*>(r.host + o_q);
    struct PL {
        PropLaunch pl;
        size_t q0;
        int nq, grid, phase;
    };
    std::vector<PL> pls;
    size_t pi = 0, qi = 0, prog = groups.size();  // next progress counter
    CtxView now;  // the context's current wait limit and error word
    ctx_view(s->ctx, &now);
    for (auto& kv : groups) {
        const PropGroupKey& k = kv.first;
        const size_t q0 = qi;
        // the two directions of each request were pushed next to each other: interleave their tiles
        for (size_t g = 0; g < kv.second.size(); g += 2) {
            const int p0 = (int)(pi + g), n0 = kv.second[g].second;
            const int n1 = g + 1 < kv.second.size() ? kv.second[g + 1].second : 0;
            for (int t = 0; t < std::max(n0, n1); t++) {
                if (t < n0) hq[qi++] = make_int2(p0, t);
                if (t < n1) hq[qi++] = make_int2(p0 + 1, t);
            }
        }
        for (auto& pr : kv.second) {
            hp[pi] = pr.first;
            if (k.dataflow) {
                hp[pi].progress = reinterpret_cast<int*>(r.dev + o_cnt) + prog;
                prog += pr.second;
            }
            pi++;
        }
        const size_t smem = prop_smem_bytes(k.tw, k.th, k.dataflow ? 1 : k.n_iter);
        const int nq = (int)(qi - q0);
        PropLaunch pl{k.tw, k.th, k.dataflow ? 1 : k.n_iter, k.threads, k.spec, s->cv.cost, k.grid};
        const int slots =
            prop_blocks_per_sm(smem, k.threads, k.spec != 0, s->cv.cost, k.grid != 0, k.dataflow != 0) * s->cv.n_sms;
        if (k.dataflow) {
            pl.dataflow = k.n_iter;
            pl.affine = k.dataflow == 2;
            pl.wait_limit = now.wait_limit;
            pl.withhold = now.withhold;
            pl.err = now.err_word;
        }
        const int64_t tasks = (int64_t)nq * (k.dataflow == 1 ? k.n_iter : 1);  // affine: one CTA per tile at most
        pls.push_back({pl, q0, nq, (int)std::min<int64_t>(tasks, slots), k.phase});
    }
    cudaStream_t stm = s->cv.stream;
    if (cudaMemcpyAsync(r.dev, r.host, bytes, cudaMemcpyHostToDevice, stm) != cudaSuccess)
        return srv_fail(s, FF_ERR_CUDA, "tick table upload failed");
    int nl = 0;
    if (!seeds.empty()) {
        launch_seed(reinterpret_cast<const SeedProblem*>(r.dev + o_seed), (int)seeds.size(), seed_tiles, stm);
        nl++;
    }
    if (!hos.empty()) {
        launch_handover(reinterpret_cast<const HandoverProblem*>(r.dev + o_ho), (int)hos.size(), ho_pix, s->cv.cost,
                        stm);
        nl++;
    }
    // Within a phase, propagation launches of different configurations are independent (disjoint problems,
    // queues and counters): the largest runs on the main stream, the others on side streams, so small launches
    // (coarse levels, other frame sizes) fill the SMs that the tail of a large one leaves idle.  Phases run one
    // after the other (the groups map is ordered by phase).
    for (size_t g0 = 0; g0 < pls.size();) {
        size_t g1 = g0;
        while (g1 < pls.size() && pls[g1].phase == pls[g0].phase) g1++;
        std::vector<size_t> order;
        for (size_t g = g0; g < g1; g++) order.push_back(g);
        std::sort(order.begin(), order.end(), [&](size_t a, size_t b) { return pls[a].nq > pls[b].nq; });
        const int n_side = (int)std::min<size_t>(kSideStreams, order.size() - 1);
        if (n_side > 0) {
            st = ensure_side_streams(s);
            if (st != FF_OK) return st;
            if (cudaEventRecord(s->fork, stm) != cudaSuccess) return srv_fail(s, FF_ERR_CUDA, "event record failed");
            for (int k = 0; k < n_side; k++)
                if (cudaStreamWaitEvent(s->side[k], s->fork, 0) != cudaSuccess)
                    return srv_fail(s, FF_ERR_CUDA, "stream wait failed");
        }
        for (size_t i = 0; i < order.size(); i++) {
            const size_t g = order[i];
            cudaStream_t sg = i == 0 ? stm : s->side[(i - 1) % kSideStreams];
            launch_propagate(reinterpret_cast<const PropProblem*>(r.dev + o_prop),
                             reinterpret_cast<const int2*>(r.dev + o_q) + pls[g].q0, pls[g].nq,
                             reinterpret_cast<int*>(r.dev + o_cnt) + g, pls[g].grid, pls[g].pl, sg);
            nl++;
        }
        for (int k = 0; k < n_side; k++) {
            if (cudaEventRecord(s->join[k], s->side[k]) != cudaSuccess ||
                cudaStreamWaitEvent(stm, s->join[k], 0) != cudaSuccess)
                return srv_fail(s, FF_ERR_CUDA, "stream join failed");
        }
        g0 = g1;
    }
    for (const Cons& cs : cons) {
        launch_consistency(cs.f, cs.b, nullptr, cs.w, cs.h, s->cv.eps, cs.mask, stm);
        nl++;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return srv_fail(s, FF_ERR_CUDA, cudaGetErrorString(e));
    if (!r.done && cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming) != cudaSuccess)
        return srv_fail(s, FF_ERR_CUDA, "event creation failed");
    if (cudaEventRecord(r.done, stm) != cudaSuccess) return srv_fail(s, FF_ERR_CUDA, "event record failed");
    r.tick = s->tick;
    s->launches += nl;
    // requests whose last launches are in this tick wait for it
    for (size_t k = finished.size(); k-- > 0;) {
        size_t ri = finished[k];
        s->active[ri]->done_tick = s->tick;
        s->finishing.push_back(std::move(s->active[ri]));
        s->active.erase(s->active.begin() + ri);
    }
    s->tick++;
    return FF_OK;
}

}  // namespace

extern "C" {

ff_status ff_server_create(ff_ctx* ctx, int64_t mem_budget_bytes, int max_active, ff_server** out) {
    if (!out) return FF_ERR_ARG;
    *out = nullptr;
    CtxView cv;
    if (!ctx_view(ctx, &cv)) return FF_ERR_ARG;
    if (mem_budget_bytes <= 0 || max_active < 1 || max_active > 4096)
        return (ff_status)ctx_set_error(ctx, FF_ERR_ARG, "bad memory budget or max_active");
    if (cudaSetDevice(cv.device) != cudaSuccess || !ctx_err_word(ctx))  // for the waits of dataflow launches
        return (ff_status)ctx_set_error(ctx, FF_ERR_OOM, "no device memory for the error word");
    ff_server* s = new (std::nothrow) ff_server();
    if (!s) return FF_ERR_OOM;
    s->ctx = ctx;
    s->cv = cv;
    s->budget = mem_budget_bytes;
    s->max_active = max_active;
    *out = s;
    return FF_OK;
}

ff_status ff_server_submit(ff_server* s, uint64_t id, const ff_request* req) {
    if (!s) return FF_ERR_ARG;
    if (!req || !req->rgb_a || !req->rgb_b || !req->flow_fwd || !req->flow_bwd || !req->mask)
        return srv_fail(s, FF_ERR_ARG, "request has a NULL buffer");
    if (req->w < 1 || req->h < 1 || req->w > 8192 || req->h > 8192 || req->pitch_bytes < 3 * req->w)
        return srv_fail(s, FF_ERR_ARG, "request size or pitch out of range");
    if (((uintptr_t)req->flow_fwd & 3) || ((uintptr_t)req->flow_bwd & 3) || ((uintptr_t)req->cost_fwd & 3) ||
        ((uintptr_t)req->cost_bwd & 3))
        return srv_fail(s, FF_ERR_ARG, "request outputs must be 4-byte aligned");
    {  // the same limit ff_features applies: at most 2^20 pixels at the coarsest level
        int cw = req->w, ch = req->h;
        for (int l = 1; l < s->cv.n_scales; l++) {
            cw = std::max(1, cw / 2);
            ch = std::max(1, ch / 2);
        }
        if ((int64_t)cw * ch > (1 << 20))
            return srv_fail(s, FF_ERR_ARG, "coarsest level too large for the exhaustive initial matching");
    }
    auto q = std::make_unique<Req>();
    q->id = id;
    q->io = *req;
    q->footprint = 2 * pyr_bytes(req->w, req->h, s->cv.n_scales, s->cv.cost == FF_COST_CENSUS) +
                   (int64_t)scratch_need(req->w, req->h, s->cv.n_scales, s->cv.sub_scales);
    if (q->footprint > s->budget) return srv_fail(s, FF_ERR_ARG, "request larger than the memory budget");
    s->queued.push_back(std::move(q));
    return FF_OK;
}

ff_status ff_server_step(ff_server* s, int* n_active, int* n_queued) {
    if (!s) return FF_ERR_ARG;
    if (cudaSetDevice(s->cv.device) != cudaSuccess) return srv_fail(s, FF_ERR_CUDA, "cudaSetDevice failed");
    ff_status st = admit(s);
    if (st == FF_OK) st = tick(s);
    if (n_active) *n_active = (int)(s->active.size() + s->finishing.size());
    if (n_queued) *n_queued = (int)s->queued.size();
    return st;
}

ff_status ff_server_poll(ff_server* s, int wait, uint64_t* ids, int max_ids, int* n_done) {
    if (!s || (max_ids > 0 && !ids)) return FF_ERR_ARG;
    int n = 0;
    auto tick_done = [&](int64_t t) {
        const RingSlot& r = s->ring[t % kRing];
        if (r.tick != t) return true;  // the slot was reused, so that tick has completed
        cudaError_t e = cudaEventQuery(r.done);
        if (e == cudaErrorNotReady) return false;
        return true;
    };
    for (int pass = 0; pass < 2; pass++) {
        for (size_t i = 0; i < s->finishing.size() && n < max_ids;) {
            Req& q = *s->finishing[i];
            if (tick_done(q.done_tick)) {
                ids[n++] = q.id;
                release_req(s, q);
                s->finishing.erase(s->finishing.begin() + i);
            } else {
                i++;
            }
        }
        if (n > 0 || !wait || s->finishing.empty()) break;
        int64_t first = s->finishing.front()->done_tick;
        for (auto& q : s->finishing) first = std::min(first, q->done_tick);
        const RingSlot& r = s->ring[first % kRing];
        if (r.tick == first && cudaEventSynchronize(r.done) != cudaSuccess)
            return srv_fail(s, FF_ERR_CUDA, "tick event failed");
    }
    cudaError_t e = cudaGetLastError();
    if (n_done) *n_done = n;
    if (e != cudaSuccess && e != cudaErrorNotReady) return srv_fail(s, FF_ERR_CUDA, cudaGetErrorString(e));
    return FF_OK;
}

ff_status ff_server_cancel(ff_server* s, uint64_t id) {
    if (!s) return FF_ERR_ARG;
    for (auto it = s->queued.begin(); it != s->queued.end(); ++it)
        if ((*it)->id == id) {  // nothing of a queued request is on the device yet
            s->queued.erase(it);
            return FF_OK;
        }
    for (auto* list : {&s->active, &s->finishing})
        for (auto& q : *list)
            if (q->id == id) return srv_fail(s, FF_ERR_BUSY, "request already admitted: it completes normally");
    return srv_fail(s, FF_ERR_ARG, "no such request");
}

ff_status ff_server_stats(ff_server* s, int64_t* ticks, int64_t* launches, int64_t* bytes_in_use) {
    if (!s) return FF_ERR_ARG;
    if (ticks) *ticks = s->tick;
    if (launches) *launches = s->launches;
    if (bytes_in_use) *bytes_in_use = s->in_use;
    return FF_OK;
}

ff_status ff_server_destroy(ff_server* s) {
    if (!s) return FF_ERR_ARG;
    cudaSetDevice(s->cv.device);
    cudaStreamSynchronize(s->cv.stream);
    for (auto& q : s->active) release_req(s, *q);
    for (auto& q : s->finishing) release_req(s, *q);
    for (auto& kv : s->free_scratch) cudaFree(kv.second);
    for (RingSlot& r : s->ring) {
        if (r.host) cudaFreeHost(r.host);
        if (r.dev) cudaFree(r.dev);
        if (r.done) cudaEventDestroy(r.done);
    }
    for (int k = 0; k < kSideStreams; k++) {
        if (s->side[k]) {
            cudaStreamSynchronize(s->side[k]);
            cudaStreamDestroy(s->side[k]);
        }
        if (s->join[k]) cudaEventDestroy(s->join[k]);
    }
    if (s->fork) cudaEventDestroy(s->fork);
    delete s;
    return FF_OK;
}

}  // extern "C"
