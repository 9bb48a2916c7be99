// propagate.cu -- per-level refinement of the matches (FlowFields++, arXiv 1805.03517, Sec. 3.1): coarse-to-fine
// hand-over and propagation towards the four quadrants with random search.
//
// Schedule of one iteration t at one level (the same schedule the oracle runs): for each quadrant direction
// d = 0..3 (neighbours left+top, right+top, left+bottom, right+bottom), two half-sweeps over the pixels with
// (x + y) even, then odd.  A pixel of the active colour tries neighbour 1 (horizontal), neighbour 2 (vertical)
// and, for d >= 1, its current flow plus a hashed random offset in [-R, R]^2 (skipped if zero); a candidate
// is taken iff its cost (WHT SAD or Census Hamming distance) is strictly lower; targets outside the level are
// rejected.  Neighbours always have the other colour, so every half-sweep is a fully parallel map.
//
// Temporal blocking: one CTA owns a tile of a level and runs n_iter whole iterations (8 half-sweeps each) in
// shared memory before writing the tile back, reading the level state from one buffer and writing another.
// It loads the tile plus a halo of 4 * n_iter pixels and, before half-sweep j, recomputes every pixel whose
// value the remaining half-sweeps need: the region grows backwards from the tile by one pixel on the two
// upstream sides of each later half-sweep.  Recomputed halo pixels use exactly the inputs of the CTA that owns
// them, so every tile's output equals the global schedule bit for bit.
#include <climits>

#include "ff_internal.h"

namespace ff {

// first index violation of a debug-bounds build (see idx_ok): code, index, limit
static __device__ int g_bounds[4];

cudaError_t bounds_take_propagate(int rec[3]) {
    int h[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyFromSymbol(h, g_bounds, sizeof h);
    if (e == cudaSuccess && h[0] != 0) {
        const int z[4] = {0, 0, 0, 0};
        e = cudaMemcpyToSymbol(g_bounds, z, sizeof z);
    }
    rec[0] = h[0], rec[1] = h[1], rec[2] = h[2];
    return e;
}

// Bounds codes of this file's checks.
enum : int { kBoundsOwn = 1, kBoundsCand1, kBoundsCand2, kBoundsRandom, kBoundsSpec, kBoundsSmemOwn, kBoundsSmemN1,
             kBoundsSmemN2, kBoundsTileRead, kBoundsTileSmem, kBoundsTileWrite, kBoundsParent, kBoundsHandoverDesc,
             kBoundsBlockRead, kBoundsBlockSmem, kBoundsBlockWrite, kBoundsRingN1, kBoundsRingN2 };

__device__ __forceinline__ int flow_x(uint32_t f) { return (int)(int16_t)(f & 0xffffu); }
__device__ __forceinline__ int flow_y(uint32_t f) { return ((int)f) >> 16; }
__device__ __forceinline__ uint32_t pack_flow(int dx, int dy) { return (uint32_t)(dx & 0xffff) | ((uint32_t)dy << 16); }
__device__ __forceinline__ bool in_level(int x, int y, int w, int h) {
    return (unsigned)x < (unsigned)w && (unsigned)y < (unsigned)h;
}

// One pixel descriptor (96 B = three 32-B sectors) with three 256-bit read-only loads, one sector per load.
__device__ __forceinline__ void load_desc(const void* __restrict__ f, int idx, uint32_t (&d)[24]) {
    const char* p = reinterpret_cast<const char*>(f) + (size_t)idx * kDescBytes;
#pragma unroll
    for (int k = 0; k < 3; k++)
        asm("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
            : "=r"(d[8 * k]), "=r"(d[8 * k + 1]), "=r"(d[8 * k + 2]), "=r"(d[8 * k + 3]), "=r"(d[8 * k + 4]),
              "=r"(d[8 * k + 5]), "=r"(d[8 * k + 6]), "=r"(d[8 * k + 7])
            : "l"(p + 32 * k));
}

// Exact SAD of the 48 coefficients, two per 32-bit word.  The feature maps store every coefficient in offset
// binary (C ^ 0x8000, i.e. C + 32768 as uint16, which preserves order), so per half max - min is |a - b| in
// [0, 32640] and a plain 32-bit subtraction of the packed max/min never borrows across halves.  Two packed
// differences add without carrying (2 * 32640 < 65536); __dp2a_lo then adds both 16-bit halves into the int32
// sum.
__device__ __forceinline__ int sad_words(const uint32_t (&a)[24], const uint32_t (&b)[24]) {
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < 24; k += 2) {
        uint32_t d0 = __vmaxu2(a[k], b[k]) - __vminu2(a[k], b[k]);
        uint32_t d1 = __vmaxu2(a[k + 1], b[k + 1]) - __vminu2(a[k + 1], b[k + 1]);
        s = __dp2a_lo(d0 + d1, 0x0101u, s);
    }
    return (int)s;
}

// The two matching costs (Sec. 3.1), as policies of the hand-over and propagation kernels: descriptor size in
// 32-bit words, load of one pixel's descriptor, one-time preparation of the source pixel's descriptor, distance.
struct CostSad {  // SAD of the 48 WHT coefficients (stored in offset binary)
    static constexpr int kWords = 24;
    __device__ __forceinline__ static void load(const void* __restrict__ f, int idx, uint32_t (&d)[kWords]) {
        load_desc(f, idx, d);
    }
    __device__ __forceinline__ static void prep(uint32_t (&)[kWords]) {}
    __device__ __forceinline__ static int dist(const uint32_t (&a)[kWords], const uint32_t (&b)[kWords]) {
        return sad_words(a, b);
    }
};

struct CostCensus {  // Hamming distance of the three 48-bit Census patterns (one 32-B sector per pixel)
    static constexpr int kWords = 8;
    __device__ __forceinline__ static void load(const void* __restrict__ f, int idx, uint32_t (&d)[kWords]) {
        const char* p = reinterpret_cast<const char*>(f) + (size_t)idx * kCensusBytes;
        asm("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
            : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7])
            : "l"(p));
    }
    __device__ __forceinline__ static void prep(uint32_t (&)[kWords]) {}
    __device__ __forceinline__ static int dist(const uint32_t (&a)[kWords], const uint32_t (&b)[kWords]) {
        int s = 0;
#pragma unroll
        for (int k = 0; k < 6; k++) s += __popc(a[k] ^ b[k]);  // words 6 and 7 are zero
        return s;
    }
};

// A descriptor load that a debug-bounds build checks against the map's n descriptors (zeros if outside).
template <class C>
__device__ __forceinline__ void load_chk(const void* __restrict__ f, int idx, int n, int code, uint32_t (&d)[C::kWords]) {
    if (idx_ok(g_bounds, code, idx, n)) {
        C::load(f, idx, d);
    } else {
#pragma unroll
        for (int k = 0; k < C::kWords; k++) d[k] = 0;
    }
}

// Cost of the descriptor at (x, y) of fa against (tx, ty) of fb (both inside the w x h level).
template <class C>
__device__ __forceinline__ int cost_at(const void* __restrict__ fa, const void* __restrict__ fb, int w, int h, int x,
                                       int y, int tx, int ty) {
    uint32_t a[C::kWords], b[C::kWords];
    load_chk<C>(fa, feat_index(x, y, w), w * h, kBoundsHandoverDesc, a);
    load_chk<C>(fb, feat_index(tx, ty, w), w * h, kBoundsHandoverDesc, b);
    C::prep(a);
    return C::dist(a, b);
}

// ---------------------------------------------------------------------------------------------------------
// hand-over: flow = 2 x parent flow (parent = (min(x/2, pw-1), min(y/2, ph-1))) or the given flow; cost of it.

template <class C>
__global__ __launch_bounds__(256) void k_handover(const HandoverProblem* __restrict__ probs, int n_probs,
                                                  int64_t total) {
    grid_dependency_sync();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_probs - 1;
        while (lo < hi) {  // last problem with pix_base <= i
            int mid = (lo + hi + 1) >> 1;
            if (probs[mid].pix_base <= i) lo = mid; else hi = mid - 1;
        }
        const HandoverProblem& P = probs[lo];
        int p = (int)(i - P.pix_base);
        const int u = p % P.w, v = p / P.w;
        const bool grid = P.g > 1;
        const int g = grid ? P.g : 1, lw = grid ? P.lw : P.w, lh = grid ? P.lh : P.h;
        const int x = g * u, y = g * v;  // level coordinates
        uint32_t f;
        if (P.parent && P.same_level) {  // from the grid of stride 2g: the same flow, its target clamped
            const int pi = min(v >> 1, P.ph - 1) * P.pw + min(u >> 1, P.pw - 1);
            uint32_t pf = idx_ok(g_bounds, kBoundsParent, pi, P.pw * P.ph) ? P.parent[pi] : 0u;
            f = pack_flow(min(max(x + flow_x(pf), 0), lw - 1) - x, min(max(y + flow_y(pf), 0), lh - 1) - y);
        } else if (P.parent) {  // from the level above: twice the parent pixel's flow
            int px = min(x >> 1, P.pw - 1), py = min(y >> 1, P.ph - 1);
            uint32_t pf = idx_ok(g_bounds, kBoundsParent, py * P.pw + px, P.pw * P.ph) ? P.parent[py * P.pw + px] : 0u;
            f = pack_flow(2 * flow_x(pf), 2 * flow_y(pf));
        } else {
            f = P.flow_in[p];
        }
        int tx = x + flow_x(f), ty = y + flow_y(f);
        int c = INT_MAX;  // unreachable for valid inputs: a handed-over flow always lands inside the level
        if (in_level(tx, ty, lw, lh)) c = cost_at<C>(P.fa, P.fb, lw, lh, x, y, tx, ty);
        P.flow_out[p] = f;
        P.cost_out[p] = c;
    }
}

void launch_handover(const HandoverProblem* probs_dev, int n_probs, int64_t total_pix, int cost, cudaStream_t st) {
    int64_t blocks = (total_pix + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    if (cost == FF_COST_CENSUS)
        launch_k(k_handover<CostCensus>, dim3((int)blocks), dim3(256), 0, st, probs_dev, n_probs, total_pix);
    else
        launch_k(k_handover<CostSad>, dim3((int)blocks), dim3(256), 0, st, probs_dev, n_probs, total_pix);
}

// ---------------------------------------------------------------------------------------------------------
// propagation + random search

// Extra pixels (left, up, right, down) recomputed before half-sweep j = 2*d + colour of the last fused
// iteration; earlier iterations add kHaloPerIter on every side per remaining iteration.
__constant__ int8_t c_grow[8][4] = {{3, 3, 4, 4}, {2, 2, 4, 4}, {2, 1, 3, 4}, {2, 0, 2, 4},
                                    {1, 0, 2, 3}, {0, 0, 2, 2}, {0, 0, 1, 1}, {0, 0, 0, 0}};

size_t prop_smem_bytes(int tw, int th, int n_iter) {
    int H = kHaloPerIter * n_iter;
    return (size_t)(tw + 2 * H) * (th + 2 * H) * 8;
}


// Geometry of the tile a CTA is working on (all coordinates are level coordinates).
struct TileGeom {
    int x0, y0, x1, y1;      // tile interior
    int lx0, ly0, RW, RH;    // loaded region (tile + halo, clipped to the level)
};

// Region of half-sweep j (colour j&1 of direction j>>1) with `rem` halo pixels still to be consumed.
__device__ __forceinline__ void halfsweep_region(const TileGeom& G, int w, int h, int j, int rem, int& rx0, int& ry0,
                                                 int& rx1, int& ry1) {
    rx0 = max(G.x0 - c_grow[j][0] - rem, 0);
    ry0 = max(G.y0 - c_grow[j][1] - rem, 0);
    rx1 = min(G.x1 + c_grow[j][2] + rem, w);
    ry1 = min(G.y1 + c_grow[j][3] + rem, h);
}

// Pixel i of the active colour of a region, row-major over (row, slot); false past the row's end.
__device__ __forceinline__ bool region_pixel(int i, int HW, int rx0, int ry0, int rx1, int colour, int& x, int& y) {
    const int row = i / HW, slot = i - row * HW;
    y = ry0 + row;
    x = rx0 + 2 * slot + ((rx0 + y + colour) & 1);
    return x < rx1;
}

// The candidates of one pixel (x, y) of a grid in a half-sweep of direction d, one thread per pixel (the whole
// descriptor per thread: 96 B WHT, 32 B Census): neighbour 1 (horizontal, flow f1, valid if v1), neighbour 2
// (vertical, f2, v2) and, for d >= 1, the hashed random offset around the flow after them.  cur / c hold the
// pixel's flow and cost and are updated; false if there was nothing to try (they are unchanged).  With SPEC the
// random candidate of directions 1..3 is fetched together with the neighbour candidates, assuming the neighbours
// will not change the pixel's flow; if one of them is taken, the random candidate is fetched again from the new
// flow.  Either way the candidate evaluated is the one the schedule defines, so results are identical.
// (Fetching it early only into a buffer no neighbour needs, without SPEC, measured 16 % slower on the 1242x375
// pair.)
// Per-launch constants of update_pixel, read from the problem once per half-sweep.
struct SweepConst {
    int g, lw, lh;  // grid stride and level size: grid pixel (x, y) is level pixel (g*x, g*y)
    int R;          // random-search radius
    uint32_t span;  // 2R + 1
};
template <bool GRID>
__device__ __forceinline__ SweepConst sweep_const(const PropProblem& P) {
    const int R = P.rs_radius;
    return {GRID ? P.g : 1, GRID ? P.lw : P.w, GRID ? P.lh : P.h, R, 2u * R + 1u};
}

template <class C, bool SPEC, bool GRID>
__device__ __forceinline__ bool update_pixel(const PropProblem& P, const SweepConst& K, int x, int y, int d,
                                             uint32_t k1, bool v1, uint32_t f1, bool v2, uint32_t f2, uint32_t& cur,
                                             int& c) {
    // flows and targets are in level pixels
    const int g = K.g, lw = K.lw, lh = K.lh, R = K.R;
    const uint32_t span = K.span;
    const int n_d = lw * lh;  // descriptors of the level
    // a candidate equal to the current flow (or to an already tried one) cannot be strictly cheaper
    const int X = g * x, Y = g * y;  // level coordinates
    const bool e1 = v1 && f1 != cur && in_level(X + flow_x(f1), Y + flow_y(f1), lw, lh);
    const bool e2 = v2 && f2 != cur && !(v1 && f2 == f1) && in_level(X + flow_x(f2), Y + flow_y(f2), lw, lh);
    if (!(e1 || e2 || d >= 1)) return false;
    int ox = 0, oy = 0;
    if (d >= 1) {
        const uint32_t k2 = mix32(k1 ^ ((uint32_t)Y * 65536u + (uint32_t)X));
        ox = (int)(mix32(k2 ^ (uint32_t)(2 * d)) % span) - R;
        oy = (int)(mix32(k2 ^ (uint32_t)(2 * d + 1)) % span) - R;
    }
    const bool rnd = ox != 0 || oy != 0;
    const uint32_t cur0 = cur;
    // issue every independent load (own descriptor, neighbour candidates, speculative random) before compute
    uint32_t a[C::kWords], b1[C::kWords], b2[C::kWords];
    uint32_t b3[SPEC ? C::kWords : 1];
    load_chk<C>(P.fa, feat_index(X, Y, lw), n_d, kBoundsOwn, a);
    if (e1) load_chk<C>(P.fb, feat_index(X + flow_x(f1), Y + flow_y(f1), lw), n_d, kBoundsCand1, b1);
    if (e2) load_chk<C>(P.fb, feat_index(X + flow_x(f2), Y + flow_y(f2), lw), n_d, kBoundsCand2, b2);
    if constexpr (SPEC) {
        const int sx = flow_x(cur) + ox, sy = flow_y(cur) + oy;
        if (rnd && in_level(X + sx, Y + sy, lw, lh))
            load_chk<C>(P.fb, feat_index(X + sx, Y + sy, lw), n_d, kBoundsSpec, b3);
    }
    C::prep(a);
    if (e1) {
        int s1 = C::dist(a, b1);
        if (s1 < c) { cur = f1; c = s1; }
    }
    if (e2) {
        int s2 = C::dist(a, b2);
        if (s2 < c) { cur = f2; c = s2; }
    }
    if (rnd) {
        const int fx = flow_x(cur) + ox, fy = flow_y(cur) + oy;
        if (in_level(X + fx, Y + fy, lw, lh)) {
            int s3;
            if constexpr (SPEC) {
                if (cur == cur0) {
                    s3 = C::dist(a, b3);  // same target as speculated (which was then in the level)
                } else {
                    load_chk<C>(P.fb, feat_index(X + fx, Y + fy, lw), n_d, kBoundsRandom, b1);
                    s3 = C::dist(a, b1);
                }
            } else {
                load_chk<C>(P.fb, feat_index(X + fx, Y + fy, lw), n_d, kBoundsRandom, b1);
                s3 = C::dist(a, b1);
            }
            if (s3 < c) { cur = pack_flow(fx, fy); c = s3; }
        }
    }
    return true;
}

// One half-sweep of a tile's region (tile form).
template <class C, bool SPEC, bool GRID>
__device__ __forceinline__ void halfsweep(const PropProblem& P, const TileGeom& G, uint32_t* sflow, int32_t* scost,
                                          int j, int rem, uint32_t k1) {
    const int w = P.w, h = P.h;  // the grid (the level itself unless GRID)
    const int d = j >> 1, colour = j & 1;
    int rx0, ry0, rx1, ry1;
    halfsweep_region(G, w, h, j, rem, rx0, ry0, rx1, ry1);
    const int HW = (rx1 - rx0 + 1) >> 1;
    const int total = HW * (ry1 - ry0);
    const SweepConst K = sweep_const<GRID>(P);
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        int x, y;
        if (!region_pixel(i, HW, rx0, ry0, rx1, colour, x, y)) continue;
        const int sidx = (y - G.ly0) * G.RW + (x - G.lx0);
        const int n_s = G.RW * G.RH;  // shared-memory entries
        if (!idx_ok(g_bounds, kBoundsSmemOwn, sidx, n_s)) continue;
        uint32_t cur = sflow[sidx];
        int c = scost[sidx];
        const int n1x = x + ((d & 1) ? 1 : -1);
        const int n2y = y + ((d & 2) ? 1 : -1);
        const bool v1 = (unsigned)n1x < (unsigned)w;
        const bool v2 = (unsigned)n2y < (unsigned)h;
        const uint32_t f1 = v1 && idx_ok(g_bounds, kBoundsSmemN1, sidx + (n1x - x), n_s) ? sflow[sidx + (n1x - x)] : 0u;
        const uint32_t f2 =
            v2 && idx_ok(g_bounds, kBoundsSmemN2, sidx + (n2y - y) * G.RW, n_s) ? sflow[sidx + (n2y - y) * G.RW] : 0u;
        if (!update_pixel<C, SPEC, GRID>(P, K, x, y, d, k1, v1, f1, v2, f2, cur, c)) continue;
        sflow[sidx] = cur;
        scost[sidx] = c;
    }
}

// Where a tile task reads the state of its region and writes its interior, and which iterations it runs.
struct TileIO {
    const uint32_t* flow_in;
    const int32_t* cost_in;
    uint32_t* flow_out;
    int32_t* cost_out;
    int t0, n_iter;
};

// One tile of one problem: load the tile and its halo, run n_iter iterations in shared memory, write the tile.
// The buffers and iterations are the problem's (tile form) or, with DF, those of `io`, a dataflow task whose
// state was written by other CTAs of the running launch and is therefore read from L2.
template <class C, bool SPEC, bool GRID, bool DF = false>
__device__ __forceinline__ void propagate_tile(const PropProblem& P, int tile, const PropLaunch& L, uint32_t* smem,
                                               const TileIO* io = nullptr) {
    const int w = P.w, h = P.h;
    const int n_iter = DF ? io->n_iter : P.n_iter;
    TileGeom G;
    G.x0 = (tile % P.tiles_x) * L.tw;
    G.y0 = (tile / P.tiles_x) * L.th;
    G.x1 = min(G.x0 + L.tw, w);
    G.y1 = min(G.y0 + L.th, h);
    const int H = kHaloPerIter * n_iter;
    G.lx0 = max(G.x0 - H, 0);
    G.ly0 = max(G.y0 - H, 0);
    G.RW = min(G.x1 + H, w) - G.lx0;
    G.RH = min(G.y1 + H, h) - G.ly0;
    uint32_t* sflow = smem;
    int32_t* scost = reinterpret_cast<int32_t*>(smem + G.RW * G.RH);

    for (int i = threadIdx.x; i < G.RW * G.RH; i += blockDim.x) {
        int r = i / G.RW, c = i - r * G.RW;
        size_t g = (size_t)(G.ly0 + r) * w + G.lx0 + c;
        // flow and cost of the region (2 words per pixel) must fit the launch's dynamic shared memory
        const bool ok = idx_ok(g_bounds, kBoundsTileRead, (long long)g, (long long)w * h) &&
                        (!FF_DEBUG_BOUNDS || idx_ok(g_bounds, kBoundsTileSmem, 2 * G.RW * G.RH - 1, dyn_smem_bytes() / 4));
        if constexpr (DF) {
            sflow[i] = ok ? __ldcg(io->flow_in + g) : 0u;
            scost[i] = ok ? __ldcg(io->cost_in + g) : 0;
        } else {
            sflow[i] = ok ? P.flow_in[g] : 0u;
            scost[i] = ok ? P.cost_in[g] : 0;
        }
    }
    __syncthreads();
    for (int it = 0; it < n_iter; it++) {
        const int t = (DF ? io->t0 : P.t0) + it;
        const int rem = kHaloPerIter * (n_iter - 1 - it);
        const uint32_t k1 = mix32(P.seed ^ mix32((uint32_t)P.dir * 65536u + (uint32_t)P.level * 256u + (uint32_t)t));
        for (int j = 0; j < 8; j++) {
            halfsweep<C, SPEC, GRID>(P, G, sflow, scost, j, rem, k1);
            __syncthreads();
        }
    }
    const int TW = G.x1 - G.x0;
    for (int i = threadIdx.x; i < TW * (G.y1 - G.y0); i += blockDim.x) {
        int r = i / TW, c = i - r * TW;
        int sidx = (G.y0 + r - G.ly0) * G.RW + (G.x0 + c - G.lx0);
        size_t g = (size_t)(G.y0 + r) * w + G.x0 + c;
        if (!idx_ok(g_bounds, kBoundsTileWrite, (long long)g, (long long)w * h) ||
            !idx_ok(g_bounds, kBoundsTileSmem, sidx, G.RW * G.RH))
            continue;
        (DF ? io->flow_out : P.flow_out)[g] = sflow[sidx];
        (DF ? io->cost_out : P.cost_out)[g] = scost[sidx];
    }
}

// Persistent launch: each CTA takes tiles from the launch's queue (an atomic counter, zeroed before the launch)
// until it is empty, so the last wave has no idle tail.  queue[i] = (problem index, tile index in problem).
// Instantiated for 128, 256 and 512 threads, with and without speculative random-candidate loads, per cost, for
// levels and for sub-scale grids (GRID).
template <int THREADS, bool SPEC, class C, bool GRID = false>
__global__ __launch_bounds__(THREADS, SPEC ? 1 : 512 / THREADS) void k_propagate(
    const PropProblem* __restrict__ probs, const int2* __restrict__ queue, int n_tiles, int* __restrict__ counter,
    PropLaunch L) {
    grid_dependency_sync();
    extern __shared__ uint32_t smem[];
    __shared__ int s_next;
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(counter, 1);
        __syncthreads();
        const int q = s_next;
        if (q >= n_tiles) return;
        const int2 e = queue[q];
        propagate_tile<C, SPEC, GRID>(probs[e.x], e.y, L, smem);
        __syncthreads();
    }
}

// Dataflow form: every iteration of a level in one persistent launch.  Task q is iteration t = q / n_tiles of
// queue entry q % n_tiles (tasks are taken in that order); it starts once the 3x3 tiles around its tile, itself
// included, have finished iteration t - 1, so no launch boundary separates the iterations and a CTA that
// finishes early goes on with the next iteration's tiles.  A task of iteration t reads its region (the tile and
// a halo of one iteration, kHaloPerIter <= tile size, so inside those nine tiles) from the buffer iteration t - 1
// wrote and writes its tile to the next: flow_alt for even t, flow_in for odd t, flow_out for the last (a buffer
// the host keeps apart from the one the iteration before wrote).  A tile overwrites a buffer its neighbours read
// one iteration earlier only after they finished that iteration, by the same rule.  Progress is published with
// a release after the tile's stores and read with an acquire; the region is then read from L2.  A task waits
// only for tasks taken before it by running CTAs, so there is no deadlock whatever the residency; every wait is
// bounded (wait_limit polls; on expiry kErrDataflow goes to the error word and the CTA stops waiting).
// Affine variant (L.affine): no queue counter; CTA b owns entries b, b + G, ... of every iteration (G CTAs, at
// most the resident ones) and runs them iteration by iteration, keeping its tiles' descriptors in its L1.  Its
// waits are for iteration t - 1 of tiles other CTAs own, which wait only for earlier iterations, so every CTA
// makes progress once the grid is resident (with the grid sized to the resident CTAs, it is).
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int THREADS, bool SPEC, class C, bool GRID = false>
__global__ __launch_bounds__(THREADS, SPEC ? 1 : 512 / THREADS) void k_propagate_df(
    const PropProblem* __restrict__ probs, const int2* __restrict__ queue, int n_tiles, int* __restrict__ counter,
    PropLaunch L) {
    grid_dependency_sync();
    extern __shared__ uint32_t smem[];
    __shared__ int s_next;
    const int T = L.dataflow, n_tasks = n_tiles * T;
    bool failed = false;  // a wait of this CTA expired: stop waiting (CTA-uniform)
    // affine: CTA b owns queue entries b, b + G, b + 2G, ... (G CTAs) for every iteration and runs them
    // iteration by iteration, so a tile's region stays in the same SM's L1 from one iteration to the next
    const int G = (int)gridDim.x, per_iter = (n_tiles - (int)blockIdx.x + G - 1) / G;  // entries this CTA owns
    for (int k = 0;; k++) {
        int q;
        if (L.affine) {
            if (k >= per_iter * T) return;
            const int ti = k / per_iter;
            q = ti * n_tiles + (int)blockIdx.x + (k - ti * per_iter) * G;
        } else {
            if (threadIdx.x == 0) s_next = atomicAdd(counter, 1);
            __syncthreads();
            q = s_next;
            if (q >= n_tasks) return;
        }
        const int t = q / n_tiles;
        const int2 e = queue[q - t * n_tiles];
        const PropProblem& P = probs[e.x];
        bool ok = true;
        if (t > 0 && !failed && threadIdx.x < 9) {  // one waiting thread per tile of the 3x3 neighbourhood
            const int tiles_y = (P.h + L.th - 1) / L.th;
            const int nx = e.y % P.tiles_x + (int)threadIdx.x % 3 - 1, ny = e.y / P.tiles_x + (int)threadIdx.x / 3 - 1;
            if (nx >= 0 && nx < P.tiles_x && ny >= 0 && ny < tiles_y) {
                const int* f = P.progress + ny * P.tiles_x + nx;
                ok = false;
                for (uint32_t i = 0; i < L.wait_limit && !ok; i++) {
                    ok = ld_acquire_gpu(f) >= t;
                    if (!ok && i > 64) __nanosleep(128);
                }
                if (!ok) atomicCAS(L.err, 0, kErrDataflow);
            }
        }
        failed = __syncthreads_or(!ok) != 0 || failed;
        TileIO io;
        io.t0 = P.t0 + t;
        io.n_iter = 1;
        const bool src_alt = t > 0 && ((t - 1) & 1) == 0;  // iteration t - 1 wrote flow_alt iff t - 1 is even
        io.flow_in = t == 0 ? P.flow_in : src_alt ? P.flow_alt : P.flow_in;
        io.cost_in = t == 0 ? P.cost_in : src_alt ? P.cost_alt : P.cost_in;
        io.flow_out = t == T - 1 ? P.flow_out : (t & 1) == 0 ? P.flow_alt : P.flow_in;
        io.cost_out = t == T - 1 ? P.cost_out : (t & 1) == 0 ? P.cost_alt : P.cost_in;
        propagate_tile<C, SPEC, GRID, true>(P, e.y, L, smem, &io);
        __syncthreads();  // every store of the tile is issued
        if (threadIdx.x == 0 && !L.withhold) {
            __threadfence();
            st_release_gpu(P.progress + e.y, t + 1);
        }
    }
}

// ---------------------------------------------------------------------------------------------------------
// Cluster form: one cluster of n CTAs per problem runs every iteration of the launch over the whole grid, with no
// halo recomputation.  CTA r owns block r of the partition cluster_partition() gives and keeps the block's flow
// and cost in shared memory, with a one-pixel ring of the neighbouring blocks' edge flows.  After computing an
// edge pixel of the active colour, a CTA stores its flow straight into the ring of each CTA beside that edge
// (st.async into the neighbour's shared memory, completing 4 bytes on the neighbour's mbarrier of that
// half-sweep), and before the next half-sweep reads its ring it waits on its own mbarrier for the edges it
// receives.  The waits are CTA-scope: a cluster-wide barrier per half-sweep, an acquire at cluster scope, also
// emptied the L1 that the next half-sweep's gathers reuse (8 % L1 hits instead of 83 % at level 4 of the
// 1242x375 pair).  A half-sweep reads exactly the state the previous one left, so the schedule is the tile
// form's, evaluated once per pixel.  Every wait is bounded (wait_limit polls); one that expires records
// kErrClusterEdges in the error word and the CTA stops waiting (the launch runs to its end; ff_sync then fails).
// An alternative for small levels of a few problems, where the tile form's halo is most of the work; the
// autotuner weighs the two forms per level.

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ int cluster_rank() {
    uint32_t r;
    asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
}
__device__ __forceinline__ int cluster_ctas() {
    uint32_t n;
    asm("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
    return (int)n;
}
// Address, in the cluster's shared-memory window, of `p` (this CTA's shared memory) in CTA `rank`.
__device__ __forceinline__ uint32_t cluster_addr(const void* p, int rank) {
    uint32_t a;
    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(smem_u32(p)), "r"(rank));
    return a;
}
// 4-byte store into another CTA's shared memory that completes 4 bytes on the mbarrier `bar` (cluster window).
__device__ __forceinline__ void st_async_u32(uint32_t addr, uint32_t v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(addr), "r"(v),
                 "r"(bar)
                 : "memory");
}
// Number of v in [a, b) with (k + v) of colour c ((k + v) & 1 == c).
__device__ __forceinline__ int colour_count(int k, int a, int b, int c) {
    const int first = a + ((c - k - a) & 1);
    return first < b ? (b - 1 - first) / 2 + 1 : 0;
}

// (no speculative variant: measured slower at every coarse level in this form)
template <int THREADS, class C, bool GRID = false>
__global__ __launch_bounds__(THREADS, 1) void k_propagate_cl(const PropProblem* __restrict__ probs, PropLaunch L) {
    grid_dependency_sync();
    extern __shared__ __align__(16) uint32_t smem[];
    const int n = cluster_ctas(), r = cluster_rank();
    const PropProblem& P = probs[blockIdx.x / n];
    const int w = P.w, h = P.h;
    int bx = 1, by = 1;
    cluster_partition(w, h, n, bx, by);  // the host launches only problems that have a partition
    const int bi = r % bx, bj = r / bx;
    const int x0 = bi * w / bx, x1 = (bi + 1) * w / bx, y0 = bj * h / by, y1 = (bj + 1) * h / by;
    const int bw = x1 - x0, bh = y1 - y0, nb = bw * bh;
    const int mw = (w + bx - 1) / bx, mh = (h + by - 1) / by;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);  // [2]: the edges received in even / odd half-sweeps
    uint32_t* ring_l = smem + 4;                         // [mh] flows of column x0 - 1
    uint32_t* ring_r = ring_l + mh;                      // [mh] column x1
    uint32_t* ring_u = ring_r + mh;                      // [mw] row y0 - 1
    uint32_t* ring_d = ring_u + mw;                      // [mw] row y1
    uint32_t* sflow = ring_d + mw;                       // [mw * mh] the block, row-major with width bw
    int32_t* scost = reinterpret_cast<int32_t*>(sflow + mw * mh);
    const bool has_l = bi > 0, has_r = bi + 1 < bx, has_u = bj > 0, has_d = bj + 1 < by;
    // an edge pixel's flow goes to the opposite ring of the CTA beside it, completing on that CTA's mbarrier
    const uint32_t to_l = has_l ? cluster_addr(ring_r, r - 1) : 0u, mb_l = has_l ? cluster_addr(mbar, r - 1) : 0u;
    const uint32_t to_r = has_r ? cluster_addr(ring_l, r + 1) : 0u, mb_r = has_r ? cluster_addr(mbar, r + 1) : 0u;
    const uint32_t to_u = has_u ? cluster_addr(ring_d, r - bx) : 0u, mb_u = has_u ? cluster_addr(mbar, r - bx) : 0u;
    const uint32_t to_d = has_d ? cluster_addr(ring_u, r + bx) : 0u, mb_d = has_d ? cluster_addr(mbar, r + bx) : 0u;
    // bytes received per half-sweep of colour c: the neighbours' edge pixels of that colour next to this block
    uint32_t rx_bytes[2];
#pragma unroll
    for (int c = 0; c < 2; c++)
        rx_bytes[c] = 4u * (uint32_t)((has_l ? colour_count(x0 - 1, y0, y1, c) : 0) +
                                      (has_r ? colour_count(x1, y0, y1, c) : 0) +
                                      (has_u ? colour_count(y0 - 1, x0, x1, c) : 0) +
                                      (has_d ? colour_count(y1, x0, x1, c) : 0));
    const bool fits = !FF_DEBUG_BOUNDS ||
                      idx_ok(g_bounds, kBoundsBlockSmem, (long long)cluster_smem_bytes(w, h, bx, by) - 1,
                             dyn_smem_bytes());
    const int J = 8 * P.n_iter;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&mbar[0]), 1);
        mbar_init(smem_u32(&mbar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // half-sweeps 0 and 1: the first phase of each mbarrier (a colour with no edges to receive never waits)
        if (rx_bytes[0] != 0) mbar_expect_tx(smem_u32(&mbar[0]), rx_bytes[0]);
        if (J > 1 && rx_bytes[1] != 0) mbar_expect_tx(smem_u32(&mbar[1]), rx_bytes[1]);
    }
    // the block and the ring from the launch's input state
    const long long n_in = (long long)w * h;
    for (int i = threadIdx.x; i < nb; i += THREADS) {
        const long long gi = (long long)(y0 + i / bw) * w + x0 + i % bw;
        const bool ok = fits && idx_ok(g_bounds, kBoundsBlockRead, gi, n_in);
        sflow[i] = ok ? P.flow_in[gi] : 0u;
        scost[i] = ok ? P.cost_in[gi] : 0;
    }
    for (int i = threadIdx.x; i < bh; i += THREADS) {
        const long long left = (long long)(y0 + i) * w + x0 - 1, right = (long long)(y0 + i) * w + x1;
        if (has_l && fits && idx_ok(g_bounds, kBoundsBlockRead, left, n_in)) ring_l[i] = P.flow_in[left];
        if (has_r && fits && idx_ok(g_bounds, kBoundsBlockRead, right, n_in)) ring_r[i] = P.flow_in[right];
    }
    for (int i = threadIdx.x; i < bw; i += THREADS) {
        const long long up = (long long)(y0 - 1) * w + x0 + i, down = (long long)y1 * w + x0 + i;
        if (has_u && fits && idx_ok(g_bounds, kBoundsBlockRead, up, n_in)) ring_u[i] = P.flow_in[up];
        if (has_d && fits && idx_ok(g_bounds, kBoundsBlockRead, down, n_in)) ring_d[i] = P.flow_in[down];
    }
    cluster_sync_all();  // every CTA of the cluster running, its block loaded and its mbarriers armed
    const int HW = (bw + 1) >> 1, total = HW * bh;
    const SweepConst K = sweep_const<GRID>(P);
    bool failed = false;  // a wait expired: stop waiting (CTA-uniform)
    uint32_t k1 = 0;
    for (int j = 0; j < J; j++) {
        if ((j & 7) == 0) {
            const uint32_t t = (uint32_t)(P.t0 + (j >> 3));
            k1 = mix32(P.seed ^ mix32((uint32_t)P.dir * 65536u + (uint32_t)P.level * 256u + t));
        }
        const int d = (j & 7) >> 1, colour = j & 1;
        const uint32_t slot = 8u * (uint32_t)(j & 1);  // byte offset of this half-sweep's mbarrier
        for (int i = threadIdx.x; i < total; i += THREADS) {
            const int row = i / HW, slot_x = i - row * HW;
            const int y = y0 + row;
            const int x = x0 + 2 * slot_x + ((x0 + y + colour) & 1);
            if (x >= x1 || !fits) continue;
            const int sidx = row * bw + (x - x0);
            uint32_t cur = sflow[sidx];
            int c = scost[sidx];
            const int n1x = x + ((d & 1) ? 1 : -1);
            const int n2y = y + ((d & 2) ? 1 : -1);
            const bool v1 = (unsigned)n1x < (unsigned)w;
            const bool v2 = (unsigned)n2y < (unsigned)h;
            uint32_t f1 = 0u, f2 = 0u;
            if (v1) {
                if (n1x < x0)
                    f1 = idx_ok(g_bounds, kBoundsRingN1, row, mh) ? ring_l[row] : 0u;
                else if (n1x >= x1)
                    f1 = idx_ok(g_bounds, kBoundsRingN1, row, mh) ? ring_r[row] : 0u;
                else
                    f1 = sflow[sidx + (n1x - x)];
            }
            if (v2) {
                if (n2y < y0)
                    f2 = idx_ok(g_bounds, kBoundsRingN2, x - x0, mw) ? ring_u[x - x0] : 0u;
                else if (n2y >= y1)
                    f2 = idx_ok(g_bounds, kBoundsRingN2, x - x0, mw) ? ring_d[x - x0] : 0u;
                else
                    f2 = sflow[sidx + (n2y - y) * bw];
            }
            if (update_pixel<C, false, GRID>(P, K, x, y, d, k1, v1, f1, v2, f2, cur, c)) {
                sflow[sidx] = cur;
                scost[sidx] = c;
            }
            if (!L.withhold) {  // every edge pixel of the colour is sent, changed or not (fixed byte counts)
                if (has_l && x == x0) st_async_u32(to_l + 4u * row, cur, mb_l + slot);
                if (has_r && x == x1 - 1) st_async_u32(to_r + 4u * row, cur, mb_r + slot);
                if (has_u && y == y0) st_async_u32(to_u + 4u * (x - x0), cur, mb_u + slot);
                if (has_d && y == y1 - 1) st_async_u32(to_d + 4u * (x - x0), cur, mb_d + slot);
            }
        }
        // the neighbours' edges of this colour, read by the next half-sweep
        const bool rx = rx_bytes[j & 1] != 0;
        // (this wait is on the critical path of every half-sweep: spin for the first 4096 polls, then sleep)
        const bool ok =
            failed || !rx || mbar_wait(smem_u32(&mbar[j & 1]), (uint32_t)(j >> 1) & 1u, L.wait_limit, 4096);
        if (!ok) atomicCAS(L.err, 0, kErrClusterEdges);
        // the same mbarrier's next phase, half-sweep j + 2, armed before this CTA sends any edge of half-sweep
        // j + 1 (which the neighbours' sends of j + 2 wait for); as it expects bytes, it cannot complete before
        // every thread here has seen this phase complete, for the same reason
        if (threadIdx.x == 0 && rx && ok && !failed && j + 2 < J)
            mbar_expect_tx(smem_u32(&mbar[j & 1]), rx_bytes[j & 1]);
        failed = __syncthreads_or(!ok) != 0 || failed;
    }
    for (int i = threadIdx.x; i < nb; i += THREADS) {
        const long long gi = (long long)(y0 + i / bw) * w + x0 + i % bw;
        if (!fits || !idx_ok(g_bounds, kBoundsBlockWrite, gi, n_in)) continue;
        P.flow_out[gi] = sflow[i];
        P.cost_out[gi] = scost[i];
    }
    cluster_sync_all();  // no CTA leaves while edge stores of its neighbours may still target its shared memory
}

using PropKernel = void (*)(const PropProblem*, const int2*, int, int*, PropLaunch);
using PropClusterKernel = void (*)(const PropProblem*, PropLaunch);

template <class C, bool SPEC, bool GRID>
PropKernel prop_kernel_t(int threads) {
    return threads == 128   ? k_propagate<128, SPEC, C, GRID>
           : threads == 512 ? k_propagate<512, SPEC, C, GRID>
                            : k_propagate<256, SPEC, C, GRID>;
}

template <class C>
PropKernel prop_kernel_c(int threads, bool spec, bool grid) {
    if (grid) return spec ? prop_kernel_t<C, true, true>(threads) : prop_kernel_t<C, false, true>(threads);
    return spec ? prop_kernel_t<C, true, false>(threads) : prop_kernel_t<C, false, false>(threads);
}

PropKernel prop_kernel(int threads, bool spec, int cost, bool grid = false) {
    return cost == FF_COST_CENSUS ? prop_kernel_c<CostCensus>(threads, spec, grid)
                                  : prop_kernel_c<CostSad>(threads, spec, grid);
}

// The dataflow form is instantiated for 128, 256 and 512 threads without speculation, per cost, for levels and
// for sub-scale grids.
template <class C, bool GRID>
PropKernel prop_df_kernel_t(int threads) {
    return threads == 128   ? k_propagate_df<128, false, C, GRID>
           : threads == 512 ? k_propagate_df<512, false, C, GRID>
                            : k_propagate_df<256, false, C, GRID>;
}

PropKernel prop_df_kernel(int threads, int cost, bool grid) {
    if (cost == FF_COST_CENSUS) return grid ? prop_df_kernel_t<CostCensus, true>(threads) : prop_df_kernel_t<CostCensus, false>(threads);
    return grid ? prop_df_kernel_t<CostSad, true>(threads) : prop_df_kernel_t<CostSad, false>(threads);
}

// The cluster form is instantiated for 256 and 512 threads, per cost, for levels and for sub-scale grids.
template <class C, bool GRID>
PropClusterKernel prop_cl_kernel_t(int threads) {
    return threads == 512 ? k_propagate_cl<512, C, GRID> : k_propagate_cl<256, C, GRID>;
}

template <class C>
PropClusterKernel prop_cl_kernel_c(int threads, bool grid) {
    return grid ? prop_cl_kernel_t<C, true>(threads) : prop_cl_kernel_t<C, false>(threads);
}

PropClusterKernel prop_cl_kernel(int threads, int cost, bool grid) {
    return cost == FF_COST_CENSUS ? prop_cl_kernel_c<CostCensus>(threads, grid) : prop_cl_kernel_c<CostSad>(threads, grid);
}

cudaLaunchConfig_t cluster_config(int n_ctas, int cluster, int threads, size_t smem, cudaStream_t st,
                                  cudaLaunchAttribute (&attr)[2]) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_ctas);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = FF_PDL;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cfg;
}

cudaError_t init_kernel_attributes() {
    cudaFuncAttributes fa;
    cudaError_t e0 = cudaFuncGetAttributes(&fa, k_handover<CostSad>);
    if (e0 == cudaSuccess) e0 = cudaFuncGetAttributes(&fa, k_handover<CostCensus>);
    if (e0 != cudaSuccess) return e0;
    for (int cost : {FF_COST_WHT_SAD, FF_COST_CENSUS})
        for (int t : {128, 256, 512})
            for (bool sp : {false, true})
                for (bool grid : {false, true}) {
                    cudaError_t e = cudaFuncSetAttribute(prop_kernel(t, sp, cost, grid),
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         (int)kMaxPropSmem);
                    if (e == cudaSuccess && !sp)
                        e = cudaFuncSetAttribute(prop_df_kernel(t, cost, grid),
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxPropSmem);
                    if (e != cudaSuccess) return e;
                }
    for (int cost : {FF_COST_WHT_SAD, FF_COST_CENSUS})
        for (int t : {256, 512})
            for (bool grid : {false, true}) {
                PropClusterKernel k = prop_cl_kernel(t, cost, grid);
                cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxPropSmem);
                if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
                if (e != cudaSuccess) return e;
            }
    return cudaSuccess;
}

bool prop_threads_ok(int threads) { return threads == 128 || threads == 256 || threads == 512; }

int prop_blocks_per_sm(size_t smem, int threads, bool spec, int cost, bool grid, bool dataflow) {
    int n = 0;
    PropKernel k = dataflow ? prop_df_kernel(threads, cost, grid) : prop_kernel(threads, spec, cost, grid);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

int prop_cluster_capacity(int cluster, int threads, int cost, bool grid, size_t smem) {
    if (cluster < 1 || cluster > kMaxCluster || (threads != 256 && threads != 512) || smem > kMaxPropSmem) return 0;
    cudaLaunchAttribute attr[2];
    cudaLaunchConfig_t cfg = cluster_config(cluster, cluster, threads, smem, nullptr, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, prop_cl_kernel(threads, cost, grid), &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

void launch_propagate(const PropProblem* probs_dev, const int2* queue_dev, int n_tiles, int* counter_dev, int grid,
                      const PropLaunch& L, cudaStream_t st) {
    if (L.cluster > 0) {
        cudaLaunchAttribute attr[2];
        cudaLaunchConfig_t cfg = cluster_config(grid, L.cluster, L.threads, (size_t)L.cl_smem, st, attr);
        cudaLaunchKernelEx(&cfg, prop_cl_kernel(L.threads, L.cost, L.grid != 0), probs_dev, L);
        return;
    }
    size_t smem = prop_smem_bytes(L.tw, L.th, L.max_iter);
    PropKernel k = L.dataflow > 0 ? prop_df_kernel(L.threads, L.cost, L.grid != 0)
                                  : prop_kernel(L.threads, L.spec != 0, L.cost, L.grid != 0);
    launch_k(k, dim3(grid), dim3(L.threads), smem, st, probs_dev, queue_dev, n_tiles, counter_dev, L);
}

}  // namespace ff
