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
             kBoundsSmemN2, kBoundsTileRead, kBoundsTileSmem, kBoundsTileWrite, kBoundsParent, kBoundsHandoverDesc };

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

// One half-sweep with one thread per pixel (the whole descriptor per thread: 96 B WHT, 32 B Census).  With SPEC
// the random candidate of directions 1..3 is fetched together with the neighbour candidates, assuming the
// neighbours will not change the pixel's flow; if one of them is taken, the random candidate is fetched again
// from the new flow.  Either way the candidate evaluated is the one the schedule defines, so results are
// identical.  (Fetching it early only into a buffer no neighbour needs, without SPEC, measured 16 % slower on
// the 1242x375 pair.)
template <class C, bool SPEC, bool GRID>
__device__ __forceinline__ void halfsweep(const PropProblem& P, const TileGeom& G, uint32_t* sflow, int32_t* scost,
                                          int j, int rem, uint32_t k1) {
    const int w = P.w, h = P.h;  // the grid (the level itself unless GRID)
    // GRID: grid pixel (x, y) is level pixel (g*x, g*y) of a lw x lh level; flows and targets are in level pixels
    const int g = GRID ? P.g : 1, lw = GRID ? P.lw : w, lh = GRID ? P.lh : h;
    const int d = j >> 1, colour = j & 1;
    int rx0, ry0, rx1, ry1;
    halfsweep_region(G, w, h, j, rem, rx0, ry0, rx1, ry1);
    const int HW = (rx1 - rx0 + 1) >> 1;
    const int total = HW * (ry1 - ry0);
    const int R = P.rs_radius;
    const uint32_t span = 2u * R + 1u;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        int x, y;
        if (!region_pixel(i, HW, rx0, ry0, rx1, colour, x, y)) continue;
        const int sidx = (y - G.ly0) * G.RW + (x - G.lx0);
        const int n_s = G.RW * G.RH, n_d = lw * lh;  // shared-memory entries, descriptors of the level
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
        // a candidate equal to the current flow (or to an already tried one) cannot be strictly cheaper
        const int X = g * x, Y = g * y;  // level coordinates
        const bool e1 = v1 && f1 != cur && in_level(X + flow_x(f1), Y + flow_y(f1), lw, lh);
        const bool e2 = v2 && f2 != cur && !(v1 && f2 == f1) && in_level(X + flow_x(f2), Y + flow_y(f2), lw, lh);
        if (!(e1 || e2 || d >= 1)) continue;
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
        sflow[sidx] = cur;
        scost[sidx] = c;
    }
}

// One tile of one problem: load the tile and its halo, run n_iter iterations in shared memory, write the tile.
template <class C, bool SPEC, bool GRID>
__device__ __forceinline__ void propagate_tile(const PropProblem& P, int tile, const PropLaunch& L, uint32_t* smem) {
    const int w = P.w, h = P.h;
    TileGeom G;
    G.x0 = (tile % P.tiles_x) * L.tw;
    G.y0 = (tile / P.tiles_x) * L.th;
    G.x1 = min(G.x0 + L.tw, w);
    G.y1 = min(G.y0 + L.th, h);
    const int H = kHaloPerIter * P.n_iter;
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
        sflow[i] = ok ? P.flow_in[g] : 0u;
        scost[i] = ok ? P.cost_in[g] : 0;
    }
    __syncthreads();
    for (int it = 0; it < P.n_iter; it++) {
        const int t = P.t0 + it;
        const int rem = kHaloPerIter * (P.n_iter - 1 - it);
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
        P.flow_out[g] = sflow[sidx];
        P.cost_out[g] = scost[sidx];
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

using PropKernel = void (*)(const PropProblem*, const int2*, int, int*, PropLaunch);

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
                    if (e != cudaSuccess) return e;
                }
    return cudaSuccess;
}

bool prop_threads_ok(int threads) { return threads == 128 || threads == 256 || threads == 512; }

int prop_blocks_per_sm(size_t smem, int threads, bool spec, int cost, bool grid) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, prop_kernel(threads, spec, cost, grid),
                                                      threads, smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

void launch_propagate(const PropProblem* probs_dev, const int2* queue_dev, int n_tiles, int* counter_dev, int grid,
                      const PropLaunch& L, cudaStream_t st) {
    size_t smem = prop_smem_bytes(L.tw, L.th, L.max_iter);
    launch_k(prop_kernel(L.threads, L.spec != 0, L.cost, L.grid != 0), dim3(grid), dim3(L.threads),
             smem, st, probs_dev, queue_dev, n_tiles, counter_dev, L);
}

}  // namespace ff
