// features.cu -- image pyramid and Walsh-Hadamard patch descriptors (FlowFields++, arXiv 1805.03517, Sec. 3
// and Sec. 3.1), plus the Census patterns (Census cost) and the packed descriptors of the coarsest level used by
// the initial matching.
#include <cuda_fp16.h>

#include "ff_internal.h"

namespace ff {

// first index violation of a debug-bounds build (see idx_ok): code, index, limit
static __device__ int g_bounds[4];
enum : int { kBoundsImage = 40, kBoundsWin, kBoundsRowt, kBoundsFeat, kBoundsCensus, kBoundsSeed, kBoundsPyr };

cudaError_t bounds_take_features(int rec[3]) {
    int h[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyFromSymbol(h, g_bounds, sizeof h);
    if (e == cudaSuccess && h[0] != 0) {
        const int z[4] = {0, 0, 0, 0};
        e = cudaMemcpyToSymbol(g_bounds, z, sizeof z);
    }
    rec[0] = h[0], rec[1] = h[1], rec[2] = h[2];
    return e;
}

// One pyramid step (Sec. 3): 2x2 box average per channel, rounded half up; source coordinates clamped so
// that a 1-pixel-wide or -high level averages its only column/row.  One thread per output pixel.
__global__ void k_downsample(const uint8_t* __restrict__ src, int sw, int sh, int spitch, uint8_t* __restrict__ dst,
                             int dw, int dh) {
    grid_dependency_sync();
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    if (x >= dw || y >= dh) return;
    int x0 = min(2 * x, sw - 1), x1 = min(2 * x + 1, sw - 1);
    int y0 = min(2 * y, sh - 1), y1 = min(2 * y + 1, sh - 1);
    const uint8_t* r0 = src + (size_t)y0 * spitch;
    const uint8_t* r1 = src + (size_t)y1 * spitch;
    uint8_t* o = dst + ((size_t)y * dw + x) * 3;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        int s = r0[x0 * 3 + c] + r0[x1 * 3 + c] + r1[x0 * 3 + c] + r1[x1 * 3 + c];
        o[c] = (uint8_t)((s + 2) >> 2);
    }
}

void launch_downsample(const uint8_t* src, int sw, int sh, int spitch, uint8_t* dst, int dw, int dh,
                       cudaStream_t st) {
    dim3 grid((dw + 127) / 128, dh);
    launch_k(k_downsample, grid, dim3(128), 0, st, src, sw, sh, spitch, dst, dw, dh);
}

// Levels 1..a.top of the pyramid of one frame in one launch (same arithmetic as k_downsample).  A CTA owns a
// 32x32 block of level 1 (computed from level 0 in global memory) and derives the co-located blocks of the next
// levels from it in shared memory: level sizes are floor(w/2), so both sources 2x, 2x+1 of a level-s pixel lie
// in the parent block (the clamp only matters when the parent level is 1 pixel wide or high, and its single
// pixel is in block 0).  A 32x32 level-1 block halves down to one pixel at level 6, hence a.top <= 6.
__device__ __forceinline__ void pyramid_block(const PyrArgs& a, int bx, int by,
                                              uint8_t (&buf)[2][kPyrBlock][kPyrBlock][3]) {
    int size = kPyrBlock, ox = bx * kPyrBlock, oy = by * kPyrBlock;
    for (int i = threadIdx.x; i < size * size; i += blockDim.x) {
        const int lx = i % size, ly = i / size, x = ox + lx, y = oy + ly;
        if (x >= a.w[1] || y >= a.h[1]) continue;
        const int x0 = min(2 * x, a.w[0] - 1), x1 = min(2 * x + 1, a.w[0] - 1);
        const int y0 = min(2 * y, a.h[0] - 1), y1 = min(2 * y + 1, a.h[0] - 1);
        if (!idx_ok(g_bounds, kBoundsPyr, (long long)y1 * a.w[0] + x1, (long long)a.w[0] * a.h[0])) continue;
        const uint8_t* r0 = a.src + (size_t)y0 * a.spitch;
        const uint8_t* r1 = a.src + (size_t)y1 * a.spitch;
        uint8_t* o = a.dst[1] + ((size_t)y * a.w[1] + x) * 3;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const int v = (r0[x0 * 3 + c] + r0[x1 * 3 + c] + r1[x0 * 3 + c] + r1[x1 * 3 + c] + 2) >> 2;
            o[c] = (uint8_t)v;
            buf[0][ly][lx][c] = (uint8_t)v;
        }
    }
    int cur = 0;
    for (int s = 2; s <= a.top; s++) {
        __syncthreads();
        const int pox = ox, poy = oy;  // parent block origin (level s-1)
        size >>= 1;
        ox >>= 1;
        oy >>= 1;
        for (int i = threadIdx.x; i < size * size; i += blockDim.x) {
            const int lx = i % size, ly = i / size, x = ox + lx, y = oy + ly;
            if (x >= a.w[s] || y >= a.h[s]) continue;
            const int x0 = min(2 * x, a.w[s - 1] - 1) - pox, x1 = min(2 * x + 1, a.w[s - 1] - 1) - pox;
            const int y0 = min(2 * y, a.h[s - 1] - 1) - poy, y1 = min(2 * y + 1, a.h[s - 1] - 1) - poy;
            uint8_t* o = a.dst[s] + ((size_t)y * a.w[s] + x) * 3;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const int v = (buf[cur][y0][x0][c] + buf[cur][y0][x1][c] + buf[cur][y1][x0][c] +
                               buf[cur][y1][x1][c] + 2) >> 2;
                o[c] = (uint8_t)v;
                buf[cur ^ 1][ly][lx][c] = (uint8_t)v;
            }
        }
        cur ^= 1;
    }
}

__global__ __launch_bounds__(256) void k_pyramid(PyrArgs a) {
    grid_dependency_sync();
    __shared__ uint8_t buf[2][kPyrBlock][kPyrBlock][3];
    pyramid_block(a, blockIdx.x, blockIdx.y, buf);
}

// The pyramids of many frames in one launch: CTA b works on frame f (the last with cta_base <= b), block
// b - cta_base of its level-1 block grid (bx blocks per row).
__global__ __launch_bounds__(256) void k_pyramid_tab(const PyrArgs* __restrict__ tab, int n) {
    grid_dependency_sync();
    __shared__ uint8_t buf[2][kPyrBlock][kPyrBlock][3];
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab[mid].cta_base <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const PyrArgs& a = tab[lo];
    const int b = (int)blockIdx.x - a.cta_base;
    pyramid_block(a, b % a.bx, b / a.bx, buf);
}

int pyramid_blocks_x(int w1) { return (w1 + kPyrBlock - 1) / kPyrBlock; }
int pyramid_blocks(int w1, int h1) { return pyramid_blocks_x(w1) * ((h1 + kPyrBlock - 1) / kPyrBlock); }

void launch_pyramid(const PyrArgs& a, cudaStream_t st) {
    dim3 grid((a.w[1] + kPyrBlock - 1) / kPyrBlock, (a.h[1] + kPyrBlock - 1) / kPyrBlock);
    launch_k(k_pyramid, grid, dim3(256), 0, st, a);
}

void launch_pyramid_tab(const PyrArgs* tab_dev, int n, int total_ctas, cudaStream_t st) {
    launch_k(k_pyramid_tab, dim3(total_ctas), dim3(256), 0, st, tab_dev, n);
}

// Walsh-Hadamard descriptor (Sec. 3.1): for every pixel and channel, the 4x4 lowest-sequency coefficients of
// the 8x8 patch over rows y-3..y+4, columns x-3..x+4 (edge pixels repeated), unnormalised.  The length-8
// sequency-ordered Walsh functions are sums of the pair sums s01, s23, s45, s67 with signs
//   W0 = + + + +,  W1 = + + - -,  W2 = + - - +,  W3 = + - + -
// so the transform is separable: a row pass (4 outputs per patch row) then a column pass.
// CTA = 32x16 output pixels: its 39x23 input window (clamped halo) is staged in shared memory, the row pass is
// computed once per (window row, output column, channel) into shared memory (|value| <= 8*255 fits int16), and
// the column pass slides down each column (per channel, half a tile at a time).  Coefficients are stored in
// offset binary (C ^ 0x8000), the form the SAD of the propagation kernels works on.
constexpr int kWtx = 32, kWty = 16;
constexpr int kWinX = kWtx + 8, kWinY = kWty + 7;  // 39 window columns used, one more keeps rows word-aligned

// One 32-byte sector with a single 256-bit store (the sector of a descriptor a thread writes).
__device__ __forceinline__ void st_sector(void* p, const uint32_t (&v)[8]) {
    asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(v[0]), "r"(v[1]), "r"(v[2]),
                 "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

__device__ __forceinline__ void walsh4(int a0, int a1, int a2, int a3, int a4, int a5, int a6, int a7, int& c0,
                                       int& c1, int& c2, int& c3) {
    int s01 = a0 + a1, s23 = a2 + a3, s45 = a4 + a5, s67 = a6 + a7;
    int p = s01 + s23, q = s45 + s67, r = s01 - s23, t = s45 - s67;
    c0 = p + q;  // + + + + + + + +
    c1 = p - q;  // + + + + - - - -
    c2 = r - t;  // + + - - - - + +
    c3 = r + t;  // + + - - + + - -
}

// Census pattern (Sec. 3.1, Census cost) of the output pixel at (lx, ly) of the tile from the same clamped input
// window: the 7x7 neighbourhood is window rows ly..ly+6, columns lx..lx+6 (the WHT window reaches one row and
// column further).  Bit k of channel c: the k-th neighbour in row-major order, centre skipped, is strictly
// darker than the centre.  Written as 8 words: (low, high) 32 bits of channels 0, 1, 2, then two zero words.
// Per window row, the eight bytes at columns lx..lx+7 come from three aligned words and two funnel shifts; a
// per-byte compare against the replicated centre gives 0xff / 0x00 bytes, and one multiply gathers the four
// byte flags of a word into four adjacent bits (flag bits 0, 8, 16, 24 land on 28..31, every cross product
// on a distinct lower bit, so nothing carries).
__device__ __forceinline__ uint32_t darker_bits4(uint32_t v, uint32_t centre4) {
    return ((__vcmpltu4(v, centre4) & 0x01010101u) * 0x10204080u) >> 28;
}

__device__ __forceinline__ void census_pixel(const uint8_t (&win)[3][kWinY][kWinX], int lx, int ly,
                                             uint32_t* __restrict__ dst) {
    uint32_t w[6];
    const int wx = lx >> 2, sh = 8 * (lx & 3);
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        const uint32_t centre4 = (uint32_t)win[ch][ly + 3][lx + 3] * 0x01010101u;
        unsigned long long bits = 0;
#pragma unroll
        for (int r = 0; r < 7; r++) {
            const uint32_t* row = reinterpret_cast<const uint32_t*>(&win[ch][ly + r][0]);
            const uint32_t a = row[wx], b = row[wx + 1], c = row[wx + 2];
            const uint32_t m = darker_bits4(__funnelshift_r(a, b, sh), centre4) |
                               (darker_bits4(__funnelshift_r(b, c, sh), centre4) << 4);  // columns lx..lx+7
            if (r < 3) bits |= (unsigned long long)(m & 0x7fu) << (7 * r);
            else if (r == 3) bits |= (unsigned long long)((m & 0x7u) | ((m >> 1) & 0x38u)) << 21;
            else bits |= (unsigned long long)(m & 0x7fu) << (7 * r - 1);
        }
        w[2 * ch] = (uint32_t)bits;
        w[2 * ch + 1] = (uint32_t)(bits >> 32);
    }
    const uint32_t sec[8] = {w[0], w[1], w[2], w[3], w[4], w[5], 0u, 0u};
    st_sector(dst, sec);
}

// The initial-matching descriptors of a coarsest-level pixel (row p = y*w + x), from its stored coefficient
// words: 8-bit C >> 7 (floor, in [-128, 127]) zero-padded to 64 with its squared norm, and the same values as
// f16 (exact) for the tensor-core seed.  Padding rows past the level's pixel count stay zero from allocation.
__device__ __forceinline__ void seed_rows(const uint32_t (&out)[24], int p, const WhtLevel& L) {
    uint32_t w8[16], w16[32];
    int norm = 0;
#pragma unroll
    for (int k = 0; k < 24; k++) {
        const int q0 = feature_coef((int16_t)(out[k] & 0xffffu)) >> 7;
        const int q1 = feature_coef((int16_t)(out[k] >> 16)) >> 7;
        norm += q0 * q0 + q1 * q1;
        const uint32_t pair8 = (uint32_t)(q0 & 0xff) | ((uint32_t)(q1 & 0xff) << 8);
        if (k & 1) w8[k >> 1] |= pair8 << 16;
        else w8[k >> 1] = pair8;
        const __half2 h = __halves2half2(__int2half_rn(q0), __int2half_rn(q1));
        w16[k] = *reinterpret_cast<const uint32_t*>(&h);
    }
#pragma unroll
    for (int k = 12; k < 16; k++) w8[k] = 0u;
#pragma unroll
    for (int k = 24; k < 32; k++) w16[k] = 0u;
    uint4* d8 = reinterpret_cast<uint4*>(L.seed_desc + (size_t)p * kSeedK);
#pragma unroll
    for (int k = 0; k < 4; k++) d8[k] = make_uint4(w8[4 * k], w8[4 * k + 1], w8[4 * k + 2], w8[4 * k + 3]);
    uint4* d16 = reinterpret_cast<uint4*>(static_cast<char*>(L.desc16) + (size_t)p * kSeedK * 2);
#pragma unroll
    for (int k = 0; k < 8; k++) d16[k] = make_uint4(w16[4 * k], w16[4 * k + 1], w16[4 * k + 2], w16[4 * k + 3]);
    L.seed_norm[p] = norm;
}

// One 32x16 tile t of one level (shared memory: the clamped input window and the row pass).
__device__ __forceinline__ void wht_tile(const WhtLevel& L, int t, uint8_t (&win)[3][kWinY][kWinX],
                                         short4 (&rowt)[3][kWinY][kWtx]) {
    int tx0 = (t % L.tiles_x) * kWtx, ty0 = (t / L.tiles_x) * kWty;
    for (int i = threadIdx.x; i < kWinX * kWinY; i += blockDim.x) {
        int r = i / kWinX, c = i - r * kWinX;
        int gy = min(max(ty0 - 3 + r, 0), L.h - 1);
        int gx = min(max(tx0 - 3 + c, 0), L.w - 1);
        if (!idx_ok(g_bounds, kBoundsImage, (long long)gy * L.w + gx, (long long)L.w * L.h)) gy = gx = 0;
        const uint8_t* px = L.img + (size_t)gy * L.pitch + gx * 3;
        win[0][r][c] = px[0];
        win[1][r][c] = px[1];
        win[2][r][c] = px[2];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * kWinY * kWtx; i += blockDim.x) {
        const int ch = i / (kWinY * kWtx), rem = i - ch * kWinY * kWtx, r = rem / kWtx, c = rem - r * kWtx;
        // bytes c..c+7 of the window row from three aligned words
        const uint32_t* rw = reinterpret_cast<const uint32_t*>(&win[ch][r][0]) + (c >> 2);
        if (!idx_ok(g_bounds, kBoundsWin, (c >> 2) + 2, kWinX / 4)) continue;
        const uint32_t sh = 8u * (uint32_t)(c & 3);
        const uint32_t lo = __funnelshift_r(rw[0], rw[1], sh), hi = __funnelshift_r(rw[1], rw[2], sh);
        int v0, v1, v2, v3;
        walsh4(lo & 0xff, (lo >> 8) & 0xff, (lo >> 16) & 0xff, lo >> 24, hi & 0xff, (hi >> 8) & 0xff,
               (hi >> 16) & 0xff, hi >> 24, v0, v1, v2, v3);
        rowt[ch][r][c] = make_short4((short)v0, (short)v1, (short)v2, (short)v3);
    }
    __syncthreads();
    // Column pass: one thread per (channel, output column, half of the tile's rows) slides down 8 output rows,
    // loading each row-pass value once (15 per 8 outputs) and writing the channel's 32-B sector of each pixel.
    for (int i = threadIdx.x; i < 3 * kWtx * 2; i += blockDim.x) {
        const int col = i % kWtx, rest = i / kWtx, seg = rest & 1, ch = rest >> 1;
        const int x = tx0 + col;
        if (x >= L.w) continue;
        if (!idx_ok(g_bounds, kBoundsRowt, seg * (kWty / 2) + kWty / 2 + 6, kWinY)) continue;
        short4 R[kWty / 2 + 7];
#pragma unroll
        for (int k = 0; k < kWty / 2 + 7; k++) R[k] = rowt[ch][seg * (kWty / 2) + k][col];
#pragma unroll
        for (int rr = 0; rr < kWty / 2; rr++) {
            const int y = ty0 + seg * (kWty / 2) + rr;
            if (y >= L.h) break;
            int C[4][4];
            walsh4(R[rr].x, R[rr + 1].x, R[rr + 2].x, R[rr + 3].x, R[rr + 4].x, R[rr + 5].x, R[rr + 6].x, R[rr + 7].x,
                   C[0][0], C[1][0], C[2][0], C[3][0]);
            walsh4(R[rr].y, R[rr + 1].y, R[rr + 2].y, R[rr + 3].y, R[rr + 4].y, R[rr + 5].y, R[rr + 6].y, R[rr + 7].y,
                   C[0][1], C[1][1], C[2][1], C[3][1]);
            walsh4(R[rr].z, R[rr + 1].z, R[rr + 2].z, R[rr + 3].z, R[rr + 4].z, R[rr + 5].z, R[rr + 6].z, R[rr + 7].z,
                   C[0][2], C[1][2], C[2][2], C[3][2]);
            walsh4(R[rr].w, R[rr + 1].w, R[rr + 2].w, R[rr + 3].w, R[rr + 4].w, R[rr + 5].w, R[rr + 6].w, R[rr + 7].w,
                   C[0][3], C[1][3], C[2][3], C[3][3]);
            uint32_t out[8];
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int v = 0; v < 4; v += 2)
                    out[u * 2 + v / 2] =
                        ((uint32_t)(C[u][v] & 0xffff) | ((uint32_t)C[u][v + 1] << 16)) ^ 0x80008000u;  // offset binary
            if (!idx_ok(g_bounds, kBoundsFeat, feat_index(x, y, L.w), (long long)L.w * L.h)) continue;
            st_sector(L.feat + (size_t)feat_index(x, y, L.w) * kNF + ch * 16, out);
        }
    }
    if (!L.census && !L.seed_desc) return;
    __syncthreads();  // the tile's descriptors written above are visible to the whole CTA
    const int lx = threadIdx.x % kWtx;
    for (int ly = threadIdx.x / kWtx; ly < kWty; ly += blockDim.x / kWtx) {
        const int x = tx0 + lx, y = ty0 + ly;
        if (x >= L.w || y >= L.h) continue;
        if (!idx_ok(g_bounds, kBoundsCensus, ly + 6, kWinY) || !idx_ok(g_bounds, kBoundsCensus, (lx >> 2) + 2, kWinX / 4))
            continue;
        if (L.census) census_pixel(win, lx, ly, L.census + (size_t)feat_index(x, y, L.w) * (kCensusBytes / 4));
        if (L.seed_desc && idx_ok(g_bounds, kBoundsSeed, y * L.w + x, (long long)L.w * L.h)) {
            uint32_t out[24];
            const uint4* src = reinterpret_cast<const uint4*>(L.feat + (size_t)feat_index(x, y, L.w) * kNF);
#pragma unroll
            for (int k = 0; k < 6; k++) {
                const uint4 v = src[k];
                out[4 * k] = v.x;
                out[4 * k + 1] = v.y;
                out[4 * k + 2] = v.z;
                out[4 * k + 3] = v.w;
            }
            seed_rows(out, y * L.w + x, L);
        }
    }
}

__global__ __launch_bounds__(256) void k_wht(WhtArgs args) {
    grid_dependency_sync();
    __shared__ __align__(16) uint8_t win[3][kWinY][kWinX];
    __shared__ short4 rowt[3][kWinY][kWtx];  // row pass: 4 horizontal Walsh sums per window row and output column
    int b = blockIdx.x, li = 0;
    while (li + 1 < args.n && b >= args.lv[li + 1].tile_base) li++;
    const WhtLevel L = args.lv[li];
    wht_tile(L, b - L.tile_base, win, rowt);
}

// The levels of many frames in one launch: CTA b works on entry e (the last with tile_base <= b).
__global__ __launch_bounds__(256) void k_wht_tab(const WhtLevel* __restrict__ tab, int n) {
    grid_dependency_sync();
    __shared__ __align__(16) uint8_t win[3][kWinY][kWinX];
    __shared__ short4 rowt[3][kWinY][kWtx];
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab[mid].tile_base <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const WhtLevel L = tab[lo];
    wht_tile(L, (int)blockIdx.x - L.tile_base, win, rowt);
}

int wht_tiles_x(int w) { return (w + kWtx - 1) / kWtx; }
int wht_tiles(int w, int h) { return wht_tiles_x(w) * ((h + kWty - 1) / kWty); }

void launch_wht(const WhtArgs& a, int total_tiles, cudaStream_t st) {
    launch_k(k_wht, dim3(total_tiles), dim3(256), 0, st, a);
}

const void* wht_tab_kernel() { return reinterpret_cast<const void*>(k_wht_tab); }

void launch_wht_tab(const WhtLevel* tab_dev, int n, int total_tiles, cudaStream_t st, bool after_kernel) {
    if (after_kernel)
        launch_k(k_wht_tab, dim3(total_tiles), dim3(256), 0, st, tab_dev, n);
    else  // after an event wait: an ordinary launch (no programmatic dependency on an earlier kernel)
        k_wht_tab<<<total_tiles, 256, 0, st>>>(tab_dev, n);
}

}  // namespace ff
