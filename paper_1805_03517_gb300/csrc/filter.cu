// filter.cu -- outlier filtering of the matches (FlowFields++, arXiv 1805.03517, Sec. 3.1; eps and s in Table 3):
// the forward/backward consistency check (with one or two inverse fields) and the 3x3 sparsification.
#include "ff_internal.h"

namespace ff {

// first index violation of a debug-bounds build (see idx_ok): code, index, limit
static __device__ int g_bounds[4];
enum : int { kBoundsBwd = 20, kBoundsSparseBwd, kBoundsSparseKey };

cudaError_t bounds_take_filter(int rec[3]) {
    int h[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyFromSymbol(h, g_bounds, sizeof h);
    if (e == cudaSuccess && h[0] != 0) {
        const int z[4] = {0, 0, 0, 0};
        e = cudaMemcpyToSymbol(g_bounds, z, sizeof z);
    }
    rec[0] = h[0], rec[1] = h[1], rec[2] = h[2];
    return e;
}

__device__ __forceinline__ int flow_x(uint32_t f) { return (int)(int16_t)(f & 0xffffu); }
__device__ __forceinline__ int flow_y(uint32_t f) { return ((int)f) >> 16; }
__device__ __forceinline__ bool in_level(int x, int y, int w, int h) {
    return (unsigned)x < (unsigned)w && (unsigned)y < (unsigned)h;
}

// Sparsification (Sec. 3.1; s in Table 3): per 3x3 block (tiling from (0, 0), partial blocks at the edges)
// holding at least s consistent matches, keep the one with the lowest squared consistency error (first in
// row-major order on ties).  A match counts only where the filter mask `keep` (may be null) is set.
// One thread per pixel: every pixel's loads are in flight at once.  A CTA covers 32 x 2 whole blocks; each pixel
// posts a key (error << 4 | its row-major index in the block, or ~0 if it does not count) to shared memory, and
// every pixel then reads its block's nine keys: the count, and whether its own key is the block's minimum.
constexpr int kSparsePx = 96, kSparsePy = 6;

__global__ void __launch_bounds__(kSparsePx* kSparsePy)
    k_sparsify(const uint32_t* __restrict__ fwd, const uint32_t* __restrict__ bwd, const uint8_t* __restrict__ keep,
               int w, int h, int eps, int s, uint8_t* __restrict__ out) {
    grid_dependency_sync();
    __shared__ unsigned long long key[kSparsePy][kSparsePx];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x = blockIdx.x * kSparsePx + tx, y = blockIdx.y * kSparsePy + ty;
    const bool inside = x < w && y < h;
    unsigned long long k = ~0ull;
    if (inside && (!keep || keep[y * w + x])) {
        const uint32_t f = fwd[y * w + x];
        const int fx = flow_x(f), fy = flow_y(f), qx = x + fx, qy = y + fy;
        if (in_level(qx, qy, w, h) && idx_ok(g_bounds, kBoundsSparseBwd, qy * w + qx, w * h)) {
            const uint32_t b = bwd[qy * w + qx];
            const long long ex = fx + flow_x(b), ey = fy + flow_y(b), e = ex * ex + ey * ey;
            if (e <= (long long)eps * eps) k = ((unsigned long long)e << 4) | (unsigned)((ty % 3) * 3 + tx % 3);
        }
    }
    key[ty][tx] = k;
    __syncthreads();
    if (!inside) return;
    const int bx0 = tx - tx % 3, by0 = ty - ty % 3;
    int count = 0;
    unsigned long long best = ~0ull;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            if (!idx_ok(g_bounds, kBoundsSparseKey, (by0 + i) * kSparsePx + bx0 + j, kSparsePx * kSparsePy)) continue;
            const unsigned long long kk = key[by0 + i][bx0 + j];
            count += kk != ~0ull;
            best = kk < best ? kk : best;
        }
    out[y * w + x] = (count >= s && k == best && k != ~0ull) ? 1 : 0;
}

void launch_sparsify(const uint32_t* fwd, const uint32_t* bwd, const uint8_t* keep, int w, int h, int eps, int s,
                     uint8_t* out, cudaStream_t st) {
    dim3 grid((w + kSparsePx - 1) / kSparsePx, (h + kSparsePy - 1) / kSparsePy);
    launch_k(k_sparsify, grid, dim3(kSparsePx, kSparsePy), 0, st, fwd, bwd, keep, w, h, eps, s, out);
}

// ---------------------------------------------------------------------------------------------------------
// forward/backward consistency (Sec. 3.1; eps in Table 3): keep p iff q = p + f(p) is inside the image and
// (f_x(p) + b_x(q))^2 + (f_y(p) + b_y(q))^2 <= eps^2; with a second inverse field b2, the same must hold for it.

__device__ __forceinline__ bool consistent(uint32_t f, const uint32_t* __restrict__ bwd, int x, int y, int w, int h,
                                           int eps) {
    const int fx = flow_x(f), fy = flow_y(f), qx = x + fx, qy = y + fy;
    if (!in_level(qx, qy, w, h) || !idx_ok(g_bounds, kBoundsBwd, qy * w + qx, w * h)) return false;
    const uint32_t b = bwd[qy * w + qx];
    const long long ex = fx + flow_x(b), ey = fy + flow_y(b);
    return ex * ex + ey * ey <= (long long)eps * eps;
}

__global__ void k_consistency(const uint32_t* __restrict__ fwd, const uint32_t* __restrict__ bwd,
                              const uint32_t* __restrict__ bwd2, int w, int h, int eps, uint8_t* __restrict__ mask) {
    grid_dependency_sync();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= w * h) return;
    const int x = i % w, y = i / w;
    const uint32_t f = fwd[i];
    bool ok = consistent(f, bwd, x, y, w, h, eps);
    if (bwd2) ok = ok && consistent(f, bwd2, x, y, w, h, eps);
    mask[i] = ok ? 1 : 0;
}

void launch_consistency(const uint32_t* fwd, const uint32_t* bwd, const uint32_t* bwd2, int w, int h, int eps,
                        uint8_t* mask, cudaStream_t st) {
    int n = w * h;
    launch_k(k_consistency, dim3((n + 255) / 256), dim3(256), 0, st, fwd, bwd, bwd2, w, h, eps, mask);
}

// Every pair of a batch in one grid-stride launch: pixel i belongs to the last pair with pix_base <= i.
__global__ void k_consistency_tab(const ConsProblem* __restrict__ probs, int n, int64_t total, int eps) {
    grid_dependency_sync();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (probs[mid].pix_base <= i) lo = mid; else hi = mid - 1;
        }
        const ConsProblem& P = probs[lo];
        const int p = (int)(i - P.pix_base);
        const int x = p % P.w, y = p / P.w;
        const uint32_t f = P.fwd[p];
        bool ok = consistent(f, P.bwd, x, y, P.w, P.h, eps);
        if (P.bwd2) ok = ok && consistent(f, P.bwd2, x, y, P.w, P.h, eps);
        P.mask[p] = ok ? 1 : 0;
    }
}

void launch_consistency_tab(const ConsProblem* probs_dev, int n, int64_t total_pix, int eps, cudaStream_t st) {
    int64_t blocks = (total_pix + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    launch_k(k_consistency_tab, dim3((int)blocks), dim3(256), 0, st, probs_dev, n, total_pix, eps);
}

}  // namespace ff
