// filter.cu -- outlier filtering of the matches (FlowFields++, arXiv 1805.03517, Sec. 3.1; eps and s in Table 3):
// the forward/backward consistency check (with one or two inverse fields) and the 3x3 sparsification.
#include "ff_internal.h"

namespace ff {

__device__ __forceinline__ int flow_x(uint32_t f) { return (int)(int16_t)(f & 0xffffu); }
__device__ __forceinline__ int flow_y(uint32_t f) { return ((int)f) >> 16; }
__device__ __forceinline__ bool in_level(int x, int y, int w, int h) {
    return (unsigned)x < (unsigned)w && (unsigned)y < (unsigned)h;
}

// Sparsification (Sec. 3.1; s in Table 3): per 3x3 block (tiling from (0, 0), partial blocks at the edges)
// holding at least s consistent matches, keep the one with the lowest squared consistency error (first in
// row-major order on ties).  A match counts only where the filter mask `keep` (may be null) is set.  One
// thread per block.
__global__ void k_sparsify(const uint32_t* __restrict__ fwd, const uint32_t* __restrict__ bwd,
                           const uint8_t* __restrict__ keep, int w, int h, int eps, int s, uint8_t* __restrict__ out) {
    grid_dependency_sync();
    const int bx = blockIdx.x * blockDim.x + threadIdx.x, by = blockIdx.y;
    if (3 * bx >= w) return;
    const int x0 = 3 * bx, y0 = 3 * by, x1 = min(x0 + 3, w), y1 = min(y0 + 3, h);
    int count = 0, best_p = -1;
    long long best_e = 0;
    for (int y = y0; y < y1; y++)
        for (int x = x0; x < x1; x++) {
            if (keep && !keep[y * w + x]) continue;
            const uint32_t f = fwd[y * w + x];
            const int fx = flow_x(f), fy = flow_y(f), qx = x + fx, qy = y + fy;
            if (!in_level(qx, qy, w, h)) continue;
            const uint32_t b = bwd[qy * w + qx];
            const long long ex = fx + flow_x(b), ey = fy + flow_y(b), e = ex * ex + ey * ey;
            if (e > (long long)eps * eps) continue;
            count++;
            if (best_p < 0 || e < best_e) {
                best_p = y * w + x;
                best_e = e;
            }
        }
    for (int y = y0; y < y1; y++)
        for (int x = x0; x < x1; x++) out[y * w + x] = (count >= s && y * w + x == best_p) ? 1 : 0;
}

void launch_sparsify(const uint32_t* fwd, const uint32_t* bwd, const uint8_t* keep, int w, int h, int eps, int s,
                     uint8_t* out, cudaStream_t st) {
    const int nbx = (w + 2) / 3, nby = (h + 2) / 3;
    dim3 grid((nbx + 127) / 128, nby);
    launch_k(k_sparsify, grid, dim3(128), 0, st, fwd, bwd, keep, w, h, eps, s, out);
}

// ---------------------------------------------------------------------------------------------------------
// forward/backward consistency (Sec. 3.1; eps in Table 3): keep p iff q = p + f(p) is inside the image and
// (f_x(p) + b_x(q))^2 + (f_y(p) + b_y(q))^2 <= eps^2; with a second inverse field b2, the same must hold for it.

__device__ __forceinline__ bool consistent(uint32_t f, const uint32_t* __restrict__ bwd, int x, int y, int w, int h,
                                           int eps) {
    const int fx = flow_x(f), fy = flow_y(f), qx = x + fx, qy = y + fy;
    if (!in_level(qx, qy, w, h)) return false;
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

}  // namespace ff
