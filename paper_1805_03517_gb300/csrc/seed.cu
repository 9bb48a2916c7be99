// seed.cu -- initial matches at the coarsest level (FlowFields++, arXiv 1805.03517, Sec. 3.1: the paper matches
// Walsh-Hadamard descriptors with kD-trees; here the exact nearest neighbour that a kD-tree approximates).
//
// For every source pixel p: q* = argmin_q |a_p - b_q|^2 over all target pixels q, ties to the smallest q.
// Since |a_p|^2 does not depend on q, q* = argmin_q (|b_q|^2 - 2 a_p.b_q): a dense 8-bit contraction A.B^T
// followed by an argmin epilogue, computed exactly in int32 on the tensor cores (m16n8k32 s8 x s8 -> s32).
// (tcgen05.mma has no 8-bit integer kind on sm_103a: ptxas rejects .kind::i8 for that target.)
#include <climits>

#include "ff_internal.h"

namespace ff {

__device__ __forceinline__ void mma_s8_16832(int (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void argmin_take(int& s, int& i, int s2, int i2) {
    if (s2 < s || (s2 == s && i2 < i)) {
        s = s2;
        i = i2;
    }
}

// One CTA of 8 warps per 16 source rows; warp k sweeps the target column tiles k, k+8, k+16, ... (8 columns
// each), so every thread still meets its columns in increasing order, then the 8 partial minima are reduced
// through shared memory (smaller index on equal score: the column slices are disjoint, so this keeps the
// first-index tie rule).  Fragment layout of m16n8k32 (8-bit): lane = 4*g + t; A regs {row g, row g+8} x
// {k 4t..4t+3, k 16+4t..}; B regs col g, k 4t.. and 16+4t..; C regs (row g, cols 2t, 2t+1), (row g+8, ...).
constexpr int kSeedWarps = 8;

__global__ __launch_bounds__(32 * kSeedWarps) void k_seed(const SeedProblem* __restrict__ probs, int n_probs,
                                                          int total_tiles) {
    grid_dependency_sync();
    __shared__ int s_best[kSeedWarps][16], s_idx[kSeedWarps][16];
    const int tile = blockIdx.x;
    int pi = 0;
    while (pi + 1 < n_probs && tile >= probs[pi + 1].warp_base) pi++;
    const SeedProblem P = probs[pi];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int r0 = (tile - P.warp_base) * 16;
    const uint32_t* A0 = reinterpret_cast<const uint32_t*>(P.A + (size_t)(r0 + g) * kSeedK);
    const uint32_t* A1 = reinterpret_cast<const uint32_t*>(P.A + (size_t)(r0 + g + 8) * kSeedK);
    uint32_t a[2][4];
#pragma unroll
    for (int kk = 0; kk < 2; kk++) {
        a[kk][0] = A0[kk * 8 + t];
        a[kk][1] = A1[kk * 8 + t];
        a[kk][2] = A0[kk * 8 + 4 + t];
        a[kk][3] = A1[kk * 8 + 4 + t];
    }
    int best0 = INT_MAX, best1 = INT_MAX, idx0 = 0, idx1 = 0;
    for (int n0 = warp * 8; n0 < P.n; n0 += 8 * kSeedWarps) {
        const uint32_t* Bq = reinterpret_cast<const uint32_t*>(P.B + (size_t)(n0 + g) * kSeedK);
        uint32_t b[2][2];
#pragma unroll
        for (int kk = 0; kk < 2; kk++) {
            b[kk][0] = Bq[kk * 8 + t];
            b[kk][1] = Bq[kk * 8 + 4 + t];
        }
        int c[4] = {0, 0, 0, 0};
        mma_s8_16832(c, a[0], b[0][0], b[0][1]);
        mma_s8_16832(c, a[1], b[1][0], b[1][1]);
        int col = n0 + 2 * t;
#pragma unroll
        for (int e = 0; e < 2; e++) {
            if (col + e < P.n) {
                int nb = P.normB[col + e];
                int s0 = nb - 2 * c[e], s1 = nb - 2 * c[2 + e];
                if (s0 < best0) { best0 = s0; idx0 = col + e; }
                if (s1 < best1) { best1 = s1; idx1 = col + e; }
            }
        }
    }
#pragma unroll
    for (int off = 1; off <= 2; off <<= 1) {
        int s = __shfl_xor_sync(0xffffffffu, best0, off), i = __shfl_xor_sync(0xffffffffu, idx0, off);
        argmin_take(best0, idx0, s, i);
        s = __shfl_xor_sync(0xffffffffu, best1, off);
        i = __shfl_xor_sync(0xffffffffu, idx1, off);
        argmin_take(best1, idx1, s, i);
    }
    if (t == 0) {
        s_best[warp][g] = best0;
        s_idx[warp][g] = idx0;
        s_best[warp][g + 8] = best1;
        s_idx[warp][g + 8] = idx1;
    }
    __syncthreads();
    if (threadIdx.x < 16) {
        const int r = threadIdx.x, p = r0 + r;
        int best = s_best[0][r], q = s_idx[0][r];
        for (int k = 1; k < kSeedWarps; k++) argmin_take(best, q, s_best[k][r], s_idx[k][r]);
        if (p < P.n) {
            int dx = q % P.w - p % P.w, dy = q / P.w - p / P.w;
            P.flow[p] = (uint32_t)(dx & 0xffff) | ((uint32_t)dy << 16);
            if (P.dist) P.dist[p] = P.normA[p] + best;
        }
    }
}

cudaError_t seed_load_kernel() {
    cudaFuncAttributes fa;
    return cudaFuncGetAttributes(&fa, k_seed);
}

void launch_seed(const SeedProblem* probs_dev, int n_probs, int total_row_tiles, cudaStream_t st) {
    launch_k(k_seed, dim3(total_row_tiles), dim3(32 * kSeedWarps), 0, st, probs_dev, n_probs, total_row_tiles);
}

}  // namespace ff
