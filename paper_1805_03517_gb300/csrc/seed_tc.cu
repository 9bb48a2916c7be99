// seed_tc.cu -- initial matches at the coarsest level on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// FlowFields++ (arXiv 1805.03517, Sec. 3.1) matches the coarsest level's Walsh-Hadamard descriptors with
// kD-trees; here the exact nearest neighbour, q* = argmin_q |a_p - b_q|^2 = argmin_q (|b_q|^2 - 2 a_p.b_q),
// ties to the smallest q.  The dot products form a dense contraction A.B^T with K = 48 (padded to 64).
//
// tcgen05.mma has no 8-bit integer kind on sm_103a, so the 8-bit descriptor values (C >> 7, in [-128, 127])
// are stored as f16, which represents them exactly; every product (|.| <= 2^14) and every partial sum
// (|.| <= 48 * 2^14 < 2^24) is an integer that f32 represents exactly, so the f32 accumulators in tensor memory
// hold the exact integer dot products and the argmin is the same as in integer arithmetic.
//
// One CTA (4 warps) computes a 128 x 256 block of scores: TMA loads the 128 source rows and 256 target rows
// (K-major, 128-byte rows, 128-byte swizzle) into shared memory, one thread issues four K=16 MMAs into a
// 128 x 256 f32 accumulator in TMEM, and each warp reads its 32 rows back with tcgen05.ld, forms
// score = |b|^2 - 2 a.b and keeps the per-row minimum; blocks of the same rows merge through a 64-bit atomicMin
// on (score + 2^31) << 32 | q, which orders by score and then by the smaller index.  Every mbarrier wait is
// bounded: on expiry the CTA records an error code, waits (bounded) for its own copies and MMAs, frees its
// tensor memory and returns.
#include <cuda.h>
#include <cuda_fp16.h>

#include <climits>

#include "ff_internal.h"

namespace ff {

namespace {

constexpr int kTcRows = 128;         // MMA M: source rows per CTA
constexpr int kTcCols = 256;         // MMA N: target rows per CTA
constexpr int kTcK = 64;             // padded descriptor length (f16)
constexpr int kRowBytes = kTcK * 2;  // 128 B per descriptor row
constexpr uint32_t kABytes = kTcRows * kRowBytes;   // 16 KB
constexpr uint32_t kBBytes = kTcCols * kRowBytes;   // 32 KB
constexpr int kTmemCols = 256;

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms of 1024 B (stride-dimension offset).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);     // start address
    d |= (uint64_t)1 << 16;                       // leading-dimension offset (unused with 128-byte swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;             // stride-dimension offset: next 8-row group
    d |= (uint64_t)1 << 46;                       // descriptor version
    d |= (uint64_t)2 << 61;                       // swizzle: 128 B
    return d;
}

// Instruction descriptor of kind::f16: f32 accumulator, f16 A and B, both K-major, N = 256, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(kTcCols >> 3) << 17) |
                            ((uint32_t)(kTcRows >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
        "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace

constexpr size_t kSeedTcSmem = 1024 /*alignment slack*/ + kABytes + kBBytes + kTcCols * 4 + 64 + 30 * 1024;

// probs[i] covers CTAs [cta_base, cta_base + row_tiles * col_tiles).
__global__ __launch_bounds__(128) void k_seed_tc(const SeedTcProblem* __restrict__ probs, int n_probs,
                                                 uint32_t wait_limit, int withhold, int* __restrict__ err) {
    grid_dependency_sync();
    extern __shared__ uint8_t smem_raw[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int pi = 0;
    while (pi + 1 < n_probs && (int)blockIdx.x >= probs[pi + 1].cta_base) pi++;
    const SeedTcProblem& P = probs[pi];
    const CUtensorMap* map_a = reinterpret_cast<const CUtensorMap*>(P.map_a);
    const CUtensorMap* map_b = reinterpret_cast<const CUtensorMap*>(P.map_b);
    const int local = blockIdx.x - P.cta_base;
    const int r0 = (local / P.col_tiles) * kTcRows, c0 = (local % P.col_tiles) * kTcCols;

    // 1024-byte aligned tiles (128-byte swizzle atoms), then norms, barriers and the TMEM address
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - smem_u32(smem_raw));
    const uint32_t sA = base, sB = base + kABytes;
    int* s_norm = reinterpret_cast<int*>(gbase + kABytes + kBBytes);
    uint64_t* s_bar = reinterpret_cast<uint64_t*>(gbase + kABytes + kBBytes + kTcCols * 4);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(s_bar + 2);
    const uint32_t bar_load = smem_u32(&s_bar[0]), bar_mma = smem_u32(&s_bar[1]);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(bar_load, 1);
        mbar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    for (int c = tid; c < kTcCols; c += blockDim.x) s_norm[c] = c0 + c < P.n ? P.normB[c0 + c] : 0;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *s_tmem;

    bool loaded = true, done = true;
    if (tid == 0) {
        mbar_expect_tx(bar_load, kABytes + kBBytes);
        if (!withhold) {  // withhold (a test of the bounded waits): the load barrier can never complete
            tma_load_2d(sA, map_a, 0, r0, bar_load);
            tma_load_2d(sB, map_b, 0, c0, bar_load);
            tma_load_2d(sB + kBBytes / 2, map_b, 0, c0 + kTcCols / 2, bar_load);
        }
        loaded = mbar_wait(bar_load, 0, wait_limit);
        if (loaded) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int k = 0; k < kTcK / 16; k++)  // K = 16 f16 = 32 bytes per MMA inside the swizzle atom
                mma_f16(tmem, smem_desc_sw128(sA + 32 * k), smem_desc_sw128(sB + 32 * k), k > 0);
            mma_commit(bar_mma);
        } else {
            atomicExch(err, 1);                       // the copies did not arrive in time
            mbar_wait(bar_load, 0, 4 * wait_limit);   // bounded drain of the copies still in flight
        }
    }
    __syncthreads();
    if (tid == 0) s_tmem[1] = loaded ? 1u : 0u;
    __syncthreads();
    loaded = s_tmem[1] != 0;
    if (loaded) {
        done = __syncthreads_and(mbar_wait(bar_mma, 0, wait_limit)) != 0;
        if (!done && tid == 0) atomicExch(err, 2);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (loaded && done) {
        const int row = r0 + warp * 32 + lane;
        int best = INT_MAX, bidx = 0;
#pragma unroll 1
        for (int ch = 0; ch < kTcCols / 32; ch++) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ch * 32), v);
#pragma unroll
            for (int e = 0; e < 32; e++) {
                const int col = c0 + ch * 32 + e;
                const int dot = __float2int_rn(__uint_as_float(v[e]));
                const int s = s_norm[ch * 32 + e] - 2 * dot;
                if (col < P.n && s < best) {
                    best = s;
                    bidx = col;
                }
            }
        }
        if (row < P.n && best != INT_MAX) {
            const unsigned long long key =
                ((unsigned long long)((uint32_t)best ^ 0x80000000u) << 32) | (unsigned long long)(uint32_t)bidx;
            atomicMin(P.keys + row, key);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (loaded && !done && tid == 0) mbar_wait(bar_mma, 0, 4 * wait_limit);  // let the MMAs drain before freeing
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// keys -> packed flow q - p and squared distance |a_p|^2 + min score.
__global__ void k_seed_finish(const SeedTcProblem* __restrict__ probs, int n_probs, int64_t total) {
    grid_dependency_sync();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_probs - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (probs[mid].pix_base <= i) lo = mid; else hi = mid - 1;
        }
        const SeedTcProblem& P = probs[lo];
        const int p = (int)(i - P.pix_base);
        const unsigned long long key = P.keys[p];
        const int q = (int)(uint32_t)(key & 0xffffffffu);
        const int best = (int)((uint32_t)(key >> 32) ^ 0x80000000u);
        const int dx = q % P.w - p % P.w, dy = q / P.w - p / P.w;
        P.flow[p] = (uint32_t)(dx & 0xffff) | ((uint32_t)dy << 16);
        if (P.dist) P.dist[p] = P.normA[p] + best;
    }
}

cudaError_t seed_tc_init_attributes() {
    return cudaFuncSetAttribute(k_seed_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSeedTcSmem);
}

void launch_seed_tc(const SeedTcProblem* probs_dev, int n_probs, int total_ctas, int64_t total_pix, uint32_t wait_limit,
                    int withhold, int* err_dev, cudaStream_t st) {
    launch_k(k_seed_tc, dim3(total_ctas), dim3(128), kSeedTcSmem, st, probs_dev, n_probs, wait_limit, withhold, err_dev);
    int64_t blocks = (total_pix + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    launch_k(k_seed_finish, dim3((int)(blocks < 1 ? 1 : blocks)), dim3(256), 0, st, probs_dev, n_probs, total_pix);
}

// Tensor map of a [n_pad][64] f16 descriptor array: boxes of 64 x 128 (one 128-byte row per descriptor),
// 128-byte swizzle, rows past n_pad read as zeros.
bool seed_tc_encode_map(void* map_out, const void* desc16_dev, int n_pad) {
    using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeFn encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return false;
        }
        encode = reinterpret_cast<EncodeFn>(fn);
    }
    cuuint64_t dims[2] = {(cuuint64_t)kTcK, (cuuint64_t)n_pad};
    cuuint64_t strides[1] = {(cuuint64_t)kRowBytes};
    cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)kTcRows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                        const_cast<void*>(desc16_dev), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace ff
