/*
 * ff_oracle.h -- plain CPU oracle of the Flow Fields dense-matching stage of FlowFields++
 * (Schuster et al., "FlowFields++: Accurate Optical Flow Correspondences Meet Robust Interpolation",
 * arXiv 1805.03517, Sec. 3 and Sec. 3.1 "Matches").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call this code: only the
 * test-suite, the smoke check and the CPU-baseline leg of the benchmark do.  It shares no source,
 * header, table or helper with the CUDA library; it is single-threaded, unblocked and written to be
 * read against the paper.
 *
 * All arithmetic is integer; results are exact, so "parity" with the GPU path means bit-for-bit equal.
 *
 * Layouts (row-major, pixel (x, y) at index y*w + x):
 *   image    uint8 [h][w][3]    RGB
 *   features int16 [h][w][48]   channel c (R=0,G=1,B=2), Walsh row index u, column index v at c*16 + u*4 + v
 *   flow     int16 [h][w][2]    (dx, dy), integer pixel displacement at the flow's own scale
 *   cost     int32 [h][w]       patch SAD of the pixel's current flow
 *   mask     uint8 [h][w]       1 = consistent (inlier)
 *   census   uint64 [h][w][3]   48-bit Census pattern per colour channel
 */
#ifndef FF_ORACLE_H
#define FF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FFO_NF 48 /* 3 channels x 16 Walsh-Hadamard coefficients */

typedef struct {
    int n_scales;  /* pyramid levels L >= 1 (level 0 = full resolution) */
    int iters;     /* propagation iterations T per level */
    int rs_radius; /* random-search radius R: offsets drawn uniformly from [-R, R] per component */
    int eps;       /* consistency threshold in pixels */
    uint32_t seed; /* random-search hash seed */
    int cost;      /* 0: SAD of the WHT descriptors, 1: Hamming distance of the Census patterns */
    int sub_scales; /* 0: none; 1: sub-scales; 2: sub-scales and sub-sub-scales (grids of every 2nd / 4th pixel) */
} ffo_params;

/* 0 on success; negative on an argument error or a broken internal assertion. */
int ffo_level_dims(int w, int h, int n_scales, int* ws, int* hs);
void ffo_downsample(const uint8_t* src, int w, int h, uint8_t* dst);
void ffo_wht(const uint8_t* img, int w, int h, int16_t* feat);
void ffo_census(const uint8_t* img, int w, int h, uint64_t* desc);
int32_t ffo_hamming(const uint64_t* ca, const uint64_t* cb, int w, int h, int x, int y, int fx, int fy);
long ffo_propagate_census(const uint64_t* ca, const uint64_t* cb, int w, int h, int16_t* flow, int32_t* cost,
                          int iters, int rs_radius, uint32_t seed, int dir, int level, long max_halfsweeps);
int ffo_match_dir_census(const int16_t* const* feat_a, const int16_t* const* feat_b, const uint64_t* const* cen_a,
                         const uint64_t* const* cen_b, const int* ws, const int* hs, const ffo_params* prm, int dir,
                         int16_t* flow, int32_t* cost);
uint32_t ffo_mix32(uint32_t x);
uint32_t ffo_hash(uint32_t seed, int dir, int level, int t, int d, int x, int y, int comp);
int32_t ffo_sad(const int16_t* fa, const int16_t* fb, int w, int h, int x, int y, int fx, int fy);
void ffo_seed(const int16_t* fa, const int16_t* fb, int w, int h, int16_t* flow, int32_t* dist);
void ffo_init_cost(const int16_t* fa, const int16_t* fb, int w, int h, const int16_t* flow, int32_t* cost);
int ffo_upsample(const int16_t* fa, const int16_t* fb, int w, int h, const int16_t* flow_coarse, int wc, int hc,
                 int16_t* flow, int32_t* cost);
long ffo_propagate(const int16_t* fa, const int16_t* fb, int w, int h, int16_t* flow, int32_t* cost, int iters,
                   int rs_radius, uint32_t seed, int dir, int level, long max_halfsweeps);
int ffo_upsample_grid(const int16_t* fa, const int16_t* fb, int w, int h, int g, const int16_t* flow_coarse, int wc,
                      int hc, int16_t* flow, int32_t* cost);
void ffo_grid_handover(const int16_t* fa, const int16_t* fb, int w, int h, int g, const int16_t* flow_parent, int pw,
                       int ph, int16_t* flow, int32_t* cost);
long ffo_propagate_grid(const int16_t* fa, const int16_t* fb, int w, int h, int g, int16_t* flow, int32_t* cost,
                        int iters, int rs_radius, uint32_t seed, int dir, int stream, long max_halfsweeps);
int ffo_match_dir(const int16_t* const* feat_a, const int16_t* const* feat_b, const int* ws, const int* hs,
                  const ffo_params* prm, int dir, int16_t* flow, int32_t* cost);
void ffo_consistency(const int16_t* fwd, const int16_t* bwd, int w, int h, int eps, uint8_t* mask);
int ffo_match_bidir2(const uint8_t* rgb_a, const uint8_t* rgb_b, int w, int h, const ffo_params* prm, int rs_radius2,
                     int16_t* flow_fwd, int16_t* flow_bwd, int16_t* flow_bwd2, uint8_t* mask);
void ffo_sparsify(const int16_t* fwd, const int16_t* bwd, const uint8_t* keep, int w, int h, int eps, int s,
                  uint8_t* out);
int ffo_match_bidir(const uint8_t* rgb_a, const uint8_t* rgb_b, int w, int h, const ffo_params* prm,
                    int16_t* flow_fwd, int16_t* flow_bwd, int32_t* cost_fwd, int32_t* cost_bwd, uint8_t* mask);

#ifdef __cplusplus
}
#endif
#endif
