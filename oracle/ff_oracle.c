/*
 * ff_oracle.c -- plain CPU oracle of the Flow Fields dense-matching stage of FlowFields++
 * (arXiv 1805.03517, Sec. 3 "Method" and Sec. 3.1 "Matches").
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU-baseline leg of the benchmark.
 * The product path never calls it.  It shares no code with the CUDA library.
 *
 * What it computes, step by step in the paper's order (Sec. 3.1):
 *   1. an image pyramid of both frames, matched from the coarsest level to the finest (Sec. 3);
 *   2. Walsh-Hadamard patch descriptors at every level (Sec. 3.1);
 *   3. initial matches at the lowest resolution (Sec. 3.1: kD-tree matching of the WHT descriptors; here an
 *      exact nearest-neighbour search, which the kD-tree approximates);
 *   4. per scale: i iterations of propagation towards the four quadrants; in every iteration, the last
 *      three propagation steps are each followed by a random search that perturbs both flow components by a
 *      small random amount (Sec. 3.1);
 *   5. an inverse flow field, and the consistency check that removes a match whose consistency error exceeds
 *      the threshold eps (Sec. 3.1; eps in Table 3).
 * The paper leaves the cost, descriptor size, filter, schedule and tie rules to cited work that is not
 * restated here; the readings taken are listed beside each function.  Parity of the end-to-end schedule is
 * pinned only through invariants (monotone cost, exact seed, exact translation recovery), since the paper
 * prints no matching output to compare with: for the composed stage (ffo_match_dir, ffo_match_bidir,
 * ffo_match_bidir2) parity is unpinned beyond those invariants; every step it composes is pinned on its own.
 */
#include "ff_oracle.h"

#include <limits.h>
#include <stdlib.h>
#include <string.h>

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
static int mini(int a, int b) { return a < b ? a : b; }

/* Level sizes of the image pyramid (Sec. 3): each level halves the previous one, rounding down,
 * never below 1 pixel.  Reading: the paper does not give the filter or odd-size rule. */
int ffo_level_dims(int w, int h, int n_scales, int* ws, int* hs) {
    if (w < 1 || h < 1 || n_scales < 1) return -1;
    ws[0] = w;
    hs[0] = h;
    for (int s = 1; s < n_scales; s++) {
        ws[s] = ws[s - 1] / 2 > 0 ? ws[s - 1] / 2 : 1;
        hs[s] = hs[s - 1] / 2 > 0 ? hs[s - 1] / 2 : 1;
    }
    return 0;
}

/* One pyramid step (Sec. 3).  Reading: 2x2 box average per channel, rounded half up,
 * source coordinates clamped to the image (only matters for a 1-pixel-wide or -high level). */
void ffo_downsample(const uint8_t* src, int w, int h, uint8_t* dst) {
    int w2 = w / 2 > 0 ? w / 2 : 1;
    int h2 = h / 2 > 0 ? h / 2 : 1;
    for (int y = 0; y < h2; y++) {
        for (int x = 0; x < w2; x++) {
            int x0 = mini(2 * x, w - 1), x1 = mini(2 * x + 1, w - 1);
            int y0 = mini(2 * y, h - 1), y1 = mini(2 * y + 1, h - 1);
            for (int c = 0; c < 3; c++) {
                int a = src[(y0 * w + x0) * 3 + c];
                int b = src[(y0 * w + x1) * 3 + c];
                int d = src[(y1 * w + x0) * 3 + c];
                int e = src[(y1 * w + x1) * 3 + c];
                dst[(y * w2 + x) * 3 + c] = (uint8_t)((a + b + d + e + 2) / 4);
            }
        }
    }
}

/* The four lowest-sequency Walsh functions of length 8, in sequency order (0, 1, 2, 3 sign changes). */
static const int WALSH8[4][8] = {
    {1, 1, 1, 1, 1, 1, 1, 1},
    {1, 1, 1, 1, -1, -1, -1, -1},
    {1, 1, -1, -1, -1, -1, 1, 1},
    {1, 1, -1, -1, 1, 1, -1, -1},
};

/* Walsh-Hadamard patch descriptor (Sec. 3.1).  Reading: for every pixel and colour channel, the 4x4
 * lowest-sequency coefficients of the 8x8 patch covering rows y-3..y+4 and columns x-3..x+4 (edge pixels
 * repeated), unnormalised:
 *     C_c[u][v](x, y) = sum_i sum_j W_u(i) W_v(j) I_c(clamp(x-3+j), clamp(y-3+i)),
 * u indexing the vertical (row) Walsh function and v the horizontal one. |C| <= 64*255 fits int16. */
void ffo_wht(const uint8_t* img, int w, int h, int16_t* feat) {
    for (int y = 0; y < h; y++) {
        for (int x = 0; x < w; x++) {
            int16_t* out = feat + ((long)y * w + x) * FFO_NF;
            for (int c = 0; c < 3; c++) {
                for (int u = 0; u < 4; u++) {
                    for (int v = 0; v < 4; v++) {
                        int acc = 0;
                        for (int i = 0; i < 8; i++) {
                            int yy = clampi(y - 3 + i, 0, h - 1);
                            for (int j = 0; j < 8; j++) {
                                int xx = clampi(x - 3 + j, 0, w - 1);
                                acc += WALSH8[u][i] * WALSH8[v][j] * img[((long)yy * w + xx) * 3 + c];
                            }
                        }
                        out[c * 16 + u * 4 + v] = (int16_t)acc;
                    }
                }
            }
        }
    }
}

/* 32-bit integer finaliser "lowbias32" (C. Wellons, hash-prospector, 2018): the counter-based generator
 * behind the random search.  The paper only asks for small random offsets (Sec. 3.1); a counter-based
 * hash makes the offsets independent of execution order. */
uint32_t ffo_mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

/* Random-search draw for pixel (x, y) at level `level`, iteration t, propagation direction d, flow
 * component comp, matching direction dir (0 = frame 1 -> frame 2, 1 = inverse). */
uint32_t ffo_hash(uint32_t seed, int dir, int level, int t, int d, int x, int y, int comp) {
    uint32_t k0 = ffo_mix32((uint32_t)dir * 65536u + (uint32_t)level * 256u + (uint32_t)t);
    uint32_t k1 = ffo_mix32(seed ^ k0);
    uint32_t k2 = ffo_mix32(k1 ^ ((uint32_t)y * 65536u + (uint32_t)x));
    return ffo_mix32(k2 ^ (uint32_t)(d * 2 + comp));
}

/* Matching cost (Sec. 3.1 defines it as a distance between feature descriptors).  Reading: sum of absolute
 * differences over the 48 WHT coefficients of pixel (x, y) in frame A and pixel (x+fx, y+fy) in frame B.
 * Returns -1 when the target lies outside the level (the candidate is rejected). */
int32_t ffo_sad(const int16_t* fa, const int16_t* fb, int w, int h, int x, int y, int fx, int fy) {
    int qx = x + fx, qy = y + fy;
    if (qx < 0 || qx >= w || qy < 0 || qy >= h) return -1;
    const int16_t* a = fa + ((long)y * w + x) * FFO_NF;
    const int16_t* b = fb + ((long)qy * w + qx) * FFO_NF;
    int32_t s = 0;
    for (int k = 0; k < FFO_NF; k++) s += abs((int)a[k] - (int)b[k]);
    return s;
}

/* Census transform (Sec. 3.1: binary patterns of the Census transform in a 7x7 patch for all colour channels).
 * Reading: the RGB channels stand in for CIELab (integer, exact); bit k of channel c is 1 iff the k-th neighbour
 * -- row-major over rows y-3..y+3 and columns x-3..x+3, centre skipped, edge pixels repeated -- is strictly darker
 * than the centre pixel.  desc[(y*w + x)*3 + c] holds the 48 bits of channel c. */
void ffo_census(const uint8_t* img, int w, int h, uint64_t* desc) {
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++)
            for (int c = 0; c < 3; c++) {
                int centre = img[((long)y * w + x) * 3 + c];
                uint64_t bits = 0;
                int k = 0;
                for (int dy = -3; dy <= 3; dy++)
                    for (int dx = -3; dx <= 3; dx++) {
                        if (dy == 0 && dx == 0) continue;
                        int v = img[((long)clampi(y + dy, 0, h - 1) * w + clampi(x + dx, 0, w - 1)) * 3 + c];
                        if (v < centre) bits |= (uint64_t)1 << k;
                        k++;
                    }
                desc[((long)y * w + x) * 3 + c] = bits;
            }
}

static int popcount64(uint64_t v) {
    int n = 0;
    while (v) {
        v &= v - 1;
        n++;
    }
    return n;
}

/* Census matching cost (Sec. 3.1): Hamming distance of the three 48-bit patterns of pixel (x, y) in frame A
 * and (x+fx, y+fy) in frame B; -1 when the target lies outside the level. */
int32_t ffo_hamming(const uint64_t* ca, const uint64_t* cb, int w, int h, int x, int y, int fx, int fy) {
    int qx = x + fx, qy = y + fy;
    if (qx < 0 || qx >= w || qy < 0 || qy >= h) return -1;
    int32_t s = 0;
    for (int c = 0; c < 3; c++) s += popcount64(ca[((long)y * w + x) * 3 + c] ^ cb[((long)qy * w + qx) * 3 + c]);
    return s;
}

/* The descriptors a level is matched with: WHT coefficients (cost = SAD) or, if ca is set, Census patterns
 * (cost = Hamming distance), and the grid of source pixels a flow field lives on: every g-th pixel of the level
 * in both directions (g = 1: every pixel; g = 2, 4: a sub-scale or sub-sub-scale, see match_dir_c).  Grid pixel
 * (x, y) is level pixel (g*x, g*y); flows are in level pixels and may point to any pixel of the target level. */
typedef struct {
    const int16_t* fa;
    const int16_t* fb;
    const uint64_t* ca;
    const uint64_t* cb;
    int w, h; /* the level */
    int g;    /* grid stride */
} costsrc;

static int grid_w(const costsrc* cs) { return (cs->w + cs->g - 1) / cs->g; }
static int grid_h(const costsrc* cs) { return (cs->h + cs->g - 1) / cs->g; }

/* Cost of grid pixel (x, y) with flow (fx, fy); -1 when the target lies outside the level. */
static int32_t cost_of(const costsrc* cs, int x, int y, int fx, int fy) {
    return cs->ca ? ffo_hamming(cs->ca, cs->cb, cs->w, cs->h, cs->g * x, cs->g * y, fx, fy)
                  : ffo_sad(cs->fa, cs->fb, cs->w, cs->h, cs->g * x, cs->g * y, fx, fy);
}

/* floor(c / 128), the arithmetic shift C >> 7 written without relying on signed shifts. */
static int quant7(int c) { return c >= 0 ? c / 128 : -((-c + 127) / 128); }

/* Initial matches at the coarsest level (Sec. 3.1: WHT descriptors matched with kD-trees).  Reading: the
 * exact nearest neighbour that a kD-tree approximates.  The descriptor is quantised to 8 bits (C >> 7,
 * in [-128, 127]); distance = squared Euclidean; ties go to the smallest row-major index of frame B.
 * flow = q - p; dist = the winning squared distance. */
void ffo_seed(const int16_t* fa, const int16_t* fb, int w, int h, int16_t* flow, int32_t* dist) {
    long n = (long)w * h;
    for (long p = 0; p < n; p++) {
        long best_q = 0;
        int32_t best = INT32_MAX;
        for (long q = 0; q < n; q++) {
            int32_t d2 = 0;
            for (int k = 0; k < FFO_NF; k++) {
                int e = quant7(fa[p * FFO_NF + k]) - quant7(fb[q * FFO_NF + k]);
                d2 += e * e;
            }
            if (d2 < best) {
                best = d2;
                best_q = q;
            }
        }
        flow[p * 2 + 0] = (int16_t)(best_q % w - p % w);
        flow[p * 2 + 1] = (int16_t)(best_q / w - p / w);
        dist[p] = best;
    }
}

/* cost(p) = matching cost of p's current flow; every flow handed in must point inside the level. */
static void init_cost_c(const costsrc* cs, const int16_t* flow, int32_t* cost) {
    for (int y = 0; y < grid_h(cs); y++)
        for (int x = 0; x < grid_w(cs); x++) {
            long p = (long)y * grid_w(cs) + x;
            cost[p] = cost_of(cs, x, y, flow[2 * p], flow[2 * p + 1]);
        }
}

void ffo_init_cost(const int16_t* fa, const int16_t* fb, int w, int h, const int16_t* flow, int32_t* cost) {
    costsrc cs = {fa, fb, NULL, NULL, w, h, 1};
    init_cost_c(&cs, flow, cost);
}

/* Coarse-to-fine hand-over (Sec. 3): a pixel starts from twice the flow of its parent pixel one level up,
 * parent = (min(x/2, wc-1), min(y/2, hc-1)), and its cost is recomputed at the finer level.  (x, y) are level
 * coordinates: on a grid of stride g, grid pixel (u, v) is level pixel (g*u, g*v).  Such a flow always lands
 * inside the finer level; returns -2 if one does not (a broken assertion). */
static int upsample_c(const costsrc* cs, const int16_t* flow_coarse, int wc, int hc, int16_t* flow, int32_t* cost) {
    const int gw = grid_w(cs), gh = grid_h(cs);
    for (int v = 0; v < gh; v++)
        for (int u = 0; u < gw; u++) {
            int x = cs->g * u, y = cs->g * v;
            int px = mini(x / 2, wc - 1), py = mini(y / 2, hc - 1);
            long pc = (long)py * wc + px, p = (long)v * gw + u;
            int fx = 2 * flow_coarse[2 * pc], fy = 2 * flow_coarse[2 * pc + 1];
            flow[2 * p] = (int16_t)fx;
            flow[2 * p + 1] = (int16_t)fy;
            cost[p] = cost_of(cs, u, v, fx, fy);
            if (cost[p] < 0) return -2;
        }
    return 0;
}

int ffo_upsample(const int16_t* fa, const int16_t* fb, int w, int h, const int16_t* flow_coarse, int wc, int hc,
                 int16_t* flow, int32_t* cost) {
    costsrc cs = {fa, fb, NULL, NULL, w, h, 1};
    return upsample_c(&cs, flow_coarse, wc, hc, flow, cost);
}

int ffo_upsample_grid(const int16_t* fa, const int16_t* fb, int w, int h, int g, const int16_t* flow_coarse, int wc,
                      int hc, int16_t* flow, int32_t* cost) {
    costsrc cs = {fa, fb, NULL, NULL, w, h, g};
    return upsample_c(&cs, flow_coarse, wc, hc, flow, cost);
}

/* Hand-over between two grids of one level (reading of the sub-scales of Sec. 3.1, see match_dir_c): grid pixel
 * (u, v) of stride g starts from the flow of grid pixel (min(u/2, pw-1), min(v/2, ph-1)) of the grid of stride 2g
 * (pw x ph), unchanged (both are in level pixels), except that its target is clamped into the level: the child
 * pixel lies up to g pixels right of / below its parent, so the parent's flow may point past the edge.  The cost
 * is recomputed. */
static void grid_handover_c(const costsrc* cs, const int16_t* flow_parent, int pw, int ph, int16_t* flow,
                            int32_t* cost) {
    const int gw = grid_w(cs), gh = grid_h(cs);
    for (int v = 0; v < gh; v++)
        for (int u = 0; u < gw; u++) {
            long pp = (long)mini(v / 2, ph - 1) * pw + mini(u / 2, pw - 1), p = (long)v * gw + u;
            int x = cs->g * u, y = cs->g * v;
            int fx = clampi(x + flow_parent[2 * pp], 0, cs->w - 1) - x;
            int fy = clampi(y + flow_parent[2 * pp + 1], 0, cs->h - 1) - y;
            flow[2 * p] = (int16_t)fx;
            flow[2 * p + 1] = (int16_t)fy;
            cost[p] = cost_of(cs, u, v, fx, fy);
        }
}

void ffo_grid_handover(const int16_t* fa, const int16_t* fb, int w, int h, int g, const int16_t* flow_parent, int pw,
                       int ph, int16_t* flow, int32_t* cost) {
    costsrc cs = {fa, fb, NULL, NULL, w, h, g};
    grid_handover_c(&cs, flow_parent, pw, ph, flow, cost);
}

/* The two neighbours a pixel looks at in propagation direction d (one direction per quadrant, Sec. 3.1).
 * Reading: one sweep direction per quadrant -- d=0 from the left/top, d=1 right/top, d=2 left/bottom,
 * d=3 right/bottom -- with the horizontal neighbour tried first. */
static void neighbours(int d, int x, int y, int* n1x, int* n1y, int* n2x, int* n2y) {
    *n1x = (d == 0 || d == 2) ? x - 1 : x + 1;
    *n1y = y;
    *n2x = x;
    *n2y = (d == 0 || d == 1) ? y - 1 : y + 1;
}

/* Propagation with random search at one level (Sec. 3.1), on the grid of cs (every pixel, or every g-th pixel
 * of a sub-scale; x, y below are grid coordinates, neighbours are grid neighbours, flows and offsets are in level
 * pixels, and the hash is keyed with the level coordinates (g*x, g*y) and the stream id `level`).  For
 * t = 0..iters-1, for each direction d = 0..3,
 * two half-sweeps (pixels with (x+y) even, then odd); within a half-sweep every pixel of that colour is
 * updated from the state at the start of the half-sweep, so their order does not matter.
 * A pixel tries, in order: the flow of neighbour 1, the flow of neighbour 2 (neighbours outside the level
 * are skipped), and for d >= 1 (the last three propagation steps of the iteration) its current flow plus a
 * random offset (ox, oy), each component uniform in [-R, R] from the hash, skipped if (0, 0).  A candidate
 * replaces the current flow iff its cost is strictly lower; candidates outside the level are rejected.
 * Stops after max_halfsweeps half-sweeps if max_halfsweeps >= 0; returns the number run. */
static long propagate_c(const costsrc* cs, int16_t* flow, int32_t* cost, int iters, int rs_radius, uint32_t seed,
                        int dir, int level, long max_halfsweeps) {
    const int w = grid_w(cs), h = grid_h(cs);
    long n = (long)w * h, done = 0;
    int16_t* prev = (int16_t*)malloc(sizeof(int16_t) * 2 * (size_t)n);
    if (!prev) return -1;
    int span = 2 * rs_radius + 1;
    for (int t = 0; t < iters; t++) {
        for (int d = 0; d < 4; d++) {
            for (int colour = 0; colour < 2; colour++) {
                if (max_halfsweeps >= 0 && done >= max_halfsweeps) {
                    free(prev);
                    return done;
                }
                memcpy(prev, flow, sizeof(int16_t) * 2 * (size_t)n);
                for (int y = 0; y < h; y++) {
                    for (int x = 0; x < w; x++) {
                        if ((x + y) % 2 != colour) continue;
                        long p = (long)y * w + x;
                        int fx = flow[2 * p], fy = flow[2 * p + 1];
                        int32_t c = cost[p];
                        int nx[2], ny[2];
                        neighbours(d, x, y, &nx[0], &ny[0], &nx[1], &ny[1]);
                        for (int k = 0; k < 2; k++) {
                            if (nx[k] < 0 || nx[k] >= w || ny[k] < 0 || ny[k] >= h) continue;
                            long q = (long)ny[k] * w + nx[k];
                            int cx = prev[2 * q], cy = prev[2 * q + 1];
                            int32_t cc = cost_of(cs, x, y, cx, cy);
                            if (cc >= 0 && cc < c) {
                                fx = cx;
                                fy = cy;
                                c = cc;
                            }
                        }
                        if (d >= 1) {
                            int lx = cs->g * x, ly = cs->g * y;
                            int ox = (int)(ffo_hash(seed, dir, level, t, d, lx, ly, 0) % (uint32_t)span) - rs_radius;
                            int oy = (int)(ffo_hash(seed, dir, level, t, d, lx, ly, 1) % (uint32_t)span) - rs_radius;
                            if (ox != 0 || oy != 0) {
                                int32_t cc = cost_of(cs, x, y, fx + ox, fy + oy);
                                if (cc >= 0 && cc < c) {
                                    fx += ox;
                                    fy += oy;
                                    c = cc;
                                }
                            }
                        }
                        flow[2 * p] = (int16_t)fx;
                        flow[2 * p + 1] = (int16_t)fy;
                        cost[p] = c;
                    }
                }
                done++;
            }
        }
    }
    free(prev);
    return done;
}

long ffo_propagate(const int16_t* fa, const int16_t* fb, int w, int h, int16_t* flow, int32_t* cost, int iters,
                   int rs_radius, uint32_t seed, int dir, int level, long max_halfsweeps) {
    costsrc cs = {fa, fb, NULL, NULL, w, h, 1};
    return propagate_c(&cs, flow, cost, iters, rs_radius, seed, dir, level, max_halfsweeps);
}

long ffo_propagate_grid(const int16_t* fa, const int16_t* fb, int w, int h, int g, int16_t* flow, int32_t* cost,
                        int iters, int rs_radius, uint32_t seed, int dir, int stream, long max_halfsweeps) {
    costsrc cs = {fa, fb, NULL, NULL, w, h, g};
    return propagate_c(&cs, flow, cost, iters, rs_radius, seed, dir, stream, max_halfsweeps);
}

long ffo_propagate_census(const uint64_t* ca, const uint64_t* cb, int w, int h, int16_t* flow, int32_t* cost,
                          int iters, int rs_radius, uint32_t seed, int dir, int level, long max_halfsweeps) {
    costsrc cs = {NULL, NULL, ca, cb, w, h, 1};
    return propagate_c(&cs, flow, cost, iters, rs_radius, seed, dir, level, max_halfsweeps);
}

/* One matching direction over a prepared pyramid of features (Sec. 3.1): exact seed at the coarsest level,
 * then for every level from coarse to fine: hand-over from the level above (except the coarsest), cost,
 * propagation with random search.  Writes the level-0 flow and cost.  feat_a/feat_b[s] are the level-s
 * feature maps of the source and target frames; both frames have the sizes ws[s] x hs[s].
 *
 * Sub-scales and sub-sub-scales (Sec. 3.1 uses them "as in" Flow Fields+, which is not restated; reading):
 * with prm->sub_scales = n (0, 1 or 2), every level below the coarsest is first matched on the grid of every
 * 2^n-th pixel, then of every 2^(n-1)-th, ..., then on every pixel -- the same descriptors, so a sparse grid
 * reaches across 2^k level pixels per propagation step with the fine level's detail.  The first grid of a level
 * takes the hand-over from the level above; each later grid takes its parent grid pixel's flow (clamped into the
 * level, grid_handover_c).  Every grid runs the level's whole propagation schedule on its own random stream,
 * stream id s + 8k for the grid of stride 2^k (k = 0: the level itself, as without sub-scales).  The coarsest
 * level starts from exact matches and has no sub-scales. */
static int match_dir_c(const int16_t* const* feat_a, const int16_t* const* feat_b, const uint64_t* const* cen_a,
                       const uint64_t* const* cen_b, const int* ws, const int* hs, const ffo_params* prm, int dir,
                       int16_t* flow, int32_t* cost) {
    int L = prm->n_scales, n_sub = prm->sub_scales;
    if (n_sub < 0 || n_sub > 2) return -1;
    int16_t* f_prev = NULL; /* the last field: of the level above, or of a sparser grid of this level */
    int w_prev = 0, h_prev = 0; /* its grid size */
    for (int s = L - 1; s >= 0; s--) {
        const int k_first = s == L - 1 ? 0 : n_sub;
        for (int k = k_first; k >= 0; k--) {
            costsrc cs = {feat_a[s], feat_b[s], cen_a ? cen_a[s] : NULL, cen_b ? cen_b[s] : NULL, ws[s], hs[s], 1 << k};
            int gw = grid_w(&cs), gh = grid_h(&cs);
            long n = (long)gw * gh;
            int16_t* f = (int16_t*)malloc(sizeof(int16_t) * 2 * (size_t)n);
            int32_t* c = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
            if (!f || !c) {
                free(f);
                free(c);
                free(f_prev);
                return -1;
            }
            if (s == L - 1) {
                ffo_seed(feat_a[s], feat_b[s], gw, gh, f, c);  /* initial matches on the WHT descriptors in both modes */
                init_cost_c(&cs, f, c);
            } else if (k == k_first) {
                if (upsample_c(&cs, f_prev, w_prev, h_prev, f, c) != 0) {
                    free(f);
                    free(c);
                    free(f_prev);
                    return -2;
                }
            } else {
                grid_handover_c(&cs, f_prev, w_prev, h_prev, f, c);
            }
            propagate_c(&cs, f, c, prm->iters, prm->rs_radius, prm->seed, dir, s + 8 * k, -1);
            free(f_prev);
            f_prev = f;
            w_prev = gw;
            h_prev = gh;
            if (s == 0 && k == 0) {
                memcpy(flow, f, sizeof(int16_t) * 2 * (size_t)n);
                memcpy(cost, c, sizeof(int32_t) * (size_t)n);
            }
            free(c);
        }
    }
    free(f_prev);
    return 0;
}

int ffo_match_dir(const int16_t* const* feat_a, const int16_t* const* feat_b, const int* ws, const int* hs,
                  const ffo_params* prm, int dir, int16_t* flow, int32_t* cost) {
    return match_dir_c(feat_a, feat_b, NULL, NULL, ws, hs, prm, dir, flow, cost);
}

int ffo_match_dir_census(const int16_t* const* feat_a, const int16_t* const* feat_b, const uint64_t* const* cen_a,
                         const uint64_t* const* cen_b, const int* ws, const int* hs, const ffo_params* prm, int dir,
                         int16_t* flow, int32_t* cost) {
    return match_dir_c(feat_a, feat_b, cen_a, cen_b, ws, hs, prm, dir, flow, cost);
}

/* Forward/backward consistency check (Sec. 3.1; eps in Table 3).  p is kept iff q = p + f(p) lies in the
 * image and the consistency error |f(p) + b(q)| (Euclidean) does not exceed eps; compared as squares. */
void ffo_consistency(const int16_t* fwd, const int16_t* bwd, int w, int h, int eps, uint8_t* mask) {
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            long p = (long)y * w + x;
            int fx = fwd[2 * p], fy = fwd[2 * p + 1];
            int qx = x + fx, qy = y + fy;
            if (qx < 0 || qx >= w || qy < 0 || qy >= h) {
                mask[p] = 0;
                continue;
            }
            long q = (long)qy * w + qx;
            long ex = fx + bwd[2 * q], ey = fy + bwd[2 * q + 1];
            mask[p] = (uint8_t)(ex * ex + ey * ey <= (long)eps * eps);
        }
}

/* Pyramid, WHT features and (for the Census cost) Census patterns of one frame, all levels. */
static int frame_features(const uint8_t* rgb, int L, const int* ws, const int* hs, int census, uint8_t** img,
                          int16_t** feat, uint64_t** cen) {
    for (int s = 0; s < L; s++) {
        long ns = (long)ws[s] * hs[s];
        img[s] = (uint8_t*)malloc((size_t)ns * 3);
        feat[s] = (int16_t*)malloc((size_t)ns * FFO_NF * sizeof(int16_t));
        cen[s] = census ? (uint64_t*)malloc((size_t)ns * 3 * sizeof(uint64_t)) : NULL;
        if (!img[s] || !feat[s] || (census && !cen[s])) return -1;
        if (s == 0)
            memcpy(img[s], rgb, (size_t)ns * 3);
        else
            ffo_downsample(img[s - 1], ws[s - 1], hs[s - 1], img[s]);
        ffo_wht(img[s], ws[s], hs[s], feat[s]);
        if (census) ffo_census(img[s], ws[s], hs[s], cen[s]);
    }
    return 0;
}

static void free_features(int L, uint8_t** img, int16_t** feat, uint64_t** cen) {
    for (int s = 0; s < L; s++) {
        free(img[s]);
        free(feat[s]);
        free(cen[s]);
    }
}

/* Two consistency checks (Sec. 3.1): the forward field is compared with two inverse fields computed with
 * different matching parameters, and kept only if it passes both.  Reading: the second inverse field uses the
 * random-search radius rs_radius2 and its own random stream (direction id 2); everything else is shared. */
int ffo_match_bidir2(const uint8_t* rgb_a, const uint8_t* rgb_b, int w, int h, const ffo_params* prm, int rs_radius2,
                     int16_t* flow_fwd, int16_t* flow_bwd, int16_t* flow_bwd2, uint8_t* mask) {
    long n = (long)w * h;
    int L = prm->n_scales, rc = 0;
    int ws[16], hs[16];
    if (L < 1 || L > 16 || ffo_level_dims(w, h, L, ws, hs) != 0) return -1;
    int32_t* cf = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* cb = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    uint8_t* m2 = (uint8_t*)malloc((size_t)n);
    uint8_t* img[2][16] = {{0}};
    int16_t* feat[2][16] = {{0}};
    uint64_t* cen[2][16] = {{0}};
    if (!cf || !cb || !m2) rc = -1;
    for (int f = 0; f < 2 && rc == 0; f++)
        rc = frame_features(f == 0 ? rgb_a : rgb_b, L, ws, hs, prm->cost, img[f], feat[f], cen[f]);
    const uint64_t* const* ca = prm->cost ? (const uint64_t* const*)cen[0] : NULL;
    const uint64_t* const* cb2 = prm->cost ? (const uint64_t* const*)cen[1] : NULL;
    const ffo_params* p1 = prm;
    ffo_params p2 = *prm;
    p2.rs_radius = rs_radius2;
    if (rc == 0) rc = match_dir_c((const int16_t* const*)feat[0], (const int16_t* const*)feat[1], ca, cb2, ws, hs, p1, 0,
                                  flow_fwd, cf);
    if (rc == 0) rc = match_dir_c((const int16_t* const*)feat[1], (const int16_t* const*)feat[0], cb2, ca, ws, hs, p1, 1,
                                  flow_bwd, cb);
    if (rc == 0) rc = match_dir_c((const int16_t* const*)feat[1], (const int16_t* const*)feat[0], cb2, ca, ws, hs, &p2, 2,
                                  flow_bwd2, cb);
    if (rc == 0) {
        ffo_consistency(flow_fwd, flow_bwd, w, h, prm->eps, mask);
        ffo_consistency(flow_fwd, flow_bwd2, w, h, prm->eps, m2);
        for (long p = 0; p < n; p++) mask[p] = (uint8_t)(mask[p] & m2[p]);
    }
    for (int f = 0; f < 2; f++) free_features(L, img[f], feat[f], cen[f]);
    free(cf);
    free(cb);
    free(m2);
    return rc;
}

/* Sparsification (Sec. 3.1; s in Table 3): in each 3x3 block that contains at least s matches that pass the
 * consistency check, keep only the match with the lowest consistency error; drop every other match.
 * Reading: blocks tile the image from (0, 0) (blocks at the right and bottom edges may be smaller); the error is
 * the squared Euclidean consistency error |f(p) + b(p + f(p))|^2; ties go to the first pixel in row-major order
 * within the block.  The paper sparsifies what is left after both consistency checks: `keep` (may be NULL) is
 * that filter's mask, and a match counts only where keep[p] != 0 as well.  out[p] = 1 for kept matches, 0
 * elsewhere. */
void ffo_sparsify(const int16_t* fwd, const int16_t* bwd, const uint8_t* keep, int w, int h, int eps, int s,
                  uint8_t* out) {
    for (long p = 0; p < (long)w * h; p++) out[p] = 0;
    for (int by = 0; by < h; by += 3)
        for (int bx = 0; bx < w; bx += 3) {
            int count = 0;
            long best_p = -1, best_e = 0;
            for (int y = by; y < by + 3 && y < h; y++)
                for (int x = bx; x < bx + 3 && x < w; x++) {
                    long p = (long)y * w + x;
                    if (keep && !keep[p]) continue;
                    int fx = fwd[2 * p], fy = fwd[2 * p + 1];
                    int qx = x + fx, qy = y + fy;
                    if (qx < 0 || qx >= w || qy < 0 || qy >= h) continue;
                    long q = (long)qy * w + qx;
                    long ex = (long)fx + bwd[2 * q], ey = (long)fy + bwd[2 * q + 1];
                    long e = ex * ex + ey * ey;
                    if (e > (long)eps * eps) continue;
                    count++;
                    if (best_p < 0 || e < best_e) {
                        best_p = p;
                        best_e = e;
                    }
                }
            if (count >= s && best_p >= 0) out[best_p] = 1;
        }
}

/* The whole stage for one frame pair: pyramids and features of both frames, matching frame 1 -> 2
 * (dir 0) and the inverse field 2 -> 1 (dir 1), then the consistency mask of the forward field.  prm->cost
 * selects the matching cost: 0 = SAD of the WHT descriptors, 1 = Hamming distance of the Census patterns. */
int ffo_match_bidir(const uint8_t* rgb_a, const uint8_t* rgb_b, int w, int h, const ffo_params* prm,
                    int16_t* flow_fwd, int16_t* flow_bwd, int32_t* cost_fwd, int32_t* cost_bwd, uint8_t* mask) {
    int L = prm->n_scales;
    if (L < 1 || L > 16) return -1;
    int ws[16], hs[16];
    if (ffo_level_dims(w, h, L, ws, hs) != 0) return -1;
    uint8_t* img[2][16] = {{0}};
    int16_t* feat[2][16] = {{0}};
    uint64_t* cen[2][16] = {{0}};
    int rc = 0;
    for (int f = 0; f < 2 && rc == 0; f++)
        rc = frame_features(f == 0 ? rgb_a : rgb_b, L, ws, hs, prm->cost, img[f], feat[f], cen[f]);
    const uint64_t* const* ca = prm->cost ? (const uint64_t* const*)cen[0] : NULL;
    const uint64_t* const* cb = prm->cost ? (const uint64_t* const*)cen[1] : NULL;
    if (rc == 0) rc = match_dir_c((const int16_t* const*)feat[0], (const int16_t* const*)feat[1], ca, cb, ws, hs, prm, 0,
                                  flow_fwd, cost_fwd);
    if (rc == 0) rc = match_dir_c((const int16_t* const*)feat[1], (const int16_t* const*)feat[0], cb, ca, ws, hs, prm, 1,
                                  flow_bwd, cost_bwd);
    if (rc == 0) ffo_consistency(flow_fwd, flow_bwd, w, h, prm->eps, mask);
    for (int f = 0; f < 2; f++) free_features(L, img[f], feat[f], cen[f]);
    return rc;
}
