/*
 * Seeded synthetic inputs for the GraphMat workloads (Section 5.1 of the paper
 * describes RMAT graphs from the Graph500 generator and a synthetic bipartite
 * rating graph).  This file holds only input synthesis: random edge lists,
 * edge values, source picks and random vectors.  It contains none of the
 * vertex-program arithmetic, so both the FP64 oracle and the CUDA library can
 * consume its output.
 *
 * Every random number comes from one counter-based generator: the SplitMix64
 * output function (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014) applied to a (seed, stream, counter) triple, so the
 * output is identical for any thread count and on any host architecture.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define SY_EXPORT __attribute__((visibility("default")))

/* SplitMix64 output function: add the golden gamma, then two xor-shift-multiply
 * rounds and a final xor-shift. */
static inline uint64_t sy_mix(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Counter-based draw: a 64-bit word for (seed, stream, counter). */
static inline uint64_t sy_draw(uint64_t seed, uint64_t stream, uint64_t counter) {
    uint64_t key = sy_mix(seed ^ sy_mix(stream * 0xD1B54A32D192ED03ULL));
    return sy_mix(key ^ (counter * 0x9E3779B97F4A7C15ULL));
}

/* Uniform double in [0, 1) with 53 random bits. */
static inline double sy_unit(uint64_t w) { return (double)(w >> 11) * (1.0 / 9007199254740992.0); }

enum { SY_STREAM_RMAT = 1, SY_STREAM_WEIGHT = 2, SY_STREAM_SOURCE = 3, SY_STREAM_UNIFORM = 4,
       SY_STREAM_CL_USER = 5, SY_STREAM_CL_ITEM = 6, SY_STREAM_SCALES = 7 };

SY_EXPORT int sy_version(void) { return 1; }

SY_EXPORT uint64_t sy_draw_u64(uint64_t seed, uint64_t stream, uint64_t counter) {
    return sy_draw(seed, stream, counter);
}

/*
 * RMAT (Chakrabarti, Zhan, Faloutsos, SDM 2004): every edge descends `scale`
 * levels of the adjacency matrix, picking quadrant (0,0) with probability a,
 * (0,1) with b, (1,0) with c and (1,1) with d = 1-a-b-c.  The first coordinate
 * bit goes to the source id, the second to the destination id, most
 * significant level first.  No vertex permutation and no per-level noise.
 * Self-loops and duplicates are left in; cleaning is the consumer's job.
 */
SY_EXPORT void sy_rmat(int32_t scale, int64_t m, double a, double b, double c, uint64_t seed,
                       int32_t* src, int32_t* dst) {
    const double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        uint32_t s = 0, d = 0;
        for (int32_t l = 0; l < scale; ++l) {
            double u = sy_unit(sy_draw(seed, SY_STREAM_RMAT, (uint64_t)e * 64u + (uint64_t)l));
            uint32_t sb, db;
            if (u < a)        { sb = 0; db = 0; }
            else if (u < ab)  { sb = 0; db = 1; }
            else if (u < abc) { sb = 1; db = 0; }
            else              { sb = 1; db = 1; }
            s = (s << 1) | sb;
            d = (d << 1) | db;
        }
        src[e] = (int32_t)s;
        dst[e] = (int32_t)d;
    }
}

/* Integer edge weight in [lo, hi] that depends only on (seed, src, dst), so a
 * duplicate edge always carries the same weight whichever copy is kept. */
SY_EXPORT void sy_edge_weights_u32(int64_t m, const int32_t* src, const int32_t* dst, uint64_t seed,
                                   uint32_t lo, uint32_t hi, uint32_t* w) {
    const uint64_t span = (uint64_t)hi - (uint64_t)lo + 1u;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        uint64_t key = ((uint64_t)(uint32_t)src[e] << 32) | (uint32_t)dst[e];
        w[e] = lo + (uint32_t)(sy_draw(seed, SY_STREAM_WEIGHT, key) % span);
    }
}

/* `count` floats uniform in [lo, hi) for stream counter offset `offset`. */
SY_EXPORT void sy_uniform_f32(int64_t count, uint64_t seed, uint64_t stream, float lo, float hi,
                              float* out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; ++i) {
        double u = sy_unit(sy_draw(seed, SY_STREAM_UNIFORM + 16u * stream, (uint64_t)i));
        out[i] = (float)(lo + (hi - lo) * u);
    }
}

/* Integers uniform in [lo, hi] (used for per-graph scales and ratings). */
SY_EXPORT void sy_uniform_int(int64_t count, uint64_t seed, uint64_t stream, int64_t lo, int64_t hi,
                              int64_t* out) {
    const uint64_t span = (uint64_t)(hi - lo) + 1u;
    for (int64_t i = 0; i < count; ++i)
        out[i] = lo + (int64_t)(sy_draw(seed, SY_STREAM_SCALES + 16u * stream, (uint64_t)i) % span);
}

/*
 * Pick `count` distinct sources with at least one out-edge that is not a
 * self-loop ("non-isolated").  Candidates are drawn in counter order; the
 * function returns how many were found (fewer only if the graph has fewer such
 * vertices or `max_draws` runs out).
 */
SY_EXPORT int64_t sy_pick_sources(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                                  int64_t count, uint64_t seed, int64_t max_draws, int32_t* out) {
    uint8_t* has_out = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!has_out) return -1;
    for (int64_t e = 0; e < m; ++e)
        if (src[e] != dst[e]) has_out[src[e]] = 1;
    int64_t found = 0;
    for (int64_t k = 0; k < max_draws && found < count && n > 0; ++k) {
        int32_t v = (int32_t)(sy_draw(seed, SY_STREAM_SOURCE, (uint64_t)k) % (uint64_t)n);
        if (has_out[v] != 1) continue;
        has_out[v] = 2; /* taken */
        out[found++] = v;
    }
    free(has_out);
    return found;
}

/*
 * Bipartite Chung-Lu rating graph: users [0, n_users), items [n_users,
 * n_users + n_items).  User of rank i (1-based) has weight i^-alpha, item of
 * rank j has weight j^-alpha, and the pair is an edge with probability
 * min(1, scale_c * wu * wv).  Each user row is sampled with geometric skips over
 * the items sorted by decreasing weight, which is exact for a run of items whose
 * probability stays at or below the first item's.  For each user we walk the
 * items in blocks of equal-probability ceiling; to keep the sampler exact and
 * simple, the skip uses the bound p_max of the block start and accepts each
 * candidate with probability p/p_max (thinning).
 *
 * Called twice: with out == NULL it only counts (returns the edge count), then
 * with arrays of that size.  The rating is 1 + draw % 5.
 */
SY_EXPORT int64_t sy_chung_lu_bipartite(int64_t n_users, int64_t n_items, double alpha, double scale_c,
                                        uint64_t seed, int32_t* out_src, int32_t* out_dst,
                                        uint32_t* out_rating, int64_t capacity) {
    double* wv = (double*)malloc(sizeof(double) * (size_t)(n_items > 0 ? n_items : 1));
    if (!wv) return -1;
    for (int64_t j = 0; j < n_items; ++j) wv[j] = pow((double)(j + 1), -alpha);
    int64_t total = 0;
    for (int64_t i = 0; i < n_users; ++i) {
        const double wu = pow((double)(i + 1), -alpha);
        uint64_t ctr = 0;
        int64_t j = 0;
        while (j < n_items) {
            double pmax = scale_c * wu * wv[j];
            if (pmax >= 1.0) { /* certain edge */
                if (out_src && total < capacity) {
                    out_src[total] = (int32_t)i;
                    out_dst[total] = (int32_t)(n_users + j);
                    out_rating[total] = 1u + (uint32_t)(sy_draw(seed, SY_STREAM_CL_ITEM,
                                                 ((uint64_t)i << 24) ^ (uint64_t)j) % 5u);
                }
                ++total;
                ++j;
                continue;
            }
            /* geometric skip with success probability pmax */
            double u = sy_unit(sy_draw(seed, SY_STREAM_CL_USER, ((uint64_t)i << 32) + ctr++));
            if (u <= 0.0) u = 1e-300;
            double skip = floor(log(u) / log1p(-pmax));
            if (skip >= (double)(n_items - j)) break;
            j += (int64_t)skip;
            double p = scale_c * wu * wv[j];
            double acc = sy_unit(sy_draw(seed, SY_STREAM_CL_USER, ((uint64_t)i << 32) + ctr++));
            if (acc * pmax < p) {
                if (out_src && total < capacity) {
                    out_src[total] = (int32_t)i;
                    out_dst[total] = (int32_t)(n_users + j);
                    out_rating[total] = 1u + (uint32_t)(sy_draw(seed, SY_STREAM_CL_ITEM,
                                                 ((uint64_t)i << 24) ^ (uint64_t)j) % 5u);
                }
                ++total;
            }
            ++j;
        }
    }
    free(wv);
    return total;
}

/* Expected edge count of the Chung-Lu model above, for calibrating scale_c:
 * per user, the items with p >= 1 count fully and the rest contribute their
 * probabilities (a suffix sum of item weights). */
SY_EXPORT double sy_chung_lu_expected(int64_t n_users, int64_t n_items, double alpha, double scale_c) {
    double* suffix = (double*)malloc(sizeof(double) * (size_t)(n_items + 1));
    double* wv = (double*)malloc(sizeof(double) * (size_t)(n_items > 0 ? n_items : 1));
    if (!suffix || !wv) { free(suffix); free(wv); return -1.0; }
    for (int64_t j = 0; j < n_items; ++j) wv[j] = pow((double)(j + 1), -alpha);
    suffix[n_items] = 0.0;
    for (int64_t j = n_items - 1; j >= 0; --j) suffix[j] = suffix[j + 1] + wv[j];
    double total = 0.0;
    int64_t jcert = n_items; /* items [0, jcert) are certain; shrinks as wu falls */
    for (int64_t i = 0; i < n_users; ++i) {
        const double wu = pow((double)(i + 1), -alpha);
        while (jcert > 0 && scale_c * wu * wv[jcert - 1] < 1.0) --jcert;
        total += (double)jcert + scale_c * wu * suffix[jcert];
    }
    free(suffix);
    free(wv);
    return total;
}
