/*
 * graphgen.c -- seeded synthetic directed graphs (R-MAT, Erdos-Renyi) and the
 * CSR/CSC builders used by both the oracle tests and the CUDA library tests.
 *
 * This file holds no PageRank arithmetic: it only draws edges, filters them,
 * relabels vertices and sorts edge lists into compressed rows.  Every random
 * draw is a pure function of (seed, stream, index) through a counter-based
 * hash (SplitMix64 finaliser, Steele/Lea/Flood 2014), so the output does not
 * depend on the number of OpenMP threads.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* one 64-bit draw for (seed, stream, index) */
static inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t idx) {
    return mix64(mix64(seed * 0x2545F4914F6CDD1DULL + stream) ^ idx);
}

/* uniform double in [0,1) with 53 random bits */
static inline double draw_u01(uint64_t seed, uint64_t stream, uint64_t idx) {
    return (double)(draw(seed, stream, idx) >> 11) * (1.0 / 9007199254740992.0);
}

double gg_u01(uint64_t seed, uint64_t stream, uint64_t idx) { return draw_u01(seed, stream, idx); }

/*
 * R-MAT edge sampler (Chakrabarti, Zhan, Faloutsos 2004): each of the `scale`
 * levels picks one quadrant of the adjacency matrix with probabilities
 * (a, b, c, 1-a-b-c); quadrant b sets the column (target) bit, c the row
 * (source) bit, d both.  No noise is added.  Four levels are drawn from one
 * 64-bit hash, 16 bits each.
 */
void gg_rmat(int scale, int64_t m, double a, double b, double c, uint64_t seed,
             int32_t *src, int32_t *dst) {
    const uint32_t ta = (uint32_t)(a * 65536.0 + 0.5);
    const uint32_t tb = (uint32_t)((a + b) * 65536.0 + 0.5);
    const uint32_t tc = (uint32_t)((a + b + c) * 65536.0 + 0.5);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; e++) {
        uint32_t s = 0, d = 0;
        uint64_t bits = 0;
        for (int lv = 0; lv < scale; lv++) {
            if ((lv & 3) == 0) bits = draw(seed, 1 + (uint64_t)(lv >> 2), (uint64_t)e);
            uint32_t u = (uint32_t)(bits & 0xFFFFu);
            bits >>= 16;
            uint32_t sb, db;
            if (u < ta)      { sb = 0; db = 0; }
            else if (u < tb) { sb = 0; db = 1; }
            else if (u < tc) { sb = 1; db = 0; }
            else             { sb = 1; db = 1; }
            s = (s << 1) | sb;
            d = (d << 1) | db;
        }
        src[e] = (int32_t)s;
        dst[e] = (int32_t)d;
    }
}

/* Erdos-Renyi G(n, m) with replacement: m independent uniform (src, dst) pairs. */
void gg_er(int32_t n, int64_t m, uint64_t seed, int32_t *src, int32_t *dst) {
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; e++) {
        uint64_t h = draw(seed, 100, (uint64_t)e);
        src[e] = (int32_t)(((h & 0xFFFFFFFFULL) * (uint64_t)n) >> 32);
        dst[e] = (int32_t)(((h >> 32) * (uint64_t)n) >> 32);
    }
}

/* mask[i] = 1 with probability frac, independently per vertex (stream separates uses). */
void gg_vertex_mask(int32_t n, double frac, uint64_t seed, uint64_t stream, uint8_t *mask) {
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; i++) mask[i] = draw_u01(seed, 200 + stream, (uint64_t)i) < frac;
}

/*
 * Uniformly random permutation of [0, n): vertex i gets as its new id the rank
 * of its 63-bit key draw(seed, 300 + stream, i) >> 1 among all keys (ties,
 * which have probability about n^2 / 2^64, go to the smaller i).  Defined by
 * sorting so that a data-parallel generator can produce the same permutation.
 */
typedef struct {
    uint64_t k;
    int32_t i;
} gg_key_idx;

static int cmp_key_idx(const void *x, const void *y) {
    const gg_key_idx *a = (const gg_key_idx *)x, *b = (const gg_key_idx *)y;
    if (a->k != b->k) return a->k < b->k ? -1 : 1;
    return (a->i > b->i) - (a->i < b->i);
}

void gg_permutation(int32_t n, uint64_t seed, uint64_t stream, int32_t *perm) {
    gg_key_idx *a = (gg_key_idx *)malloc(sizeof(gg_key_idx) * ((size_t)n + 1));
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; i++) {
        a[i].k = draw(seed, 300 + stream, (uint64_t)i) >> 1;
        a[i].i = i;
    }
    qsort(a, (size_t)n, sizeof(gg_key_idx), cmp_key_idx);
#pragma omp parallel for schedule(static)
    for (int32_t r = 0; r < n; r++) perm[a[r].i] = r;
    free(a);
}

/* Apply a vertex relabelling to an edge list in place: v -> perm[v]. */
void gg_relabel(int64_t m, const int32_t *perm, int32_t *src, int32_t *dst) {
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; e++) { src[e] = perm[src[e]]; dst[e] = perm[dst[e]]; }
}

/*
 * DAG-heavy orientation: with probability frac an edge is turned so that it
 * points forward in the order `rank` (rank[src] < rank[dst]), swapping its
 * endpoints if needed; the rest keep their direction.
 */
void gg_orient(int64_t m, const int32_t *rank, double frac, uint64_t seed,
               int32_t *src, int32_t *dst) {
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; e++) {
        if (draw_u01(seed, 400, (uint64_t)e) < frac && rank[src[e]] > rank[dst[e]]) {
            int32_t t = src[e]; src[e] = dst[e]; dst[e] = t;
        }
    }
}

/*
 * Keep edge e unless its source is in drop_out or its target in drop_in (either
 * mask may be NULL), or it is a self-loop and drop_loops is set.  Compacts in
 * place and returns the new edge count.
 */
int64_t gg_filter(int64_t m, int32_t *src, int32_t *dst, const uint8_t *drop_out,
                  const uint8_t *drop_in, int drop_loops) {
    int64_t k = 0;
    for (int64_t e = 0; e < m; e++) {
        int32_t s = src[e], d = dst[e];
        if (drop_loops && s == d) continue;
        if (drop_out && drop_out[s]) continue;
        if (drop_in && drop_in[d]) continue;
        src[k] = s; dst[k] = d; k++;
    }
    return k;
}

static int cmp_i32(const void *x, const void *y) {
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

/* sort a short row: insertion sort below 32 entries, qsort above */
static void sort_row(int32_t *v, int64_t len) {
    if (len > 32) { qsort(v, (size_t)len, sizeof(int32_t), cmp_i32); return; }
    for (int64_t i = 1; i < len; i++) {
        int32_t t = v[i]; int64_t j = i - 1;
        while (j >= 0 && v[j] > t) { v[j + 1] = v[j]; j--; }
        v[j + 1] = t;
    }
}

/*
 * Group an edge list by `key` (counting sort), sort each group by `val`, drop
 * repeated (key, val) pairs, and write compressed rows: off[n+1] (int64) and
 * col[<= m].  Returns the number of distinct pairs.  `tmp` must hold m int32.
 */
int64_t gg_compress(int32_t n, int64_t m, const int32_t *key, const int32_t *val,
                    int64_t *off, int32_t *col, int32_t *tmp) {
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    memset(off, 0, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t e = 0; e < m; e++) off[key[e] + 1]++;
    for (int32_t i = 0; i < n; i++) off[i + 1] += off[i];
    memcpy(cur, off, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t e = 0; e < m; e++) tmp[cur[key[e]]++] = val[e];
    int64_t *cnt = cur; /* reuse: distinct count per row */
#pragma omp parallel for schedule(dynamic, 4096)
    for (int32_t i = 0; i < n; i++) {
        int32_t *row = tmp + off[i];
        int64_t len = off[i + 1] - off[i];
        sort_row(row, len);
        int64_t k = 0;
        for (int64_t j = 0; j < len; j++)
            if (k == 0 || row[j] != row[k - 1]) row[k++] = row[j];
        cnt[i] = k;
    }
    /* compact rows to the front */
    int64_t pos = 0;
    for (int32_t i = 0; i < n; i++) {
        int64_t start = off[i], k = cnt[i];
        memmove(col + pos, tmp + start, sizeof(int32_t) * (size_t)k);
        off[i] = pos;
        pos += k;
    }
    off[n] = pos;
    free(cur);
    return pos;
}

/* CSC from CSR: in-lists come out sorted by source because rows are scanned in order. */
void gg_transpose(int32_t n, const int64_t *out_off, const int32_t *out_dst,
                  int64_t *in_off, int32_t *in_src) {
    int64_t m = out_off[n];
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    memset(in_off, 0, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t e = 0; e < m; e++) in_off[out_dst[e] + 1]++;
    for (int32_t i = 0; i < n; i++) in_off[i + 1] += in_off[i];
    memcpy(cur, in_off, sizeof(int64_t) * ((size_t)n + 1));
    for (int32_t i = 0; i < n; i++)
        for (int64_t e = out_off[i]; e < out_off[i + 1]; e++) in_src[cur[out_dst[e]]++] = i;
    free(cur);
}

int gg_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
