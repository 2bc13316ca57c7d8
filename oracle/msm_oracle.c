/*
 * msm_oracle.c -- plain CPU restatement of the epsilon-neighbour-graph method
 * of Uno, Sugiyama and Tsuda, "Efficient Construction of Neighborhood Graphs
 * by the Multiple Sorting Method".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg load it.  It is written to be read against
 * the paper, not to be fast: single thread, double precision for every
 * floating-point decision, sequential fma accumulation, qsort for grouping.
 *
 * Conventions (readings of the paper, each also listed in the design notes):
 *   - bit c of a string is bit (c & 63) of word (c >> 6); words per string
 *     W = ceil(ell / 64); unused high bits are zero.
 *   - sign(t) is 1 iff t > 0 (Eq. 3), so t == 0 gives 0.
 *   - block b (0-based) of a string covers bits [floor(b*ell/k),
 *     floor((b+1)*ell/k)) (Sec. 2.2 asks only for blocks of nearly the same size).
 *   - a pair co-grouped under kept block set K is reported under K only if
 *     K is the set of its k-d lowest-index equal blocks (the per-mask
 *     de-duplication Sec. 2.2 leaves to the original MSM paper), and only in
 *     the first replicate where its Hamming distance is <= d (Appendix,
 *     first trick).
 *   - pairs are encoded as (uint64)i << 32 | j with i < j.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------
 * Counter-based generator: Philox4x64-10 (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC 2011), restated from
 * its published definition.  Used only to restate the device-side
 * generation of the Gaussian projection matrix R of Eq. 3.
 * ---------------------------------------------------------------------- */
void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2],
                       uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        unsigned __int128 p0 = (unsigned __int128)M0 * c0;
        unsigned __int128 p1 = (unsigned __int128)M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Standard normal samples for element indices [0, count): element e comes
 * from Philox block e/4 (counter {e/4, 0, 0, 0}, key {seed, 0}); words
 * (w0, w1) feed one Box-Muller pair for lanes 0 and 1, (w2, w3) for lanes 2
 * and 3.  u1 = (w>>11 + 1) * 2^-53 lies in (0, 1], u2 = (w>>11) * 2^-53 in
 * [0, 1); z = sqrt(-2 ln u1) * (cos | sin)(2 pi u2), computed in double and
 * rounded to float. */
void orc_gaussian(uint64_t seed, int64_t count, float* out) {
    const double two_pi = 2.0 * 3.14159265358979323846;
    for (int64_t e0 = 0; e0 < count; e0 += 4) {
        uint64_t ctr[4] = {(uint64_t)(e0 / 4), 0, 0, 0};
        uint64_t key[2] = {seed, 0};
        uint64_t w[4];
        orc_philox4x64_10(ctr, key, w);
        for (int pair = 0; pair < 2; ++pair) {
            double u1 = (double)((w[2 * pair] >> 11) + 1) * 0x1.0p-53;
            double u2 = (double)(w[2 * pair + 1] >> 11) * 0x1.0p-53;
            double rad = sqrt(-2.0 * log(u1));
            double ang = two_pi * u2;
            double z0 = rad * cos(ang), z1 = rad * sin(ang);
            if (e0 + 2 * pair < count) out[e0 + 2 * pair] = (float)z0;
            if (e0 + 2 * pair + 1 < count) out[e0 + 2 * pair + 1] = (float)z1;
        }
    }
}

/* ------------------------------------------------------------------------
 * Eq. 3: s_ic = sign(r_c^T x_i), one string pool per replicate (Sec. 4.1).
 * X: double [n][D] (exact copies of the stored values), R: double
 * [Q][D][ell].  Output S: uint64 [Q][n][W].  t is accumulated in double by
 * sequential fma over the D coordinates, starting from 0.
 * ---------------------------------------------------------------------- */
void orc_project(const double* X, int64_t n, int D, const double* R, int Q,
                 int ell, uint64_t* S) {
    int W = (ell + 63) / 64;
    memset(S, 0, sizeof(uint64_t) * (size_t)Q * (size_t)n * (size_t)W);
    for (int q = 0; q < Q; ++q)
        for (int64_t i = 0; i < n; ++i)
            for (int c = 0; c < ell; ++c) {
                double t = 0.0;
                for (int dd = 0; dd < D; ++dd)
                    t = fma(X[i * D + dd], R[((size_t)q * D + dd) * ell + c], t);
                if (t > 0.0)
                    S[((size_t)q * n + i) * W + (c >> 6)] |= 1ULL << (c & 63);
            }
}

/* The projection value t itself (same arithmetic as orc_project). */
double orc_project_value(const double* x, int D, const double* Rq, int ell,
                         int c) {
    double t = 0.0;
    for (int dd = 0; dd < D; ++dd) t = fma(x[dd], Rq[(size_t)dd * ell + c], t);
    return t;
}

/* ------------------------------------------------------------------------
 * Hamming distance (Sec. 2.1): number of positions where two strings differ.
 * ---------------------------------------------------------------------- */
static int ham(const uint64_t* a, const uint64_t* b, int W) {
    int h = 0;
    for (int w = 0; w < W; ++w) h += __builtin_popcountll(a[w] ^ b[w]);
    return h;
}

/* Eq. 1, by definition: every pair i < j of one pool with Hamming distance
 * <= d, in increasing (i, j) order.  Returns the number of pairs; writes at
 * most cap of them. */
int64_t orc_ham_pairs(const uint64_t* S, int64_t n, int ell, int d,
                      uint64_t* out, int64_t cap) {
    int W = (ell + 63) / 64;
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            if (ham(S + i * W, S + j * W, W) <= d) {
                if (m < cap) out[m] = ((uint64_t)i << 32) | (uint64_t)j;
                ++m;
            }
    return m;
}

/* ------------------------------------------------------------------------
 * Blockwise MSM (Sec. 2.2) over Q replicate pools (Eq. 5, Sec. 4.1) with
 * the replicate de-duplication of the Appendix.
 * ---------------------------------------------------------------------- */
typedef struct {
    uint64_t key[4]; /* the string with its masked-out blocks cleared */
    uint32_t idx;
} orc_item;

static int g_cmp_words; /* words compared by cmp_item (single-threaded) */

static int cmp_item(const void* pa, const void* pb) {
    const orc_item* a = (const orc_item*)pa;
    const orc_item* b = (const orc_item*)pb;
    for (int w = 0; w < g_cmp_words; ++w) {
        if (a->key[w] < b->key[w]) return -1;
        if (a->key[w] > b->key[w]) return 1;
    }
    return (a->idx > b->idx) - (a->idx < b->idx);
}

static int cmp_u64(const void* pa, const void* pb) {
    uint64_t a = *(const uint64_t*)pa, b = *(const uint64_t*)pb;
    return (a > b) - (a < b);
}

/* Bit mask (over W words) of block b. */
static void block_mask(int ell, int k, int b, uint64_t* m, int W) {
    int lo = (int)((int64_t)b * ell / k), hi = (int)((int64_t)(b + 1) * ell / k);
    for (int w = 0; w < W; ++w) m[w] = 0;
    for (int c = lo; c < hi; ++c) m[c >> 6] |= 1ULL << (c & 63);
}

/* Next k-subset of {0..k-1} in lexicographic order, as a sorted index
 * list; returns 0 after the last one. */
static int next_combination(int* a, int r, int k) {
    int i = r - 1;
    while (i >= 0 && a[i] == k - r + i) --i;
    if (i < 0) return 0;
    ++a[i];
    for (int j = i + 1; j < r; ++j) a[j] = a[j - 1] + 1;
    return 1;
}

/* stats (may be NULL): [0] masks run, [1] pairs inspected inside groups of
 * equal kept blocks, [2] pairs reported.  Returns the number of reported
 * pairs; writes at most cap of them, sorted ascending. */
int64_t orc_msm(const uint64_t* S, int64_t n, int ell, int k, int d, int Q,
                uint64_t* out, int64_t cap, int64_t* stats) {
    int W = (ell + 63) / 64;
    int r = k - d; /* kept blocks per mask */
    if (d < 0 || r < 1 || k > ell || W > 4) return -1;
    uint64_t bmask[64][4];
    for (int b = 0; b < k; ++b) block_mask(ell, k, b, bmask[b], W);

    orc_item* items = (orc_item*)malloc(sizeof(orc_item) * (size_t)(n > 0 ? n : 1));
    int64_t masks = 0, checks = 0, m = 0;
    int kept[64];

    for (int q = 0; q < Q; ++q) {
        const uint64_t* Sq = S + (size_t)q * n * W;
        for (int j = 0; j < r; ++j) kept[j] = j;
        do {
            /* K as a bit set over blocks, and the kept-bit mask. */
            uint64_t K = 0, keep[4] = {0, 0, 0, 0};
            for (int j = 0; j < r; ++j) {
                K |= 1ULL << kept[j];
                for (int w = 0; w < W; ++w) keep[w] |= bmask[kept[j]][w];
            }
            ++masks;
            /* Sort the K-restricted strings (Sec. 2.1 / Fig. 1). */
            for (int64_t i = 0; i < n; ++i) {
                memset(items[i].key, 0, sizeof(items[i].key));
                for (int w = 0; w < W; ++w) items[i].key[w] = Sq[i * W + w] & keep[w];
                items[i].idx = (uint32_t)i;
            }
            g_cmp_words = W;
            qsort(items, (size_t)n, sizeof(orc_item), cmp_item);
            /* Walk the equivalence classes and inspect every pair in each. */
            int64_t s = 0;
            while (s < n) {
                int64_t e = s + 1;
                while (e < n && memcmp(items[e].key, items[s].key, sizeof(uint64_t) * W) == 0) ++e;
                for (int64_t a = s; a < e; ++a)
                    for (int64_t b = a + 1; b < e; ++b) {
                        ++checks;
                        uint32_t i = items[a].idx, jj = items[b].idx;
                        if (i > jj) { uint32_t t = i; i = jj; jj = t; }
                        const uint64_t* si = Sq + (size_t)i * W;
                        const uint64_t* sj = Sq + (size_t)jj * W;
                        if (ham(si, sj, W) > d) continue; /* Sec. 2.2 filter */
                        /* equal-block set and its r lowest members */
                        uint64_t low = 0;
                        int cnt = 0;
                        for (int b2 = 0; b2 < k && cnt < r; ++b2) {
                            int eq = 1;
                            for (int w = 0; w < W; ++w)
                                if ((si[w] ^ sj[w]) & bmask[b2][w]) eq = 0;
                            if (eq) { low |= 1ULL << b2; ++cnt; }
                        }
                        if (low != K) continue; /* reported under another mask */
                        int earlier = 0;        /* Appendix, first trick */
                        for (int g = 0; g < q && !earlier; ++g) {
                            const uint64_t* Sg = S + (size_t)g * n * W;
                            if (ham(Sg + (size_t)i * W, Sg + (size_t)jj * W, W) <= d) earlier = 1;
                        }
                        if (earlier) continue;
                        if (m < cap) out[m] = ((uint64_t)i << 32) | jj;
                        ++m;
                    }
                s = e;
            }
        } while (next_combination(kept, r, k));
    }
    free(items);
    if (out && cap > 0) qsort(out, (size_t)(m < cap ? m : cap), sizeof(uint64_t), cmp_u64);
    if (stats) { stats[0] = masks; stats[1] = checks; stats[2] = m; }
    return m;
}

/* Position masking of Sec. 2.1 (every C of size d over the ell positions),
 * pairs merged over all C; the comparison point for blockwise masking.
 * Returns the number of distinct pairs; writes at most cap, sorted. */
int64_t orc_msm_positions(const uint64_t* S, int64_t n, int ell, int d,
                          uint64_t* out, int64_t cap, int64_t* sorts) {
    int W = (ell + 63) / 64;
    int r = ell - d;
    if (r < 1 || W > 4) return -1;
    orc_item* items = (orc_item*)malloc(sizeof(orc_item) * (size_t)(n > 0 ? n : 1));
    size_t bufcap = 1024, nb = 0;
    uint64_t* buf = (uint64_t*)malloc(sizeof(uint64_t) * bufcap);
    int kept[256];
    int64_t nsorts = 0;
    for (int j = 0; j < r; ++j) kept[j] = j;
    do {
        uint64_t keep[4] = {0, 0, 0, 0};
        for (int j = 0; j < r; ++j) keep[kept[j] >> 6] |= 1ULL << (kept[j] & 63);
        ++nsorts;
        for (int64_t i = 0; i < n; ++i) {
            memset(items[i].key, 0, sizeof(items[i].key));
            for (int w = 0; w < W; ++w) items[i].key[w] = S[i * W + w] & keep[w];
            items[i].idx = (uint32_t)i;
        }
        g_cmp_words = W;
        qsort(items, (size_t)n, sizeof(orc_item), cmp_item);
        int64_t s = 0;
        while (s < n) {
            int64_t e = s + 1;
            while (e < n && memcmp(items[e].key, items[s].key, sizeof(uint64_t) * W) == 0) ++e;
            for (int64_t a = s; a < e; ++a)
                for (int64_t b = a + 1; b < e; ++b) {
                    uint32_t i = items[a].idx, jj = items[b].idx;
                    if (i > jj) { uint32_t t = i; i = jj; jj = t; }
                    if (nb == bufcap) { bufcap *= 2; buf = (uint64_t*)realloc(buf, sizeof(uint64_t) * bufcap); }
                    buf[nb++] = ((uint64_t)i << 32) | jj;
                }
            s = e;
        }
    } while (next_combination(kept, r, ell));
    qsort(buf, nb, sizeof(uint64_t), cmp_u64);
    int64_t m = 0;
    for (size_t t = 0; t < nb; ++t)
        if (t == 0 || buf[t] != buf[t - 1]) {
            if (m < cap) out[m] = buf[t];
            ++m;
        }
    free(buf);
    free(items);
    if (sorts) *sorts = nsorts;
    return m;
}

/* ------------------------------------------------------------------------
 * Distances.  metric 0: cosine distance, Eq. 2, evaluated as
 *   1 - dot / (sqrt(|x_i|^2) * sqrt(|x_j|^2))
 * with dot and the squared norms accumulated by sequential fma in double.
 * metric 1: Euclidean distance sqrt(sum_c (x_ic - x_jc)^2), same style.
 * ---------------------------------------------------------------------- */
double orc_distance(const double* xi, const double* xj, int D, int metric) {
    if (metric == 0) {
        double dot = 0.0, ni = 0.0, nj = 0.0;
        for (int c = 0; c < D; ++c) dot = fma(xi[c], xj[c], dot);
        for (int c = 0; c < D; ++c) ni = fma(xi[c], xi[c], ni);
        for (int c = 0; c < D; ++c) nj = fma(xj[c], xj[c], nj);
        return 1.0 - dot / (sqrt(ni) * sqrt(nj));
    }
    double s = 0.0;
    for (int c = 0; c < D; ++c) {
        double t = xi[c] - xj[c];
        s = fma(t, t, s);
    }
    return sqrt(s);
}

void orc_dist(const double* X, int64_t n, int D, int metric,
              const uint64_t* pairs, int64_t m, double* dist) {
    (void)n;
    for (int64_t t = 0; t < m; ++t) {
        uint64_t i = pairs[t] >> 32, j = pairs[t] & 0xffffffffULL;
        dist[t] = orc_distance(X + i * D, X + j * D, D, metric);
    }
}

/* Def. 1.1 by exhaustive comparison: every pair i < j with distance <= eps,
 * in increasing (i, j) order.  Returns the count; writes at most cap. */
int64_t orc_eps_bruteforce(const double* X, int64_t n, int D, int metric,
                           double eps, uint64_t* out, double* dist,
                           int64_t cap) {
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            double v = orc_distance(X + i * D, X + j * D, D, metric);
            if (v <= eps) {
                if (m < cap) {
                    out[m] = ((uint64_t)i << 32) | (uint64_t)j;
                    if (dist) dist[m] = v;
                }
                ++m;
            }
        }
    return m;
}

/* ========================================================================
 * E2LSH symbol strings (Sec. 3.1: an LSH family turns each vector into a
 * sequence of integer symbols; here the Euclidean family of Datar et al.
 * 2004, whose width w Sec. 4.3 tunes).
 * ---------------------------------------------------------------------- */

/* Offsets of the buckets: u_{q,c} in [0, 1), one per (replicate, symbol):
 * the top 24 bits of word 0 of Philox4x64-10 block q * ell + c under key
 * {seed, 2}, times 2^-24 (exactly representable in float). */
void orc_e2lsh_offsets(uint64_t seed, int Q, int ell, float* out) {
    for (int64_t e = 0; e < (int64_t)Q * ell; ++e) {
        uint64_t ctr[4] = {(uint64_t)e, 0, 0, 0}, key[2] = {seed, 2}, o[4];
        orc_philox4x64_10(ctr, key, o);
        out[e] = (float)((double)(o[0] >> 40) * 0x1.0p-24);
    }
}

/* Symbol c of replicate q for point x: h = floor(t / width + u_{q,c}) with
 * t = r_{q,c}^T x accumulated in double by sequential fma (as Eq. 3) and the
 * division and addition done in double; the stored symbol is the low sw
 * bits of h (two's complement).  Symbols are packed LSB first: symbol c
 * occupies bits [c sw, (c + 1) sw) of the string. */
void orc_project_e2lsh(const double* X, int64_t n, int D, const double* R, int Q,
                       int ell, const float* u, double width, int sw, uint64_t* S) {
    int W = (ell * sw + 63) / 64;
    uint64_t mask = (sw >= 64) ? ~0ULL : ((1ULL << sw) - 1);
    memset(S, 0, sizeof(uint64_t) * (size_t)Q * (size_t)n * (size_t)W);
    for (int q = 0; q < Q; ++q)
        for (int64_t i = 0; i < n; ++i)
            for (int c = 0; c < ell; ++c) {
                double t = 0.0;
                for (int dd = 0; dd < D; ++dd)
                    t = fma(X[i * D + dd], R[((size_t)q * D + dd) * ell + c], t);
                double z = t / width + (double)u[(size_t)q * ell + c];
                int64_t h = (int64_t)floor(z);
                uint64_t sym = (uint64_t)h & mask;
                int bit = c * sw;
                S[((size_t)q * n + i) * W + (bit >> 6)] |= sym << (bit & 63);
            }
}

/* Symbol c (sw bits) of a string. */
static uint64_t sym_at(const uint64_t* s, int c, int sw) {
    int bit = c * sw;
    uint64_t v = s[bit >> 6] >> (bit & 63);
    return sw >= 64 ? v : (v & ((1ULL << sw) - 1));
}

/* Symbol Hamming distance: number of symbols that differ. */
static int mism(const uint64_t* a, const uint64_t* b, int ell, int sw) {
    int h = 0;
    for (int c = 0; c < ell; ++c) h += sym_at(a, c, sw) != sym_at(b, c, sw);
    return h;
}

/* Eq. 1 over symbols, by definition: pairs i < j of one pool with at most
 * d differing symbols, in increasing order; returns the count. */
int64_t orc_sym_pairs(const uint64_t* S, int64_t n, int ell, int sw, int d,
                      uint64_t* out, int64_t cap) {
    int W = (ell * sw + 63) / 64;
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            if (mism(S + i * W, S + j * W, ell, sw) <= d) {
                if (m < cap) out[m] = ((uint64_t)i << 32) | (uint64_t)j;
                ++m;
            }
    return m;
}

/* Blockwise MSM (Sec. 2.2) over symbol strings: block b holds symbols
 * [floor(b ell / k), floor((b + 1) ell / k)); a pair is inspected in every
 * group of equal kept blocks, kept if at most d symbols differ, reported
 * under the kept set made of its k - d lowest-index equal blocks, and only
 * in the first replicate where it is within d (Appendix).  stats as
 * orc_msm.  Returns the number of reported pairs, sorted ascending. */
int64_t orc_msm_sym(const uint64_t* S, int64_t n, int ell, int sw, int k, int d, int Q,
                    uint64_t* out, int64_t cap, int64_t* stats) {
    int W = (ell * sw + 63) / 64;
    int r = k - d;
    if (d < 0 || r < 1 || k > ell || W > 4 || k > 64) return -1;
    int blo[65];
    for (int b = 0; b <= k; ++b) blo[b] = (int)((int64_t)b * ell / k);
    orc_item* items = (orc_item*)malloc(sizeof(orc_item) * (size_t)(n > 0 ? n : 1));
    int64_t masks = 0, checks = 0, m = 0;
    int kept[64];
    for (int q = 0; q < Q; ++q) {
        const uint64_t* Sq = S + (size_t)q * n * W;
        for (int j = 0; j < r; ++j) kept[j] = j;
        do {
            uint64_t K = 0;
            for (int j = 0; j < r; ++j) K |= 1ULL << kept[j];
            ++masks;
            /* key: the string with the masked-out blocks' symbols cleared */
            for (int64_t i = 0; i < n; ++i) {
                memset(items[i].key, 0, sizeof(items[i].key));
                for (int j = 0; j < r; ++j)
                    for (int c = blo[kept[j]]; c < blo[kept[j] + 1]; ++c) {
                        int bit = c * sw;
                        items[i].key[bit >> 6] |= sym_at(Sq + i * W, c, sw) << (bit & 63);
                    }
                items[i].idx = (uint32_t)i;
            }
            g_cmp_words = W;
            qsort(items, (size_t)n, sizeof(orc_item), cmp_item);
            int64_t s = 0;
            while (s < n) {
                int64_t e = s + 1;
                while (e < n && memcmp(items[e].key, items[s].key, sizeof(uint64_t) * W) == 0) ++e;
                for (int64_t a = s; a < e; ++a)
                    for (int64_t b = a + 1; b < e; ++b) {
                        ++checks;
                        uint32_t i = items[a].idx, jj = items[b].idx;
                        if (i > jj) { uint32_t t = i; i = jj; jj = t; }
                        const uint64_t* si = Sq + (size_t)i * W;
                        const uint64_t* sj = Sq + (size_t)jj * W;
                        if (mism(si, sj, ell, sw) > d) continue;
                        uint64_t low = 0;
                        int cnt = 0;
                        for (int b2 = 0; b2 < k && cnt < r; ++b2) {
                            int eq = 1;
                            for (int c = blo[b2]; c < blo[b2 + 1]; ++c)
                                if (sym_at(si, c, sw) != sym_at(sj, c, sw)) eq = 0;
                            if (eq) { low |= 1ULL << b2; ++cnt; }
                        }
                        if (low != K) continue;
                        int earlier = 0;
                        for (int g = 0; g < q && !earlier; ++g) {
                            const uint64_t* Sg = S + (size_t)g * n * W;
                            if (mism(Sg + (size_t)i * W, Sg + (size_t)jj * W, ell, sw) <= d)
                                earlier = 1;
                        }
                        if (earlier) continue;
                        if (m < cap) out[m] = ((uint64_t)i << 32) | jj;
                        ++m;
                    }
                s = e;
            }
        } while (next_combination(kept, r, k));
    }
    free(items);
    if (out && cap > 0) qsort(out, (size_t)(m < cap ? m : cap), sizeof(uint64_t), cmp_u64);
    if (stats) { stats[0] = masks; stats[1] = checks; stats[2] = m; }
    return m;
}
