/*
 * Seeded synthetic web-like graph generator.
 *
 * This file produces INPUTS only (edge lists and personalised seed sets). It holds none of the
 * D-iteration's arithmetic, so both the CPU oracle and the CUDA library may consume what it
 * writes. The graphs stand in for the paper's web graphs (uk-2007-05 prefixes, Section 2.6,
 * Table 1: L/N 12-41, a few percent dangling nodes, 10-24% loop nodes, max_in >> max_out),
 * which are not available here.
 *
 * Random numbers: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014) used as a counter-based generator: draw(key, c) is the c-th output
 * of a SplitMix64 stream whose state starts at `key`. Every draw is addressed by (purpose, node,
 * slot), so the output does not depend on the number of threads.
 *
 * Recipe (one call per graph):
 *   1. Zero-in-degree chains: about chain_frac*N nodes form chains of length
 *      chain_min..chain_max laid out on contiguous ascending ids; a chain node's only in-link
 *      comes from its predecessor, so no other link may point at a chain node.
 *   2. Dangling nodes: exactly floor(p_dangling*N) non-chain nodes, picked by a seeded partial
 *      Fisher-Yates shuffle, get no out-links.
 *   3. Out-degree of every other node: discrete power law P(k) ~ k^-alpha on [a, cap]; a mix of
 *      a and a+1 as the lower end hits the requested mean out-degree (mean_out <= 0: a = 1).
 *   4. Self-loops: with probability p_loop a non-chain node spends one of its links on itself.
 *   5. Destinations: with probability p_local uniform in [i-window, i+window] (host locality,
 *      retried when it lands outside [0,N), on i itself or on a chain node); otherwise static
 *      preferential attachment: rank r drawn from a continuous power law with density
 *      ~ x^(-1/(alpha-1)), mapped through a seeded permutation of the non-chain nodes, which
 *      gives a power-law in-degree with exponent alpha.
 *   Duplicate links are kept; the consumer removes them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
/* c-th output of the SplitMix64 stream whose state starts at key */
static inline uint64_t draw(uint64_t key, uint64_t c) { return sm64_mix(key + (c + 1) * GOLDEN); }
static inline double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }
/* uniform integer in [0, range) without division: high half of a 64x64 product */
static inline uint64_t below(uint64_t x, uint64_t range) {
    return (uint64_t)(((__uint128_t)x * (__uint128_t)range) >> 64);
}
static uint64_t purpose_key(uint64_t seed, uint64_t purpose) {
    return sm64_mix(seed ^ (purpose * 0xD1B54A32D192ED03ULL + 0x2545F4914F6CDD1DULL));
}

enum { P_CHAIN = 1, P_DANGLE = 2, P_DEG = 3, P_LOOP = 4, P_DST = 5, P_PERM = 6, P_SEEDS = 7 };

typedef struct {
    int64_t n;
    double p_dangling;
    double alpha;
    int32_t cap;
    double mean_out;   /* target mean out-degree of non-dangling nodes; <= 0 means a = 1 */
    double p_local;
    int32_t window;
    double chain_frac;
    int32_t chain_min, chain_max;
    double p_loop;
    uint64_t seed;
} gen_params;

/* Generator state shared by the count and fill passes. */
typedef struct {
    gen_params p;
    uint8_t *role;      /* 0 plain, 1 dangling, 2 chain (not last), 3 chain last */
    int32_t *deg;       /* out-links generated per node (before dedupe) */
    uint8_t *has_loop;
    int32_t *pa_perm;   /* rank -> node over non-chain nodes */
    int64_t n_pa;
    double *cdf_a, *cdf_b; /* CDFs over k = a..cap and a+1..cap */
    int32_t a;
    double q;           /* probability of using the a+1 table */
} gen_state;

static double zipf_mean(int32_t a, int32_t cap, double alpha) {
    double s0 = 0.0, s1 = 0.0;
    for (int32_t k = a; k <= cap; k++) {
        double w = pow((double)k, -alpha);
        s0 += w;
        s1 += w * k;
    }
    return s1 / s0;
}
static double *zipf_cdf(int32_t a, int32_t cap, double alpha) {
    int32_t m = cap - a + 1;
    double *c = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double s = 0.0;
    for (int32_t k = a; k <= cap; k++) s += pow((double)k, -alpha);
    double acc = 0.0;
    for (int32_t k = a; k <= cap; k++) {
        acc += pow((double)k, -alpha) / s;
        c[k - a] = acc;
    }
    c[m - 1] = 1.0;
    return c;
}
static int32_t zipf_draw(const double *cdf, int32_t a, int32_t cap, double u) {
    int32_t lo = 0, hi = cap - a; /* first index with cdf >= u */
    while (lo < hi) {
        int32_t mid = (lo + hi) >> 1;
        if (cdf[mid] >= u) hi = mid; else lo = mid + 1;
    }
    return a + lo;
}

static void free_state(gen_state *s) {
    free(s->role); free(s->deg); free(s->has_loop); free(s->pa_perm);
    free(s->cdf_a); free(s->cdf_b);
    memset(s, 0, sizeof(*s));
}

static int init_state(gen_state *s, const gen_params *p) {
    memset(s, 0, sizeof(*s));
    s->p = *p;
    int64_t n = p->n;
    s->role = (uint8_t *)calloc((size_t)n + 1, 1);
    s->deg = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    s->has_loop = (uint8_t *)calloc((size_t)n + 1, 1);
    s->pa_perm = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    if (!s->role || !s->deg || !s->has_loop || !s->pa_perm) { free_state(s); return -1; }

    /* 1. chains on contiguous ascending ids */
    uint64_t kc = purpose_key(p->seed, P_CHAIN);
    if (p->chain_frac > 0.0 && p->chain_max >= 2 && n >= 4 * (int64_t)p->chain_max) {
        double mean_len = 0.5 * (p->chain_min + p->chain_max);
        int64_t n_chains = (int64_t)floor(p->chain_frac * (double)n / mean_len);
        if (n_chains < 1) n_chains = 1;
        int64_t seg = n / n_chains;
        if (seg >= p->chain_max + 2) {
            for (int64_t c = 0; c < n_chains; c++) {
                int64_t len = p->chain_min + (int64_t)below(draw(kc, 2 * c), (uint64_t)(p->chain_max - p->chain_min + 1));
                int64_t start = c * seg + (int64_t)below(draw(kc, 2 * c + 1), (uint64_t)(seg - len));
                for (int64_t v = start; v < start + len; v++) s->role[v] = (v == start + len - 1) ? 3 : 2;
            }
        }
    }
    /* 2. dangling: exactly floor(p_dangling*n) non-chain nodes (partial Fisher-Yates) */
    int64_t m = 0;
    for (int64_t v = 0; v < n; v++) if (s->role[v] == 0) s->pa_perm[m++] = (int32_t)v;
    int64_t nd = (int64_t)floor(p->p_dangling * (double)n);
    if (nd > m) nd = m;
    uint64_t kd = purpose_key(p->seed, P_DANGLE);
    for (int64_t k = 0; k < nd; k++) {
        int64_t j = k + (int64_t)below(draw(kd, (uint64_t)k), (uint64_t)(m - k));
        int32_t t = s->pa_perm[k]; s->pa_perm[k] = s->pa_perm[j]; s->pa_perm[j] = t;
        s->role[s->pa_perm[k]] = 1;
    }
    /* preferential-attachment permutation over all non-chain nodes (dangling ones included) */
    m = 0;
    for (int64_t v = 0; v < n; v++) if (s->role[v] <= 1) s->pa_perm[m++] = (int32_t)v;
    s->n_pa = m;
    uint64_t kp = purpose_key(p->seed, P_PERM);
    for (int64_t k = 0; k + 1 < m; k++) {
        int64_t j = k + (int64_t)below(draw(kp, (uint64_t)k), (uint64_t)(m - k));
        int32_t t = s->pa_perm[k]; s->pa_perm[k] = s->pa_perm[j]; s->pa_perm[j] = t;
    }
    /* 3. out-degree law: lower end a, mixed with a+1 to hit mean_out */
    int32_t cap = p->cap < 1 ? 1 : p->cap;
    s->a = 1; s->q = 0.0;
    if (p->mean_out > 0.0) {
        int32_t a = 1;
        double ma = zipf_mean(1, cap, p->alpha);
        if (p->mean_out <= ma) { a = 1; s->q = 0.0; }
        else {
            double mb = ma;
            while (a < cap) {
                mb = zipf_mean(a + 1, cap, p->alpha);
                if (mb >= p->mean_out) break;
                a++; ma = mb;
            }
            if (a >= cap) { a = cap; s->q = 0.0; }
            else s->q = (p->mean_out - ma) / (mb - ma);
        }
        s->a = a;
    }
    s->cdf_a = zipf_cdf(s->a, cap, p->alpha);
    s->cdf_b = zipf_cdf(s->a < cap ? s->a + 1 : cap, cap, p->alpha);
    uint64_t kg = purpose_key(p->seed, P_DEG);
    uint64_t kl = purpose_key(p->seed, P_LOOP);
    for (int64_t v = 0; v < n; v++) {
        if (s->role[v] == 1) { s->deg[v] = 0; continue; }
        double u_mix = u01(draw(kg, 2 * (uint64_t)v));
        double u = u01(draw(kg, 2 * (uint64_t)v + 1));
        int32_t k = (u_mix < s->q && s->a < cap) ? zipf_draw(s->cdf_b, s->a + 1, cap, u)
                                                 : zipf_draw(s->cdf_a, s->a, cap, u);
        s->deg[v] = k;
        if (s->role[v] == 0 && p->p_loop > 0.0 && u01(draw(kl, (uint64_t)v)) < p->p_loop) s->has_loop[v] = 1;
    }
    return 0;
}

/* Destination of the link with global index `link`, sent by node i (regular links only). */
static int32_t pick_dst(const gen_state *s, uint64_t kdst, int64_t i, int64_t link) {
    const gen_params *p = &s->p;
    int64_t n = p->n;
    for (int attempt = 0; attempt < 16; attempt++) {
        uint64_t c = (uint64_t)link * 64 + (uint64_t)attempt * 3;
        double u = u01(draw(kdst, c));
        int64_t j;
        if (u < p->p_local && attempt < 8) {
            int64_t off = (int64_t)below(draw(kdst, c + 1), (uint64_t)(2 * p->window + 1)) - p->window;
            j = i + off;
            if (j < 0 || j >= n || j == i || s->role[j] >= 2) continue;
            return (int32_t)j;
        }
        double gam = 1.0 / (p->alpha - 1.0);
        double M = (double)s->n_pa;
        double x;
        double uu = u01(draw(kdst, c + 2));
        if (fabs(1.0 - gam) < 1e-12) x = exp(uu * log(M + 1.0));
        else x = pow(1.0 + uu * (pow(M + 1.0, 1.0 - gam) - 1.0), 1.0 / (1.0 - gam));
        int64_t r = (int64_t)floor(x) - 1;
        if (r < 0) r = 0;
        if (r >= s->n_pa) r = s->n_pa - 1;
        j = s->pa_perm[r];
        if (j == i) continue;
        return (int32_t)j;
    }
    /* give up: nearest non-chain node other than i (deterministic) */
    for (int64_t t = 1; t < n; t++) {
        int64_t j = (i + t) % n;
        if (s->role[j] < 2) return (int32_t)j;
    }
    return (int32_t)i;
}

/* Pass 1: per-node out-link counts (before dedupe) into deg_out[n]; returns total links. */
int64_t gen_graph_count(const gen_params *p, int32_t *deg_out) {
    gen_state s;
    if (p->n <= 0 || init_state(&s, p) != 0) return -1;
    int64_t total = 0;
    for (int64_t v = 0; v < p->n; v++) { deg_out[v] = s.deg[v]; total += s.deg[v]; }
    free_state(&s);
    return total;
}

/* Pass 2: fill src/dst (length = sum of deg_out from pass 1). Returns links written. */
int64_t gen_graph_fill(const gen_params *p, int32_t *src, int32_t *dst) {
    gen_state s;
    if (p->n <= 0 || init_state(&s, p) != 0) return -1;
    int64_t n = p->n;
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!off) { free_state(&s); return -1; }
    off[0] = 0;
    for (int64_t v = 0; v < n; v++) off[v + 1] = off[v] + s.deg[v];
    uint64_t kdst = purpose_key(p->seed, P_DST);
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < n; v++) {
        int64_t o = off[v];
        int32_t k = s.deg[v];
        int32_t slot = 0;
        if (k == 0) continue;
        if (s.role[v] == 2) { src[o] = (int32_t)v; dst[o] = (int32_t)(v + 1); o++; slot++; }
        else if (s.has_loop[v]) { src[o] = (int32_t)v; dst[o] = (int32_t)v; o++; slot++; }
        for (; slot < k; slot++, o++) {
            src[o] = (int32_t)v;
            dst[o] = pick_dst(&s, kdst, v, o);
        }
    }
    int64_t total = off[n];
    free(off);
    free_state(&s);
    return total;
}

/* Personalised seed sets: k sets with sizes floor(exp(U(0, ln max_size))) clamped to
 * [1, max_size], members uniform over [0, n) without replacement (rejection on a small set).
 * sizes_out[k], seeds_out[sum sizes] (caller gives room for k*max_size). Returns total seeds. */
int64_t gen_seed_sets(int64_t n, int32_t k, int32_t max_size, uint64_t seed,
                      int32_t *sizes_out, int32_t *seeds_out) {
    uint64_t ks = purpose_key(seed, P_SEEDS);
    int64_t pos = 0;
    if (max_size > n) max_size = (int32_t)n;
    for (int32_t r = 0; r < k; r++) {
        double u = u01(draw(ks, (uint64_t)r * 1000003ULL));
        int64_t sz = (int64_t)floor(exp(u * log((double)max_size)));
        if (sz < 1) sz = 1;
        if (sz > max_size) sz = max_size;
        sizes_out[r] = (int32_t)sz;
        uint64_t c = (uint64_t)r * 1000003ULL + 1;
        for (int64_t t = 0; t < sz; t++) {
            for (;;) {
                int32_t cand = (int32_t)below(draw(ks, c++), (uint64_t)n);
                int dup = 0;
                for (int64_t q = 0; q < t; q++) if (seeds_out[pos + q] == cand) { dup = 1; break; }
                if (!dup) { seeds_out[pos + t] = cand; break; }
            }
        }
        pos += sz;
    }
    return pos;
}

/* Uniform u64 stream for tests that need extra seeded integers (e.g. edge permutations). */
/* raw stream outputs draw(key, first + i), for checking the generator against SplitMix64's
   published sequence */
void gen_draw(uint64_t key, uint64_t first, int64_t count, uint64_t *out) {
    for (int64_t i = 0; i < count; i++) out[i] = draw(key, first + (uint64_t)i);
}

void gen_u64(uint64_t seed, uint64_t purpose, int64_t count, uint64_t *out) {
    uint64_t k = purpose_key(seed, 100 + purpose);
    for (int64_t i = 0; i < count; i++) out[i] = draw(k, (uint64_t)i);
}
