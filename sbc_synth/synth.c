/*
 * Seeded synthetic bipartite graphs (input generation only): the Chung-Lu
 * sampler and the CSR builder of sbc_synth, in C for large graphs and large
 * batches. Holds none of the counting method's arithmetic.
 *
 * Randomness is counter-based: draw i of stream s for seed S is
 * splitmix64(key(S, s) + i * 0x9E3779B97F4A7C15), key(S, s) =
 * splitmix64(splitmix64(S) ^ s), with splitmix64 the public-domain mixer of
 * S. Vigna (Steele, Lea, Flood 2014). Uniform doubles take the top 53 bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ull

static inline uint64_t mix(uint64_t x) {
    uint64_t z = x + GOLDEN;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline uint64_t stream_key(uint64_t seed, uint64_t stream) { return mix(mix(seed) ^ stream); }

static inline double unif(uint64_t key, uint64_t i) {
    return (double)(mix(key + i * GOLDEN) >> 11) * (1.0 / 9007199254740992.0);
}

/* Expected degrees (i+1)^(-1/(gamma-1)), summing to total, each at most cap
 * (the excess is spread over the others by rescaling, up to 64 rounds). */
static void weights(int64_t n, double gamma, double total, double cap, double *w) {
    double s = 0;
    for (int64_t i = 0; i < n; i++) {
        w[i] = pow((double)(i + 1), -1.0 / (gamma - 1.0));
        s += w[i];
    }
    for (int64_t i = 0; i < n; i++) w[i] *= total / s;
    if (cap < total / (double)n) cap = total / (double)n;
    for (int it = 0; it < 64; it++) {
        int64_t over = 0;
        double fs = 0;
        for (int64_t i = 0; i < n; i++) {
            if (w[i] > cap) {
                w[i] = cap;
                over++;
            }
        }
        if (!over) break;
        for (int64_t i = 0; i < n; i++)
            if (w[i] < cap) fs += w[i];
        double rest = total - cap * (double)over;
        /* clipped entries equal cap exactly; the rest are rescaled */
        int64_t nfree = 0;
        for (int64_t i = 0; i < n; i++) nfree += w[i] < cap;
        if (fs <= 0 || rest <= 0 || nfree == 0) break;
        for (int64_t i = 0; i < n; i++)
            if (w[i] < cap) w[i] *= rest / fs;
    }
}

/* First index with cdf[idx] > x (cdf ascending), clamped to n-1. */
static inline int64_t upper(const double *cdf, int64_t n, double x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (cdf[mid] > x) hi = mid; else lo = mid + 1;
    }
    return lo < n ? lo : n - 1;
}

typedef struct {
    uint64_t key;
    uint64_t idx;
} kp_t;

static int cmp_kp(const void *a, const void *b) {
    const kp_t *x = (const kp_t *)a, *y = (const kp_t *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* perm[i] = rank of draw i of stream `stream` among n draws (a random
 * permutation of 0..n-1: ids are relabelled by it). */
static int permutation(uint64_t seed, uint64_t stream, int64_t n, int64_t *perm) {
    kp_t *kp = (kp_t *)malloc(sizeof(kp_t) * (size_t)(n > 0 ? n : 1));
    if (!kp) return -1;
    uint64_t key = stream_key(seed, stream);
    for (int64_t i = 0; i < n; i++) {
        kp[i].key = mix(key + (uint64_t)i * GOLDEN);
        kp[i].idx = (uint64_t)i;
    }
    qsort(kp, (size_t)n, sizeof(kp_t), cmp_kp);
    /* argsort: perm[j] = index of the j-th smallest key; id i -> perm[i] */
    for (int64_t j = 0; j < n; j++) perm[j] = (int64_t)kp[j].idx;
    free(kp);
    return 0;
}

/*
 * m distinct (u, v) pairs of a bipartite Chung-Lu graph in draw order of
 * their first occurrence; U ends from stream 1, V ends from stream 2, drawn in
 * rounds of 1.25 * (missing) + 64; ids relabelled by the permutations of
 * streams 3 (U) and 4 (V). Returns 0, -1 on allocation failure, -2 when m
 * distinct pairs cannot be drawn.
 */
int synth_chung_lu(uint64_t seed, int64_t n_u, int64_t n_v, int64_t m, double gamma_u,
                   double gamma_v, double cap_u, double cap_v, int64_t *out_u, int64_t *out_v) {
    if (m > n_u * n_v) return -2;
    double *cu = (double *)malloc(sizeof(double) * (size_t)(n_u > 0 ? n_u : 1));
    double *cv = (double *)malloc(sizeof(double) * (size_t)(n_v > 0 ? n_v : 1));
    int64_t cap = 1;
    while (cap < 2 * m + 2) cap <<= 1;
    uint64_t *set = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)cap);
    int64_t *pu = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_u > 0 ? n_u : 1));
    int64_t *pv = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_v > 0 ? n_v : 1));
    int rc = 0;
    if (!cu || !cv || !set || !pu || !pv) {
        rc = -1;
        goto done;
    }
    weights(n_u, gamma_u, (double)m, cap_u, cu);
    weights(n_v, gamma_v, (double)m, cap_v, cv);
    for (int64_t i = 1; i < n_u; i++) cu[i] += cu[i - 1];
    for (int64_t i = 1; i < n_v; i++) cv[i] += cv[i - 1];
    memset(set, 0xFF, sizeof(uint64_t) * (size_t)cap);
    {
        const uint64_t ku = stream_key(seed, 1), kv = stream_key(seed, 2);
        int64_t have = 0;
        uint64_t drawn = 0;
        for (int round = 0; round < 200 && have < m; round++) {
            int64_t k = (int64_t)((double)(m - have) * 1.25) + 64;
            for (int64_t i = 0; i < k && have < m; i++) {
                uint64_t t = drawn + (uint64_t)i;
                int64_t u = upper(cu, n_u, unif(ku, t) * cu[n_u - 1]);
                int64_t v = upper(cv, n_v, unif(kv, t) * cv[n_v - 1]);
                uint64_t key = (uint64_t)u * (uint64_t)n_v + (uint64_t)v;
                uint64_t h = mix(key) & (uint64_t)(cap - 1);
                for (;;) {
                    if (set[h] == ~0ull) {
                        set[h] = key;
                        out_u[have] = u;
                        out_v[have] = v;
                        have++;
                        break;
                    }
                    if (set[h] == key) break;
                    h = (h + 1) & (uint64_t)(cap - 1);
                }
            }
            drawn += (uint64_t)k;
        }
        if (have < m) {
            rc = -2;
            goto done;
        }
    }
    if (permutation(seed, 3, n_u, pu) || permutation(seed, 4, n_v, pv)) {
        rc = -1;
        goto done;
    }
    for (int64_t e = 0; e < m; e++) {
        out_u[e] = pu[out_u[e]];
        out_v[e] = pv[out_v[e]];
    }
done:
    free(cu);
    free(cv);
    free(set);
    free(pu);
    free(pv);
    return rc;
}

typedef struct {
    int32_t v;
    int8_t s;
} vs_t;

static int cmp_vs(const void *a, const void *b) {
    int32_t x = ((const vs_t *)a)->v, y = ((const vs_t *)b)->v;
    return (x > y) - (x < y);
}

/* CSR over U from edge arrays: rows by u, each row sorted by v, signs
 * carried along. off: n_u+1, col/sgn: m. */
int synth_csr(int64_t n_u, int64_t m, const int64_t *u, const int64_t *v, const int8_t *s,
              int64_t *off, int32_t *col, int8_t *sgn) {
    vs_t *buf = (vs_t *)malloc(sizeof(vs_t) * (size_t)(m > 0 ? m : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_u + 1));
    if (!buf || !fill) {
        free(buf);
        free(fill);
        return -1;
    }
    memset(off, 0, sizeof(int64_t) * (size_t)(n_u + 1));
    for (int64_t e = 0; e < m; e++) off[u[e] + 1]++;
    for (int64_t i = 0; i < n_u; i++) off[i + 1] += off[i];
    memcpy(fill, off, sizeof(int64_t) * (size_t)(n_u + 1));
    for (int64_t e = 0; e < m; e++) {
        int64_t p = fill[u[e]]++;
        buf[p].v = (int32_t)v[e];
        buf[p].s = s[e];
    }
    for (int64_t i = 0; i < n_u; i++)
        qsort(buf + off[i], (size_t)(off[i + 1] - off[i]), sizeof(vs_t), cmp_vs);
    for (int64_t e = 0; e < m; e++) {
        col[e] = buf[e].v;
        sgn[e] = buf[e].s;
    }
    free(buf);
    free(fill);
    return 0;
}
