/*
 * Second CPU counter of balanced (p,q)-bicliques: the wedge-centric method
 * (BBWC, Algorithm 1, Section 4.2), as an independent cross-check of the
 * oracle in sbc_oracle.c.
 *
 * TEST INFRASTRUCTURE ONLY, like sbc_oracle.c: nothing on the product path
 * calls, links or loads it. It shares no code with sbc_oracle.c nor with the
 * CUDA path (its own adjacency lists, priorities, hashing and binomials).
 *
 * Method (Section 4.2). Vertices of the anchor side S are ordered by the
 * priority rho of Definition 4 (degree, then id). A signed p-wedge is
 * <u, w_1, ..., w_{p-1}, v> with u, w_i in S, v adjacent to all of them and
 * rho(u) > rho(w_1) > ... > rho(w_{p-1}). Its type is the word c_1 ... c_{p-1}
 * with c_i = s when sign(u, v) = sign(w_i, v) and d otherwise. By Lemma 1 all
 * p-wedges of a balanced biclique have one type, and conversely the p-wedges
 * of one anchor set {u, w_1, ..., w_{p-1}} and one type share their common
 * neighbours' sign pattern relative to u, so any q of those neighbours close
 * a balanced biclique. For each u the method counts, per type and per set
 * (w_1, ..., w_{p-1}), the wedges through every v in Gamma(u) (each v adds
 * one wedge per (p-1)-subset of its lower-priority neighbours), then adds
 * binom(count, q) for every (type, set) bucket. Every balanced biclique is
 * counted once: from its member of highest priority, in the bucket of its
 * type.
 *
 * Exact arithmetic: binomials by the multiplicative formula in unsigned
 * 128-bit integers (the running value after step i is binom(n - k + i, i)),
 * sums in unsigned 128 bits; a term or a sum that does not fit sets the
 * overflow status. OpenMP threads take anchors u, each with its own buckets
 * and partial sum.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

enum { BB_OK = 0, BB_OVERFLOW = 1, BB_NOMEM = 2, BB_INVALID = 3 };
#define BB_MAXP 8

/* Neighbour of an S vertex (an id on the other side) or of an other-side
 * vertex (an S vertex by priority rank), with the edge sign. */
typedef struct {
    int32_t to;
    int8_t neg; /* 1 when the edge is negative */
} nb_t;

typedef struct {
    int64_t ns, no;                 /* vertices of S and of the other side */
    int64_t *s_off, *o_off;         /* CSR offsets */
    nb_t *s_adj, *o_adj;            /* S -> other side; other side -> S (by rank, ascending) */
} graph_t;

static void graph_free(graph_t *g) {
    free(g->s_off);
    free(g->o_off);
    free(g->s_adj);
    free(g->o_adj);
    memset(g, 0, sizeof(*g));
}

typedef struct {
    int64_t deg, id;
} prio_t;

static int cmp_prio(const void *a, const void *b) {
    const prio_t *x = (const prio_t *)a, *y = (const prio_t *)b;
    if (x->deg != y->deg) return x->deg < y->deg ? -1 : 1;
    return x->id < y->id ? -1 : (x->id > y->id);
}

static int cmp_nb(const void *a, const void *b) {
    const nb_t *x = (const nb_t *)a, *y = (const nb_t *)b;
    return x->to < y->to ? -1 : (x->to > y->to);
}

/* Builds the lists with S vertices renamed by priority rank (rank 0 = lowest
 * rho), so that "lower priority than u" is "smaller rank". side 0: S = U (the
 * CSR rows); side 1: S = V. */
static int graph_build(graph_t *g, int64_t n_u, int64_t n_v, const int64_t *off,
                       const int32_t *col, const int8_t *sgn, int side) {
    memset(g, 0, sizeof(*g));
    const int64_t m = off[n_u];
    g->ns = side == 0 ? n_u : n_v;
    g->no = side == 0 ? n_v : n_u;
    /* each edge as (S vertex, other vertex, sign) */
    int64_t *es = malloc(sizeof(int64_t) * (size_t)(m + 1));
    int64_t *eo = malloc(sizeof(int64_t) * (size_t)(m + 1));
    int8_t *en = malloc((size_t)(m + 1));
    int64_t *sdeg = calloc((size_t)g->ns + 1, sizeof(int64_t));
    int64_t *odeg = calloc((size_t)g->no + 1, sizeof(int64_t));
    prio_t *pr = malloc(sizeof(prio_t) * (size_t)(g->ns + 1));
    int64_t *rank = malloc(sizeof(int64_t) * (size_t)(g->ns + 1));
    g->s_off = calloc((size_t)g->ns + 1, sizeof(int64_t));
    g->o_off = calloc((size_t)g->no + 1, sizeof(int64_t));
    g->s_adj = malloc(sizeof(nb_t) * (size_t)(m + 1));
    g->o_adj = malloc(sizeof(nb_t) * (size_t)(m + 1));
    int st = BB_OK;
    if (!es || !eo || !en || !sdeg || !odeg || !pr || !rank || !g->s_off || !g->o_off ||
        !g->s_adj || !g->o_adj) {
        st = BB_NOMEM;
        goto done;
    }
    for (int64_t x = 0; x < n_u; x++)
        for (int64_t e = off[x]; e < off[x + 1]; e++) {
            const int64_t y = col[e];
            if (y < 0 || y >= n_v || (sgn[e] != 1 && sgn[e] != -1)) {
                st = BB_INVALID;
                goto done;
            }
            es[e] = side == 0 ? x : y;
            eo[e] = side == 0 ? y : x;
            en[e] = sgn[e] < 0;
            sdeg[es[e]]++;
            odeg[eo[e]]++;
        }
    for (int64_t s = 0; s < g->ns; s++) {
        pr[s].deg = sdeg[s];
        pr[s].id = s;
    }
    qsort(pr, (size_t)g->ns, sizeof(prio_t), cmp_prio);
    for (int64_t r = 0; r < g->ns; r++) rank[pr[r].id] = r;
    /* offsets by rank on S, by id on the other side */
    for (int64_t r = 0; r < g->ns; r++) g->s_off[r + 1] = g->s_off[r] + pr[r].deg;
    for (int64_t o = 0; o < g->no; o++) g->o_off[o + 1] = g->o_off[o] + odeg[o];
    memset(sdeg, 0, sizeof(int64_t) * (size_t)(g->ns + 1));
    memset(odeg, 0, sizeof(int64_t) * (size_t)(g->no + 1));
    for (int64_t e = 0; e < m; e++) {
        const int64_t r = rank[es[e]], o = eo[e];
        g->s_adj[g->s_off[r] + sdeg[r]++] = (nb_t){(int32_t)o, en[e]};
        g->o_adj[g->o_off[o] + odeg[o]++] = (nb_t){(int32_t)r, en[e]};
    }
    for (int64_t o = 0; o < g->no; o++)
        qsort(g->o_adj + g->o_off[o], (size_t)(g->o_off[o + 1] - g->o_off[o]), sizeof(nb_t), cmp_nb);
done:
    free(es);
    free(eo);
    free(en);
    free(sdeg);
    free(odeg);
    free(pr);
    free(rank);
    if (st != BB_OK) graph_free(g);
    return st;
}

/* ---- exact binomials */

static uint64_t gcd64(uint64_t a, uint64_t b) {
    while (b) {
        const uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

/* binom(n, k) in 128 bits; *ovf set when it does not fit. */
static u128 choose(uint64_t n, int k, int *ovf) {
    if ((uint64_t)k > n) return 0;
    u128 r = 1;
    for (int i = 1; i <= k; i++) {
        /* r = binom(n - k + i - 1, i - 1); next = r * (n - k + i) / i */
        uint64_t f = n - (uint64_t)k + (uint64_t)i, d = (uint64_t)i;
        const uint64_t g1 = gcd64(f, d);
        f /= g1;
        d /= g1;
        /* d divides r (the product is divisible by i and gcd(f, d) = 1) */
        r /= d;
        if (f && r > ((u128)0 - 1) / f) {
            *ovf = 1;
            return 0;
        }
        r *= f;
    }
    return r;
}

static void add128(u128 *acc, u128 v, int *ovf) {
    const u128 s = *acc + v;
    if (s < *acc) *ovf = 1;
    *acc = s;
}

/* ---- buckets: (type, w_1 .. w_{p-1}) -> wedge count, open addressing */

typedef struct {
    int32_t w[BB_MAXP - 1];
    uint32_t type;
    uint64_t cnt; /* 0: empty slot */
} slot_t;

typedef struct {
    slot_t *s;
    uint64_t *occ; /* indices of the filled slots, `used` of them */
    uint64_t cap, used;
    int k; /* members w per key (p - 1) */
} buckets_t;

static uint64_t key_hash(const int32_t *w, int k, uint32_t type) {
    uint64_t h = 0x243F6A8885A308D3ull ^ type;
    for (int i = 0; i < k; i++) {
        h ^= (uint64_t)(uint32_t)w[i] + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
        h *= 0xBF58476D1CE4E5B9ull;
    }
    return h ^ (h >> 31);
}

static int buckets_grow(buckets_t *b) {
    const uint64_t ncap = b->cap ? 2 * b->cap : 1024;
    slot_t *ns = calloc((size_t)ncap, sizeof(slot_t));
    uint64_t *nocc = malloc(sizeof(uint64_t) * (size_t)ncap);
    if (!ns || !nocc) {
        free(ns);
        free(nocc);
        return BB_NOMEM;
    }
    for (uint64_t j = 0; j < b->used; j++) {
        const slot_t *o = &b->s[b->occ[j]];
        uint64_t h = key_hash(o->w, b->k, o->type) & (ncap - 1);
        while (ns[h].cnt) h = (h + 1) & (ncap - 1);
        ns[h] = *o;
        nocc[j] = h;
    }
    free(b->s);
    free(b->occ);
    b->s = ns;
    b->occ = nocc;
    b->cap = ncap;
    return BB_OK;
}

/* Empties the buckets (only the filled slots are touched). */
static void buckets_clear(buckets_t *b) {
    for (uint64_t j = 0; j < b->used; j++) b->s[b->occ[j]].cnt = 0;
    b->used = 0;
}

static int buckets_add(buckets_t *b, const int32_t *w, uint32_t type) {
    if (4 * (b->used + 1) > 3 * b->cap && buckets_grow(b)) return BB_NOMEM;
    uint64_t h = key_hash(w, b->k, type) & (b->cap - 1);
    for (;;) {
        slot_t *s = &b->s[h];
        if (!s->cnt) {
            memcpy(s->w, w, sizeof(int32_t) * (size_t)b->k);
            s->type = type;
            s->cnt = 1;
            b->occ[b->used++] = h;
            return BB_OK;
        }
        if (s->type == type && !memcmp(s->w, w, sizeof(int32_t) * (size_t)b->k)) {
            s->cnt++;
            return BB_OK;
        }
        h = (h + 1) & (b->cap - 1);
    }
}

/* ---- the count */

/* Wedges of anchor u through v: every (p-1)-subset of v's neighbours of rank
 * below u, in decreasing priority, with its type. */
static int wedges_through(buckets_t *b, const nb_t *nv, int64_t below, int8_t neg_uv, int k) {
    if (below < k) return BB_OK;
    int64_t idx[BB_MAXP];
    int32_t w[BB_MAXP];
    /* subsets as decreasing index tuples below[-1] > idx[0] > ... > idx[k-1] >= 0 */
    for (int i = 0; i < k; i++) idx[i] = below - 1 - i;
    for (;;) {
        uint32_t type = 0;
        for (int i = 0; i < k; i++) {
            const nb_t *x = &nv[idx[i]];
            w[i] = x->to;
            if (x->neg != neg_uv) type |= 1u << i; /* c_i = d */
        }
        if (buckets_add(b, w, type)) return BB_NOMEM;
        /* next tuple in decreasing lexicographic order */
        int i = k - 1;
        while (i >= 0 && idx[i] == (int64_t)(k - 1 - i)) i--;
        if (i < 0) break;
        idx[i]--;
        for (int j = i + 1; j < k; j++) idx[j] = idx[j - 1] - 1;
    }
    return BB_OK;
}

int sbc_bbwc_count(int64_t n_u, int64_t n_v, const int64_t *off, const int32_t *col,
                   const int8_t *sgn, int p, int q, int side, int nthreads, uint64_t out[2]) {
    out[0] = out[1] = 0;
    if (n_u < 0 || n_v < 0 || (side != 0 && side != 1)) return BB_INVALID;
    /* k members of S per biclique, l vertices of the other side */
    const int k = side == 0 ? p : q, l = side == 0 ? q : p;
    if (k < 1 || k > BB_MAXP || l < 1) return BB_INVALID;
    graph_t g;
    int st = graph_build(&g, n_u, n_v, off, col, sgn, side);
    if (st) return st;
    u128 total = 0;
    int ovf = 0, nomem = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads) reduction(| : ovf, nomem)
#endif
    {
        buckets_t b = {NULL, NULL, 0, 0, k - 1};
        u128 part = 0;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t u = 0; u < g.ns; u++) {
            if (nomem) continue;
            if (k == 1) { /* no wedges: the bicliques of u are its l-subsets */
                add128(&part, choose((uint64_t)(g.s_off[u + 1] - g.s_off[u]), l, &ovf), &ovf);
                continue;
            }
            buckets_clear(&b);
            for (int64_t e = g.s_off[u]; e < g.s_off[u + 1] && !nomem; e++) {
                const int32_t v = g.s_adj[e].to;
                const nb_t *nv = g.o_adj + g.o_off[v];
                const int64_t dv = g.o_off[v + 1] - g.o_off[v];
                int64_t below = 0; /* neighbours of v with rank below u */
                while (below < dv && nv[below].to < u) below++;
                if (wedges_through(&b, nv, below, g.s_adj[e].neg, k - 1)) nomem = 1;
            }
            for (uint64_t j = 0; j < b.used && !nomem; j++) {
                const uint64_t c = b.s[b.occ[j]].cnt;
                if (c >= (uint64_t)l) add128(&part, choose(c, l, &ovf), &ovf);
            }
        }
        free(b.s);
        free(b.occ);
#ifdef _OPENMP
#pragma omp critical
#endif
        add128(&total, part, &ovf);
    }
    graph_free(&g);
    if (nomem) return BB_NOMEM;
    if (ovf) return BB_OVERFLOW;
    out[0] = (uint64_t)total;
    out[1] = (uint64_t)(total >> 64);
    return BB_OK;
}
