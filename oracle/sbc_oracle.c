/*
 * Plain CPU oracle for counting balanced (p,q)-bicliques in a signed
 * bipartite graph.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or
 * load this file: only the tests, the smoke check and the benchmark's CPU
 * baseline legs use it. It shares no code, header or table with the CUDA path.
 *
 * What it counts (Section 3: Definitions 1-4 and the problem statement):
 * pairs (L, R), L a p-subset of U and R a q-subset of V, with every (x, v) in
 * L x R an edge and no butterfly of L x R holding an odd number of negative
 * edges.
 *
 * Two counters live here, written independently of each other:
 *
 * sbc_oracle_brute -- the definition itself: every p-subset L of U, every
 *   q-subset R of its common neighbourhood, every butterfly of L x R tested
 *   for an even number of negative edges. Tiny graphs only.
 *
 * sbc_oracle_count -- the same number for graphs of real size, through the
 *   sign-vector characterisation of a balanced biclique (Lemma 1 and its
 *   converse, Section 4.2): a complete L x R is balanced exactly when every
 *   v in R has the same sign vector relative to one fixed x1 in L, i.e. the
 *   same bits kappa_x(v) = [sign(x1,v) != sign(x,v)] over x in L \ {x1}.
 *   (Each butterfly (x1, x, v, v') is balanced iff kappa_x(v) = kappa_x(v');
 *   a butterfly (x, y, v, v') without x1 has the product of the signs of
 *   (x1,x,v,v') and (x1,y,v,v'), so it is balanced when both are.)
 *   Hence, for a fixed L with common neighbourhood N(L), the balanced R are
 *   the q-subsets of one class of N(L) under kappa, and the count is the sum
 *   over L of sum over classes c of binom(|c|, q).
 *
 *   Every L is visited once, from its member x1 of lowest priority rho
 *   (Definition 4: degree, then id), by a depth-first extension: a node is a
 *   set L = {x1, ..., xd} in increasing priority together with N(L) as a list
 *   of (v, sign(x1,v), kappa bits so far) in increasing v. Its children are
 *   the vertices x of higher priority than xd adjacent to some v in N(L);
 *   scanning N(L) once and appending each v to the bucket of every such x
 *   gives each child's N(L + x) directly, in increasing v. A child with fewer
 *   than q common neighbours has no q-subset below it (N only shrinks) and is
 *   not visited. At |L| = p the classes of N(L) are tallied.
 *
 *   The anchor side S (the side L is drawn from) may be either side: the
 *   count with p from U and q from V equals the count of the transposed
 *   graph with q from V and p from U.
 *
 * Counts are exact: unsigned 128-bit sums, binomials by the exact
 * multiplicative formula; a binomial or a sum that would not fit 128 bits
 * sets the overflow flag. The loop over anchors x1 may run on several OpenMP
 * threads, each with its own partial sum (integer addition: order-free).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

/* ORACLE_MUTANT plants one known mistake (tests only, built into a separate
 * library) so that the test suite can show that its pins catch it:
 *   1 priority compares degrees only (equal degrees admitted both ways)
 *   2 kappa from sign(x,v) alone instead of relative to x1
 *   3 children need more than q common neighbours
 *   4 one class (all bits set) dropped at the leaf
 *   5 binomial with q-1
 *   6 a vertex may extend a set that ends with itself
 *   7 the kappa bit of the 5th and later members lands on the 4th's bit */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

/* One adjacency entry: neighbour id and edge sign (+1 / -1). */
typedef struct {
    int32_t id;
    int8_t sign;
} adj_t;

typedef struct {
    int64_t n;    /* vertices on this side */
    int64_t *off; /* n+1 */
    adj_t *adj;   /* off[n] entries */
} side_t;

/* Entry of N(L): common neighbour v, sign(x1, v), kappa bits. */
typedef struct {
    int32_t v;
    int8_t s1;
    uint32_t kappa;
} nent_t;

static void free_side(side_t *s) {
    free(s->off);
    free(s->adj);
    s->off = NULL;
    s->adj = NULL;
}

/* Transpose-style build: lists of `side` (n_side vertices) from the edge list
 * (a[e], b[e], sgn[e]); entry of a[e] is (b[e], sign). */
static int build_lists(int64_t n_side, int64_t m, const int32_t *a, const int32_t *b,
                       const int8_t *sgn, side_t *out) {
    out->n = n_side;
    out->off = (int64_t *)calloc((size_t)(n_side + 1), sizeof(int64_t));
    out->adj = (adj_t *)malloc(sizeof(adj_t) * (size_t)(m > 0 ? m : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_side + 1));
    if (!out->off || !out->adj || !fill) {
        free(fill);
        return -1;
    }
    for (int64_t e = 0; e < m; e++) out->off[a[e] + 1]++;
    for (int64_t x = 0; x < n_side; x++) out->off[x + 1] += out->off[x];
    memcpy(fill, out->off, sizeof(int64_t) * (size_t)(n_side + 1));
    for (int64_t e = 0; e < m; e++) {
        adj_t t;
        t.id = b[e];
        t.sign = sgn[e];
        out->adj[fill[a[e]]++] = t;
    }
    free(fill);
    return 0;
}

/* Sorting helpers (qsort with a file-scope key array: the sorts run before
 * any thread starts). */
static const int64_t *g_key;
static int cmp_by_key(const void *pa, const void *pb) {
    int64_t x = g_key[((const adj_t *)pa)->id], y = g_key[((const adj_t *)pb)->id];
    return (x > y) - (x < y);
}
static int cmp_by_id(const void *pa, const void *pb) {
    int32_t x = ((const adj_t *)pa)->id, y = ((const adj_t *)pb)->id;
    return (x > y) - (x < y);
}

static uint64_t gcd_u64(uint64_t a, uint64_t b) {
    while (b) {
        uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

/* binom(n, k) exactly; sets *ovf if the value does not fit 128 bits.
 * Multiplicative form r_i = r_{i-1} * (n-k+i) / i, where i divides
 * r_{i-1} * (n-k+i) (r_i is itself a binomial). With g = gcd(n-k+i, i), i/g
 * divides r_{i-1}, so r_i = (r_{i-1} / (i/g)) * ((n-k+i)/g) never builds an
 * intermediate larger than r_i. */
static u128 binom_u128(int64_t n, int k, int *ovf) {
    if (k < 0 || n < k) return 0;
    u128 r = 1;
    for (int i = 1; i <= k; i++) {
        uint64_t f = (uint64_t)(n - k + i);
        uint64_t g = gcd_u64(f, (uint64_t)i);
        u128 div = (u128)((uint64_t)i / g);
        u128 mul = (u128)(f / g);
        r /= div;
        if (r > (~(u128)0) / mul) {
            *ovf = 1;
            return 0;
        }
        r *= mul;
    }
    return r;
}

/* *acc += v, flagging a sum that leaves 128 bits. */
static void add_u128(u128 *acc, u128 v, int *ovf) {
    u128 s = *acc + v;
    if (s < v) *ovf = 1;
    *acc = s;
}

/* Per-thread work space: one level of the extension per set size. */
typedef struct {
    nent_t *ent;  /* the children's N lists, back to back */
    int64_t ecap;
    int32_t *cx;  /* child vertices */
    int64_t ccap;
    int64_t *cb;  /* child list begins (nchild + 1) */
    int64_t bcap;
} level_t;

typedef struct {
    const side_t *s, *o; /* anchor side (lists by id), other side (lists by rank) */
    const int64_t *rank; /* rank of each S vertex in rho order */
    const int64_t *deg;  /* degree of each S vertex */
    int p, q;            /* set size on S, subset size on the other side */
    int32_t *mark;       /* n_S, zero between uses */
    int32_t *touched;    /* n_S */
    level_t lv[17];
    u128 *xcnt;          /* class sizes, 2^(p-1) */
    int ovf, err;
} ctx_t;

/* First entry of the other-side list `a[0..n)` (ascending rank) whose vertex
 * may follow `last` in a set. */
static int64_t first_later(const ctx_t *c, const adj_t *a, int64_t n, int32_t last) {
#if ORACLE_MUTANT == 1
    int64_t key = c->deg[last]; /* degree only: ties on both sides */
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (c->deg[a[mid].id] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
#else
    int64_t key = c->rank[last];
#if ORACLE_MUTANT == 6
    key -= 1; /* admits `last` itself */
#endif
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (c->rank[a[mid].id] <= key) lo = mid + 1; else hi = mid;
    }
    return lo;
#endif
}

static int grow(void **p, int64_t *cap, int64_t need, size_t elem) {
    if (need <= *cap) return 0;
    int64_t nc = *cap ? *cap : 256;
    while (nc < need) nc *= 2;
    void *q = realloc(*p, (size_t)nc * elem);
    if (!q) return -1;
    *p = q;
    *cap = nc;
    return 0;
}

/* Bit of member number d (0-based; member 0 is x1) in kappa. */
static uint32_t kappa_bit(int d) {
#if ORACLE_MUTANT == 7
    if (d >= 4) return 1u << 2;
#endif
    return 1u << (d - 1);
}

/* Sum over the classes of N(L), |L| = p: binom(|class|, q). */
static u128 leaf(ctx_t *c, const nent_t *n, int64_t nn) {
    u128 b = 0;
    uint32_t ncls = 1u << (c->p - 1);
    for (uint32_t k = 0; k < ncls; k++) c->xcnt[k] = 0;
    for (int64_t t = 0; t < nn; t++) c->xcnt[n[t].kappa] += 1;
    for (uint32_t k = 0; k < ncls; k++) {
#if ORACLE_MUTANT == 4
        if (k == ncls - 1) continue;
#endif
#if ORACLE_MUTANT == 5
        add_u128(&b, binom_u128((int64_t)c->xcnt[k], c->q - 1, &c->ovf), &c->ovf);
#else
        add_u128(&b, binom_u128((int64_t)c->xcnt[k], c->q, &c->ovf), &c->ovf);
#endif
    }
    return b;
}

/* Children of the set whose last member is `last` (d members so far) and
 * whose common neighbourhood is n[0..nn): fills level d with each child x and
 * its N(L + x). Returns the number of children. */
static int64_t children(ctx_t *c, int d, const nent_t *n, int64_t nn, int32_t last) {
    const side_t *o = c->o;
    level_t *L = &c->lv[d];
    int64_t ntouch = 0;
    /* bucket sizes */
    for (int64_t t = 0; t < nn; t++) {
        const adj_t *a = o->adj + o->off[n[t].v];
        int64_t len = o->off[n[t].v + 1] - o->off[n[t].v];
        for (int64_t f = first_later(c, a, len, last); f < len; f++) {
            int32_t x = a[f].id;
#if ORACLE_MUTANT == 1
            if (x == last) continue;
#endif
            if (c->mark[x]++ == 0) c->touched[ntouch++] = x;
        }
    }
    /* keep the children with at least q common neighbours; mark[x] becomes
     * the child's index + 1 (0: not a child) */
    int64_t nch = 0, tot = 0;
    if (grow((void **)&L->cx, &L->ccap, ntouch + 1, sizeof(int32_t)) ||
        grow((void **)&L->cb, &L->bcap, ntouch + 1, sizeof(int64_t))) {
        c->err = 1;
        for (int64_t i = 0; i < ntouch; i++) c->mark[c->touched[i]] = 0;
        return 0;
    }
    for (int64_t i = 0; i < ntouch; i++) {
        int32_t x = c->touched[i];
        int32_t cnt = c->mark[x];
#if ORACLE_MUTANT == 3
        int keep = cnt > c->q;
#else
        int keep = cnt >= c->q;
#endif
        if (keep) {
            L->cx[nch] = x;
            L->cb[nch] = tot;
            tot += cnt;
            nch++;
            c->mark[x] = (int32_t)nch;
        } else {
            c->mark[x] = 0;
        }
    }
    L->cb[nch] = tot;
    if (grow((void **)&L->ent, &L->ecap, tot + 1, sizeof(nent_t))) {
        c->err = 1;
        nch = 0;
    }
    /* fill the buckets in increasing v (n is in increasing v) */
    if (nch > 0) {
        int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)nch);
        if (!cur) {
            c->err = 1;
            nch = 0;
        } else {
            for (int64_t i = 0; i < nch; i++) cur[i] = L->cb[i];
            uint32_t bit = kappa_bit(d);
            for (int64_t t = 0; t < nn; t++) {
                const adj_t *a = o->adj + o->off[n[t].v];
                int64_t len = o->off[n[t].v + 1] - o->off[n[t].v];
                for (int64_t f = first_later(c, a, len, last); f < len; f++) {
                    int32_t x = a[f].id;
                    int32_t ci = c->mark[x];
                    if (ci == 0) continue;
#if ORACLE_MUTANT == 1
                    if (x == last) continue;
#endif
                    nent_t e = n[t];
#if ORACLE_MUTANT == 2
                    if (a[f].sign < 0) e.kappa |= bit;
#else
                    if (a[f].sign != n[t].s1) e.kappa |= bit;
#endif
                    L->ent[cur[ci - 1]++] = e;
                }
            }
            free(cur);
        }
    }
    for (int64_t i = 0; i < ntouch; i++) c->mark[c->touched[i]] = 0;
    return nch;
}

/* Balanced bicliques of the sets extending L (d members, last member `last`,
 * common neighbourhood n[0..nn)). */
static u128 extend(ctx_t *c, int d, const nent_t *n, int64_t nn, int32_t last) {
    if (d == c->p) return leaf(c, n, nn);
    int64_t nch = children(c, d, n, nn, last);
    level_t *L = &c->lv[d];
    u128 b = 0;
    for (int64_t i = 0; i < nch && !c->err; i++)
        add_u128(&b, extend(c, d + 1, L->ent + L->cb[i], L->cb[i + 1] - L->cb[i], L->cx[i]),
                 &c->ovf);
    return b;
}

/* The graph's lists, ordered for one anchor side: the anchor side's lists
 * by id, the other side's by the anchor side's priority rank. */
typedef struct {
    side_t su, sv;
    int side;
    int64_t *deg, *rank; /* of the anchor side's vertices */
} prep_t;

static void free_prep(prep_t *P) {
    free_side(&P->su);
    free_side(&P->sv);
    free(P->deg);
    free(P->rank);
    memset(P, 0, sizeof(*P));
}

/* Orders the lists for anchor side `side` and ranks its vertices by rho. */
static int order_for_side(prep_t *P, int side) {
    side_t *s = side == 0 ? &P->su : &P->sv, *o = side == 0 ? &P->sv : &P->su;
    int64_t nS = s->n;
    P->side = side;
    P->deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nS > 0 ? nS : 1));
    P->rank = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nS > 0 ? nS : 1));
    adj_t *ord = (adj_t *)malloc(sizeof(adj_t) * (size_t)(nS > 0 ? nS : 1));
    int64_t *key = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nS > 0 ? nS : 1));
    if (!P->deg || !P->rank || !ord || !key) {
        free(ord), free(key);
        return -1;
    }
    /* Definition 4: rho orders by degree, then by id */
    for (int64_t x = 0; x < nS; x++) {
        P->deg[x] = s->off[x + 1] - s->off[x];
        key[x] = P->deg[x] * (nS + 1) + x;
        ord[x].id = (int32_t)x;
    }
    g_key = key;
    qsort(ord, (size_t)nS, sizeof(adj_t), cmp_by_key);
    for (int64_t i = 0; i < nS; i++) P->rank[ord[i].id] = i;
    /* the other side's lists in increasing rank, the anchor side's by id */
    for (int64_t v = 0; v < o->n; v++)
        qsort(o->adj + o->off[v], (size_t)(o->off[v + 1] - o->off[v]), sizeof(adj_t), cmp_by_key);
    for (int64_t x = 0; x < nS; x++)
        qsort(s->adj + s->off[x], (size_t)(s->off[x + 1] - s->off[x]), sizeof(adj_t), cmp_by_id);
    free(ord);
    free(key);
    return 0;
}

/*
 * Count on the prepared anchor side S against the other side.
 * p = set size on S, q = subset size on the other side.
 */
static int count_side(const prep_t *P, int p, int q, int nthreads,
                      const uint8_t *anchor_mask, uint64_t max_subsets, uint8_t *skipped,
                      uint64_t out[2], uint64_t *anchor_out, uint64_t *tuples_out, int *ovf_out) {
    const side_t *s = P->side == 0 ? &P->su : &P->sv, *o = P->side == 0 ? &P->sv : &P->su;
    const int64_t *deg = P->deg, *rank = P->rank;
    int64_t nS = s->n;

    int nt = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    nt = omp_get_max_threads();
#else
    (void)nthreads;
#endif
    u128 *part = (u128 *)calloc((size_t)nt, sizeof(u128));
    u128 *tup = (u128 *)calloc((size_t)nt, sizeof(u128));
    int ovf = 0, err = 0;
    if (!part || !tup) err = 1;

#pragma omp parallel reduction(| : ovf, err)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        ctx_t c;
        memset(&c, 0, sizeof(c));
        c.s = s;
        c.o = o;
        c.rank = rank;
        c.deg = deg;
        c.p = p;
        c.q = q;
        c.mark = (int32_t *)calloc((size_t)(nS > 0 ? nS : 1), sizeof(int32_t));
        c.touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nS > 0 ? nS : 1));
        c.xcnt = (u128 *)malloc(sizeof(u128) * ((size_t)1 << (p - 1)));
        nent_t *n1 = NULL;
        int64_t n1cap = 0;
        if (!c.mark || !c.touched || !c.xcnt || err) c.err = 1;

#pragma omp for schedule(dynamic, 16)
        for (int64_t u = 0; u < nS; u++) {
            if (c.err) continue;
            if (anchor_mask && !anchor_mask[u]) continue; /* test subset of anchors */
            /* N({u}) = Gamma(u), in increasing v */
            int64_t du = s->off[u + 1] - s->off[u];
            if (grow((void **)&n1, &n1cap, du + 1, sizeof(nent_t))) {
                c.err = 1;
                continue;
            }
            for (int64_t e = 0; e < du; e++) {
                n1[e].v = s->adj[s->off[u] + e].id;
                n1[e].s1 = s->adj[s->off[u] + e].sign;
                n1[e].kappa = 0;
            }
            u128 b_u = 0, tuples_u = 0;
            {
                int64_t nch = children(&c, 1, n1, du, (int32_t)u);
                /* the (p-1)-subsets of u's first-level children are the sets
                 * Algorithm 2 enumerates for anchor u (reported, not used) */
                int dummy = 0;
                tuples_u = binom_u128(nch, p - 1, &dummy);
                if (max_subsets && (tuples_u > (u128)max_subsets || dummy)) {
                    /* test option: leave out anchors with too many subsets */
                    if (skipped) skipped[u] = 1;
                    nch = 0;
                }
                level_t *L = &c.lv[1];
                for (int64_t i = 0; i < nch && !c.err; i++)
                    add_u128(&b_u, extend(&c, 2, L->ent + L->cb[i], L->cb[i + 1] - L->cb[i], L->cx[i]),
                             &c.ovf);
            }
            add_u128(&part[tid], b_u, &c.ovf);
            tup[tid] += tuples_u;
            if (anchor_out) {
                anchor_out[2 * u] = (uint64_t)b_u;
                anchor_out[2 * u + 1] = (uint64_t)(b_u >> 64);
            }
        }
        ovf |= c.ovf;
        err |= c.err;
        free(c.mark);
        free(c.touched);
        free(c.xcnt);
        free(n1);
        for (int d = 0; d < 17; d++) {
            free(c.lv[d].ent);
            free(c.lv[d].cx);
            free(c.lv[d].cb);
        }
    }
    u128 total = 0, tt = 0;
    for (int i = 0; i < nt && part; i++) {
        add_u128(&total, part[i], &ovf);
        tt += tup[i];
    }
    free(part);
    free(tup);
    out[0] = (uint64_t)total;
    out[1] = (uint64_t)(total >> 64);
    if (tuples_out) {
        tuples_out[0] = (uint64_t)tt;
        tuples_out[1] = (uint64_t)(tt >> 64);
    }
    *ovf_out = ovf;
    return err ? -1 : 0;
}

/* Edge arrays of a CSR over U, checked: offsets from 0, non-decreasing, ids
 * in range, signs +1/-1. */
static int edges_of(int64_t n_u, int64_t n_v, const int64_t *off, const int32_t *col,
                    const int8_t *sgn, int32_t **ru) {
    if (off[0] != 0) return -2;
    int64_t m = off[n_u];
    *ru = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    if (!*ru) return -1;
    for (int64_t u = 0; u < n_u; u++) {
        if (off[u + 1] < off[u]) return -2;
        for (int64_t e = off[u]; e < off[u + 1]; e++) {
            if (col[e] < 0 || col[e] >= n_v || (sgn[e] != 1 && sgn[e] != -1)) return -2;
            (*ru)[e] = (int32_t)u;
        }
    }
    return 0;
}

/*
 * Count balanced bicliques with p_u vertices from U and q_v from V.
 *   anchor_side 0: L drawn from U (set size p_u, subsets of V of size q_v)
 *   anchor_side 1: L drawn from V (set size q_v, subsets of U of size p_u)
 * off/col/sgn: CSR over U, signs +1/-1. out: u128 total as {lo, hi}.
 * anchor_out (optional): each anchor's share (the sets whose member of lowest
 * priority it is), 2 u64 per vertex of the anchor side.
 * tuples_out (optional): sum over anchors u of binom(|C(u)|, p-1), C(u) the
 * vertices of higher priority sharing at least q neighbours with u (the
 * number of subsets Algorithm 2 enumerates), {lo, hi}.
 * anchor_mask (optional): one byte per anchor-side vertex; only anchors with
 * a non-zero byte are processed (the total then covers those anchors only).
 * max_subsets (test option, 0 = none): anchors whose binom(|C(u)|, p-1)
 * exceeds it are left out and flagged in `skipped` (one byte per vertex).
 * Returns 0, -1 on allocation failure, -2 on bad arguments, 1 on overflow.
 */
static int prepare(prep_t *P, int64_t n_u, int64_t n_v, const int64_t *off, const int32_t *col,
                   const int8_t *sgn, int anchor_side) {
    memset(P, 0, sizeof(*P));
    if (n_u < 0 || n_v < 0 || n_u >= INT32_MAX || n_v >= INT32_MAX ||
        (anchor_side != 0 && anchor_side != 1))
        return -2;
    int32_t *ru = NULL;
    int rc = edges_of(n_u, n_v, off, col, sgn, &ru);
    if (rc) {
        free(ru);
        return rc;
    }
    int64_t m = off[n_u];
    if (build_lists(n_u, m, ru, col, sgn, &P->su) || build_lists(n_v, m, col, ru, sgn, &P->sv) ||
        order_for_side(P, anchor_side)) {
        free(ru);
        free_prep(P);
        return -1;
    }
    free(ru);
    return 0;
}

static int count_prepared(const prep_t *P, int p_u, int q_v, int nthreads, uint64_t out[2],
                          uint64_t *anchor_out, uint64_t *tuples_out, const uint8_t *anchor_mask,
                          uint64_t max_subsets, uint8_t *skipped) {
    if (p_u < 2 || q_v < 2 || p_u > 16 || q_v > 16) return -2;
    int ovf = 0;
    int rc = P->side == 0 ? count_side(P, p_u, q_v, nthreads, anchor_mask, max_subsets, skipped,
                                       out, anchor_out, tuples_out, &ovf)
                          : count_side(P, q_v, p_u, nthreads, anchor_mask, max_subsets, skipped,
                                       out, anchor_out, tuples_out, &ovf);
    if (rc) return rc;
    return ovf ? 1 : 0;
}

/*
 * Count balanced bicliques with p_u vertices from U and q_v from V.
 *   anchor_side 0: L drawn from U (set size p_u, subsets of V of size q_v)
 *   anchor_side 1: L drawn from V (set size q_v, subsets of U of size p_u)
 * off/col/sgn: CSR over U, signs +1/-1. out: u128 total as {lo, hi}.
 * anchor_out (optional): each anchor's share (the sets whose member of lowest
 * priority it is), 2 u64 per vertex of the anchor side.
 * tuples_out (optional): sum over anchors u of binom(|C(u)|, p-1), C(u) the
 * vertices of higher priority sharing at least q neighbours with u (the
 * number of subsets Algorithm 2 enumerates), {lo, hi}.
 * anchor_mask (optional): one byte per anchor-side vertex; only anchors with
 * a non-zero byte are processed (the total then covers those anchors only).
 * max_subsets (test option, 0 = none): anchors whose binom(|C(u)|, p-1)
 * exceeds it are left out and flagged in `skipped` (one byte per vertex).
 * Returns 0, -1 on allocation failure, -2 on bad arguments, 1 on overflow.
 */
int sbc_oracle_count(int64_t n_u, int64_t n_v, const int64_t *off, const int32_t *col,
                     const int8_t *sgn, int p_u, int q_v, int anchor_side, int nthreads,
                     uint64_t out[2], uint64_t *anchor_out, uint64_t *tuples_out,
                     const uint8_t *anchor_mask, uint64_t max_subsets, uint8_t *skipped) {
    if (p_u < 2 || q_v < 2 || p_u > 16 || q_v > 16) return -2;
    prep_t P;
    int rc = prepare(&P, n_u, n_v, off, col, sgn, anchor_side);
    if (rc) return rc;
    rc = count_prepared(&P, p_u, q_v, nthreads, out, anchor_out, tuples_out, anchor_mask,
                        max_subsets, skipped);
    free_prep(&P);
    return rc;
}

/* The same count over lists built once (sbc_oracle_prepare) for repeated
 * counts of one graph from one anchor side, e.g. anchor samples. */
void *sbc_oracle_prepare(int64_t n_u, int64_t n_v, const int64_t *off, const int32_t *col,
                         const int8_t *sgn, int anchor_side, int *rc) {
    prep_t *P = (prep_t *)malloc(sizeof(prep_t));
    if (!P) {
        *rc = -1;
        return NULL;
    }
    *rc = prepare(P, n_u, n_v, off, col, sgn, anchor_side);
    if (*rc) {
        free(P);
        return NULL;
    }
    return P;
}

int sbc_oracle_count_prepared(void *h, int p_u, int q_v, int nthreads, uint64_t out[2],
                              uint64_t *anchor_out, uint64_t *tuples_out,
                              const uint8_t *anchor_mask, uint64_t max_subsets, uint8_t *skipped) {
    if (!h) return -2;
    return count_prepared((const prep_t *)h, p_u, q_v, nthreads, out, anchor_out, tuples_out,
                          anchor_mask, max_subsets, skipped);
}

void sbc_oracle_release(void *h) {
    if (!h) return;
    free_prep((prep_t *)h);
    free(h);
}

/* Next k-subset of {0..n-1} in lexicographic order; 0 when done. */
static int next_subset(int *idx, int k, int n) {
    int i = k - 1;
    while (i >= 0 && idx[i] == n - k + i) i--;
    if (i < 0) return 0;
    idx[i]++;
    for (int j = i + 1; j < k; j++) idx[j] = idx[j - 1] + 1;
    return 1;
}

/*
 * The definition, by brute force (tiny graphs: n_u, n_v <= 64): every
 * p-subset L of U, every q-subset R of V with L x R complete, kept when every
 * butterfly (x, y, v, w) of L x R has an even number of negative edges.
 * Returns 0, -2 on bad arguments or sizes, 1 on overflow.
 */
int sbc_oracle_brute(int64_t n_u, int64_t n_v, const int64_t *off, const int32_t *col,
                     const int8_t *sgn, int p, int q, uint64_t out[2]) {
    if (p < 1 || q < 1 || p > 64 || q > 64 || n_u < 0 || n_v < 0 || n_u > 64 || n_v > 64)
        return -2;
    /* sign matrix: 0 = no edge */
    int8_t S[64][64];
    memset(S, 0, sizeof(S));
    for (int64_t u = 0; u < n_u; u++)
        for (int64_t e = off[u]; e < off[u + 1]; e++) {
            if (col[e] < 0 || col[e] >= n_v || (sgn[e] != 1 && sgn[e] != -1)) return -2;
            S[u][col[e]] = sgn[e];
        }
    u128 total = 0;
    int ovf = 0;
    if (p <= n_u && q <= n_v) {
        int L[64], R[64], C[64];
        for (int i = 0; i < p; i++) L[i] = i;
        do {
            /* the columns adjacent to every row of L */
            int nc = 0;
            for (int v = 0; v < n_v; v++) {
                int all = 1;
                for (int i = 0; i < p; i++)
                    if (!S[L[i]][v]) all = 0;
                if (all) C[nc++] = v;
            }
            if (nc < q) continue;
            for (int j = 0; j < q; j++) R[j] = j;
            do {
                int ok = 1;
                for (int a = 0; a < p && ok; a++)
                    for (int b = a + 1; b < p && ok; b++)
                        for (int c = 0; c < q && ok; c++)
                            for (int d = c + 1; d < q && ok; d++) {
                                int neg = (S[L[a]][C[R[c]]] < 0) + (S[L[a]][C[R[d]]] < 0) +
                                          (S[L[b]][C[R[c]]] < 0) + (S[L[b]][C[R[d]]] < 0);
                                if (neg & 1) ok = 0;
                            }
                if (ok) add_u128(&total, 1, &ovf);
            } while (next_subset(R, q, nc));
        } while (next_subset(L, p, (int)n_u));
    }
    out[0] = (uint64_t)total;
    out[1] = (uint64_t)(total >> 64);
    return ovf ? 1 : 0;
}

/* Exact binomial, exported so tests can pin it against closed forms. */
int sbc_oracle_binom(int64_t n, int k, uint64_t out[2]) {
    int ovf = 0;
    u128 r = binom_u128(n, k, &ovf);
    out[0] = (uint64_t)r;
    out[1] = (uint64_t)(r >> 64);
    return ovf;
}

int sbc_oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
