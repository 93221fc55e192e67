/*
 * Plain CPU oracle for counting balanced (p,q)-bicliques in a signed
 * bipartite graph.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or
 * load this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it. It shares no code, header or table with the CUDA path.
 *
 * It follows Algorithm 2 (BBVP, "vertex-based pruning", Section 4.3) of
 * "Counting Small Balanced (p,q)-bicliques in Signed Bipartite Graphs" step by
 * step, in the paper's notation:
 *
 *   for each anchor u in S:
 *     cnt[w] = number of v in Gamma(u) with w in Gamma(v), w in S, rho(w) > rho(u)
 *     C = { w : cnt[w] >= q };  skip u if |C| < p-1
 *     L[w] = Gamma(u) intersect Gamma(w)            for w in C
 *     for every (p-1)-subset A = (w_1 < ... < w_{p-1}) of C:
 *       T = intersection of L[w] over w in A;  skip if |T| < q
 *       x[kappa] = number of v in T with wedge type kappa, where
 *         c_i = s if sign(u,v) == sign(v,w_i), else d           (Section 4.2)
 *       b_pq += sum over kappa of binom(x[kappa], q)
 *
 * Here p is the size of the tuple drawn from the anchor side S and q the size
 * drawn from the other side. rho is the vertex priority of Definition 4
 * (degree, then id). The sum over types of binom(x[kappa], q) relies on
 * Lemma 1 (all signed p-wedges of a balanced biclique share one type) and on
 * its converse (if every v in R gives the same type, every butterfly of
 * {u, w_1..w_{p-1}} x R has an even number of negative edges); the test suite
 * pins this oracle against a brute-force check of every butterfly.
 *
 * Counts are exact: unsigned 128-bit sums, binomials by the exact
 * multiplicative formula. A binomial that would not fit 128 bits sets the
 * overflow flag.
 *
 * The loop over anchors may run on several OpenMP threads; each thread keeps
 * its own maps and partial sum, and the partial sums are added at the end
 * (integer addition, so the order does not matter).
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
 *   1 priority ties broken as "greater"   2 type from sign(w_i,v) alone
 *   3 candidates need cnt > q             4 one type class dropped
 *   5 binomial with q-1                   6 anchor included as its own partner */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

/* One adjacency entry: neighbour id and edge sign (+1 / -1). */
typedef struct {
    int32_t id;
    int8_t sign;
} adj_t;

/* L[w] entry: common neighbour v with sign(u,v) and sign(w,v). */
typedef struct {
    int32_t v;
    int8_t s_uv;
    int8_t s_wv;
} lent_t;

typedef struct {
    int64_t n;        /* vertices on this side */
    int64_t *off;     /* n+1 */
    adj_t *adj;       /* off[n] entries, sorted by id within each list */
} side_t;

static int cmp_adj(const void *a, const void *b) {
    int32_t x = ((const adj_t *)a)->id, y = ((const adj_t *)b)->id;
    return (x > y) - (x < y);
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static void free_side(side_t *s) {
    free(s->off);
    free(s->adj);
    s->off = NULL;
    s->adj = NULL;
}

/* Adjacency of U from the CSR, each list sorted by neighbour id. */
static int build_u_side(int64_t n_u, const int64_t *off, const int32_t *col,
                        const int8_t *sgn, side_t *out) {
    int64_t m = off[n_u];
    out->n = n_u;
    out->off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_u + 1));
    out->adj = (adj_t *)malloc(sizeof(adj_t) * (size_t)(m > 0 ? m : 1));
    if (!out->off || !out->adj) return -1;
    for (int64_t i = 0; i <= n_u; i++) out->off[i] = off[i];
    for (int64_t e = 0; e < m; e++) {
        out->adj[e].id = col[e];
        out->adj[e].sign = sgn[e];
    }
    for (int64_t i = 0; i < n_u; i++)
        qsort(out->adj + off[i], (size_t)(off[i + 1] - off[i]), sizeof(adj_t), cmp_adj);
    return 0;
}

/* Adjacency of V (the transpose), each list sorted by neighbour id. */
static int build_v_side(int64_t n_u, int64_t n_v, const int64_t *off,
                        const int32_t *col, const int8_t *sgn, side_t *out) {
    int64_t m = off[n_u];
    out->n = n_v;
    out->off = (int64_t *)calloc((size_t)(n_v + 1), sizeof(int64_t));
    out->adj = (adj_t *)malloc(sizeof(adj_t) * (size_t)(m > 0 ? m : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_v + 1));
    if (!out->off || !out->adj || !fill) {
        free(fill);
        return -1;
    }
    for (int64_t e = 0; e < m; e++) out->off[col[e] + 1]++;
    for (int64_t v = 0; v < n_v; v++) out->off[v + 1] += out->off[v];
    memcpy(fill, out->off, sizeof(int64_t) * (size_t)(n_v + 1));
    for (int64_t u = 0; u < n_u; u++)
        for (int64_t e = off[u]; e < off[u + 1]; e++) {
            adj_t a;
            a.id = (int32_t)u;
            a.sign = sgn[e];
            out->adj[fill[col[e]]++] = a;
        }
    free(fill);
    for (int64_t v = 0; v < n_v; v++)
        qsort(out->adj + out->off[v], (size_t)(out->off[v + 1] - out->off[v]),
              sizeof(adj_t), cmp_adj);
    return 0;
}

/* Definition 4: rho(a) > rho(b) iff deg(a) > deg(b), or equal degrees and
 * id(a) > id(b). */
static int rho_greater(const side_t *s, int64_t a, int64_t b) {
    int64_t da = s->off[a + 1] - s->off[a], db = s->off[b + 1] - s->off[b];
    if (da != db) return da > db;
#if ORACLE_MUTANT == 1
    return 1;
#else
    return a > b;
#endif
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

/* Section 4.2: c_i = d when sign(u,v) differs from sign(v,w_i). */
#if ORACLE_MUTANT == 2
#define TYPE_D(s_uv, s_wv) ((s_wv) < 0)
#else
#define TYPE_D(s_uv, s_wv) ((s_uv) != (s_wv))
#endif

/* T entry: common neighbour v with the type bits gathered so far
 * (bit i set when c_i = d). */
typedef struct {
    int32_t v;
    uint32_t kappa;
} tent_t;

typedef struct {
    int32_t *cnt;      /* n_S, zero between anchors */
    int32_t *touched;  /* ids with cnt > 0 */
    int32_t *cand;     /* C */
    int64_t *loff;     /* L[w] offsets, |C|+1 */
    lent_t *lbuf;      /* L[w] lists */
    int64_t lcap;
    tent_t *tbuf[2];   /* T work buffers */
    int64_t tcap;
    u128 *xcnt;        /* x[kappa], 2^(p-1) */
} work_t;

/*
 * Algorithm 2 on anchor side S (adjacency `s`), other side `o`.
 * p = tuple size on S, q = size on the other side.
 */
static int bbvp(const side_t *s, const side_t *o, int p, int q, int nthreads,
                const uint8_t *anchor_mask, uint64_t max_subsets, uint8_t *skipped,
                uint64_t out[2], uint64_t *anchor_out, uint64_t *tuples_out, int *ovf_out) {
    int64_t nS = s->n;
    int ovf = 0;
    int nt = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    nt = omp_get_max_threads();
#else
    (void)nthreads;
#endif
    u128 *part = (u128 *)calloc((size_t)nt, sizeof(u128));
    u128 *tup = (u128 *)calloc((size_t)nt, sizeof(u128));
    int err = 0;
    if (!part || !tup) {
        free(part);
        free(tup);
        return -1;
    }
    int64_t maxdeg = 0;
    for (int64_t u = 0; u < nS; u++) {
        int64_t d = s->off[u + 1] - s->off[u];
        if (d > maxdeg) maxdeg = d;
    }

#pragma omp parallel reduction(| : ovf, err)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        work_t w;
        memset(&w, 0, sizeof(w));
        w.cnt = (int32_t *)calloc((size_t)(nS > 0 ? nS : 1), sizeof(int32_t));
        w.touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nS > 0 ? nS : 1));
        w.cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nS > 0 ? nS : 1));
        w.loff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nS + 1));
        w.lcap = 1024;
        w.lbuf = (lent_t *)malloc(sizeof(lent_t) * (size_t)w.lcap);
        w.tcap = maxdeg + 1;
        w.tbuf[0] = (tent_t *)malloc(sizeof(tent_t) * (size_t)w.tcap);
        w.tbuf[1] = (tent_t *)malloc(sizeof(tent_t) * (size_t)w.tcap);
        w.xcnt = (u128 *)malloc(sizeof(u128) * ((size_t)1 << (p - 1)));
        int *idx = (int *)malloc(sizeof(int) * (size_t)p);
        if (!w.cnt || !w.touched || !w.cand || !w.loff || !w.lbuf || !w.tbuf[0] ||
            !w.tbuf[1] || !w.xcnt || !idx)
            err = 1;

#pragma omp for schedule(dynamic, 16)
        for (int64_t u = 0; u < nS; u++) {
            if (err) continue;
            if (anchor_mask && !anchor_mask[u]) continue; /* test subset of anchors */
            u128 b_u = 0;       /* this anchor's contribution */
            u128 tuples_u = 0;  /* (p-1)-subsets of C enumerated */
            int64_t nt_touch = 0;
            /* cnt[w]: shared neighbours of u and w, rho(w) > rho(u) */
            for (int64_t e = s->off[u]; e < s->off[u + 1]; e++) {
                int32_t v = s->adj[e].id;
                for (int64_t f = o->off[v]; f < o->off[v + 1]; f++) {
                    int32_t x = o->adj[f].id;
#if ORACLE_MUTANT == 6
                    if (x != u && !rho_greater(s, x, u)) continue;
#else
                    if (x == u || !rho_greater(s, x, u)) continue;
#endif
                    if (w.cnt[x]++ == 0) w.touched[nt_touch++] = x;
                }
            }
            /* C = { w : cnt[w] >= q } (necessary pairwise condition) */
            int64_t nc = 0;
            for (int64_t i = 0; i < nt_touch; i++)
#if ORACLE_MUTANT == 3
                if (w.cnt[w.touched[i]] > q) w.cand[nc++] = w.touched[i];
#else
                if (w.cnt[w.touched[i]] >= q) w.cand[nc++] = w.touched[i];
#endif
            for (int64_t i = 0; i < nt_touch; i++) w.cnt[w.touched[i]] = 0;
            if (nc >= p - 1 && max_subsets) {
                /* test option: leave out anchors with too many subsets */
                int dummy = 0;
                if (binom_u128(nc, p - 1, &dummy) > (u128)max_subsets || dummy) {
                    if (skipped) skipped[u] = 1;
                    nc = 0;
                }
            }
            if (nc >= p - 1) {
                /* w_1 < ... < w_{p-1}: order C by vertex id */
                qsort(w.cand, (size_t)nc, sizeof(int32_t), cmp_i32);
                /* L[w] = Gamma(u) intersect Gamma(w), sorted by v */
                int64_t du = s->off[u + 1] - s->off[u];
                if (w.lcap < nc * du) {
                    free(w.lbuf);
                    w.lcap = nc * du;
                    w.lbuf = (lent_t *)malloc(sizeof(lent_t) * (size_t)w.lcap);
                    if (!w.lbuf) {
                        err = 1;
                        continue;
                    }
                }
                int64_t pos = 0;
                for (int64_t c = 0; c < nc; c++) {
                    int32_t x = w.cand[c];
                    w.loff[c] = pos;
                    int64_t a = s->off[u], ae = s->off[u + 1];
                    int64_t bb = s->off[x], be = s->off[x + 1];
                    while (a < ae && bb < be) {
                        if (s->adj[a].id < s->adj[bb].id) a++;
                        else if (s->adj[a].id > s->adj[bb].id) bb++;
                        else {
                            w.lbuf[pos].v = s->adj[a].id;
                            w.lbuf[pos].s_uv = s->adj[a].sign;
                            w.lbuf[pos].s_wv = s->adj[bb].sign;
                            pos++;
                            a++;
                            bb++;
                        }
                    }
                }
                w.loff[nc] = pos;
                /* every (p-1)-subset A of C, as increasing index tuples */
                int k = p - 1;
                for (int i = 0; i < k; i++) idx[i] = i;
                for (;;) {
                    tuples_u += 1;
                    /* T = intersection of L[w_i] over A, each v carrying its
                     * type bits: bit i set when c_i = d, i.e.
                     * sign(u,v) != sign(v,w_i) */
                    int64_t tn = 0;
                    tent_t *cur = w.tbuf[0], *nxt = w.tbuf[1];
                    {
                        const lent_t *l1 = w.lbuf + w.loff[idx[0]];
                        int64_t ln = w.loff[idx[0] + 1] - w.loff[idx[0]];
                        for (int64_t t = 0; t < ln; t++) {
                            cur[tn].v = l1[t].v;
                            cur[tn].kappa = TYPE_D(l1[t].s_uv, l1[t].s_wv) ? 1u : 0u;
                            tn++;
                        }
                    }
                    for (int i = 1; i < k; i++) {
                        const lent_t *lw = w.lbuf + w.loff[idx[i]];
                        int64_t ln = w.loff[idx[i] + 1] - w.loff[idx[i]];
                        int64_t a = 0, bb = 0, nn = 0;
                        while (a < tn && bb < ln) {
                            if (cur[a].v < lw[bb].v) a++;
                            else if (cur[a].v > lw[bb].v) bb++;
                            else {
                                nxt[nn].v = cur[a].v;
                                nxt[nn].kappa = cur[a].kappa |
                                    (TYPE_D(lw[bb].s_uv, lw[bb].s_wv) ? (1u << i) : 0u);
                                nn++;
                                a++;
                                bb++;
                            }
                        }
                        tent_t *t = cur;
                        cur = nxt;
                        nxt = t;
                        tn = nn;
                    }
                    if (tn >= q) {
                        /* x[kappa] counts, then sum of binom(x[kappa], q) */
                        for (uint32_t kk = 0; kk < (1u << k); kk++) w.xcnt[kk] = 0;
                        for (int64_t t = 0; t < tn; t++) w.xcnt[cur[t].kappa] += 1;
                        for (uint32_t kk = 0; kk < (1u << k); kk++) {
#if ORACLE_MUTANT == 4
                            if (kk == (1u << k) - 1) continue;
#endif
#if ORACLE_MUTANT == 5
                            b_u += binom_u128((int64_t)w.xcnt[kk], q - 1, &ovf);
#else
                            b_u += binom_u128((int64_t)w.xcnt[kk], q, &ovf);
#endif
                        }
                    }
                    /* next subset */
                    int i = k - 1;
                    while (i >= 0 && idx[i] == nc - k + i) i--;
                    if (i < 0) break;
                    idx[i]++;
                    for (int j = i + 1; j < k; j++) idx[j] = idx[j - 1] + 1;
                }
            }
            part[tid] += b_u;
            tup[tid] += tuples_u;
            if (anchor_out) {
                anchor_out[2 * u] = (uint64_t)b_u;
                anchor_out[2 * u + 1] = (uint64_t)(b_u >> 64);
            }
        }
        free(w.cnt);
        free(w.touched);
        free(w.cand);
        free(w.loff);
        free(w.lbuf);
        free(w.tbuf[0]);
        free(w.tbuf[1]);
        free(w.xcnt);
        free(idx);
    }
    u128 total = 0, tt = 0;
    for (int i = 0; i < nt; i++) {
        total += part[i];
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

/*
 * Count balanced bicliques with p_u vertices from U and q_v from V.
 *   anchor_side 0: S = U (tuple size p_u, other size q_v)
 *   anchor_side 1: S = V (tuple size q_v, other size p_u)
 * off/col/sgn: CSR over U, signs +1/-1. out: u128 total as {lo, hi}.
 * anchor_out (optional): per-anchor contribution, 2 u64 per vertex of S.
 * tuples_out (optional): number of (p-1)-subsets enumerated, {lo, hi}.
 * anchor_mask (optional): one byte per vertex of S; only anchors with a
 * non-zero byte are processed (the total then covers those anchors only).
 * max_subsets (test option, 0 = none): anchors whose (p-1)-subsets of C
 * number more are left out and flagged in `skipped` (one byte per vertex).
 * Returns 0, -1 on allocation failure, -2 on bad arguments, 1 on overflow.
 */
int sbc_oracle_count(int64_t n_u, int64_t n_v, const int64_t *off,
                     const int32_t *col, const int8_t *sgn, int p_u, int q_v,
                     int anchor_side, int nthreads, uint64_t out[2],
                     uint64_t *anchor_out, uint64_t *tuples_out,
                     const uint8_t *anchor_mask, uint64_t max_subsets, uint8_t *skipped) {
    if (p_u < 2 || q_v < 2 || p_u > 16 || q_v > 16 || n_u < 0 || n_v < 0) return -2;
    side_t su, sv;
    memset(&su, 0, sizeof(su));
    memset(&sv, 0, sizeof(sv));
    if (build_u_side(n_u, off, col, sgn, &su) || build_v_side(n_u, n_v, off, col, sgn, &sv)) {
        free_side(&su);
        free_side(&sv);
        return -1;
    }
    int ovf = 0, rc;
    if (anchor_side == 0)
        rc = bbvp(&su, &sv, p_u, q_v, nthreads, anchor_mask, max_subsets, skipped, out,
                  anchor_out, tuples_out, &ovf);
    else
        rc = bbvp(&sv, &su, q_v, p_u, nthreads, anchor_mask, max_subsets, skipped, out,
                  anchor_out, tuples_out, &ovf);
    free_side(&su);
    free_side(&sv);
    if (rc) return rc;
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
