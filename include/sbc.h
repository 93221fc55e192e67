/*
 * sbc.h -- balanced (p,q)-biclique counting in signed bipartite graphs on one
 * NVIDIA GB300 GPU (sm_103a).
 *
 * The operation: given a signed bipartite graph G = (U, V, E) (Section 3:
 * every edge (u,v) carries a sign + or -), count the balanced
 * (p,q)-bicliques: pairs (L, R) with L a p-subset of U, R a q-subset of V,
 * every (l, r) in L x R an edge, and no butterfly (2x2 sub-biclique) of L x R
 * with an odd number of negative edges (Definitions 1-4 and the problem
 * statement, Section 3). p and q are both at least 2 (the problem statement
 * excludes p = 1 and q = 1).
 *
 * Convention: p vertices are taken from U (the rows of the input CSR) and q
 * from V (its column ids). The paper draws p from the anchor side S of
 * Algorithm 2 (the smaller partition); that count is count(G^T, p, q) here
 * when S = V, and count(G, p, q) = count(G^T, q, p) always holds.
 *
 * The counting method is Algorithm 2 of the paper (vertex-based pruning,
 * Section 4.3) executed by CUDA kernels: anchors u with the lowest vertex
 * priority (Definition 4) in their tuple, 2-hop counts cnt[w], the candidate
 * filter cnt[w] >= q, (p-1)-subsets of candidates, signed p-wedge types
 * (Section 4.2, Lemma 1) and sums of binom(x[type], q). All counts are exact
 * unsigned 128-bit integers.
 *
 * Conventions of this interface:
 *  - Every function returns an sbc_status; on a non-OK status,
 *    sbc_last_error() gives a message for the calling thread. No function
 *    aborts the process or throws across the ABI.
 *  - "stream" arguments are cudaStream_t values passed as void*; NULL means
 *    the legacy default stream. Host pointers are ordinary pageable or pinned
 *    memory; device pointers must be on the current device.
 *  - The library copies every input. The caller keeps ownership of its
 *    buffers and may free them as soon as the call returns.
 *  - Handles are owned by the caller and freed only by the *_destroy calls.
 *  - All entry points work on the CUDA device that is current on the calling
 *    thread; a graph must be used on the device it was created on.
 *  - Device memory comes from cudaMallocAsync on the call's stream unless an
 *    allocator is installed with sbc_set_allocator.
 *  - Environment variables read at each count: SBC_DEBUG=1 (device
 *    self-checks, as SBC_COUNT_CHECK), SBC_POS_NODE_COST (unit of the
 *    position-side cost model), SBC_TC_MIN_CANDIDATES (candidates an anchor
 *    needs for the tensor-core pair step), SBC_POOL_BUDGET_KB (candidate-mask
 *    pool per anchor group); for tests only, SBC_HASH_SLOTS_CAP (2-hop table
 *    size cap, to make tables overflow) and SBC_TWOHOP_WINDOW (wedges of a
 *    one-window anchor, to force the bucketed 2-hop strategy on small graphs).
 */
#ifndef SBC_H
#define SBC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sbc_graph sbc_graph;   /* opaque, immutable after creation */
typedef struct sbc_server sbc_server; /* opaque request server */
typedef struct sbc_batch sbc_batch;   /* opaque planned batch of graphs */

/* Unsigned 128-bit integer, little-endian limbs: value = lo + hi * 2^64. */
typedef struct {
    uint64_t lo, hi;
} sbc_u128;

typedef enum {
    SBC_OK = 0,
    SBC_E_INVAL = 1,       /* bad argument (NULL pointer, p or q out of range) */
    SBC_E_GRAPH = 2,       /* malformed graph (offsets, column ids, signs, duplicates) */
    SBC_E_NOMEM = 3,       /* device or host allocation failed */
    SBC_E_CUDA = 4,        /* a CUDA call or kernel failed */
    SBC_E_TIMEOUT = 5,     /* a bounded wait ran out */
    SBC_E_BUSY = 6,        /* server admission refused (memory or slots) */
    SBC_E_UNSUPPORTED = 7, /* feature not available on this device or build */
    SBC_E_OVERFLOW = 8     /* the exact count does not fit 128 bits */
} sbc_status;

/* sbc_graph_create flags */
#define SBC_OFFS_I64 (1u << 0)    /* row_offsets are int64_t (else int32_t) */
#define SBC_SIGN_BITS (1u << 1)   /* signs are packed bits, 1 per edge in CSR
                                     order, bit (e & 7) of byte e >> 3, set =
                                     negative (else one int8_t per edge, +1/-1) */
#define SBC_DEVICE_PTRS (1u << 2) /* row_offsets, cols and signs are device pointers */

/*
 * Build a device-resident graph from a signed CSR over U (Section 3's input
 * model): row u lists the V-neighbours of u in cols[row_offsets[u] ..
 * row_offsets[u+1]), with one sign per edge. Rows need not be sorted.
 *   n_u, n_v     vertex counts (>= 0, each < 2^31)
 *   nnz          number of edges (must equal row_offsets[n_u]; < 2^31)
 *   row_offsets  n_u+1 entries, int32 or int64 (SBC_OFFS_I64), row_offsets[0] = 0,
 *                non-decreasing
 *   cols         nnz int32 column ids in [0, n_v)
 *   signs        nnz int8 (+1 / -1), or ceil(nnz/8) bytes of packed bits
 * The graph is validated on the device: offsets, column range, sign values
 * and duplicate (u, v) pairs give SBC_E_GRAPH. The call returns after the
 * graph is built (it synchronises `stream`). Empty graphs are allowed.
 */
sbc_status sbc_graph_create(sbc_graph **out, int64_t n_u, int64_t n_v, int64_t nnz,
                            const void *row_offsets, const int32_t *cols, const void *signs,
                            uint32_t flags, void *stream);

/* Free a graph and its device memory (synchronises the device first). */
sbc_status sbc_graph_destroy(sbc_graph *g);

typedef struct {
    int64_t n_u, n_v, nnz;
    int64_t max_deg_u, max_deg_v;
    /* 2-paths through the other side, sum over y of binom(deg(y), 2): the
     * number of 2-hop visits of Algorithm 2 when anchoring on that side */
    uint64_t wedges_anchor_u, wedges_anchor_v;
    uint64_t device_bytes; /* device memory held by the graph now */
} sbc_graph_info_t;

sbc_status sbc_graph_info(const sbc_graph *g, sbc_graph_info_t *out);

/* Anchor side choice (Algorithm 2 anchors on a side S; see sbc_count_opts). */
#define SBC_SIDE_AUTO (-1) /* the side with fewer 2-paths to visit (ties: U); when p != q and
                              one side gives tuples of 3 against tuples of 4 or more on the
                              other, that side (its pairs run on the tensor cores) unless it
                              visits over 64 times the other side's 2-paths */
#define SBC_SIDE_U 0       /* anchors in U: tuples of p, q from V */
#define SBC_SIDE_V 1       /* anchors in V: tuples of q, p from U */

/* sbc_count_opts flags */
#define SBC_COUNT_PAPER_TUPLES (1 << 0) /* also count the candidate sets of Algorithm 2
                                           exactly as printed (cnt over every neighbour)
                                           and report sum binom(|C(u)|, k-1) in
                                           sbc_count_stats.anchor_tuples */
#define SBC_COUNT_CANDIDATE_SIDE (1 << 1) /* enumerate candidate subsets for every anchor */
#define SBC_COUNT_POSITION_SIDE (1 << 2)  /* enumerate position subsets wherever they fit
                                             (default: the cheaper side per anchor) */
#define SBC_COUNT_CHECK (1 << 3) /* device self-checks: after the 2-hop step every kept
                                    candidate's mask popcounts are compared with the
                                    counters of its hash-table entry; a mismatch gives
                                    SBC_E_CUDA. Also enabled for every count by the
                                    environment variable SBC_DEBUG=1. Slower. */

/*
 * Launch parameters of the counting kernels: the search space of the
 * autotuner (sbc_autotune). They change how the work is spread over the GPU,
 * never the count. Zero in a field selects the built-in default.
 *   small_wedges   anchors whose 2-hop visit (Algorithm 2's cnt loop) covers
 *                  at most this many wedges take the warp-per-anchor 2-hop
 *                  kernel; the others take a whole CTA of 16 warps each.
 *                  1..512, default 512.
 *   pos_node_cost  cost of one prefix node of the position-side enumeration
 *                  relative to one word test of the candidate-side
 *                  enumeration; each anchor takes the cheaper side, so a
 *                  larger value favours the candidate (bitmap AND/POPC over
 *                  candidate tuples) side. 1..2^20, default 3.
 *   split_per_warp work items per warp of a full-GPU tuple launch: heavy
 *                  anchors are split into items of about (estimated total
 *                  cost) / (resident warps x split_per_warp). 1..64, default 4.
 *   tc_min_words   anchors with two partners (tuple size 3 on the anchor side)
 *                  whose candidate masks have at least this many 32-bit words
 *                  (and at least 128 candidates) take the tensor-core pair
 *                  step: the four type-class sizes of every candidate pair are
 *                  entries of a Gram matrix of the candidates' 0/1 masks,
 *                  computed by tcgen05 MMAs. -1 turns the step off, 1..65536
 *                  sets the threshold, default 2.
 * SBC_E_INVAL for a field outside its range.
 */
typedef struct {
    int32_t small_wedges;
    int32_t pos_node_cost;
    int32_t split_per_warp;
    int32_t tc_min_words;
    float ms; /* sbc_autotune: time of one count with the chosen parameters */
} sbc_tune_t;

typedef struct {
    int32_t anchor_side;  /* SBC_SIDE_AUTO, SBC_SIDE_U or SBC_SIDE_V */
    int32_t flags;        /* SBC_COUNT_* bits, 0 for a plain count */
    /* optional per-anchor contributions, host memory, indexed by vertex id of
     * the anchor side: n_u entries (side U), n_v (side V), max(n_u, n_v) with
     * SBC_SIDE_AUTO (sbc_count_stats.anchor_side then tells the side); or NULL */
    sbc_u128 *per_anchor;
    /* first shard of anchors and number of shards: anchors with
     * (rank of the anchor) % shard_count == shard are counted. 0/0 or 0/1 = all. */
    int32_t shard, shard_count;
    const sbc_tune_t *tune; /* launch parameters, or NULL for the defaults */
} sbc_count_opts;

typedef struct {
    sbc_u128 count;         /* the balanced (p,q)-biclique count */
    /* anchor tuples: sum over anchors u of binom(|C(u)|, k-1), k the tuple
     * size on the anchor side. With SBC_COUNT_PAPER_TUPLES, C(u) is the
     * candidate set of Algorithm 2 (cnt >= other-side size over all of
     * Gamma(u)), i.e. the number of (p-1)-subsets the algorithm enumerates;
     * without it, C(u) is the smaller set the kernels keep (cnt counted only
     * over neighbours v that can close a tuple) */
    sbc_u128 anchor_tuples;
    uint64_t candidates;    /* sum over anchors of |C(u)| */
    uint64_t wedges;        /* 2-hop entries visited */
    uint64_t work_items;    /* tuple-phase work items launched */
    uint64_t tuples_tested; /* tuples whose common-neighbour mask was tested (after
                               nested pruning) */
    uint64_t tuples_typed;  /* tuples with at least q common neighbours (type counts taken) */
    uint64_t popc_words;    /* mask words popcounted by the tuple kernel: one per word of
                               every tested tuple, 2^(k-1) per word of every typed tuple */
    int32_t anchor_side;    /* side used */
    int32_t kernels;        /* kernel launches issued by the call */
    float ms_prepare;       /* orientation build (first use of a side) + plan */
    float ms_twohop;        /* 2-hop candidate kernel */
    float ms_tuples;        /* tuple / type-count kernel */
    float ms_total;
    float ms_tc;            /* tensor-core pair step (mask expansion + MMA kernel) */
    uint64_t tc_anchors;    /* anchors whose pairs the tensor-core step counted */
    uint64_t tc_tiles;      /* 128 x 256 Gram-matrix tiles it computed */
    uint64_t tc_kblocks;    /* K steps of 128 positions over those tiles: the step made
                               tc_kblocks x 128 x 256 x 128 multiply-adds */
    /* CTA-wide 2-hop kernel (anchors with more than the warp tier's wedges), by
     * strategy: [0] one hash window, [1] wedges bucketed once by hash class,
     * [2] the 2-hop re-read once per hash class (fallback), [3] bucketed, then
     * scattered a second time at exact class offsets (a class overflowed its
     * capacity) */
    uint64_t twohop_reads;      /* 2-hop entries it read, all passes */
    uint64_t twohop_anchors[4]; /* its anchors per strategy */
    float twohop_share[4];      /* share of its SM time per strategy */
    float twohop_tail_ms;       /* last minus first finish of its CTAs (load imbalance) */
    uint64_t pool_bytes;        /* candidate-mask pool: bytes reserved over all anchor groups */
    uint64_t twohop_split_classes; /* hash classes whose distinct partners overflowed one
                                      table and were hashed in sub-class windows */
} sbc_count_stats;

/*
 * Count balanced (p,q)-bicliques (p from U, q from V), 2 <= p, q <= 8.
 * Writes the exact count to *out (host memory) and returns when it is known
 * (synchronises `stream`). SBC_E_OVERFLOW if the count needs more than 128 bits.
 */
sbc_status sbc_count(const sbc_graph *g, int p, int q, sbc_u128 *out, void *stream);

/* sbc_count with options (anchor side, per-anchor output, sharding) and
 * statistics; opts and stats may be NULL. */
sbc_status sbc_count_ex(const sbc_graph *g, int p, int q, const sbc_count_opts *opts,
                        sbc_count_stats *stats, void *stream);

/*
 * One-call convenience for callers holding a host CSR: uploads the graph
 * (sbc_graph_create with host pointers), counts, frees. Same arguments as
 * sbc_graph_create followed by sbc_count.
 */
sbc_status sbc_count_csr(int64_t n_u, int64_t n_v, int64_t nnz, const void *row_offsets,
                         const int32_t *cols, const void *signs, uint32_t flags, int p, int q,
                         sbc_u128 *out, void *stream);

/*
 * Batched counting. A batch of independent graphs is counted as their
 * disjoint union: a biclique is connected, so each balanced (p,q)-biclique
 * lies in one graph (Section 3's definitions), and one pass of the counting
 * kernels over the union (Algorithm 2 per graph, each graph on its preferred
 * anchor side) yields every graph's count. The graphs must be on the current
 * device; they are only read.
 *
 * sbc_count_batch: count the n graphs once; out[i] = count of graphs[i]
 * (p from U, q from V). Synchronises `stream`.
 */
sbc_status sbc_count_batch(const sbc_graph *const *graphs, size_t n, int p, int q, sbc_u128 *out,
                           void *stream);

/*
 * A planned batch for repeated counts of the same resident graphs: creation
 * plans the union and counts it once; sbc_batch_run re-executes the counting
 * kernels (2-hop and tuple kernels of every graph) from a CUDA graph captured
 * at creation and writes out[i] for each graph. The graphs must outlive the
 * batch and stay unchanged. Runs on one batch must not overlap.
 */
sbc_status sbc_batch_create(const sbc_graph *const *graphs, size_t n, int p, int q,
                            sbc_batch **out, void *stream);
/* sbc_batch_create with launch parameters (NULL: defaults), e.g. from sbc_autotune. */
sbc_status sbc_batch_create_ex(const sbc_graph *const *graphs, size_t n, int p, int q,
                               const sbc_tune_t *tune, sbc_batch **out, void *stream);
sbc_status sbc_batch_run(sbc_batch *b, sbc_u128 *out, void *stream);
sbc_status sbc_batch_destroy(sbc_batch *b);

/*
 * Autotuner (the paper has no counterpart: its algorithm has no launch
 * parameters). Times the counting kernels of the batch `graphs` (n >= 1; a
 * single graph is a batch of one) for (p, q) under candidate launch
 * parameters and writes the fastest to *out (out->ms = its time per count).
 * The search is coordinate descent from the defaults over split_per_warp
 * {1, 2, 4, 8, 16}, small_wedges {32, 64, 128, 256, 512} and pos_node_cost
 * {2, 4, 6, 10, 16, 64, 2^20}; each candidate is planned once and its
 * counting kernels timed (best of `reps`, 0 = 3) with CUDA events on
 * `stream`. Every candidate must produce the same counts, or the call fails
 * with SBC_E_CUDA. Synchronises `stream`; allocates and frees device memory
 * like sbc_batch_create.
 */
sbc_status sbc_autotune(const sbc_graph *const *graphs, size_t n, int p, int q, int32_t reps,
                        sbc_tune_t *out, void *stream);

/*
 * sbc_autotune with a per-GPU cache (no counterpart in the paper). The cache
 * is a text file at cache_path, one line per tuning: a key made of the GPU's
 * name and SM count, p, q, and the powers of two just above the batch's graph
 * count and total edges, then the chosen parameters and their time. When the
 * file holds the key, *out is read from it and *from_cache = 1 (no kernel
 * runs); else the search of sbc_autotune runs, its result is appended to the
 * file and *from_cache = 0. from_cache may be NULL. SBC_E_INVAL when the file
 * cannot be written or holds invalid parameters for the key. Writers that
 * share one file should not append at the same time.
 */
sbc_status sbc_autotune_cached(const sbc_graph *const *graphs, size_t n, int p, int q,
                               int32_t reps, const char *cache_path, sbc_tune_t *out,
                               int32_t *from_cache, void *stream);

/*
 * Serving. A server answers count requests (graph, p, q) on resident graphs
 * as they arrive. A scheduler thread forms jobs for a set of device lanes
 * (one stream and worker thread each): requests on small graphs that wait
 * together with the same (p, q) are fused into one batched count
 * (sbc_count_batch semantics), requests on large graphs run alone; a job
 * starts when a lane is free and the estimated device bytes of the jobs in
 * flight plus its own stay within mem_budget_bytes (a job larger than the
 * budget runs when nothing else does). Requests that arrive while others
 * run are admitted as lanes and memory free up, and jobs on different lanes
 * overlap on the device. Results are exact and never cached across requests.
 * Graphs must stay alive and unchanged while the server uses them.
 */
typedef struct {
    uint64_t mem_budget_bytes; /* device bytes for jobs in flight; 0 = 80% of free memory */
    int32_t lanes;             /* concurrent device lanes; 0 = 4 */
    int32_t max_batch;         /* most requests fused into one job; 0 = 64 */
    int64_t small_edges;       /* graphs with at most this many edges are fused; 0 = 200000 */
} sbc_server_opts;

typedef struct {
    uint64_t submitted, completed, failed;
    uint64_t jobs;                /* counts dispatched to lanes */
    uint64_t fused_requests;      /* requests that ran inside a multi-request job */
    uint64_t peak_admitted_bytes; /* largest estimated footprint in flight */
    uint64_t mem_budget_bytes;
    double p50_ms, p99_ms, mean_ms, max_ms; /* latency from submit to completion */
    double throughput_rps;        /* completed / (last completion - first submit) */
} sbc_server_stats_t;

sbc_status sbc_server_create(const sbc_server_opts *opts, sbc_server **out);
/* Register a resident graph; *gid identifies it in requests. */
sbc_status sbc_server_add_graph(sbc_server *s, const sbc_graph *g, uint32_t *gid);
/* Queue a request (thread-safe, returns at once); *ticket identifies it. */
sbc_status sbc_server_submit(sbc_server *s, uint32_t gid, int p, int q, uint64_t *ticket);
/* Wait for a request (timeout_us < 0: no limit; SBC_E_TIMEOUT when it runs
 * out, the request stays pending). On return the ticket is released; the
 * request's own status is returned (its count in *out, submit-to-finish time
 * in *latency_s). */
sbc_status sbc_server_wait(sbc_server *s, uint64_t ticket, int64_t timeout_us, sbc_u128 *out,
                           double *latency_s);
sbc_status sbc_server_stats(sbc_server *s, sbc_server_stats_t *out);
sbc_status sbc_server_reset_stats(sbc_server *s);
/* Stop the server: jobs already on a lane finish; waiting requests are dropped. */
sbc_status sbc_server_destroy(sbc_server *s);

/*
 * sbc_count_csr without any device allocation, for callers that cannot call
 * cudaMalloc (a fixed device-memory plan, a loop that must not enter the
 * allocator). No counterpart in the paper: same arguments and result as
 * sbc_count_csr, but every device buffer of the call is carved from one
 * fixed array of SBC_NOALLOC_SCRATCH_BYTES in device memory that the library
 * holds on every GPU it is loaded on, and the call makes no cudaMalloc,
 * cudaFree or other allocating call. Inputs may be host or device pointers
 * (SBC_DEVICE_PTRS). Limits: at most SBC_NOALLOC_MAX_VERTICES per side and
 * SBC_NOALLOC_MAX_EDGES edges (else SBC_E_INVAL); a graph whose counting
 * needs more scratch than the array holds gives SBC_E_NOMEM. The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture. Calls share the array and
 * are serialised by a lock inside the library; calls from other processes
 * that overlap on the same GPU memory would race.
 */
#define SBC_NOALLOC_SCRATCH_BYTES (32u << 20)
#define SBC_NOALLOC_MAX_VERTICES 65536
#define SBC_NOALLOC_MAX_EDGES 65536
sbc_status sbc_count_csr_noalloc(int64_t n_u, int64_t n_v, int64_t nnz, const void *row_offsets,
                                 const int32_t *cols, const void *signs, uint32_t flags, int p,
                                 int q, sbc_u128 *out, void *stream);

/*
 * Measurement helper (no counterpart in the paper): the current device's
 * sustained rates of 32-bit population counts and of three-input logic
 * operations (LOP3), the operations of the tuple step's mask tests, in
 * operations per second. Each is the best of three timed launches (CUDA
 * events on `stream`, after one warm-up launch) of a kernel that keeps every
 * SM busy with eight independent dependency chains per thread; about 30 ms in
 * all. Synchronises `stream`.
 */
sbc_status sbc_measure_alu_rates(double *popc_per_s, double *lop3_per_s, void *stream);

/* Human-readable message for the last non-OK status on this thread. */
/*
 * Dynamic graphs (the setting the paper leaves to future work, Section 6): a
 * balanced (p,q) count kept exact while edges are inserted, deleted or change
 * sign. An update of edge (u, v) changes the count by the balanced bicliques
 * that contain it; these are the complete (p-1, q-1) subgraphs of the local
 * graph H(u, v) on Gamma(v) - {u} (rows) and Gamma(u) - {v} (columns) whose
 * edges are the (w, x) with sign(u,v) sign(u,x) sign(w,v) sign(w,x) = +1 (a
 * biclique through (u, v) is balanced exactly when its butterflies through
 * (u, v) are). H is assembled on the host from the handle's adjacency (kept
 * there, sorted per vertex) and counted by the GPU kernels (its balanced
 * (p-1, q-1) count with every sign positive); p and q are in [3, 8].
 */
typedef struct sbc_dyn sbc_dyn; /* opaque, owned by the caller; one thread at a time per handle */
#define SBC_DYN_INSERT 0   /* add edge (u, v) with `sign`; the edge must be absent */
#define SBC_DYN_DELETE 1   /* remove edge (u, v); it must be present (`sign` unused) */
#define SBC_DYN_SET_SIGN 2 /* give the present edge (u, v) the sign `sign` */

/* Start from a host CSR over U (int64 offsets, int32 columns, int8 signs +1 /
 * -1; validated like sbc_graph_create) and count it on the GPU. SBC_E_INVAL
 * when p or q is outside [3, 8]. */
sbc_status sbc_dyn_create(sbc_dyn **out, int64_t n_u, int64_t n_v, int64_t nnz,
                          const int64_t *row_offsets, const int32_t *cols, const int8_t *signs,
                          int p, int q, void *stream);
/* Apply one update and write the new count to *count (host, may be NULL).
 * SBC_E_INVAL for an absent edge (delete, set sign), a present one (insert), a
 * vertex outside the graph or a sign other than +1 / -1; the handle is
 * unchanged on any error. */
sbc_status sbc_dyn_update(sbc_dyn *d, int op, int64_t u, int64_t v, int8_t sign, sbc_u128 *count,
                          void *stream);
/* The current count and edge number (nnz may be NULL). */
sbc_status sbc_dyn_count(const sbc_dyn *d, sbc_u128 *count, int64_t *nnz);
sbc_status sbc_dyn_destroy(sbc_dyn *d);
/* H(u, v) of the graph in the given host CSR for edge (u, v) with sign `sign`
 * (the edge itself need not be present), host only: writes its row and column
 * numbers and edge number; with h_offsets non-NULL also its CSR (n_l + 1
 * offsets; h_cols of `capacity` entries, SBC_E_INVAL when it holds fewer than
 * the edges). Rows follow Gamma(v) - {u} and columns Gamma(u) - {v} in
 * increasing vertex id. */
sbc_status sbc_edge_local_graph(int64_t n_u, int64_t n_v, int64_t nnz, const int64_t *row_offsets,
                                const int32_t *cols, const int8_t *signs, int64_t u, int64_t v,
                                int8_t sign, int64_t *n_l, int64_t *n_r, int64_t *h_nnz,
                                int64_t *h_offsets, int32_t *h_cols, int64_t capacity);

const char *sbc_last_error(void);

/* Library version string. */
const char *sbc_version(void);

/* Kernel launches issued by the library in this process so far (all
 * threads); the difference around a call counts its launches. */
uint64_t sbc_launch_count(void);

/*
 * Route the library's device allocations through caller functions (for
 * example a framework's caching allocator). alloc returns a device pointer of
 * at least `bytes` bytes usable on `stream`, or NULL; free releases it.
 * Passing NULL functions restores cudaMallocAsync / cudaFreeAsync.
 */
typedef void *(*sbc_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*sbc_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
sbc_status sbc_set_allocator(sbc_alloc_fn alloc, sbc_free_fn free, void *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SBC_H */
