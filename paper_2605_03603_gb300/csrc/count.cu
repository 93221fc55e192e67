// Counting kernels: Algorithm 2 (BBVP, vertex-based pruning, Section 4.3) on
// the device.
//
// Notation. The anchor side X plays S of Algorithm 2; its vertices are
// renumbered by rank in the vertex priority rho (Definition 4). k is the tuple
// size on X and l the size on the other side Y (k = p, l = q when X = U;
// k = q, l = p when X = V); R = k - 1 partners join each anchor.
//
// Per anchor u (rank r):
//   position j of u's list Gamma(u) = (v_0, v_1, ...) is "useful" when the
//   suffix of v_j's list above r holds at least R entries: only then can v_j
//   be a common neighbour of u and R partners of higher rank. Useful
//   positions are numbered 0..d'-1 and become bit positions.
//   2-hop step (Algorithm 2, cnt and L maps): for every useful position j and
//   every w in the suffix of v_j: cnt[w] += 1, P_w[j] = 1 and
//   D_w[j] = (sign(u,v_j) != sign(w,v_j)). P_w is L[w] as a bitmask over
//   Gamma(u); D_w holds the type letter of Section 4.2 (set = d, clear = s).
//   Candidate filter (Algorithm 2): C = { w : cnt[w] >= l }.
//   Tuple step: every R-subset A of C with T = AND of P_w over A (nested
//   pruning: a prefix whose T already has fewer than l bits is dropped, which
//   drops only subsets with |T| < l). The type of v_j is the vector of D_w[j]
//   over A; x[type] = popc(T AND the matching D / NOT D masks), and the
//   anchor adds sum over types of binom(x[type], l).
// Positions that are not useful can never be in T, so leaving them out of
// cnt changes no term of the sum; the paper's own candidate set (counted
// over all positions) is also computed on request to report the number of
// subsets Algorithm 2 enumerates.
#include <algorithm>
#include <vector>

#include "sbc_internal.cuh"

namespace sbc {

namespace {

constexpr uint32_t VMASK = 0x7FFFFFFFu;
constexpr uint32_t EMPTY = 0xFFFFFFFFu;
constexpr unsigned FULL = 0xFFFFFFFFu;

// ------------------------------------------------------------------ counters

// Device-side scalars of one count. Fields up to `run_begin` are set while
// planning (they stay valid when the counting kernels are replayed); the
// rest are accumulators and queue heads of one execution.
struct Counters {
    unsigned long long tuples_paper[2];// u128, sum binom(|C_paper|, R)
    unsigned long long tuples_ours[2]; // u128, sum binom(|C'|, R)
    unsigned long long candidates;     // sum |C'| (or |C_paper| in stats mode)
    unsigned long long cost_total;     // tuple-phase cost estimate
    unsigned long long e_max;          // largest visited-wedge count of a large anchor
    unsigned int n_active;             // anchors with work
    unsigned int n_big;                // anchors for the CTA-wide 2-hop kernel
    unsigned int n_items;
    unsigned int n_tc;                 // anchors of the group for the tensor-core pair step
    // ---- per execution
    unsigned long long run_begin;      // marker (unused)
    unsigned long long total[2];       // u128 count
    unsigned long long wedges;         // 2-hop entries visited
    unsigned long long tested;         // tuples whose common-neighbour mask was tested
    unsigned long long leaves;         // tuples with |T| >= l (type counts taken)
    unsigned long long popc_words;     // mask words popcounted: W per test, 2^R W per leaf
    // CTA-wide 2-hop kernel, by strategy (one window, bucketed, re-read windows,
    // bucketed with a second scatter)
    unsigned long long tw_reads;       // 2-hop entries read, all passes
    unsigned long long tw_cyc[4];      // SM cycles spent on its anchors
    unsigned long long tw_anchors[4];
    unsigned long long tw_fin_max, tw_fin_min_n;  // CTA finish times (global ns; min kept as ~t)
    unsigned long long tw_split;       // hash classes hashed in sub-class windows
    unsigned int head_large;           // 2-hop queue heads
    unsigned int head_small;
    unsigned int head_b;               // tuple queue head
    unsigned int err;                  // error bits
};

enum : unsigned {
    CERR_OVERFLOW = kErrOverflow,  // a binomial or the sum left 128 bits
    CERR_TIMEOUT = kErrTimeout,    // a bounded wait of the tensor-core kernel ran out
    CERR_RESERVE = 2u,    // candidate reservation exceeded (cannot happen)
    CERR_HASH = 4u,       // 2-hop table overflow after all retries
    CERR_MASK = 8u,       // self-check: a candidate mask disagrees with its 2-hop counters
};

// Thresholds: the largest x for which binom(x, l) is computed exactly in 64
// bits by the multiplicative formula (index l, 0..8).
__constant__ unsigned long long c_binom64_max[9];

// ------------------------------------------------------------------ binomials

__device__ __forceinline__ void div_u128_small(unsigned long long &lo, unsigned long long &hi,
                                               unsigned d) {
    unsigned long long qh = hi / d;
    unsigned long long r = hi % d;
    unsigned long long a = (r << 32) | (lo >> 32);
    unsigned long long q1 = a / d;
    r = a % d;
    unsigned long long b = (r << 32) | (lo & 0xFFFFFFFFull);
    unsigned long long q0 = b / d;
    hi = qh;
    lo = (q1 << 32) | q0;
}

// (lo, hi) *= m; returns false on 128-bit overflow.
__device__ __forceinline__ bool mul_u128_u64(unsigned long long &lo, unsigned long long &hi,
                                             unsigned long long m) {
    unsigned long long l0 = lo * m;
    unsigned long long c = __umul64hi(lo, m);
    unsigned long long h0 = hi * m;
    unsigned long long hh = __umul64hi(hi, m);
    unsigned long long nh = h0 + c;
    bool ovf = hh != 0 || nh < h0;
    lo = l0;
    hi = nh;
    return !ovf;
}

__device__ __forceinline__ unsigned gcd_u32(unsigned a, unsigned b) {
    while (b) {
        unsigned t = a % b;
        a = b;
        b = t;
    }
    return a;
}

template <int L>
__device__ __forceinline__ unsigned long long binom_u64(unsigned long long x) {
    unsigned long long r = 1;
#pragma unroll
    for (int i = 1; i <= L; i++) r = r * (x - L + i) / (unsigned long long)i;
    return r;
}

// binom(x, l) in 128 bits, exact (returned by value so that callers'
// accumulators stay in registers). Sets CERR_OVERFLOW if it needs more.
__device__ __noinline__ U128 binom_slow(unsigned long long x, int l, unsigned *err) {
    U128 t;
    unsigned long long lo = 1, hi = 0;
    for (int i = 1; i <= l; i++) {
        unsigned long long f = x - l + i;
        unsigned g = gcd_u32((unsigned)(f % (unsigned)i), (unsigned)i);
        if (g == 0) g = (unsigned)i;
        div_u128_small(lo, hi, (unsigned)i / g);
        if (!mul_u128_u64(lo, hi, f / g)) {
            atomicOr(err, CERR_OVERFLOW);
            return t;
        }
    }
    t.lo = lo;
    t.hi = hi;
    return t;
}

__device__ __forceinline__ void binom_add(U128 &acc, unsigned x, int l, unsigned *err) {
    if ((int)x < l) return;
    if (x > c_binom64_max[l]) {
        if (acc.add(binom_slow(x, l, err))) atomicOr(err, CERR_OVERFLOW);
        return;
    }
    unsigned long long v;
    switch (l) {
        case 2: v = binom_u64<2>(x); break;
        case 3: v = binom_u64<3>(x); break;
        case 4: v = binom_u64<4>(x); break;
        case 5: v = binom_u64<5>(x); break;
        case 6: v = binom_u64<6>(x); break;
        case 7: v = binom_u64<7>(x); break;
        default: v = binom_u64<8>(x); break;
    }
    acc.add(v);
}

// ------------------------------------------------------------------ plan

// Warp per anchor: useful positions, wedge counts, reservation, sort key.
__global__ void k_plan(const int64_t *__restrict__ A_off, const uint32_t *__restrict__ A_ent,
                       const uint32_t *__restrict__ A_pos, const int64_t *__restrict__ B_off,
                       int64_t nX, int R, int l, int shard, int nshard, int stats,
                       uint32_t *__restrict__ A_bit, uint32_t *__restrict__ dprime,
                       unsigned long long *__restrict__ e_use, unsigned long long *__restrict__ e_all,
                       uint32_t *__restrict__ rsv_c, int64_t *__restrict__ rsv_w,
                       uint32_t *__restrict__ skey, uint32_t *__restrict__ sval,
                       Counters *cnt, int small_e) {
    const int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    for (int64_t r = warp; r < nX; r += nwarps) {
        int64_t e0 = A_off[r], e1 = A_off[r + 1];
        uint32_t dp = 0;
        unsigned long long eu = 0, ea = 0;
        for (int64_t b = e0; b < e1; b += 32) {
            int64_t e = b + lane;
            bool in = e < e1;
            unsigned long long suf = 0;
            if (in) {
                uint32_t y = A_ent[e] & VMASK;
                suf = (unsigned long long)(B_off[y + 1] - B_off[y] - (int64_t)A_pos[e] - 1);
            }
            bool useful = in && suf >= (unsigned long long)R;
            uint32_t bal = __ballot_sync(FULL, useful);
            if (in) A_bit[e] = useful ? dp + __popc(bal & lt) : EMPTY;
            dp += __popc(bal);
            eu += useful ? suf : 0ull;
            ea += suf;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            eu += __shfl_xor_sync(FULL, eu, o);
            ea += __shfl_xor_sync(FULL, ea, o);
        }
        if (lane == 0) {
            bool mine = nshard <= 1 || (r % nshard) == shard;
            int64_t d = e1 - e0;
            bool act_count = dp >= (uint32_t)l && eu >= (unsigned long long)R * l;
            bool act_stats = d >= l && ea >= (unsigned long long)R * l;
            bool active = mine && (stats ? act_stats : act_count);
            unsigned long long rc = 0;
            if (active) {
                rc = eu / (unsigned long long)l;  // each candidate owns >= l useful wedges
                unsigned long long above = (unsigned long long)(nX - 1 - r);
                rc = rc < above ? rc : above;
            }
            uint32_t W = (dp + 31) / 32;
            dprime[r] = dp;
            e_use[r] = eu;
            e_all[r] = ea;
            rsv_c[r] = (uint32_t)rc;
            rsv_w[r] = (int64_t)(2ull * W * rc);
            unsigned long long cost = stats ? ea : eu;
            skey[r] = active ? 0xFFFFFFFEu - (uint32_t)(cost < 0xFFFFFFFEull ? cost : 0xFFFFFFFEull)
                             : 0xFFFFFFFFu;
            sval[r] = (uint32_t)r;
            if (active) atomicAdd(&cnt->n_active, 1u);
            if (active && cost > (unsigned long long)small_e) {
                atomicAdd(&cnt->n_big, 1u);
                atomicMax(&cnt->e_max, cost);
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) rsv_w[nX] = 0;
}

// ------------------------------------------------------------------ 2-hop

// Hash value: three 21-bit counters of one 2-hop partner w of the anchor.
//   bits  0..20  cnt over all positions (Algorithm 2's cnt[w])
//   bits 21..41  cnt over useful positions (|P_w|)
//   bits 42..62  useful positions with sign(u,v) != sign(w,v) (|D_w|)
//   bit  63      set once w is kept; bits 0..20 then hold its candidate index
//                (the other two counters stay, for the mask self-check)
constexpr unsigned long long F_ALL = 1ull, F_USE = 1ull << 21, F_DIFF = 1ull << 42;
constexpr unsigned long long M21 = (1ull << 21) - 1;
constexpr unsigned long long CAND = 1ull << 63;
constexpr uint32_t NOBIT = 0x7FFFFFFFu;

__device__ __forceinline__ uint32_t hash_slot(uint32_t w, uint32_t hs) {
    return __umulhi(w * 0x9E3779B1u, hs);
}
__device__ __forceinline__ uint32_t class_mix(uint32_t w) {
    return ((w * 0x85EBCA6Bu) ^ (w >> 15)) * 0xC2B2AE35u;
}
// Hash class of w among 2^lg (the top lg bits of its mix) ...
__device__ __forceinline__ uint32_t class_of(uint32_t w, int lg) {
    return lg ? class_mix(w) >> (32 - lg) : 0u;
}
// ... and its sub-class among 2^lg2 within that class (the next lg2 bits).
__device__ __forceinline__ uint32_t subclass_of(uint32_t w, int lg, int lg2) {
    return lg2 ? (class_mix(w) << lg) >> (32 - lg2) : 0u;
}

// Add `add` to w's counters (open addressing, linear probing, at most hs
// probes). Returns false when the table is full.
__device__ __forceinline__ bool tab_insert(uint32_t *keys, unsigned long long *vals, uint32_t hs,
                                           uint32_t w, unsigned long long add) {
    uint32_t sl = hash_slot(w, hs);
    for (uint32_t probes = 0; probes < hs; probes++) {
        uint32_t k = keys[sl];
        if (k == EMPTY) {
            uint32_t old = atomicCAS(&keys[sl], EMPTY, w);
            if (old == EMPTY || old == w) {
                atomicAdd(&vals[sl], add);
                return true;
            }
            k = old;
        }
        if (k == w) {
            atomicAdd(&vals[sl], add);
            return true;
        }
        sl = (sl + 1 == hs) ? 0u : sl + 1;
    }
    return false;
}

__device__ __forceinline__ int tab_find(const uint32_t *keys, uint32_t hs, uint32_t w) {
    uint32_t sl = hash_slot(w, hs);
    for (uint32_t probes = 0; probes < hs; probes++) {
        uint32_t k = keys[sl];
        if (k == w) return (int)sl;
        if (k == EMPTY) return -1;
        sl = (sl + 1 == hs) ? 0u : sl + 1;
    }
    return -1;
}

// Candidate filter. Algorithm 2 keeps w when cnt[w] >= l. Every type class
// of a tuple through w lies inside the same-sign or the different-sign part
// of L[w] (the letter c_w is constant on a class), so only w with one part of
// at least l useful common neighbours can add a non-zero binomial; the others
// are dropped here, which changes no term of the sum.
__device__ __forceinline__ bool keep_candidate(unsigned long long v, int l) {
    uint32_t use = (uint32_t)((v >> 21) & M21), diff = (uint32_t)((v >> 42) & M21);
    return use - diff >= (uint32_t)l || diff >= (uint32_t)l;
}

__device__ __forceinline__ unsigned long long pass1_add(uint32_t sdiff, uint32_t bit) {
    return bit != EMPTY ? (F_ALL | F_USE | (sdiff ? F_DIFF : 0ull)) : F_ALL;
}

// Kept candidate: index `c` in bits 0..20, the two useful-position counters
// kept, CAND set.
__device__ __forceinline__ unsigned long long cand_value(unsigned long long v, uint32_t c) {
    return CAND | (v & ~(CAND | M21)) | (unsigned long long)c;
}
__device__ __forceinline__ uint32_t cand_index(unsigned long long v) { return (uint32_t)(v & M21); }

// Self-check of one kept candidate after its masks are written: popc(P_w)
// must equal its useful common neighbours and popc(D_w) its different-sign
// ones (both counted by the hash table in the first pass). `P` and `D` are
// the candidate's first words; consecutive words are `stride` apart. Reads
// bypass L1 (the words were written by atomics at L2).
__device__ __forceinline__ bool masks_match(const uint32_t *P, const uint32_t *D, size_t stride,
                                            uint32_t W, unsigned long long v, bool global) {
    uint32_t np = 0, nd = 0;
    for (uint32_t w = 0; w < W; w++) {
        np += __popc(global ? __ldcg(P + w * stride) : P[w * stride]);
        nd += __popc(global ? __ldcg(D + w * stride) : D[w * stride]);
    }
    return np == (uint32_t)((v >> 21) & M21) && nd == (uint32_t)((v >> 42) & M21);
}

struct TwohopArgs {
    const int64_t *A_off;
    const uint32_t *A_ent, *A_pos, *A_bit;
    const int64_t *B_off;
    const uint32_t *B_ent;
    const uint32_t *dprime;
    const unsigned long long *e_use, *e_all;
    const uint32_t *rsv_c;
    const int64_t *pool_off;
    const uint32_t *order;
    uint32_t *pool;
    uint32_t *ncand, *npaper;
    Counters *cnt;
    unsigned long long *bucket;     // per-CTA bucket slots of the large-anchor kernel
    unsigned long long bucket_slot; // entries per slot
    unsigned large_begin, large_end;  // order[] ranges of the two kernels
    unsigned small_begin, small_end;
    int l;
    int check;                      // run the candidate-mask self-check
    uint32_t hs_cap;                // test override: most hash slots per table (0: none)
    uint32_t wcap;                  // most visited wedges of a one-window anchor
};

// Table size after the test override (which makes tables overflow on purpose,
// to drive the CERR_HASH path).
__device__ __forceinline__ uint32_t cap_slots(uint32_t hs, const TwohopArgs &a) {
    return (a.hs_cap && hs > a.hs_cap) ? a.hs_cap : hs;
}

// ---- small anchors: one warp per anchor, private table in shared memory

constexpr int PS_THREADS = 256;
constexpr int PS_WARPS = PS_THREADS / 32;
constexpr int PS_HS = 1024;            // slots per warp
// Default and largest tier threshold in visited wedges (table load <= 1/2).
constexpr int SMALL_E_MAX = PS_HS / 2;
constexpr size_t PS_SMEM = (size_t)PS_WARPS * PS_HS * 12;

// Visit the anchor's 2-hop entries with one warp. fn(w, sdiff, bit).
template <typename F>
__device__ __forceinline__ void visit_warp(int64_t ebase, int d, bool useful_only,
                                           const uint32_t *__restrict__ A_ent,
                                           const uint32_t *__restrict__ A_pos,
                                           const uint32_t *__restrict__ A_bit,
                                           const int64_t *__restrict__ B_off,
                                           const uint32_t *__restrict__ B_ent, F fn) {
    const int lane = threadIdx.x & 31;
    for (int g = 0; g < d; g += 32) {
        int j = g + lane;
        int64_t start = 0;
        uint32_t len = 0, su = 0, bit = EMPTY;
        if (j < d) {
            int64_t e = ebase + j;
            uint32_t av = A_ent[e];
            uint32_t y = av & VMASK;
            su = av >> 31;
            bit = A_bit[e];
            start = B_off[y] + (int64_t)A_pos[e] + 1;
            len = (uint32_t)(B_off[y + 1] - start);
            if (useful_only && bit == EMPTY) len = 0;
        }
        uint32_t incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        uint32_t total = __shfl_sync(FULL, incl, 31);
        uint32_t excl = incl - len;
        for (uint32_t base = 0; base < total; base += 32) {
            uint32_t idx = base + lane;
            int s = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                uint32_t ex = __shfl_sync(FULL, excl, s + step);
                if (ex <= idx) s += step;
            }
            long long st = __shfl_sync(FULL, (long long)start, s);
            uint32_t exs = __shfl_sync(FULL, excl, s);
            uint32_t sus = __shfl_sync(FULL, su, s);
            uint32_t bits = __shfl_sync(FULL, bit, s);
            if (idx < total) {
                uint32_t ent = B_ent[st + (idx - exs)];
                fn(ent & VMASK, sus ^ (ent >> 31), bits);
            }
        }
    }
}

template <bool STATS>
__global__ void __launch_bounds__(PS_THREADS) k_twohop_small(TwohopArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *keys = (uint32_t *)(smem_raw + (size_t)warp * PS_HS * 4);
    unsigned long long *vals =
        (unsigned long long *)(smem_raw + (size_t)PS_WARPS * PS_HS * 4 + (size_t)warp * PS_HS * 8);
    const int l = a.l;
    const uint32_t lt = (1u << lane) - 1u;
    unsigned long long wedges = 0;
    for (;;) {
        unsigned item = 0;
        if (lane == 0) item = atomicAdd(&a.cnt->head_small, 1u);
        item = __shfl_sync(FULL, item, 0) + a.small_begin;
        if (item >= a.small_end) break;
        const uint32_t r = a.order[item];
        const int64_t ebase = a.A_off[r];
        const int d = (int)(a.A_off[r + 1] - ebase);
        const uint32_t W = (a.dprime[r] + 31) / 32;
        const uint32_t rsv = a.rsv_c[r];
        uint32_t *region = a.pool + a.pool_off[r];
        const unsigned long long e_vis = STATS ? a.e_all[r] : a.e_use[r];
        uint32_t hs = (uint32_t)(2 * e_vis + 31) & ~31u;
        hs = hs < 64 ? 64 : (hs > PS_HS ? PS_HS : hs);
        hs = cap_slots(hs, a);
        for (uint32_t i = lane; i < hs; i += 32) {
            keys[i] = EMPTY;
            vals[i] = 0;
        }
        __syncwarp();
        bool ovf = false;
        visit_warp(ebase, d, !STATS, a.A_ent, a.A_pos, a.A_bit, a.B_off, a.B_ent,
                   [&](uint32_t w, uint32_t sdiff, uint32_t bit) {
                       if (!tab_insert(keys, vals, hs, w, pass1_add(sdiff, bit))) ovf = true;
                   });
        __syncwarp();
        uint32_t ncw = 0, npaper = 0;
        if (__any_sync(FULL, ovf)) {
            if (lane == 0) atomicOr(&a.cnt->err, CERR_HASH);
        } else {
            for (uint32_t base = 0; base < hs; base += 32) {
                uint32_t i = base + lane;
                bool cand = false, pap = false;
                unsigned long long v = 0;
                if (i < hs && keys[i] != EMPTY) {
                    v = vals[i];
                    pap = STATS && (v & M21) >= (unsigned long long)l;
                    cand = keep_candidate(v, l);
                }
                uint32_t bal = __ballot_sync(FULL, cand);
                if (cand) vals[i] = cand_value(v, ncw + __popc(bal & lt));
                ncw += __popc(bal);
                npaper += __popc(__ballot_sync(FULL, pap));
            }
            __syncwarp();
            if (ncw > rsv) {
                if (lane == 0) atomicOr(&a.cnt->err, CERR_RESERVE);
                ncw = 0;
            }
            if (ncw > 0) {
                // The pool is zeroed on the stream before the 2-hop launches,
                // so the masks are built by atomicOr alone (no zeroing stores
                // of this kernel ever meet its atomics on the same words).
                visit_warp(ebase, d, true, a.A_ent, a.A_pos, a.A_bit, a.B_off, a.B_ent,
                           [&](uint32_t w, uint32_t sdiff, uint32_t bit) {
                               int sl = tab_find(keys, hs, w);
                               if (sl < 0) return;
                               unsigned long long v = vals[sl];
                               if (!(v & CAND)) return;
                               uint32_t c = cand_index(v);
                               uint32_t m = 1u << (bit & 31);
                               size_t wd = bit >> 5;
                               atomicOr(&region[wd * rsv + c], m);
                               if (sdiff) atomicOr(&region[(W + wd) * rsv + c], m);
                           });
                if (a.check) {
                    __syncwarp();
                    bool bad = false;
                    for (uint32_t i = lane; i < hs; i += 32) {
                        if (keys[i] == EMPTY) continue;
                        unsigned long long v = vals[i];
                        if (!(v & CAND)) continue;
                        uint32_t c = cand_index(v);
                        if (!masks_match(region + c, region + (size_t)W * rsv + c, rsv, W, v, true))
                            bad = true;
                    }
                    if (__any_sync(FULL, bad) && lane == 0) atomicOr(&a.cnt->err, CERR_MASK);
                }
            }
        }
        if (lane == 0) {
            a.ncand[r] = ncw;
            if (STATS) a.npaper[r] = npaper;
        }
        wedges += e_vis;
        __syncwarp();
    }
    if (lane == 0 && wedges) atomicAdd(&a.cnt->wedges, wedges);
}

// ---- large anchors: one CTA per anchor, wedges flattened over the CTA

constexpr int PL_THREADS = 512;
constexpr int PL_WARPS = PL_THREADS / 32;
constexpr int PL_HS = 7168;             // slots
constexpr int PL_WCAP = PL_HS / 2;      // visited wedges per re-read window (load <= 1/2)
constexpr int PL_BCAP = PL_HS / 3;      // expected entries per bucket (bucket <= 1.5x + 64)
constexpr int PL_MAXCLS = 1024;         // bucket classes per anchor
constexpr int PL_PCH = PL_THREADS;      // positions staged per chunk
constexpr int PL_STAGE_WORDS = 4096;    // staged P/D words
constexpr size_t PL_OFF_VALS = (size_t)PL_HS * 4;
constexpr size_t PL_OFF_PST = PL_OFF_VALS + (size_t)PL_HS * 8;
constexpr size_t PL_OFF_PPRE = PL_OFF_PST + (size_t)PL_PCH * 8;
constexpr size_t PL_OFF_PINFO = PL_OFF_PPRE + (size_t)(PL_PCH + 4) * 4;
constexpr size_t PL_OFF_STAGE = PL_OFF_PINFO + (size_t)PL_PCH * 4;
constexpr size_t PL_SMEM = PL_OFF_STAGE + (size_t)PL_STAGE_WORDS * 4;

// Bucket entry of a wedge: w (bits 0..30), sdiff (bit 31), bit index of the
// position (bits 32..52; all ones when the position is not useful).
constexpr unsigned long long BE_NOBIT = (1ull << 21) - 1;

__device__ __forceinline__ unsigned long long bucket_entry(uint32_t w, uint32_t sdiff, uint32_t bit) {
    const unsigned long long bi = bit == EMPTY ? BE_NOBIT : (unsigned long long)bit;
    return (unsigned long long)w | ((unsigned long long)sdiff << 31) | (bi << 32);
}

__host__ __device__ __forceinline__ unsigned long long bucket_cap(unsigned long long e_vis, int lg) {
    return ((e_vis >> lg) * 3) / 2 + 65;
}

// Largest bucket area one anchor can need: sum of its classes' capacities.
__host__ __device__ __forceinline__ int bucket_lg(unsigned long long e_vis) {
    int lg = 0;
    while (((unsigned long long)PL_BCAP << lg) < e_vis && lg < 10) lg++;
    return lg;
}

__device__ __forceinline__ unsigned long long block_excl_scan_u64(unsigned long long v,
                                                                  unsigned long long *warp_tot,
                                                                  unsigned long long *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = PL_WARPS;
    unsigned long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned long long wv = lane < NW ? warp_tot[lane] : 0ull;
        unsigned long long wi = wv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long t = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < NW) warp_tot[lane] = wi - wv;
        if (lane == NW - 1) *total = wi;
    }
    __syncthreads();
    return warp_tot[warp] + incl - v;
}

// Visit the anchor's 2-hop entries with the whole CTA; with lg_nw > 0 only
// entries of hash class `cls`. Positions are staged PL_PCH at a time and the
// non-empty ones compacted; each warp takes 32 consecutive entries, one
// binary search for the first and short forward walks for the others.
// fn(w, sdiff, bit).
template <typename F>
__device__ __forceinline__ void visit_block(int64_t ebase, int d, bool useful_only, int lg_nw,
                                            uint32_t cls, const TwohopArgs &a, int64_t *pst,
                                            uint32_t *ppre, uint32_t *pinfo,
                                            unsigned long long *warp_tot,
                                            unsigned long long *s_total, F fn) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int c0 = 0; c0 < d; c0 += PL_PCH) {
        const int nch = d - c0 < PL_PCH ? d - c0 : PL_PCH;
        uint32_t len = 0, info = 0;
        int64_t st = 0;
        if (tid < nch) {
            int64_t e = ebase + c0 + tid;
            uint32_t av = a.A_ent[e];
            uint32_t y = av & VMASK;
            uint32_t bit = a.A_bit[e];
            st = a.B_off[y] + (int64_t)a.A_pos[e] + 1;
            len = (uint32_t)(a.B_off[y + 1] - st);
            if (useful_only && bit == EMPTY) len = 0;
            info = (av & 0x80000000u) | (bit == EMPTY ? NOBIT : bit);
        }
        // scan of (non-empty flag, length): compact slot and entry prefix
        unsigned long long packed = len ? ((1ull << 32) | len) : 0ull;
        unsigned long long ex = block_excl_scan_u64(packed, warp_tot, s_total);
        if (len) {
            const uint32_t slot = (uint32_t)(ex >> 32);
            pst[slot] = st;
            pinfo[slot] = info;
            ppre[slot] = (uint32_t)ex;
        }
        __syncthreads();
        const uint32_t npos = (uint32_t)(*s_total >> 32);
        const uint32_t total = (uint32_t)*s_total;
        for (uint32_t base = (uint32_t)warp * 32; base < total; base += PL_THREADS) {
            uint32_t p0 = 0;
            if (lane == 0) {
                uint32_t lo = 0, hi = npos;  // largest j with ppre[j] <= base
                while (hi - lo > 1) {
                    uint32_t mid = (lo + hi) >> 1;
                    if (ppre[mid] <= base) lo = mid; else hi = mid;
                }
                p0 = lo;
            }
            uint32_t p = __shfl_sync(FULL, p0, 0);
            const uint32_t t = base + lane;
            if (t < total) {
                while (p + 1 < npos && ppre[p + 1] <= t) p++;
                uint32_t ent = a.B_ent[pst[p] + (t - ppre[p])];
                uint32_t w = ent & VMASK;
                if (lg_nw == 0 || class_of(w, lg_nw) == cls) {
                    uint32_t inf = pinfo[p];
                    uint32_t bit = inf & NOBIT;
                    fn(w, (inf >> 31) ^ (ent >> 31), bit == NOBIT ? EMPTY : bit);
                }
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <bool STATS>
__global__ void __launch_bounds__(PL_THREADS) k_twohop_large(TwohopArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *keys = (uint32_t *)smem_raw;
    unsigned long long *vals = (unsigned long long *)(smem_raw + PL_OFF_VALS);
    int64_t *pst = (int64_t *)(smem_raw + PL_OFF_PST);
    uint32_t *ppre = (uint32_t *)(smem_raw + PL_OFF_PPRE);
    uint32_t *pinfo = (uint32_t *)(smem_raw + PL_OFF_PINFO);
    uint32_t *stage = (uint32_t *)(smem_raw + PL_OFF_STAGE);
    __shared__ unsigned long long warp_tot[PL_WARPS];
    __shared__ unsigned long long s_total;
    __shared__ unsigned s_item, s_ncw, s_paper, s_ovf;
    __shared__ uint32_t s_bcnt[PL_MAXCLS];
    const int tid = threadIdx.x, lane = tid & 31;
    const int l = a.l;
    unsigned long long *bucket =
        a.bucket ? a.bucket + (size_t)blockIdx.x * a.bucket_slot : nullptr;
    unsigned long long wedges = 0;

    // Candidate filter over the table, window-local indices in vals.
    auto extract = [&](uint32_t hs) {
        for (uint32_t base = 0; base < hs; base += PL_THREADS) {
            uint32_t i = base + tid;
            bool cand = false, pap = false;
            if (i < hs && keys[i] != EMPTY) {
                unsigned long long v = vals[i];
                pap = STATS && (v & M21) >= (unsigned long long)l;
                cand = keep_candidate(v, l);
            }
            uint32_t bal = __ballot_sync(FULL, cand);
            uint32_t pb = __ballot_sync(FULL, pap);
            uint32_t wbase = 0;
            if (lane == 0 && bal) wbase = atomicAdd(&s_ncw, (unsigned)__popc(bal));
            if (lane == 0 && pb) atomicAdd(&s_paper, (unsigned)__popc(pb));
            wbase = __shfl_sync(FULL, wbase, 0);
            if (cand) vals[i] = cand_value(vals[i], wbase + __popc(bal & ((1u << lane) - 1u)));
        }
    };
    auto set_bits = [&](uint32_t hs, uint32_t *bb, uint32_t bstride, uint32_t W, uint32_t w,
                        uint32_t sdiff, uint32_t bit) {
        int sl = tab_find(keys, hs, w);
        if (sl < 0) return;
        unsigned long long v = vals[sl];
        if (!(v & CAND)) return;
        uint32_t c = cand_index(v);
        uint32_t m = 1u << (bit & 31);
        size_t wd = bit >> 5;
        atomicOr(&bb[wd * bstride + c], m);
        if (sdiff) atomicOr(&bb[(W + wd) * bstride + c], m);
    };

    for (;;) {
        if (tid == 0) s_item = a.large_begin + atomicAdd(&a.cnt->head_large, 1u);
        __syncthreads();
        const unsigned item = s_item;
        __syncthreads();
        if (item >= a.large_end) break;
        const uint32_t r = a.order[item];
        const int64_t ebase = a.A_off[r];
        const int d = (int)(a.A_off[r + 1] - ebase);
        const uint32_t W = (a.dprime[r] + 31) / 32;
        const uint32_t rsv = a.rsv_c[r];
        uint32_t *region = a.pool + a.pool_off[r];
        const unsigned long long e_vis = STATS ? a.e_all[r] : a.e_use[r];
        const unsigned long long e_use = a.e_use[r];
        const long long c0 = clock64();
        unsigned long long reads = 0;
        int path = 0;
        uint32_t nc = 0, npaper = 0;
        bool failed = false;

        // Window bookkeeping shared by both strategies: after the table of
        // one window holds its counts, keep candidates and write their bits.
        // Returns false when the reservation would overflow.
        auto finish_window = [&](uint32_t hs, auto &&pass2) -> bool {
            extract(hs);
            __syncthreads();
            const uint32_t ncw = s_ncw;
            npaper += s_paper;
            if (ncw > 0) {
                if (nc + ncw > rsv) {
                    if (tid == 0) atomicOr(&a.cnt->err, CERR_RESERVE);
                    __syncthreads();
                    return false;
                }
                const bool staged = 2ull * W * ncw <= (unsigned long long)PL_STAGE_WORDS;
                uint32_t *bb = staged ? stage : region + nc;
                const uint32_t bstride = staged ? ncw : rsv;
                for (uint32_t i = tid; i < 2 * W * ncw; i += PL_THREADS) {
                    uint32_t wd = i / ncw, c = i % ncw;
                    bb[(size_t)wd * bstride + c] = 0;
                }
                __syncthreads();
                pass2(bb, bstride);
                __syncthreads();
                if (a.check) {
                    bool bad = false;
                    for (uint32_t i = tid; i < hs; i += PL_THREADS) {
                        if (keys[i] == EMPTY) continue;
                        const unsigned long long v = vals[i];
                        if (!(v & CAND)) continue;
                        const uint32_t c = cand_index(v);
                        if (!masks_match(bb + c, bb + (size_t)W * bstride + c, bstride, W, v, !staged))
                            bad = true;
                    }
                    if (bad) atomicOr(&a.cnt->err, CERR_MASK);
                    __syncthreads();
                }
                if (staged) {
                    for (uint32_t i = tid; i < 2 * W * ncw; i += PL_THREADS) {
                        uint32_t wd = i / ncw, c = i % ncw;
                        region[(size_t)wd * rsv + nc + c] = stage[i];
                    }
                }
                nc += ncw;
            }
            __syncthreads();
            return true;
        };
        auto clear_table = [&](uint32_t hs) {
            for (uint32_t i = tid; i < hs; i += PL_THREADS) {
                keys[i] = EMPTY;
                vals[i] = 0;
            }
            if (tid == 0) {
                s_ncw = 0;
                s_paper = 0;
                s_ovf = 0;
            }
            __syncthreads();
        };

        const int lgb = bucket_lg(e_vis);
        bool bucketed = false;
        if (e_vis <= (unsigned long long)a.wcap) {
            // one window
            uint32_t hs = (uint32_t)((2 * e_vis + 31) & ~31ull);
            hs = hs < 64 ? 64 : (hs > PL_HS ? PL_HS : hs);
            hs = cap_slots(hs, a);
            clear_table(hs);
            reads = e_vis + e_use;
            visit_block(ebase, d, !STATS, 0, 0, a, pst, ppre, pinfo, warp_tot, &s_total,
                        [&](uint32_t w, uint32_t sdiff, uint32_t bit) {
                            if (!tab_insert(keys, vals, hs, w, pass1_add(sdiff, bit))) s_ovf = 1;
                        });
            if (s_ovf) {
                failed = true;
                if (tid == 0) atomicOr(&a.cnt->err, CERR_HASH);
            } else {
                failed = !finish_window(hs, [&](uint32_t *bb, uint32_t bstride) {
                    visit_block(ebase, d, true, 0, 0, a, pst, ppre, pinfo, warp_tot, &s_total,
                                [&](uint32_t w, uint32_t sdiff, uint32_t bit) {
                                    set_bits(hs, bb, bstride, W, w, sdiff, bit);
                                });
                });
            }
        } else if (bucket && lgb <= 10 &&
                   (bucket_cap(e_vis, lgb) << lgb) <= a.bucket_slot) {
            // partition the wedges once into 2^lgb hash classes, then one
            // window per class from its bucket
            const uint32_t ncls = 1u << lgb;
            const uint32_t cap = (uint32_t)bucket_cap(e_vis, lgb);
            for (uint32_t i = tid; i < ncls; i += PL_THREADS) s_bcnt[i] = 0;
            if (tid == 0) s_ovf = 0;
            __syncthreads();
            visit_block(ebase, d, !STATS, 0, 0, a, pst, ppre, pinfo, warp_tot, &s_total,
                        [&](uint32_t w, uint32_t sdiff, uint32_t bit) {
                            uint32_t c = class_of(w, lgb);
                            uint32_t pos = atomicAdd(&s_bcnt[c], 1u);
                            if (pos < cap) bucket[(size_t)c * cap + pos] = bucket_entry(w, sdiff, bit);
                            else s_ovf = 1;
                        });
            reads = e_vis;
            path = 1;
            __syncthreads();
            // A partner sharing many of the anchor's positions fills its class
            // beyond the capacity. The class sizes are exact all the same, so
            // the wedges are then scattered once more, classes back to back.
            const bool packed = s_ovf != 0;
            if (packed) {
                uint32_t *cursor = keys;  // the table is free until the windows
                const uint32_t c2 = 2 * tid;
                const uint32_t n0 = c2 < ncls ? s_bcnt[c2] : 0u;
                const uint32_t n1 = c2 + 1 < ncls ? s_bcnt[c2 + 1] : 0u;
                const unsigned long long ex = block_excl_scan_u64(n0 + n1, warp_tot, &s_total);
                if (c2 < ncls) cursor[c2] = (uint32_t)ex;
                if (c2 + 1 < ncls) cursor[c2 + 1] = (uint32_t)ex + n0;
                __syncthreads();
                visit_block(ebase, d, !STATS, 0, 0, a, pst, ppre, pinfo, warp_tot, &s_total,
                            [&](uint32_t w, uint32_t sdiff, uint32_t bit) {
                                uint32_t pos = atomicAdd(&cursor[class_of(w, lgb)], 1u);
                                bucket[pos] = bucket_entry(w, sdiff, bit);
                            });
                reads += e_vis;
                path = 3;
                __syncthreads();
            }
            bucketed = true;
            size_t base = 0;
            for (uint32_t c = 0; c < ncls && !failed; c++) {
                const uint32_t n = s_bcnt[c];
                const unsigned long long *bk = bucket + (packed ? base : (size_t)c * cap);
                base += n;
                if (n == 0) continue;
                // one window for the class; when its distinct partners overflow
                // the table, 2^lg2 windows over its sub-classes
                const uint32_t nc0 = nc, np0 = npaper;
                for (int lg2 = 0; !failed; lg2++) {
                    if (lg2 > 8) {
                        if (tid == 0) atomicOr(&a.cnt->err, CERR_HASH);
                        failed = true;
                        break;
                    }
                    const uint32_t per = (n + (1u << lg2) - 1) >> lg2;
                    uint32_t hs = (uint32_t)((2ull * per + 31) & ~31ull);
                    hs = hs < 64 ? 64 : (hs > PL_HS ? PL_HS : hs);
                    hs = cap_slots(hs, a);
                    nc = nc0;
                    npaper = np0;
                    bool over = false;
                    for (uint32_t sub = 0; sub < (1u << lg2) && !failed; sub++) {
                        __syncthreads();
                        clear_table(hs);
                        for (uint32_t i = tid; i < n; i += PL_THREADS) {
                            unsigned long long e = bk[i];
                            const uint32_t w = (uint32_t)e & VMASK;
                            if (lg2 && subclass_of(w, lgb, lg2) != sub) continue;
                            uint32_t bi = (uint32_t)(e >> 32);
                            uint32_t bit = bi == (uint32_t)BE_NOBIT ? EMPTY : bi;
                            if (!tab_insert(keys, vals, hs, w, pass1_add((uint32_t)(e >> 31) & 1u, bit)))
                                s_ovf = 1;
                        }
                        __syncthreads();
                        if (s_ovf) {
                            over = true;
                            break;
                        }
                        failed = !finish_window(hs, [&](uint32_t *bb, uint32_t bstride) {
                            for (uint32_t i = tid; i < n; i += PL_THREADS) {
                                unsigned long long e = bk[i];
                                uint32_t bi = (uint32_t)(e >> 32);
                                if (bi == (uint32_t)BE_NOBIT) continue;
                                const uint32_t w = (uint32_t)e & VMASK;
                                if (lg2 && subclass_of(w, lgb, lg2) != sub) continue;
                                set_bits(hs, bb, bstride, W, w, (uint32_t)(e >> 31) & 1u, bi);
                            }
                        });
                    }
                    if (!over) break;
                    if (lg2 == 0 && tid == 0) atomicAdd(&a.cnt->tw_split, 1ull);
                }
            }
        }
        if (!bucketed && !failed && e_vis > (unsigned long long)a.wcap) {
            // re-read windows: every pass over the 2-hop keeps one hash class
            nc = 0;
            npaper = 0;
            int lg_nw = 0;
            while (((unsigned long long)a.wcap << lg_nw) < e_vis) lg_nw++;
            path = 2;
            for (int attempt = 0; attempt < 8 && !failed; attempt++) {
                const uint32_t nw = 1u << lg_nw;
                reads += (unsigned long long)nw * (e_vis + e_use);
                const unsigned long long per = (e_vis + nw - 1) >> lg_nw;
                uint32_t hs = (uint32_t)((2 * per + 31) & ~31ull);
                hs = hs < 64 ? 64 : (hs > PL_HS ? PL_HS : hs);
                hs = cap_slots(hs, a);
                nc = 0;
                npaper = 0;
                bool restart = false;
                for (uint32_t cls = 0; cls < nw && !failed; cls++) {
                    clear_table(hs);
                    visit_block(ebase, d, !STATS, lg_nw, cls, a, pst, ppre, pinfo, warp_tot,
                                &s_total, [&](uint32_t w, uint32_t sdiff, uint32_t bit) {
                                    if (!tab_insert(keys, vals, hs, w, pass1_add(sdiff, bit)))
                                        s_ovf = 1;
                                });
                    if (s_ovf) {
                        restart = true;
                        break;
                    }
                    failed = !finish_window(hs, [&](uint32_t *bb, uint32_t bstride) {
                        visit_block(ebase, d, true, lg_nw, cls, a, pst, ppre, pinfo, warp_tot,
                                    &s_total, [&](uint32_t w, uint32_t sdiff, uint32_t bit) {
                                        set_bits(hs, bb, bstride, W, w, sdiff, bit);
                                    });
                    });
                }
                if (!restart) break;
                lg_nw++;
                if (attempt == 7) {
                    if (tid == 0) atomicOr(&a.cnt->err, CERR_HASH);
                    failed = true;
                }
                __syncthreads();
            }
        }
        if (failed) nc = 0;
        if (tid == 0) {
            a.ncand[r] = nc;
            if (STATS) a.npaper[r] = npaper;
            wedges += e_vis;
            atomicAdd(&a.cnt->tw_reads, reads);
            atomicAdd(&a.cnt->tw_cyc[path], (unsigned long long)(clock64() - c0));
            atomicAdd(&a.cnt->tw_anchors[path], 1ull);
        }
        __syncthreads();
    }
    if (tid == 0) {
        if (wedges) atomicAdd(&a.cnt->wedges, wedges);
        const unsigned long long t = global_ns();
        atomicMax(&a.cnt->tw_fin_max, t);
        atomicMax(&a.cnt->tw_fin_min_n, ~t);
    }
}

// ------------------------------------------------------------------ groups

// Candidate-mask words of the sorted anchors: gw[i] = words of order[i].
__global__ void k_gather_words(const uint32_t *order, const int64_t *words_by_rank, int64_t n,
                               int64_t *gw) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n;
         i += (int64_t)gridDim.x * blockDim.x)
        gw[i] = i < n ? words_by_rank[order[i]] : 0;
}

// Pool offsets of one group of sorted anchors [a, b): offset from cum[a].
__global__ void k_group_offsets(const uint32_t *order, const int64_t *cum, int64_t a, int64_t b,
                                int64_t *pool_off) {
    for (int64_t i = a + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < b;
         i += (int64_t)gridDim.x * blockDim.x)
        pool_off[order[i]] = cum[i] - cum[a];
}

// ------------------------------------------------------------------ items

// Saturating binom(n, k) in 64 bits (planning cost only).
__device__ __forceinline__ unsigned long long binom_sat(unsigned long long n, int k) {
    if ((long long)n < k) return 0;
    unsigned long long r = 1;
    for (int i = 1; i <= k; i++) {
        unsigned long long f = n - k + i;
        if (r > 0xFFFFFFFFFFFFFFFFull / f) return 0xFFFFFFFFFFFFFFFFull;
        r = r * f / i;
    }
    return r;
}

// A work item of one anchor. Candidate side: rows [i0, i1) of first
// partners, all their units when u1 == 0, else units [u0, u1) of row i0.
// Position side (u1 == POS_ITEM): first positions [i0, i1).
struct Item {
    uint32_t anchor, i0, i1, u0, u1;
};
constexpr uint32_t POS_ITEM = 0xFFFFFFFFu;
constexpr int POS_MAX_WORDS = 128;  // candidate words of a position-side mask (4 per lane)

constexpr int ROWS_MAX = 1024;
constexpr int PB_SMEM_WORDS_PLAN = 24576;  // staged words of the tuple kernel (PB_SMEM_WORDS)

struct ItemArgs {
    const uint32_t *ncand, *npaper, *dprime;
    const uint32_t *order;  // anchors of the group: order[begin .. begin + nX)
    int64_t begin;
    int64_t nX;             // anchors in the group
    int R, l;
    int method;  // 0: cheaper side per anchor, 1: candidate side, 2: position side where it fits
    unsigned long long pos_unit;  // cost of one position-side prefix node per candidate word-lane
    unsigned long long item_cost;
    const int64_t *item_off;  // emit pass
    int64_t *item_cnt;        // count pass (nX + 1 entries)
    Item *items;
    uint32_t *ikey, *ival;
    Counters *cnt;
    // tensor-core pair step (two partners, candidate side, wide masks)
    int tc_on;
    uint32_t tc_min_w, tc_min_nc;
    uint32_t *tc_list;
};

__device__ __forceinline__ unsigned long long row_cost(uint32_t nc, uint32_t i, int R, uint32_t W) {
    if (R == 1) return 0;
    unsigned long long t = binom_sat(nc - 1 - i, R - 1);
    unsigned long long c = t * W;
    return (W && c / W != t) ? 0xFFFFFFFFFFFFFFFFull : c;
}

__device__ __forceinline__ unsigned long long unit_cost(uint32_t nc, uint32_t i, uint32_t u, int R,
                                                        uint32_t W) {
    if (R <= 2) return 32ull * W;
    unsigned long long s = 0;
    uint32_t j0 = i + 1 + 32 * u;
    for (uint32_t j = j0; j < j0 + 32 && j < nc; j++) {
        unsigned long long t = binom_sat(nc - 1 - j, R - 2);
        s = (s + t < s) ? 0xFFFFFFFFFFFFFFFFull : s + t;
    }
    unsigned long long c = s * W;
    return (W && c / W != s) ? 0xFFFFFFFFFFFFFFFFull : c;
}

// Position-side enumeration of one anchor (see k_tuples): l-subsets Q of the
// anchor's useful positions, each with N_Q candidates whose same-sign or
// different-sign part of L[w] contains Q; the anchor adds sum over Q of
// binom(N_Q, R). Cost in the candidate-side units (mask words x tuples):
// 32 lanes x 3 steps x words per lane for every prefix node.
__device__ __forceinline__ bool pos_fits(uint32_t nc, uint32_t dp, int l) {
    const uint32_t wc = (nc + 31) / 32;
    return dp >= (uint32_t)l && wc <= (uint32_t)POS_MAX_WORDS &&
           2ull * dp * (wc | 1u) <= (unsigned long long)PB_SMEM_WORDS_PLAN;
}

__device__ __forceinline__ unsigned long long pos_row_cost(uint32_t nc, uint32_t dp, uint32_t q1,
                                                           int l, unsigned long long unit) {
    const unsigned long long wpl = ((nc + 31) / 32 + 31) / 32;
    unsigned long long nodes = 0;
    for (int i = 0; i < l; i++) {
        unsigned long long t = binom_sat(dp - 1 - q1, i);
        nodes = (nodes + t < nodes) ? 0xFFFFFFFFFFFFFFFFull : nodes + t;
    }
    unsigned long long c = nodes * unit * wpl;
    return (c / (unit * wpl) != nodes) ? 0xFFFFFFFFFFFFFFFFull : c;
}

__device__ __forceinline__ unsigned long long pos_cost(uint32_t nc, uint32_t dp, int l,
                                                       unsigned long long unit) {
    const unsigned long long wpl = ((nc + 31) / 32 + 31) / 32;
    unsigned long long nodes = 0;
    for (int i = 1; i <= l; i++) {
        unsigned long long t = binom_sat(dp, i);
        nodes = (nodes + t < nodes) ? 0xFFFFFFFFFFFFFFFFull : nodes + t;
    }
    unsigned long long c = nodes * unit * wpl;
    return (c / (unit * wpl) != nodes) ? 0xFFFFFFFFFFFFFFFFull : c;
}

__device__ __forceinline__ unsigned long long cand_cost(uint32_t nc, uint32_t W, int R) {
    unsigned long long t = binom_sat(nc, R);
    unsigned long long c = t * (W ? W : 1);
    return (W > 1 && c / W != t) ? 0xFFFFFFFFFFFFFFFFull : c;
}

// True when the anchor takes the position side (cheaper, or forced).
__device__ __forceinline__ bool use_pos(uint32_t nc, uint32_t dp, int R, int l, int method,
                                        unsigned long long unit) {
    if (method == 1 || nc < (uint32_t)R || !pos_fits(nc, dp, l)) return false;
    if (method == 2) return true;
    return pos_cost(nc, dp, l, unit) < cand_cost(nc, (dp + 31) / 32, R);
}

// True when the anchor's pairs go to the tensor-core kernel (tc_pairs.cu):
// two partners, candidate side, at least tc_min_w mask words and tc_min_nc
// candidates.
__device__ __forceinline__ bool tc_take(const ItemArgs &a, uint32_t nc, uint32_t dp) {
    return a.tc_on && a.R == 2 && nc >= a.tc_min_nc && (dp + 31) / 32 >= a.tc_min_w &&
           !use_pos(nc, dp, a.R, a.l, a.method, a.pos_unit);
}

// Anchor cost, anchor tuple counts, tensor-core anchor list. Thread per anchor.
__global__ void k_anchor_cost(ItemArgs a) {
    U128 tp, to;
    unsigned long long cand = 0, cost = 0;
    for (int64_t ix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ix < a.nX;
         ix += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = a.order[a.begin + ix];
        uint32_t nc = a.ncand[r];
        uint32_t W = (a.dprime[r] + 31) / 32;
        if (a.npaper) {
            uint32_t np = a.npaper[r];
            cand += np;
            if (np >= (uint32_t)a.R) {
                // binom(np, R) exactly: np < 2^32, R <= 7, fits 128 bits
                unsigned long long lo = 1, hi = 0;
                for (int i = 1; i <= a.R; i++) {
                    unsigned long long f = np - a.R + i;
                    unsigned g = gcd_u32((unsigned)(f % (unsigned)i), (unsigned)i);
                    if (g == 0) g = i;
                    div_u128_small(lo, hi, i / g);
                    mul_u128_u64(lo, hi, f / g);
                }
                U128 t;
                t.lo = lo;
                t.hi = hi;
                tp.add(t);
            }
        } else {
            cand += nc;
        }
        if (nc >= (uint32_t)a.R) {
            unsigned long long t = binom_sat(nc, a.R);
            to.add(t);
            if (tc_take(a, nc, a.dprime[r])) {
                a.tc_list[atomicAdd(&a.cnt->n_tc, 1u)] = r;
            } else {
                unsigned long long c = use_pos(nc, a.dprime[r], a.R, a.l, a.method, a.pos_unit)
                                           ? pos_cost(nc, a.dprime[r], a.l, a.pos_unit)
                                           : cand_cost(nc, W, a.R);
                cost = (cost + c < cost) ? 0xFFFFFFFFFFFFFFFFull : cost + c;
            }
        }
    }
    tp = warp_sum_u128(tp, nullptr);
    to = warp_sum_u128(to, nullptr);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cand += __shfl_xor_sync(FULL, cand, o);
        unsigned long long t = __shfl_xor_sync(FULL, cost, o);
        cost = (cost + t < cost) ? 0xFFFFFFFFFFFFFFFFull : cost + t;
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_add_u128(a.cnt->tuples_paper, tp.lo, tp.hi, nullptr);
        atomic_add_u128(a.cnt->tuples_ours, to.lo, to.hi, nullptr);
        atomicAdd(&a.cnt->candidates, cand);
        atomicAdd(&a.cnt->cost_total, cost);
    }
}

// Split each anchor's tuple space into items. EMIT == false counts them.
template <bool EMIT>
__global__ void k_items(ItemArgs a) {
    for (int64_t ix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ix < a.nX;
         ix += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = a.order[a.begin + ix];
        const uint32_t nc = a.ncand[r];
        const int R = a.R;
        int64_t n = 0;
        int64_t out = EMIT ? a.item_off[ix] : 0;
        const uint32_t W = (a.dprime[r] + 31) / 32;
        auto emit = [&](uint32_t i0, uint32_t i1, uint32_t u0, uint32_t u1, unsigned long long c) {
            if (EMIT) {
                Item it;
                it.anchor = (uint32_t)r;
                it.i0 = i0;
                it.i1 = i1;
                it.u0 = u0;
                it.u1 = u1;
                a.items[out + n] = it;
                uint32_t c32 = c < 0xFFFFFFFEull ? (uint32_t)c : 0xFFFFFFFEu;
                a.ikey[out + n] = 0xFFFFFFFEu - c32;
                a.ival[out + n] = (uint32_t)(out + n);
            }
            n++;
        };
        const uint32_t dp = a.dprime[r];
        if (nc >= (uint32_t)R && nc > 0 && tc_take(a, nc, dp)) {
            // the tensor-core kernel takes this anchor's pairs: no items
        } else if (nc >= (uint32_t)R && nc > 0 && use_pos(nc, dp, R, a.l, a.method, a.pos_unit)) {
            const uint32_t rows = dp - a.l + 1;
            const unsigned long long cap = 4 * a.item_cost;
            uint32_t rb = 0;
            unsigned long long acc = 0;
            for (uint32_t q1 = 0; q1 < rows; q1++) {
                unsigned long long c = pos_row_cost(nc, dp, q1, a.l, a.pos_unit);
                if (q1 > rb && (acc + c > cap || q1 - rb >= (uint32_t)ROWS_MAX)) {
                    emit(rb, q1, 0, POS_ITEM, acc);
                    rb = q1;
                    acc = 0;
                }
                acc = (acc + c < acc) ? 0xFFFFFFFFFFFFFFFFull : acc + c;
            }
            emit(rb, rows, 0, POS_ITEM, acc);
        } else if (nc >= (uint32_t)R && nc > 0) {
            if (R == 1) {
                uint32_t units = (nc + 31) / 32;
                unsigned long long per = 32ull * W, acc = 0;
                uint32_t u0 = 0;
                for (uint32_t u = 0; u < units; u++) {
                    if (acc > 0 && acc + per > a.item_cost) {
                        emit(0, 1, u0, u, acc);
                        u0 = u;
                        acc = 0;
                    }
                    acc += per;
                }
                emit(0, 1, u0, units, acc);
            } else {
                const uint32_t rows = nc - R + 1;
                uint32_t rb = 0;
                unsigned long long acc = 0;
                for (uint32_t i = 0; i < rows; i++) {
                    unsigned long long ci = row_cost(nc, i, R, W);
                    if (ci > a.item_cost) {
                        if (i > rb) emit(rb, i, 0, 0, acc);
                        uint32_t units = (nc - 1 - i + 31) / 32;
                        uint32_t u0 = 0;
                        unsigned long long ua = 0;
                        for (uint32_t u = 0; u < units; u++) {
                            unsigned long long cu = unit_cost(nc, i, u, R, W);
                            if (ua > 0 && ua + cu > a.item_cost) {
                                emit(i, i + 1, u0, u, ua);
                                u0 = u;
                                ua = 0;
                            }
                            ua = (ua + cu < ua) ? 0xFFFFFFFFFFFFFFFFull : ua + cu;
                        }
                        emit(i, i + 1, u0, units, ua);
                        rb = i + 1;
                        acc = 0;
                    } else {
                        if (i > rb && (acc + ci > a.item_cost || i - rb >= (uint32_t)ROWS_MAX)) {
                            emit(rb, i, 0, 0, acc);
                            rb = i;
                            acc = 0;
                        }
                        acc += ci;
                    }
                }
                if (rows > rb) emit(rb, rows, 0, 0, acc);
            }
        }
        if (!EMIT) a.item_cnt[ix] = n;
    }
    if (!EMIT && blockIdx.x == 0 && threadIdx.x == 0) a.item_cnt[a.nX] = 0;
}

// Inputs of the tensor-core plan: the listed anchors' sizes and pool offsets.
__global__ void k_tc_gather(const uint32_t *list, unsigned n, const uint32_t *ncand,
                            const uint32_t *dprime, const uint32_t *rsv_c, const int64_t *pool_off,
                            TcInput *out) {
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t r = list[i];
        TcInput t;
        t.r = r;
        t.nc = ncand[r];
        t.W = (dprime[r] + 31) / 32;
        t.rsv = rsv_c[r];
        t.pool_off = pool_off[r];
        out[i] = t;
    }
}

// ------------------------------------------------------------------ tuples

constexpr int PB_THREADS = 256;
constexpr int PB_WARPS = PB_THREADS / 32;
constexpr int PB_SMEM_WORDS = PB_SMEM_WORDS_PLAN;  // 96 KB of staged words
constexpr size_t PB_SMEM = PB_SMEM_WORDS * 4;
constexpr int SCRATCH_SLOTS = 7;  // per-warp mask slots for wide anchors (>= max(R, 6))

struct TupleArgs {
    const uint32_t *ncand, *dprime, *rsv_c;
    const int64_t *pool_off;
    const uint32_t *pool;
    const Item *items;
    const uint32_t *iorder;
    Counters *cnt;
    unsigned long long *per_anchor;  // u128 per anchor rank, or null
    unsigned long long *per_graph;   // u128 per graph of a batch, or null
    const int64_t *graph_x0;         // first anchor rank of each graph (n_graphs + 1)
    int n_graphs;
    uint32_t *wide_scratch;          // per warp: R * wmax words
    uint32_t wmax;
    int l;
};

// Per-lane work tally of the tuple kernel (the algorithmic operations: one
// AND+POPC per mask word of every tested tuple, 2^R masked POPCs per word of
// every tuple that reaches the type count).
struct Acc {
    U128 sum;
    unsigned long long tested = 0, leaves = 0, words = 0;
};

constexpr int BINOM_TBL = 256;

// Dynamic shared memory of the tuple kernel (staged masks) and its binomial
// table binom(x, l) for x <= BINOM_TBL (binom(256, 8) < 2^64).
extern __shared__ __align__(16) uint32_t sm_dyn[];
__shared__ unsigned long long s_bt[BINOM_TBL + 1];

// Views of an anchor's candidate masks: P(w, c) and D(w, c), word-major.
// MasksS: staged in the dynamic shared array (32-bit offsets, shared loads);
// MasksG: read from the candidate pool in global memory.
struct MasksS {
    uint32_t stride, W, nc;
    __device__ __forceinline__ uint32_t P(uint32_t w, uint32_t c) const {
        return sm_dyn[w * stride + c];
    }
    __device__ __forceinline__ uint32_t D(uint32_t w, uint32_t c) const {
        return sm_dyn[(W + w) * stride + c];
    }
};
struct MasksG {
    const uint32_t *base;
    uint32_t stride, W, nc;
    __device__ __forceinline__ uint32_t P(uint32_t w, uint32_t c) const {
        return base[(size_t)w * stride + c];
    }
    __device__ __forceinline__ uint32_t D(uint32_t w, uint32_t c) const {
        return base[(size_t)(W + w) * stride + c];
    }
};

// Type counts of a tuple and the binomial sum. T: the lane's common
// neighbourhood mask; idx[0..R-1]: the tuple's candidate indices.
template <int R, int WN, class MK>
__device__ __forceinline__ void leaf_narrow(const MK &m, const uint32_t (&T)[WN],
                                            const uint32_t (&idx)[R], int l, Acc &acc,
                                            unsigned *err) {
    acc.leaves++;
    acc.words += (unsigned long long)m.W << R;
    if constexpr (R <= 3) {
        uint32_t x[1 << R];
#pragma unroll
        for (int k = 0; k < (1 << R); k++) x[k] = 0;
#pragma unroll
        for (int w = 0; w < WN; w++) {
            if (w >= (int)m.W) break;
            uint32_t dd[R];
#pragma unroll
            for (int i = 0; i < R; i++) dd[i] = m.D(w, idx[i]);
#pragma unroll
            for (int k = 0; k < (1 << R); k++) {
                uint32_t msk = T[w];
#pragma unroll
                for (int i = 0; i < R; i++) msk &= ((k >> i) & 1) ? dd[i] : ~dd[i];
                x[k] += __popc(msk);
            }
        }
#pragma unroll
        for (int k = 0; k < (1 << R); k++) binom_add(acc.sum, x[k], l, err);
    } else {
        // split T by each partner's type letter, dropping parts below l
        uint32_t stk[R + 1][WN];
        int lev[R + 1];
        int sp = 0;
#pragma unroll
        for (int w = 0; w < WN; w++) stk[0][w] = T[w];
        lev[0] = 0;
        sp = 1;
        while (sp > 0) {
            sp--;
            int lv = lev[sp];
            uint32_t cur[WN];
#pragma unroll
            for (int w = 0; w < WN; w++) cur[w] = stk[sp][w];
            if (lv == R) {
                uint32_t n = 0;
#pragma unroll
                for (int w = 0; w < WN; w++) n += __popc(cur[w]);
                binom_add(acc.sum, n, l, err);
                continue;
            }
            uint32_t a0[WN], a1[WN];
            uint32_t n0 = 0, n1 = 0;
#pragma unroll
            for (int w = 0; w < WN; w++) {
                uint32_t dw = (w < (int)m.W) ? m.D(w, idx[lv]) : 0u;
                a0[w] = cur[w] & ~dw;
                a1[w] = cur[w] & dw;
                n0 += __popc(a0[w]);
                n1 += __popc(a1[w]);
            }
            if ((int)n0 >= l) {
#pragma unroll
                for (int w = 0; w < WN; w++) stk[sp][w] = a0[w];
                lev[sp] = lv + 1;
                sp++;
            }
            if ((int)n1 >= l) {
#pragma unroll
                for (int w = 0; w < WN; w++) stk[sp][w] = a1[w];
                lev[sp] = lv + 1;
                sp++;
            }
        }
    }
}

// Extend a warp-uniform prefix (mask `pre`, indices idx[0..L-2]) by every
// candidate m >= start, lanes over m.
template <int L, int R, int WN, class MK>
__device__ void expand_narrow(const MK &m, const uint32_t (&pre)[WN], uint32_t (&idx)[R],
                              uint32_t start, int l, Acc &acc, unsigned *err) {
    const int lane = threadIdx.x & 31;
    for (uint32_t mb = start; mb < m.nc; mb += 32) {
        uint32_t c = mb + lane;
        bool valid = c < m.nc;
        uint32_t T[WN];
        uint32_t n = 0;
#pragma unroll
        for (int w = 0; w < WN; w++) {
            T[w] = (valid && w < (int)m.W) ? (pre[w] & m.P(w, c)) : 0u;
            n += __popc(T[w]);
        }
        if (valid) {
            acc.tested++;
            acc.words += m.W;
        }
        if constexpr (L == R) {
            if (valid && (int)n >= l) {
                uint32_t id2[R];
#pragma unroll
                for (int i = 0; i < R; i++) id2[i] = idx[i];
                id2[R - 1] = c;
                leaf_narrow<R, WN>(m, T, id2, l, acc, err);
            }
        } else {
            bool ok = valid && (int)n >= l && (m.nc - 1 - c) >= (uint32_t)(R - L);
            uint32_t bal = __ballot_sync(FULL, ok);
            while (bal) {
                int s = __ffs(bal) - 1;
                bal &= bal - 1;
                uint32_t Ts[WN];
#pragma unroll
                for (int w = 0; w < WN; w++) Ts[w] = __shfl_sync(FULL, T[w], s);
                idx[L - 1] = mb + s;
                expand_narrow<L + 1, R, WN>(m, Ts, idx, mb + s + 1, l, acc, err);
            }
        }
    }
}

// One work unit: row i (first partner) and a chunk of 32 second partners;
// for R == 1 a chunk of 32 single partners.
template <int R, int WN, class MK>
__device__ void unit_narrow(const MK &m, uint32_t i, uint32_t jc, int l, Acc &acc,
                            unsigned *err) {
    const int lane = threadIdx.x & 31;
    if constexpr (R == 1) {
        uint32_t c = jc * 32 + lane;
        if (c < m.nc) {
            acc.tested++;
            acc.words += m.W;
            uint32_t T[WN];
            uint32_t n = 0;
#pragma unroll
            for (int w = 0; w < WN; w++) {
                T[w] = (w < (int)m.W) ? m.P(w, c) : 0u;
                n += __popc(T[w]);
            }
            if ((int)n >= l) {
                uint32_t id[1] = {c};
                leaf_narrow<1, WN>(m, T, id, l, acc, err);
            }
        }
    } else {
        uint32_t Pi[WN];
#pragma unroll
        for (int w = 0; w < WN; w++) Pi[w] = (w < (int)m.W) ? m.P(w, i) : 0u;
        uint32_t j = i + 1 + jc * 32 + lane;
        bool valid = j < m.nc;
        uint32_t T[WN];
        uint32_t n = 0;
#pragma unroll
        for (int w = 0; w < WN; w++) {
            T[w] = valid ? (Pi[w] & ((w < (int)m.W) ? m.P(w, j) : 0u)) : 0u;
            n += __popc(T[w]);
        }
        if (valid) {
            acc.tested++;
            acc.words += m.W;
        }
        if constexpr (R == 2) {
            if (valid && (int)n >= l) {
                uint32_t id[2] = {i, j};
                leaf_narrow<2, WN>(m, T, id, l, acc, err);
            }
        } else {
            bool ok = valid && (int)n >= l && (m.nc - 1 - j) >= (uint32_t)(R - 2);
            uint32_t bal = __ballot_sync(FULL, ok);
            uint32_t idx[R];
            idx[0] = i;
            while (bal) {
                int s = __ffs(bal) - 1;
                bal &= bal - 1;
                uint32_t Ts[WN];
#pragma unroll
                for (int w = 0; w < WN; w++) Ts[w] = __shfl_sync(FULL, T[w], s);
                uint32_t js = i + 1 + jc * 32 + s;
                idx[1] = js;
                expand_narrow<3, R, WN>(m, Ts, idx, js + 1, l, acc, err);
            }
        }
    }
}

// ---- wide anchors (more than 256 useful positions): masks streamed word by
// word; warp-uniform prefixes live in a per-warp scratch (level L-1 at
// pre + (L-2) * wmax).

template <int R, class MK>
__device__ __forceinline__ void leaf_wide(const MK &m, const uint32_t *pre, uint32_t c,
                                          const uint32_t (&idx)[R], int l, Acc &acc,
                                          unsigned *err) {
    acc.leaves++;
    acc.words += (unsigned long long)m.W << R;
    // T = pre AND P(., c); pre == nullptr means T = P(., c)
    if constexpr (R <= 3) {
        uint32_t x[1 << R];
#pragma unroll
        for (int k = 0; k < (1 << R); k++) x[k] = 0;
        for (uint32_t w = 0; w < m.W; w++) {
            uint32_t t = m.P(w, c);
            if (pre) t &= pre[w];
            if (!t) continue;
            uint32_t dd[R];
#pragma unroll
            for (int i = 0; i < R; i++) dd[i] = m.D(w, idx[i]);
#pragma unroll
            for (int k = 0; k < (1 << R); k++) {
                uint32_t msk = t;
#pragma unroll
                for (int i = 0; i < R; i++) msk &= ((k >> i) & 1) ? dd[i] : ~dd[i];
                x[k] += __popc(msk);
            }
        }
#pragma unroll
        for (int k = 0; k < (1 << R); k++) binom_add(acc.sum, x[k], l, err);
    } else {
        uint32_t x[1 << R];
        for (int k = 0; k < (1 << R); k++) x[k] = 0;
        for (uint32_t w = 0; w < m.W; w++) {
            uint32_t t = m.P(w, c);
            if (pre) t &= pre[w];
            while (t) {
                int b = __ffs(t) - 1;
                t &= t - 1;
                uint32_t kk = 0;
                for (int i = 0; i < R; i++) kk |= ((m.D(w, idx[i]) >> b) & 1u) << i;
                x[kk]++;
            }
        }
        for (int k = 0; k < (1 << R); k++) binom_add(acc.sum, x[k], l, err);
    }
}

template <int L, int R, class MK>
__device__ void expand_wide(const MK &m, uint32_t *scratch, uint32_t wmax,
                            uint32_t (&idx)[R], uint32_t start, int l, Acc &acc, unsigned *err) {
    const int lane = threadIdx.x & 31;
    const uint32_t *pre = scratch + (size_t)(L - 2) * wmax;  // prefix of L-1 partners
    for (uint32_t mb = start; mb < m.nc; mb += 32) {
        uint32_t c = mb + lane;
        bool valid = c < m.nc;
        uint32_t n = 0;
        if (valid) {
            acc.tested++;
            acc.words += m.W;
            for (uint32_t w = 0; w < m.W; w++) n += __popc(pre[w] & m.P(w, c));
        }
        if constexpr (L == R) {
            if (valid && (int)n >= l) {
                uint32_t id2[R];
#pragma unroll
                for (int i = 0; i < R; i++) id2[i] = idx[i];
                id2[R - 1] = c;
                leaf_wide<R>(m, pre, c, id2, l, acc, err);
            }
        } else {
            bool ok = valid && (int)n >= l && (m.nc - 1 - c) >= (uint32_t)(R - L);
            uint32_t bal = __ballot_sync(FULL, ok);
            while (bal) {
                int s = __ffs(bal) - 1;
                bal &= bal - 1;
                uint32_t cs = mb + s;
                uint32_t *nxt = scratch + (size_t)(L - 1) * wmax;
                __syncwarp();
                for (uint32_t w = lane; w < m.W; w += 32) nxt[w] = pre[w] & m.P(w, cs);
                __syncwarp();
                idx[L - 1] = cs;
                expand_wide<L + 1, R>(m, scratch, wmax, idx, cs + 1, l, acc, err);
            }
        }
    }
}

template <int R, class MK>
__device__ void unit_wide(const MK &m, uint32_t *scratch, uint32_t wmax, uint32_t i,
                          uint32_t jc, int l, Acc &acc, unsigned *err) {
    const int lane = threadIdx.x & 31;
    if constexpr (R == 1) {
        uint32_t c = jc * 32 + lane;
        if (c < m.nc) {
            acc.tested++;
            acc.words += m.W;
            uint32_t n = 0;
            for (uint32_t w = 0; w < m.W; w++) n += __popc(m.P(w, c));
            if ((int)n >= l) {
                uint32_t id[1] = {c};
                leaf_wide<1>(m, nullptr, c, id, l, acc, err);
            }
        }
    } else {
        // level-1 prefix P(., i) at scratch[0 .. W)
        __syncwarp();
        for (uint32_t w = lane; w < m.W; w += 32) scratch[w] = m.P(w, i);
        __syncwarp();
        uint32_t j = i + 1 + jc * 32 + lane;
        bool valid = j < m.nc;
        uint32_t n = 0;
        if (valid) {
            acc.tested++;
            acc.words += m.W;
            for (uint32_t w = 0; w < m.W; w++) n += __popc(scratch[w] & m.P(w, j));
        }
        if constexpr (R == 2) {
            if (valid && (int)n >= l) {
                uint32_t id[2] = {i, j};
                leaf_wide<2>(m, scratch, j, id, l, acc, err);
            }
        } else {
            bool ok = valid && (int)n >= l && (m.nc - 1 - j) >= (uint32_t)(R - 2);
            uint32_t bal = __ballot_sync(FULL, ok);
            uint32_t idx[R];
            idx[0] = i;
            while (bal) {
                int s = __ffs(bal) - 1;
                bal &= bal - 1;
                uint32_t js = i + 1 + jc * 32 + s;
                uint32_t *nxt = scratch + wmax;
                __syncwarp();
                for (uint32_t w = lane; w < m.W; w += 32) nxt[w] = scratch[w] & m.P(w, js);
                __syncwarp();
                idx[1] = js;
                expand_wide<3, R>(m, scratch, wmax, idx, js + 1, l, acc, err);
            }
        }
    }
}

// ---- type parts (R <= 3). By Lemma 1 and its converse, every v of a
// balanced biclique's other side has the same type relative to the anchor,
// so a prefix of partners is carried as its type parts: the masks of common
// neighbours sharing one type vector, kept only while they hold at least l
// bits. Extending by a partner m splits each part P into P & P_m & ~D_m and
// P & P_m & D_m; at the last partner each child adds binom(popc, l). Parts
// below l bits are dropped, which drops only zero binomials.

// Split one part y (already ANDed with P_m) by D_m and add the binomials.
template <int WN, class MK>
__device__ __forceinline__ void close_part(const MK &m, const uint32_t (&y)[WN], uint32_t c,
                                           int l, Acc &acc, unsigned *err) {
    uint32_t n = 0;
#pragma unroll
    for (int w = 0; w < WN; w++) n += __popc(y[w]);
    acc.words += m.W;
    if ((int)n < l) return;
    uint32_t x1 = 0;
#pragma unroll
    for (int w = 0; w < WN; w++)
        if (w < (int)m.W) x1 += __popc(y[w] & m.D(w, c));
    acc.words += m.W;
    acc.leaves++;
    if (n <= (uint32_t)BINOM_TBL) {
        acc.sum.add(s_bt[x1] + s_bt[n - x1]);
    } else {
        binom_add(acc.sum, x1, l, err);
        binom_add(acc.sum, n - x1, l, err);
    }
}

// Close part B against candidate c given S = P_c & ~D_c and T = P_c & D_c:
// the two children B & S and B & T add binom(., l) each (zero below l).
// Returns whether the part had at least l common neighbours with c.
template <int WN>
__device__ __forceinline__ bool close_st(const uint32_t (&B)[WN], const uint32_t (&S)[WN],
                                         const uint32_t (&T)[WN], int l, Acc &acc,
                                         unsigned *err) {
    uint32_t n0 = 0, n1 = 0;
#pragma unroll
    for (int w = 0; w < WN; w++) {
        n0 += __popc(B[w] & S[w]);
        n1 += __popc(B[w] & T[w]);
    }
    const uint32_t n = n0 + n1;
    const bool ok = (int)n >= l;
    if (__any_sync(FULL, ok) && ok) {
        if (n <= (uint32_t)BINOM_TBL) {
            acc.sum.add(s_bt[n0] + s_bt[n1]);
        } else {
            binom_add(acc.sum, n0, l, err);
            binom_add(acc.sum, n1, l, err);
        }
    }
    return ok;
}

template <int WN, class MK>
__device__ void parts_r1(const MK &m, uint32_t jc, int l, Acc &acc, unsigned *err) {
    const uint32_t c = jc * 32 + (threadIdx.x & 31);
    if (c >= m.nc) return;
    acc.tested++;
    uint32_t y[WN];
#pragma unroll
    for (int w = 0; w < WN; w++) y[w] = w < (int)m.W ? m.P(w, c) : 0u;
    close_part<WN>(m, y, c, l, acc, err);
}

// Type parts of candidate i: A0 = P_i & ~D_i (same sign), A1 = P_i & D_i.
template <int WN, class MK>
__device__ __forceinline__ uint32_t parts_of(const MK &m, uint32_t i, uint32_t (&A0)[WN],
                                             uint32_t (&A1)[WN], int l) {
    uint32_t n0 = 0, n1 = 0;
#pragma unroll
    for (int w = 0; w < WN; w++) {
        uint32_t p = w < (int)m.W ? m.P(w, i) : 0u;
        uint32_t d = w < (int)m.W ? m.D(w, i) : 0u;
        A0[w] = p & ~d;
        A1[w] = p & d;
        n0 += __popc(A0[w]);
        n1 += __popc(A1[w]);
    }
    return ((int)n0 >= l ? 1u : 0u) | ((int)n1 >= l ? 2u : 0u);
}

template <int WN, class MK>
__device__ void parts_r2(const MK &m, uint32_t i, uint32_t jc, int l, Acc &acc,
                         unsigned *err) {
    uint32_t A0[WN], A1[WN];
    const uint32_t va = parts_of<WN>(m, i, A0, A1, l);
    if (!va) return;
    const uint32_t j = i + 1 + jc * 32 + (threadIdx.x & 31);
    const bool jv = j < m.nc;
    uint32_t S[WN], T[WN];
#pragma unroll
    for (int w = 0; w < WN; w++) {
        const bool in = jv && w < (int)m.W;
        const uint32_t p = in ? m.P(w, j) : 0u, d = in ? m.D(w, j) : 0u;
        S[w] = p & ~d;
        T[w] = p & d;
    }
    uint32_t closes = 0, viable = 0;
    if (va & 1u) {
        closes++;
        viable += close_st<WN>(A0, S, T, l, acc, err);
    }
    if (va & 2u) {
        closes++;
        viable += close_st<WN>(A1, S, T, l, acc, err);
    }
    if (jv) {
        acc.tested++;
        acc.leaves += viable;
        acc.words += (unsigned long long)(closes + viable) * m.W;
    }
}

template <int WN, class MK>
__device__ void parts_r3(const MK &m, uint32_t i, uint32_t jc, int l, Acc &acc,
                         unsigned *err) {
    const int lane = threadIdx.x & 31;
    uint32_t A0[WN], A1[WN];
    const uint32_t va = parts_of<WN>(m, i, A0, A1, l);
    if (!va) return;
    const uint32_t j = i + 1 + jc * 32 + lane;
    const bool valid = j + 1 < m.nc;  // room for a third partner
    uint32_t vb = 0;
    if (valid) {
        acc.tested++;
        uint32_t n[4] = {0, 0, 0, 0};
#pragma unroll
        for (int w = 0; w < WN; w++) {
            uint32_t p = w < (int)m.W ? m.P(w, j) : 0u;
            uint32_t d = w < (int)m.W ? m.D(w, j) : 0u;
            n[0] += __popc(A0[w] & p & ~d);
            n[1] += __popc(A0[w] & p & d);
            n[2] += __popc(A1[w] & p & ~d);
            n[3] += __popc(A1[w] & p & d);
        }
        acc.words += 4 * m.W;
#pragma unroll
        for (int b = 0; b < 4; b++) vb |= ((int)n[b] >= l ? 1u : 0u) << b;
        vb &= ((va & 1u) ? 3u : 0u) | ((va & 2u) ? 12u : 0u);
    }
    uint32_t bal = __ballot_sync(FULL, vb != 0);
    while (bal) {
        const int s = __ffs(bal) - 1;
        bal &= bal - 1;
        const uint32_t js = i + 1 + jc * 32 + s;
        const uint32_t vbs = __shfl_sync(FULL, vb, s);
        uint32_t B[4][WN];
#pragma unroll
        for (int w = 0; w < WN; w++) {
            uint32_t p = w < (int)m.W ? m.P(w, js) : 0u;
            uint32_t d = w < (int)m.W ? m.D(w, js) : 0u;
            B[0][w] = A0[w] & p & ~d;
            B[1][w] = A0[w] & p & d;
            B[2][w] = A1[w] & p & ~d;
            B[3][w] = A1[w] & p & d;
        }
        uint32_t tested = 0, closes = 0, viable = 0;
        for (uint32_t mb = js + 1; mb < m.nc; mb += 32) {
            const uint32_t c = mb + lane;
            const bool cv = c < m.nc;
            uint32_t S[WN], T[WN];
#pragma unroll
            for (int w = 0; w < WN; w++) {
                const bool in = cv && w < (int)m.W;
                const uint32_t p = in ? m.P(w, c) : 0u, d = in ? m.D(w, c) : 0u;
                S[w] = p & ~d;
                T[w] = p & d;
            }
            tested += cv;
#pragma unroll
            for (int b = 0; b < 4; b++) {
                if (!((vbs >> b) & 1u)) continue;
                closes += cv;
                viable += close_st<WN>(B[b], S, T, l, acc, err);
            }
        }
        acc.tested += tested;
        acc.leaves += viable;
        acc.words += (unsigned long long)(closes + viable) * m.W;
    }
}

// ---- type parts for wide anchors (more words than the register paths
// hold). The words stream through registers: the first partner's parts are
// recomputed per word from its masks (warp-uniform loads), the lanes' own
// candidates' S = P & ~D and T = P & D likewise, and all parts are counted in
// one pass. For three partners the warp-uniform parts of the chosen pair live
// in a per-warp slot (shared memory up to SLOT_W words, else the warp's
// global scratch).

constexpr int SLOT_W = 32;  // words per part in the shared per-warp slot
__shared__ uint32_t s_slot[PB_WARPS][4 * SLOT_W];

// Adds binom(x0, l) + binom(x1, l) when x0 + x1 >= l; returns that test.
__device__ __forceinline__ bool close_x(uint32_t x0, uint32_t x1, int l, U128 &sum,
                                        unsigned *err) {
    const uint32_t n = x0 + x1;
    const bool ok = (int)n >= l;
    if (ok) {
        if (n <= (uint32_t)BINOM_TBL) {
            sum.add(s_bt[x0] + s_bt[x1]);
        } else {
            binom_add(sum, x0, l, err);
            binom_add(sum, x1, l, err);
        }
    }
    return ok;
}

// Viability of candidate i's parts (warp-cooperative): bit 0 same-sign part,
// bit 1 different-sign part, set when the part holds at least l positions.
template <class MK>
__device__ __forceinline__ uint32_t stream_parts_of(const MK &m, uint32_t i, int l) {
    const int lane = threadIdx.x & 31;
    uint32_t n0 = 0, n1 = 0;
    for (uint32_t w = lane; w < m.W; w += 32) {
        const uint32_t p = m.P(w, i), d = m.D(w, i);
        n0 += __popc(p & ~d);
        n1 += __popc(p & d);
    }
    n0 = __reduce_add_sync(FULL, n0);
    n1 = __reduce_add_sync(FULL, n1);
    return ((int)n0 >= l ? 1u : 0u) | ((int)n1 >= l ? 2u : 0u);
}

template <class MK>
__device__ void wide_r1(const MK &m, uint32_t jc, int l, Acc &acc, unsigned *err) {
    const uint32_t c = jc * 32 + (threadIdx.x & 31);
    if (c >= m.nc) return;
    uint32_t x0 = 0, x1 = 0;
    for (uint32_t w = 0; w < m.W; w++) {
        const uint32_t p = m.P(w, c), d = m.D(w, c);
        x0 += __popc(p & ~d);
        x1 += __popc(p & d);
    }
    const bool ok = close_x(x0, x1, l, acc.sum, err);
    acc.tested++;
    acc.leaves += ok;
    acc.words += (ok ? 2ull : 1ull) * m.W;
}

// Two partners (i, j): the four type counts of every pair in one pass.
template <class MK>
__device__ void wide_r2(const MK &m, uint32_t i, uint32_t jc, int l, Acc &acc, unsigned *err) {
    const uint32_t va = stream_parts_of(m, i, l);
    if (!va) return;
    const uint32_t j = i + 1 + jc * 32 + (threadIdx.x & 31);
    if (j >= m.nc) return;
    uint32_t x00 = 0, x01 = 0, x10 = 0, x11 = 0;
#pragma unroll 2
    for (uint32_t w = 0; w < m.W; w++) {
        const uint32_t pi = m.P(w, i), di = m.D(w, i);
        const uint32_t pj = m.P(w, j), dj = m.D(w, j);
        const uint32_t a0 = pi & ~di, a1 = pi & di, sj = pj & ~dj, tj = pj & dj;
        x00 += __popc(a0 & sj);
        x01 += __popc(a0 & tj);
        x10 += __popc(a1 & sj);
        x11 += __popc(a1 & tj);
    }
    uint32_t closes = 0, viable = 0;
    if (va & 1u) {
        closes++;
        viable += close_x(x00, x01, l, acc.sum, err);
    }
    if (va & 2u) {
        closes++;
        viable += close_x(x10, x11, l, acc.sum, err);
    }
    acc.tested++;
    acc.leaves += viable;
    acc.words += (unsigned long long)(closes + viable) * m.W;
}

// Third partners c > js of a pair whose NB viable parts sit in `slot`
// (NB parts of W words, part k at slot[k * stride ...]).
template <int NB, bool SHARED, class MK>
__device__ __forceinline__ void stream_third(const MK &m, const uint32_t *slot, uint32_t stride,
                                             uint32_t js, int l, Acc &acc, unsigned *err) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t tested = 0, viable = 0;
    for (uint32_t mb = js + 1; mb < m.nc; mb += 32) {
        const uint32_t c = mb + lane;
        if (c >= m.nc) break;
        uint32_t x0[NB], x1[NB];
#pragma unroll
        for (int k = 0; k < NB; k++) x0[k] = x1[k] = 0;
        for (uint32_t w = 0; w < m.W; w++) {
            const uint32_t p = m.P(w, c), d = m.D(w, c);
            const uint32_t sc = p & ~d, tc = p & d;
#pragma unroll
            for (int k = 0; k < NB; k++) {
                const uint32_t bw = SHARED ? s_slot[warp][k * stride + w] : slot[k * stride + w];
                x0[k] += __popc(bw & sc);
                x1[k] += __popc(bw & tc);
            }
        }
        tested++;
#pragma unroll
        for (int k = 0; k < NB; k++) viable += close_x(x0[k], x1[k], l, acc.sum, err);
    }
    acc.tested += tested;
    acc.leaves += viable;
    acc.words += (unsigned long long)(NB * tested + viable) * m.W;
}

// Three partners (i, j, c) for wide anchors. SHARED: the pair's parts fit the
// shared per-warp slot (W <= SLOT_W); otherwise they go to the warp scratch.
template <bool SHARED, class MK>
__device__ void wide_r3(const MK &m, uint32_t *scratch, uint32_t wmax, uint32_t i, uint32_t jc,
                        int l, Acc &acc, unsigned *err) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t va = stream_parts_of(m, i, l);
    if (!va) return;
    const uint32_t j = i + 1 + jc * 32 + lane;
    const bool valid = j + 1 < m.nc;  // room for a third partner
    uint32_t vb = 0;
    if (valid) {
        uint32_t n[4] = {0, 0, 0, 0};
        for (uint32_t w = 0; w < m.W; w++) {
            const uint32_t pi = m.P(w, i), di = m.D(w, i);
            const uint32_t pj = m.P(w, j), dj = m.D(w, j);
            const uint32_t a0 = pi & ~di, a1 = pi & di, sj = pj & ~dj, tj = pj & dj;
            n[0] += __popc(a0 & sj);
            n[1] += __popc(a0 & tj);
            n[2] += __popc(a1 & sj);
            n[3] += __popc(a1 & tj);
        }
        acc.tested++;
        acc.words += 4ull * m.W;
#pragma unroll
        for (int b = 0; b < 4; b++) vb |= ((int)n[b] >= l ? 1u : 0u) << b;
        vb &= ((va & 1u) ? 3u : 0u) | ((va & 2u) ? 12u : 0u);
    }
    uint32_t *slot = SHARED ? s_slot[warp] : scratch;
    const uint32_t stride = SHARED ? (uint32_t)SLOT_W : wmax;
    uint32_t bal = __ballot_sync(FULL, vb != 0);
    while (bal) {
        const int sl = __ffs(bal) - 1;
        bal &= bal - 1;
        const uint32_t js = i + 1 + jc * 32 + sl;
        const uint32_t vbs = __shfl_sync(FULL, vb, sl);
        const int nb = __popc(vbs);
        // the viable parts of (i, js), compacted into slots 0 .. nb-1
        __syncwarp();
        for (uint32_t w = lane; w < m.W; w += 32) {
            const uint32_t pi = m.P(w, i), di = m.D(w, i);
            const uint32_t pj = m.P(w, js), dj = m.D(w, js);
            const uint32_t a0 = pi & ~di, a1 = pi & di, sj = pj & ~dj, tj = pj & dj;
            const uint32_t part[4] = {a0 & sj, a0 & tj, a1 & sj, a1 & tj};
            int k = 0;
#pragma unroll
            for (int b = 0; b < 4; b++)
                if ((vbs >> b) & 1u) slot[(k++) * stride + w] = part[b];
        }
        __syncwarp();
        switch (nb) {
            case 1: stream_third<1, SHARED>(m, slot, stride, js, l, acc, err); break;
            case 2: stream_third<2, SHARED>(m, slot, stride, js, l, acc, err); break;
            case 3: stream_third<3, SHARED>(m, slot, stride, js, l, acc, err); break;
            default: stream_third<4, SHARED>(m, slot, stride, js, l, acc, err); break;
        }
        __syncwarp();
    }
}

// ---- position side. For an anchor with few useful positions and many
// candidates the same sum is taken over position subsets instead of
// candidate subsets: expanding each binom(x, l) as the number of l-subsets Q
// of a type class gives
//   sum over R-subsets A, types k of binom(x[k], l)
//     = sum over l-subsets Q of positions of binom(N_Q, R),
// where N_Q counts the candidates w with Q inside the same-sign part
// (P_w & ~D_w) or inside the different-sign part (P_w & D_w) of L[w] (the two
// parts are disjoint, so w counts at most once). CM0[q] / CM1[q] are the
// candidates whose same-sign / different-sign part holds position q (rows of
// wc candidate words at an odd stride wcp, so lanes reading different rows hit
// different banks). A warp walks Q depth first; at every node its lanes scan
// 32 children q at once, each lane intersecting the node's prefix (held one
// word per lane and broadcast by shuffles) with row q.

template <int R>
__device__ __forceinline__ void binom_add_r(U128 &acc, unsigned long long x, unsigned *err) {
    if (x < (unsigned long long)R) return;
    if constexpr (R == 1) {
        acc.add(x);
    } else {
        if (x > c_binom64_max[R]) {
            if (acc.add(binom_slow(x, R, err))) atomicOr(err, CERR_OVERFLOW);
            return;
        }
        acc.add(binom_u64<R>(x));
    }
}

// binom(x, R) for x <= BINOM_TBL, R = the anchor's tuple partners (shared).
__shared__ unsigned long long s_btR[BINOM_TBL + 1];

// A position-side node's prefix masks, word w of each at lane w % 32, slot
// w / 32 (passed by value so that it stays in registers across calls).
template <int WPL>
struct Pfx {
    uint32_t m0[WPL], m1[WPL];
};

// Partial result of a subtree of the position-side walk.
struct PosOut {
    U128 sum;
    uint32_t tested = 0, leaves = 0;
};

// Children q in [qs, qe] of a node at depth LEV - 1 with prefix M; lanes over
// q. At depth l a child is a leaf and adds binom(N_Q, R); otherwise children
// with N >= R are expanded one at a time.
template <int R, int WPL, int LEV>
__device__ __noinline__ PosOut pos_scan(uint32_t dp, uint32_t wc, uint32_t wcp, Pfx<WPL> M,
                                        uint32_t qs, uint32_t qe, int l, unsigned *err) {
    const int lane = threadIdx.x & 31;
    PosOut out;
    for (uint32_t qb = qs; qb <= qe; qb += 32) {
        const uint32_t q = qb + lane;
        const bool valid = q <= qe;
        const uint32_t o0 = (valid ? q : qs) * wcp, o1 = (dp + (valid ? q : qs)) * wcp;
        uint32_t n = 0;
#pragma unroll
        for (int k = 0; k < WPL; k++) {
            if (32u * k >= wc) break;  // WPL = 4 also serves 65..96 words
            const uint32_t wend = wc - 32u * k < 32u ? wc - 32u * k : 32u;
            for (uint32_t sl = 0; sl < wend; sl++) {
                const uint32_t m0 = __shfl_sync(FULL, M.m0[k], sl), m1 = __shfl_sync(FULL, M.m1[k], sl);
                const uint32_t w = 32u * k + sl;
                n += __popc(m0 & sm_dyn[o0 + w]) + __popc(m1 & sm_dyn[o1 + w]);
            }
        }
        out.tested += valid;
        if (LEV == l) {
            if (valid && n >= (uint32_t)R) {
                out.leaves++;
                if (n <= (uint32_t)BINOM_TBL) out.sum.add(s_btR[n]);
                else binom_add_r<R>(out.sum, n, err);
            }
        } else if constexpr (LEV < 8) {
            const uint32_t qe2 = dp - 1 - (uint32_t)(l - LEV - 1);  // room for the rest of Q
            uint32_t bal = __ballot_sync(FULL, valid && n >= (uint32_t)R);
            while (bal) {
                const int sl = __ffs(bal) - 1;
                bal &= bal - 1;
                const uint32_t qc = qb + sl;
                if (qc + 1 > qe2) continue;
                Pfx<WPL> X;
#pragma unroll
                for (int k = 0; k < WPL; k++) {
                    const uint32_t w = lane + 32u * k;
                    X.m0[k] = w < wc ? (M.m0[k] & sm_dyn[qc * wcp + w]) : 0u;
                    X.m1[k] = w < wc ? (M.m1[k] & sm_dyn[(dp + qc) * wcp + w]) : 0u;
                }
                const PosOut c = pos_scan<R, WPL, LEV + 1>(dp, wc, wcp, X, qc + 1, qe2, l, err);
                if (out.sum.add(c.sum)) atomicOr(err, CERR_OVERFLOW);
                out.tested += c.tested;
                out.leaves += c.leaves;
            }
        }
    }
    return out;
}

// A position-side unit: first position q1 and a chunk of 32 second positions.
template <int R, int WPL>
__device__ void pos_unit_scan(uint32_t dp, uint32_t wc, uint32_t wcp, uint32_t q1, uint32_t chunk,
                              int l, Acc &acc, unsigned *err) {
    const int lane = threadIdx.x & 31;
    Pfx<WPL> M;
    uint32_t n = 0;
#pragma unroll
    for (int k = 0; k < WPL; k++) {
        const uint32_t w = lane + 32u * k;
        M.m0[k] = w < wc ? sm_dyn[q1 * wcp + w] : 0u;
        M.m1[k] = w < wc ? sm_dyn[(dp + q1) * wcp + w] : 0u;
        n += __popc(M.m0[k]) + __popc(M.m1[k]);
    }
    n = __reduce_add_sync(FULL, n);
    if (n < (uint32_t)R) return;  // no Q through q1 has R candidates
    const uint32_t qe2 = dp - 1 - (uint32_t)(l - 2);
    const uint32_t qs = q1 + 1 + 32u * chunk;
    const uint32_t qe = qs + 31 < qe2 ? qs + 31 : qe2;
    if (qs > qe) return;
    const PosOut o = pos_scan<R, WPL, 2>(dp, wc, wcp, M, qs, qe, l, err);
    if (acc.sum.add(o.sum)) atomicOr(err, CERR_OVERFLOW);
    acc.tested += o.tested;
    acc.leaves += o.leaves;
    acc.words += 2ull * wc * o.tested;
}

// Second-position chunks of first position q1 (l-subsets need q2 <= dp + 1 - l).
__device__ __forceinline__ uint32_t pos_chunks(uint32_t dp, uint32_t q1, int l) {
    return (dp + 1 - (uint32_t)l - q1 + 31) / 32;
}

// ---- two partners with the masks in global memory (anchors too large to
// stage): blocks of BLK_I first partners, whose S / T words a warp keeps in
// its shared region, against 32 second partners (one per lane) whose words
// are loaded once per block instead of once per first partner.

constexpr int BLK_I = 8;
constexpr uint32_t BLK_MAX_W = PB_SMEM_WORDS / PB_WARPS / (2 * BLK_I);  // words per mask

// Tally of one block unit.
struct BlkOut {
    U128 sum;
    uint32_t tested = 0, closes = 0, viable = 0;
};

__device__ __noinline__ BlkOut block_r2(MasksG m, uint32_t *wsm, uint32_t ib, uint32_t nrows,
                                        uint32_t jc, int l, unsigned *err) {
    BlkOut out;
    const int lane = threadIdx.x & 31;
    const uint32_t W = m.W;
    // stage S = P & ~D, T = P & D of rows ib .. ib + nrows - 1; viability bits
    __syncwarp();
    for (uint32_t t = lane; t < nrows * W; t += 32) {
        const uint32_t k = t / W, w = t - k * W;
        const uint32_t p = m.P(w, ib + k), d = m.D(w, ib + k);
        wsm[(2 * k) * W + w] = p & ~d;
        wsm[(2 * k + 1) * W + w] = p & d;
    }
    __syncwarp();
    uint32_t va = 0;  // bit 2k: row k's same-sign part viable, bit 2k+1: different-sign
    for (uint32_t k = 0; k < nrows; k++) {
        uint32_t n0 = 0, n1 = 0;
        for (uint32_t w = lane; w < W; w += 32) {
            n0 += __popc(wsm[(2 * k) * W + w]);
            n1 += __popc(wsm[(2 * k + 1) * W + w]);
        }
        n0 = __reduce_add_sync(FULL, n0);
        n1 = __reduce_add_sync(FULL, n1);
        va |= ((int)n0 >= l ? 1u : 0u) << (2 * k);
        va |= ((int)n1 >= l ? 1u : 0u) << (2 * k + 1);
    }
    if (!va) return out;
    const uint32_t j = ib + 1 + jc * 32 + lane;
    if (j >= m.nc) return out;
    uint32_t x[BLK_I][4];
#pragma unroll
    for (int k = 0; k < BLK_I; k++) x[k][0] = x[k][1] = x[k][2] = x[k][3] = 0;
    for (uint32_t w = 0; w < W; w++) {
        const uint32_t p = m.P(w, j), d = m.D(w, j);
        const uint32_t sj = p & ~d, tj = p & d;
#pragma unroll
        for (int k = 0; k < BLK_I; k++) {
            if ((uint32_t)k >= nrows) break;
            const uint32_t a0 = wsm[(2 * k) * W + w], a1 = wsm[(2 * k + 1) * W + w];
            x[k][0] += __popc(a0 & sj);
            x[k][1] += __popc(a0 & tj);
            x[k][2] += __popc(a1 & sj);
            x[k][3] += __popc(a1 & tj);
        }
    }
#pragma unroll
    for (int k = 0; k < BLK_I; k++) {
        if ((uint32_t)k >= nrows || j <= ib + k) break;  // pairs i < j only
        out.tested++;
        if ((va >> (2 * k)) & 1u) {
            out.closes++;
            out.viable += close_x(x[k][0], x[k][1], l, out.sum, err);
        }
        if ((va >> (2 * k + 1)) & 1u) {
            out.closes++;
            out.viable += close_x(x[k][2], x[k][3], l, out.sum, err);
        }
    }
    return out;
}

// Units of a two-partner item with global masks: blocks of BLK_I rows and
// chunks of 32 second partners after the block's first row.
__device__ __forceinline__ void block_units(const MasksG &m, const Item &it, int l, Acc &acc,
                                            unsigned *err, uint32_t *s_unit, uint32_t *s_total,
                                            uint32_t *s_rowpre) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t nc = m.nc;
    uint32_t *wsm = sm_dyn + (size_t)warp * (2 * BLK_I) * m.W;
    const bool split = it.u1 != 0;
    const uint32_t nblk = split ? 1u : (it.i1 - it.i0 + BLK_I - 1) / BLK_I;
    if (tid == 0) {
        *s_unit = 0;
        if (split) {
            *s_total = it.u1 - it.u0;
        } else {
            uint32_t acc_u = 0;
            for (uint32_t b = 0; b < nblk; b++) {
                s_rowpre[b] = acc_u;
                acc_u += (nc - 1 - (it.i0 + b * BLK_I) + 31) / 32;
            }
            s_rowpre[nblk] = acc_u;
            *s_total = acc_u;
        }
    }
    __syncthreads();
    const uint32_t total = *s_total;
    for (;;) {
        uint32_t u = 0;
        if (lane == 0) u = atomicAdd(s_unit, 1u);
        u = __shfl_sync(FULL, u, 0);
        if (u >= total) break;
        BlkOut o;
        if (split) {
            o = block_r2(m, wsm, it.i0, 1, it.u0 + u, l, err);
        } else {
            uint32_t lo = 0, hi = nblk;  // largest b with rowpre[b] <= u
            while (hi - lo > 1) {
                uint32_t mid = (lo + hi) >> 1;
                if (s_rowpre[mid] <= u) lo = mid; else hi = mid;
            }
            const uint32_t ib = it.i0 + lo * BLK_I;
            const uint32_t nrows = it.i1 - ib < (uint32_t)BLK_I ? it.i1 - ib : (uint32_t)BLK_I;
            o = block_r2(m, wsm, ib, nrows, u - s_rowpre[lo], l, err);
        }
        if (acc.sum.add(o.sum)) atomicOr(err, CERR_OVERFLOW);
        acc.tested += o.tested;
        acc.leaves += o.viable;
        acc.words += (unsigned long long)(o.closes + o.viable) * m.W;
    }
}

// Candidate-side work units of one item (rows i of first partners, chunks of
// 32 second partners), taken by the CTA's warps from a shared counter.
template <int R, class MK>
__device__ __forceinline__ void cand_units(const MK &m, const Item &it, uint32_t *scratch,
                                           uint32_t wmax, int l, Acc &acc, unsigned *err,
                                           uint32_t *s_unit, uint32_t *s_total,
                                           uint32_t *s_rowpre) {
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t nc = m.nc;
    const uint32_t W = m.W;
    // unit layout
    const bool split = it.u1 != 0;
    if (tid == 0) {
        (*s_unit) = 0;
        if (split) {
            (*s_total) = it.u1 - it.u0;
        } else {
            uint32_t acc = 0;
            for (uint32_t i = it.i0; i < it.i1; i++) {
                s_rowpre[i - it.i0] = acc;
                acc += (nc - 1 - i + 31) / 32;
            }
            s_rowpre[it.i1 - it.i0] = acc;
            (*s_total) = acc;
        }
    }
    __syncthreads();
    const uint32_t total = (*s_total);
    for (;;) {
        uint32_t u = 0;
        if (lane == 0) u = atomicAdd(s_unit, 1u);
        u = __shfl_sync(FULL, u, 0);
        if (u >= total) break;
        uint32_t i, jc;
        if (split) {
            i = it.i0;
            jc = it.u0 + u;
        } else {
            uint32_t lo = 0, hi = it.i1 - it.i0;  // largest k with rowpre[k] <= u
            while (hi - lo > 1) {
                uint32_t mid = (lo + hi) >> 1;
                if (s_rowpre[mid] <= u) lo = mid; else hi = mid;
            }
            i = it.i0 + lo;
            jc = u - s_rowpre[lo];
        }
        if constexpr (R == 1) {
            if (W <= 1) parts_r1<1>(m, jc, l, acc, err);
            else if (W <= 2) parts_r1<2>(m, jc, l, acc, err);
            else if (W <= 4) parts_r1<4>(m, jc, l, acc, err);
            else if (W <= 8) parts_r1<8>(m, jc, l, acc, err);
            else wide_r1(m, jc, l, acc, err);
        } else if constexpr (R == 2) {
            if (W <= 1) parts_r2<1>(m, i, jc, l, acc, err);
            else if (W <= 2) parts_r2<2>(m, i, jc, l, acc, err);
            else if (W <= 4) parts_r2<4>(m, i, jc, l, acc, err);
            else if (W <= 8) parts_r2<8>(m, i, jc, l, acc, err);
            else wide_r2(m, i, jc, l, acc, err);
        } else if constexpr (R == 3) {
            if (W <= 1) parts_r3<1>(m, i, jc, l, acc, err);
            else if (W <= 2) parts_r3<2>(m, i, jc, l, acc, err);
            else if (W <= 4) parts_r3<4>(m, i, jc, l, acc, err);
            else if (W <= (uint32_t)SLOT_W) wide_r3<true>(m, scratch, wmax, i, jc, l, acc, err);
            else wide_r3<false>(m, scratch, wmax, i, jc, l, acc, err);
        } else {
            if (W <= 1) unit_narrow<R, 1>(m, i, jc, l, acc, err);
            else if (W <= 2) unit_narrow<R, 2>(m, i, jc, l, acc, err);
            else if (W <= 4) unit_narrow<R, 4>(m, i, jc, l, acc, err);
            else if (W <= 8) unit_narrow<R, 8>(m, i, jc, l, acc, err);
            else unit_wide<R>(m, scratch, wmax, i, jc, l, acc, err);
        }
    }
}

template <int R>
__global__ void __launch_bounds__(PB_THREADS, 2) k_tuples(TupleArgs a) {
    __shared__ int s_item;
    __shared__ uint32_t s_unit, s_total;
    __shared__ uint32_t s_rowpre[ROWS_MAX + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned *err = &a.cnt->err;
    for (int x = tid; x <= BINOM_TBL; x += PB_THREADS) {
        unsigned long long v = 0;
        if (x >= a.l) {
            v = 1;
            for (int i = 1; i <= a.l; i++) v = v * (unsigned long long)(x - a.l + i) / (unsigned long long)i;
        }
        s_bt[x] = v;
        unsigned long long vr = 0;
        if (x >= R) {
            vr = 1;
            for (int i = 1; i <= R; i++) vr = vr * (unsigned long long)(x - R + i) / (unsigned long long)i;
        }
        s_btR[x] = vr;
    }
    __syncthreads();
    uint32_t *scratch =
        a.wide_scratch ? a.wide_scratch + ((size_t)blockIdx.x * PB_WARPS + warp) * SCRATCH_SLOTS * a.wmax
                       : nullptr;
    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(&a.cnt->head_b, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= (int)a.cnt->n_items) break;
        const Item it = a.items[a.iorder[item]];
        const uint32_t r = it.anchor;
        const uint32_t nc = a.ncand[r];
        const uint32_t W = (a.dprime[r] + 31) / 32;
        const uint32_t rsv = a.rsv_c[r];
        const uint32_t *region = a.pool + a.pool_off[r];
        Acc acc;
        if (it.u1 == POS_ITEM) {
            // position side: CM0 / CM1 (2 * dp rows of wc words, stride wcp) in shared memory
            const uint32_t dp = a.dprime[r];
            const uint32_t wc = (nc + 31) / 32, wcp = wc | 1u;
            for (uint32_t t = tid; t < 2 * dp * wcp; t += PB_THREADS) sm_dyn[t] = 0;
            __syncthreads();
            for (uint32_t c = tid; c < nc; c += PB_THREADS) {
                const uint32_t cb = 1u << (c & 31), cw = c >> 5;
                for (uint32_t w = 0; w < W; w++) {
                    uint32_t pw = region[(size_t)w * rsv + c];
                    const uint32_t dw = region[(size_t)(W + w) * rsv + c];
                    while (pw) {
                        const int b = __ffs(pw) - 1;
                        pw &= pw - 1;
                        const uint32_t q = 32 * w + b;
                        const uint32_t part = (dw >> b) & 1u;
                        atomicOr(&sm_dyn[(part * dp + q) * wcp + cw], cb);
                    }
                }
            }
            // units: first position q1 and a chunk of 32 second positions
            if (tid == 0) {
                uint32_t acc_u = 0;
                for (uint32_t q = it.i0; q < it.i1; q++) {
                    s_rowpre[q - it.i0] = acc_u;
                    acc_u += pos_chunks(dp, q, a.l);
                }
                s_rowpre[it.i1 - it.i0] = acc_u;
                s_total = acc_u;
                s_unit = 0;
            }
            __syncthreads();
            const uint32_t total = s_total;
            for (;;) {
                uint32_t u = 0;
                if (lane == 0) u = atomicAdd(&s_unit, 1u);
                u = __shfl_sync(FULL, u, 0);
                if (u >= total) break;
                uint32_t lo = 0, hi = it.i1 - it.i0;
                while (hi - lo > 1) {
                    uint32_t mid = (lo + hi) >> 1;
                    if (s_rowpre[mid] <= u) lo = mid; else hi = mid;
                }
                const uint32_t q1 = it.i0 + lo;
                const uint32_t chunk = u - s_rowpre[lo];
                if (wc <= 32) pos_unit_scan<R, 1>(dp, wc, wcp, q1, chunk, a.l, acc, err);
                else if (wc <= 64) pos_unit_scan<R, 2>(dp, wc, wcp, q1, chunk, a.l, acc, err);
                else pos_unit_scan<R, 4>(dp, wc, wcp, q1, chunk, a.l, acc, err);
            }
        } else if (2ull * W * nc <= (unsigned long long)PB_SMEM_WORDS) {
            // candidate side, masks staged in shared memory
            for (uint32_t t = tid; t < 2 * W * nc; t += PB_THREADS) {
                uint32_t wd = t / nc, c = t % nc;
                sm_dyn[t] = region[(size_t)wd * rsv + c];
            }
            MasksS ms;
            ms.W = W;
            ms.nc = nc;
            ms.stride = nc;
            cand_units<R>(ms, it, scratch, a.wmax, a.l, acc, err, &s_unit, &s_total, s_rowpre);
        } else {
            // candidate side, masks read from the pool
            MasksG mg;
            mg.base = region;
            mg.stride = rsv;
            mg.W = W;
            mg.nc = nc;
            bool blocked = false;
            if constexpr (R == 2) {
                if (W > 8 && W <= BLK_MAX_W) {
                    block_units(mg, it, a.l, acc, err, &s_unit, &s_total, s_rowpre);
                    blocked = true;
                }
            }
            if (!blocked)
                cand_units<R>(mg, it, scratch, a.wmax, a.l, acc, err, &s_unit, &s_total, s_rowpre);
        }
        U128 ws = warp_sum_u128(acc.sum, err);
        if (lane == 0 && (ws.lo | ws.hi)) {
            // a batch's union total is not a count (its graphs' totals are)
            atomic_add_u128(a.cnt->total, ws.lo, ws.hi, a.per_graph ? nullptr : err);
            if (a.per_anchor) atomic_add_u128(a.per_anchor + 2 * (size_t)r, ws.lo, ws.hi, err);
            if (a.per_graph) {
                int lo = 0, hi = a.n_graphs;  // largest g with graph_x0[g] <= r
                while (hi - lo > 1) {
                    int mid = (lo + hi) >> 1;
                    if (a.graph_x0[mid] <= (int64_t)r) lo = mid; else hi = mid;
                }
                atomic_add_u128(a.per_graph + 2 * (size_t)lo, ws.lo, ws.hi, err);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc.tested += __shfl_xor_sync(FULL, acc.tested, o);
            acc.leaves += __shfl_xor_sync(FULL, acc.leaves, o);
            acc.words += __shfl_xor_sync(FULL, acc.words, o);
        }
        if (lane == 0 && acc.tested) {
            atomicAdd(&a.cnt->tested, acc.tested);
            atomicAdd(&a.cnt->leaves, acc.leaves);
            atomicAdd(&a.cnt->popc_words, acc.words);
        }
        __syncthreads();
    }
}

}  // namespace

// ------------------------------------------------------------------ host side

namespace {

// Relative cost of one position-side prefix node (per candidate word per
// lane) against one candidate-side tuple word; measured on GB300.
constexpr unsigned long long kPosNodeCost = 3;
// Default tuple work items per resident warp of a full launch.
constexpr unsigned long long kSplitPerWarp = 4;
// Two-partner anchors with at least this many mask words and candidates take
// the tensor-core pair step.
constexpr uint32_t kTcMinWords = 2;
constexpr uint32_t kTcMinCandidates = 128;

// Largest x with binom(x, l) computable in 64 bits by the multiplicative
// formula: every partial product binom(x-l+i, i) * i must stay below 2^64.
unsigned long long binom64_limit(int l) {
    auto fits = [l](unsigned long long x) {
        unsigned __int128 r = 1;
        for (int i = 1; i <= l; i++) {
            unsigned __int128 prod = r * (unsigned __int128)(x - l + i);
            if (prod >> 64) return false;
            r = prod / i;
        }
        return true;
    };
    unsigned long long lo = (unsigned long long)l, hi = 1ull << 40;
    while (lo < hi) {
        unsigned long long mid = lo + (hi - lo + 1) / 2;
        if (fits(mid)) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int R>
void set_tuple_attr() {
    SBC_CUDA(cudaFuncSetAttribute(k_tuples<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)PB_SMEM));
}

// Opt every large-shared-memory kernel in, and load the binomial limits,
// once per device.
void ensure_kernel_attrs() {
    static std::mutex mu;
    static bool done[64] = {};
    std::lock_guard<std::mutex> lock(mu);
    int dev = 0;
    SBC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(SBC_E_UNSUPPORTED, "device ordinal %d out of range", dev);
    if (done[dev]) return;
    // Counts allocate and free their buffers (plans, candidate pools, the
    // tensor-core Z arena) on the stream from the device's default memory
    // pool; let the pool keep up to 4 GiB of freed memory mapped between
    // counts instead of returning it at every synchronisation.
    {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = 4ull << 30, cur = 0;
            if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur) == cudaSuccess &&
                cur < keep)
                SBC_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        }
        cudaGetLastError();
    }
    unsigned long long lim[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 2; i <= 8; i++) lim[i] = binom64_limit(i);
    SBC_CUDA(cudaMemcpyToSymbol(c_binom64_max, lim, sizeof(lim)));
    SBC_CUDA(cudaFuncSetAttribute(k_twohop_small<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PS_SMEM));
    SBC_CUDA(cudaFuncSetAttribute(k_twohop_small<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PS_SMEM));
    SBC_CUDA(cudaFuncSetAttribute(k_twohop_large<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PL_SMEM));
    SBC_CUDA(cudaFuncSetAttribute(k_twohop_large<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PL_SMEM));
    tc_ensure_attrs();
    set_tuple_attr<1>();
    set_tuple_attr<2>();
    set_tuple_attr<3>();
    set_tuple_attr<4>();
    set_tuple_attr<5>();
    set_tuple_attr<6>();
    set_tuple_attr<7>();
    done[dev] = true;
}

template <int R>
void launch_tuples(int grid, cudaStream_t s, const TupleArgs &a) {
    k_tuples<R><<<grid, PB_THREADS, PB_SMEM, s>>>(a);
    SBC_LAUNCHED();
}

int blocks_per_sm(const void *fn, int threads, size_t smem) {
    int n = 0;
    SBC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem));
    return n < 1 ? 1 : n;
}


}  // namespace

struct EventTimer {
    cudaEvent_t e[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    bool on;
    explicit EventTimer(bool enable) : on(enable) {
        if (on)
            for (auto &x : e) SBC_CUDA(cudaEventCreate(&x));
    }
    void mark(int i, cudaStream_t s) {
        if (on) SBC_CUDA(cudaEventRecord(e[i], s));
    }
    float ms(int a, int b) {
        float t = 0;
        if (on) SBC_CUDA(cudaEventElapsedTime(&t, e[a], e[b]));
        return t;
    }
    ~EventTimer() {
        for (auto &x : e)
            if (x) cudaEventDestroy(x);
    }
};

struct CountRun {
    const Orient *o = nullptr;
    int64_t nnz = 0, nX = 0;
    CountSpec spec;
    int R = 0;
    cudaStream_t s = nullptr;
    DevBuf<Counters> cnt;
    DevBuf<uint32_t> A_bit, dprime, rsv_c, skey, sval, tk, tv, ncand, npaper, pool, ikey, ival, t1b,
        t2b, scratch;
    DevBuf<unsigned long long> e_use, e_all, bucket, per;
    DevBuf<int64_t> pool_off, dtot, item_off, cum_dev;
    DevBuf<Item> items;
    DevBuf<uint32_t> tc_list;
    DevBuf<unsigned char> zbuf;     // Z arena of the tensor-core pair step
    std::vector<TcPlan> tc_plans;   // per anchor group
    TwohopArgs ta;
    TupleArgs tu;
    int ga = 0, gs = 0, gt = 0;
    int64_t n_items = 0;
    unsigned h_items = 0;
    Counters hc;
    CountResult res;

    // Launches that execute a planned count (no host synchronisation, no
    // allocation): usable under stream capture. Valid when the plan has at
    // most one anchor group.
    void launch_count() {
        SBC_CUDA(cudaMemsetAsync(&cnt.ptr->run_begin, 0,
                                 sizeof(Counters) - offsetof(Counters, run_begin), s));
        if (per.ptr) SBC_CUDA(cudaMemsetAsync(per.ptr, 0, per.bytes(), s));
        if (spec.per_graph) SBC_CUDA(cudaMemsetAsync(spec.per_graph, 0, 16 * (size_t)spec.n_graphs, s));
        if (groups.empty()) return;
        zero_pool(0);
        launch_twohop((unsigned)groups[0].first, (unsigned)groups[0].second);
        if (gt > 0) launch_tuple_kernel();
        launch_tc(0);
    }

    // Tensor-core pair step of group `grp` (expansion and pair kernels of each
    // of its chunks).
    void launch_tc(size_t grp) {
        if (grp >= tc_plans.size() || tc_plans[grp].anchors == 0) return;
        TcArgs ta2;
        ta2.pool = pool.ptr;
        ta2.l = spec.l;
        ta2.total = cnt.ptr->total;
        ta2.per_anchor = per.ptr;
        ta2.per_graph = spec.per_graph;
        ta2.graph_x0 = spec.graph_x0;
        ta2.n_graphs = spec.n_graphs;
        ta2.err = &cnt.ptr->err;
        ta2.big64 = binom64_limit(spec.l);
        tc_launch(tc_plans[grp], ta2, zbuf.ptr, s);
    }

    // Bytes of Z one tensor-core chunk may take.
    int64_t tc_budget_bytes() const {
        size_t fr = 0, tot = 0;
        SBC_CUDA(cudaMemGetInfo(&fr, &tot));
        int64_t b = (int64_t)(fr / 8);
        return std::max<int64_t>(256ll << 20, std::min<int64_t>(b, 1ll << 30));
    }

    // Events around the 2-hop and tuple launches of each group (pairs).
    std::vector<cudaEvent_t> ev_twohop, ev_tuples;
    cudaEvent_t new_event(std::vector<cudaEvent_t> &v) {
        cudaEvent_t e = nullptr;
        SBC_CUDA(cudaEventCreate(&e));
        v.push_back(e);
        return e;
    }
    void drop_events() {
        for (cudaEvent_t e : ev_twohop) cudaEventDestroy(e);
        for (cudaEvent_t e : ev_tuples) cudaEventDestroy(e);
        for (cudaEvent_t e : ev_tc) cudaEventDestroy(e);
        ev_twohop.clear();
        ev_tuples.clear();
        ev_tc.clear();
    }
    static float pairs_ms(const std::vector<cudaEvent_t> &v) {
        float sum = 0;
        for (size_t i = 0; i + 1 < v.size(); i += 2) {
            float t = 0;
            SBC_CUDA(cudaEventElapsedTime(&t, v[i], v[i + 1]));
            sum += t;
        }
        return sum;
    }
    ~CountRun() { drop_events(); }

    // Device words the candidate pool may take at once.
    int64_t pool_budget_words() const {
        if (const char *e = getenv("SBC_POOL_BUDGET_KB")) {  // tuning / testing override
            long long v = atoll(e);
            if (v > 0) return (int64_t)v * 256;
        }
        // the fixed scratch of the no-allocation entry point frees only its
        // top allocation: one group there
        if (thread_arena_active()) return INT64_MAX / 8;
        size_t fr = 0, tot = 0;
        SBC_CUDA(cudaMemGetInfo(&fr, &tot));
        return (int64_t)(fr / 4 / 4);
    }

    // The 2-hop kernels build candidate masks with atomicOr into a pool that
    // is zero on entry (the CTA kernel also clears what it stages or redoes).
    void zero_pool(size_t grp) {
        const int64_t words = cum[groups[grp].second] - cum[groups[grp].first];
        if (words > 0) SBC_CUDA(cudaMemsetAsync(pool.ptr, 0, (size_t)words * 4, s));
    }

    void launch_twohop(unsigned a, unsigned b) {
        ta.large_begin = a;
        ta.large_end = b < hc.n_big ? b : hc.n_big;
        ta.small_begin = a > hc.n_big ? a : hc.n_big;
        ta.small_end = b;
        if (ga > 0 && ta.large_end > ta.large_begin) {
            int g = ga;
            if ((unsigned)g > ta.large_end - ta.large_begin) g = (int)(ta.large_end - ta.large_begin);
            if (spec.paper) k_twohop_large<true><<<g, PL_THREADS, PL_SMEM, s>>>(ta);
            else k_twohop_large<false><<<g, PL_THREADS, PL_SMEM, s>>>(ta);
            SBC_LAUNCHED();
            g_launches++;
        }
        if (gs > 0 && ta.small_end > ta.small_begin) {
            int g = gs;
            int64_t need = ((int64_t)ta.small_end - ta.small_begin + PS_WARPS - 1) / PS_WARPS;
            if ((int64_t)g > need) g = (int)need;
            if (spec.paper) k_twohop_small<true><<<g, PS_THREADS, PS_SMEM, s>>>(ta);
            else k_twohop_small<false><<<g, PS_THREADS, PS_SMEM, s>>>(ta);
            SBC_LAUNCHED();
            g_launches++;
        }
    }

    void launch_tuple_kernel() {
        switch (R) {
            case 1: launch_tuples<1>(gt, s, tu); break;
            case 2: launch_tuples<2>(gt, s, tu); break;
            case 3: launch_tuples<3>(gt, s, tu); break;
            case 4: launch_tuples<4>(gt, s, tu); break;
            case 5: launch_tuples<5>(gt, s, tu); break;
            case 6: launch_tuples<6>(gt, s, tu); break;
            default: launch_tuples<7>(gt, s, tu); break;
        }
        g_launches++;
    }

    std::vector<std::pair<int64_t, int64_t>> groups;  // ranges of the sorted anchors
    std::vector<int64_t> cum;  // pool words before each sorted anchor
    float tw_tail_ms = 0;      // largest finish spread of the CTA-wide 2-hop kernel's CTAs

    // Finish spread of the CTA-wide 2-hop launch of the last group (counters in hc).
    float group_tail_ms() const {
        return hc.tw_fin_max ? (float)((double)(hc.tw_fin_max - ~hc.tw_fin_min_n) * 1e-6) : 0.f;
    }
    float ms_twohop = 0, ms_tuples = 0, ms_tc = 0;
    std::vector<cudaEvent_t> ev_tc;

    // Plan (with host reads of sizes) and execute once. Anchors are taken in
    // heavy-first order in groups whose candidate masks fit the pool budget;
    // each group runs its 2-hop kernels, item planning and tuple kernel.
    // Tensor-core plan of group `grp` from the n anchors k_anchor_cost listed.
    void plan_tc(size_t grp, unsigned n) {
        DevBuf<TcInput> tin(n, s);
        k_tc_gather<<<grid_for(n, 256), 256, 0, s>>>(tc_list.ptr, n, ncand.ptr, dprime.ptr,
                                                    rsv_c.ptr, pool_off.ptr, tin.ptr);
        SBC_LAUNCHED();
        g_launches++;
        std::vector<TcInput> h(n);
        SBC_CUDA(cudaMemcpyAsync(h.data(), tin.ptr, sizeof(TcInput) * n, cudaMemcpyDeviceToHost, s));
        SBC_CUDA(cudaStreamSynchronize(s));
        TcPlan plan = tc_plan(h, tc_budget_bytes());
        tc_upload(plan, s);
        const size_t need = (size_t)plan.max_blocks * (size_t)kTcBlockBytes;
        if (need > zbuf.bytes()) zbuf.alloc(need, s);
        tc_anchors += (uint64_t)plan.anchors;
        tc_tiles += (uint64_t)plan.tiles;
        tc_kblocks += plan.kblocks;
        tc_plans[grp] = std::move(plan);
    }

    void run_tc_timed(size_t grp, bool timing) {
        if (grp >= tc_plans.size() || tc_plans[grp].anchors == 0) return;
        cudaEvent_t t4 = timing ? new_event(ev_tc) : nullptr;
        cudaEvent_t t5 = timing ? new_event(ev_tc) : nullptr;
        if (t4) SBC_CUDA(cudaEventRecord(t4, s));
        NvtxRange nr("sbc/tc_pairs");
        launch_tc(grp);
        if (t5) SBC_CUDA(cudaEventRecord(t5, s));
    }
    uint64_t tc_anchors = 0, tc_tiles = 0, tc_kblocks = 0;

    void plan_and_run(EventTimer *tm) {
        NvtxRange nr("sbc/count");
        const bool timing = tm != nullptr;
        const int B = 256;
        groups.clear();
        drop_events();
        tc_anchors = tc_tiles = tc_kblocks = 0;
        ta.large_begin = ta.large_end = ta.small_begin = ta.small_end = 0;
        gt = 0;
        const int l = spec.l;
        R = spec.k - 1;
        cnt.alloc(1, s);
        SBC_CUDA(cudaMemsetAsync(cnt.ptr, 0, sizeof(Counters), s));
        A_bit.alloc(nnz, s);
        dprime.alloc(nX, s);
        rsv_c.alloc(nX, s);
        skey.alloc(nX, s);
        sval.alloc(nX, s);
        tk.alloc(nX, s);
        tv.alloc(nX, s);
        ncand.alloc(nX, s);
        npaper.alloc(spec.paper ? nX : 0, s);
        e_use.alloc(nX, s);
        e_all.alloc(nX, s);
        pool_off.alloc(nX + 1, s);
        dtot.alloc(1, s);
        k_plan<<<grid_for(nX * 32, B), B, 0, s>>>(o->A_off.ptr, o->A_ent.ptr, o->A_pos.ptr,
                                                  o->B_off.ptr, nX, R, l, spec.shard, spec.nshard,
                                                  spec.paper ? 1 : 0, A_bit.ptr, dprime.ptr,
                                                  e_use.ptr, e_all.ptr, rsv_c.ptr, pool_off.ptr,
                                                  skey.ptr, sval.ptr, cnt.ptr,
                                                  spec.small_e > 0 ? spec.small_e : SMALL_E_MAX);
        SBC_LAUNCHED();
        g_launches++;
        radix_sort_pairs(skey.ptr, sval.ptr, tk.ptr, tv.ptr, nX, 32, s);
        SBC_CUDA(cudaMemsetAsync(ncand.ptr, 0, (size_t)nX * 4, s));
        if (spec.paper) SBC_CUDA(cudaMemsetAsync(npaper.ptr, 0, (size_t)nX * 4, s));
        SBC_CUDA(cudaMemcpyAsync(&hc, cnt.ptr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
        SBC_CUDA(cudaStreamSynchronize(s));
        const int64_t n_act = hc.n_active;
        // candidate-mask words in heavy-first order, prefix sums, groups
        cum.assign(n_act + 1, 0);
        {
            DevBuf<int64_t> dcum(n_act + 1, s);
            k_gather_words<<<grid_for(n_act + 1, B), B, 0, s>>>(sval.ptr, pool_off.ptr, n_act, dcum.ptr);
            SBC_LAUNCHED();
            g_launches++;
            scan_exclusive_i64(dcum.ptr, dcum.ptr, n_act + 1, nullptr, s);
            SBC_CUDA(cudaMemcpyAsync(cum.data(), dcum.ptr, 8 * (size_t)(n_act + 1),
                                     cudaMemcpyDeviceToHost, s));
            SBC_CUDA(cudaStreamSynchronize(s));
            const int64_t budget = pool_budget_words();
            int64_t most = 1;
            for (int64_t a = 0; a < n_act;) {
                int64_t b = std::upper_bound(cum.begin() + a + 1, cum.end(), cum[a] + budget) -
                            cum.begin() - 1;
                if (b <= a) b = a + 1;  // one anchor larger than the budget runs alone
                groups.emplace_back(a, b);
                most = std::max(most, cum[b] - cum[a]);
                a = b;
            }
            cum_dev = std::move(dcum);
            pool.alloc((size_t)most, s);
        }
        const int sms = sm_count();

        ta.A_off = o->A_off.ptr;
        ta.A_ent = o->A_ent.ptr;
        ta.A_pos = o->A_pos.ptr;
        ta.A_bit = A_bit.ptr;
        ta.B_off = o->B_off.ptr;
        ta.B_ent = o->B_ent.ptr;
        ta.dprime = dprime.ptr;
        ta.e_use = e_use.ptr;
        ta.e_all = e_all.ptr;
        ta.rsv_c = rsv_c.ptr;
        ta.pool_off = pool_off.ptr;
        ta.order = sval.ptr;
        ta.pool = pool.ptr;
        ta.ncand = ncand.ptr;
        ta.npaper = spec.paper ? npaper.ptr : nullptr;
        ta.cnt = cnt.ptr;
        ta.l = l;
        ta.check = spec.check ? 1 : 0;
        ta.hs_cap = hash_slots_cap();
        ta.wcap = twohop_window_wedges();
        ta.bucket = nullptr;
        ta.bucket_slot = 0;
        if (hc.n_big > 0) {
            const void *fn = spec.paper ? (const void *)k_twohop_large<true> : (const void *)k_twohop_large<false>;
            ga = sms * blocks_per_sm(fn, PL_THREADS, PL_SMEM);
            if ((int64_t)ga > (int64_t)hc.n_big) ga = (int)hc.n_big;
            if (hc.e_max > (unsigned long long)ta.wcap) {
                const int lgb = bucket_lg(hc.e_max);
                ta.bucket_slot = bucket_cap(hc.e_max, lgb) << lgb;
                bucket.alloc((size_t)ga * ta.bucket_slot, s);
                ta.bucket = bucket.ptr;
            }
        }
        if (hc.n_active > hc.n_big) {
            const void *fn = spec.paper ? (const void *)k_twohop_small<true> : (const void *)k_twohop_small<false>;
            gs = sms * blocks_per_sm(fn, PS_THREADS, PS_SMEM);
        }
        const int gb = sms * blocks_per_sm((const void *)k_tuples<1>, PB_THREADS, PB_SMEM);
        const uint32_t wmax = (uint32_t)((o->max_deg_x + 31) / 32);
        per.alloc(spec.per_anchor ? 2 * nX : 0, s);
        if (per.ptr) SBC_CUDA(cudaMemsetAsync(per.ptr, 0, per.bytes(), s));
        if (spec.per_graph) SBC_CUDA(cudaMemsetAsync(spec.per_graph, 0, 16 * (size_t)spec.n_graphs, s));
        // warp scratch of the wide paths (more words than the register paths hold)
        const uint32_t wide_from = R == 3 ? (uint32_t)SLOT_W : R <= 2 ? 0xFFFFFFFFu : 8u;
        scratch.alloc(wmax > wide_from ? (size_t)gb * PB_WARPS * SCRATCH_SLOTS * wmax : 0, s);
        tu.ncand = ncand.ptr;
        tu.dprime = dprime.ptr;
        tu.rsv_c = rsv_c.ptr;
        tu.pool_off = pool_off.ptr;
        tu.pool = pool.ptr;
        tu.cnt = cnt.ptr;
        tu.per_anchor = per.ptr;
        tu.per_graph = spec.per_graph;
        tu.graph_x0 = spec.graph_x0;
        tu.n_graphs = spec.n_graphs;
        tu.wide_scratch = scratch.ptr;
        tu.wmax = wmax;
        tu.l = l;

        ItemArgs ia;
        ia.ncand = ncand.ptr;
        ia.npaper = spec.paper ? npaper.ptr : nullptr;
        ia.dprime = dprime.ptr;
        ia.order = sval.ptr;
        ia.R = R;
        ia.l = l;
        ia.method = spec.method;
        ia.pos_unit = spec.pos_unit;
        ia.cnt = cnt.ptr;
        ia.tc_on = spec.tc_min_w >= 0 && R == 2 && !thread_arena_active();
        ia.tc_min_w = spec.tc_min_w > 0 ? (uint32_t)spec.tc_min_w : kTcMinWords;
        ia.tc_min_nc = tc_min_candidates();
        if (ia.tc_on) {
            tc_list.alloc(nX, s);
            tc_ensure_attrs();
        }
        ia.tc_list = tc_list.ptr;
        tc_plans.clear();
        tc_plans.resize(groups.size());
        n_items = 0;
        for (size_t gi = 0; gi < groups.size(); gi++) {
            const int64_t a = groups[gi].first, b = groups[gi].second, na = b - a;
            // this group's pool offsets and fresh queue heads
            k_group_offsets<<<grid_for(na, B), B, 0, s>>>(sval.ptr, cum_dev.ptr, a, b, pool_off.ptr);
            SBC_LAUNCHED();
            g_launches++;
            SBC_CUDA(cudaMemsetAsync(&cnt.ptr->head_large, 0, 3 * sizeof(unsigned), s));
            SBC_CUDA(cudaMemsetAsync(&cnt.ptr->cost_total, 0, sizeof(unsigned long long), s));
            SBC_CUDA(cudaMemsetAsync(&cnt.ptr->n_tc, 0, sizeof(unsigned), s));
            SBC_CUDA(cudaMemsetAsync(&cnt.ptr->tw_fin_max, 0, 2 * sizeof(unsigned long long), s));
            cudaEvent_t t0 = timing ? new_event(ev_twohop) : nullptr;
            cudaEvent_t t1 = timing ? new_event(ev_twohop) : nullptr;
            zero_pool(gi);
            if (t0) SBC_CUDA(cudaEventRecord(t0, s));
            {
                NvtxRange nr("sbc/twohop");
                launch_twohop((unsigned)a, (unsigned)b);
            }
            if (t1) SBC_CUDA(cudaEventRecord(t1, s));
            // tuple phase planning (needs the candidate counts)
            ia.begin = a;
            ia.nX = na;
            ia.item_cost = 0;
            ia.item_off = nullptr;
            ia.item_cnt = nullptr;
            ia.items = nullptr;
            ia.ikey = ia.ival = nullptr;
            k_anchor_cost<<<grid_for(na, B), B, 0, s>>>(ia);
            SBC_LAUNCHED();
            g_launches++;
            SBC_CUDA(cudaMemcpyAsync(&hc, cnt.ptr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
            SBC_CUDA(cudaStreamSynchronize(s));
            tw_tail_ms = std::max(tw_tail_ms, group_tail_ms());
            if (hc.n_tc > 0) plan_tc(gi, hc.n_tc);
            const unsigned long long spw =
                spec.split_per_warp > 0 ? (unsigned long long)spec.split_per_warp : kSplitPerWarp;
            unsigned long long ic = hc.cost_total / ((unsigned long long)gb * PB_WARPS * spw);
            if (ic < (1ull << 12)) ic = 1ull << 12;
            if (ic > (1ull << 30)) ic = 1ull << 30;
            ia.item_cost = ic;
            item_off.alloc(na + 1, s);
            ia.item_cnt = item_off.ptr;
            int64_t ng = 0;
            if (hc.cost_total > 0 || R == 1) {
                k_items<false><<<grid_for(na, B), B, 0, s>>>(ia);
                SBC_LAUNCHED();
                scan_exclusive_i64(item_off.ptr, item_off.ptr, na + 1, dtot.ptr, s);
                g_launches++;
                SBC_CUDA(cudaMemcpyAsync(&ng, dtot.ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
                SBC_CUDA(cudaStreamSynchronize(s));
            }
            if (ng > 0xFFFFFFF0ll) fail(SBC_E_UNSUPPORTED, "too many work items");
            if (ng == 0) {
                run_tc_timed(gi, timing);
                continue;
            }
            items.alloc(ng, s);
            ikey.alloc(ng, s);
            ival.alloc(ng, s);
            t1b.alloc(ng, s);
            t2b.alloc(ng, s);
            ia.item_off = item_off.ptr;
            ia.items = items.ptr;
            ia.ikey = ikey.ptr;
            ia.ival = ival.ptr;
            k_items<true><<<grid_for(na, B), B, 0, s>>>(ia);
            SBC_LAUNCHED();
            g_launches++;
            radix_sort_pairs(ikey.ptr, ival.ptr, t1b.ptr, t2b.ptr, ng, 32, s);
            h_items = (unsigned)ng;
            SBC_CUDA(cudaMemcpyAsync(&cnt.ptr->n_items, &h_items, sizeof(unsigned), cudaMemcpyHostToDevice, s));
            tu.items = items.ptr;
            tu.iorder = ival.ptr;
            gt = gb;
            if ((int64_t)gt > ng) gt = (int)ng;
            cudaEvent_t t2 = timing ? new_event(ev_tuples) : nullptr;
            cudaEvent_t t3 = timing ? new_event(ev_tuples) : nullptr;
            if (t2) SBC_CUDA(cudaEventRecord(t2, s));
            {
                NvtxRange nr("sbc/tuples");
                launch_tuple_kernel();
            }
            if (t3) SBC_CUDA(cudaEventRecord(t3, s));
            run_tc_timed(gi, timing);
            n_items += ng;
        }
        if (tm) tm->mark(4, s);
        collect();
        if (timing) {
            ms_twohop = pairs_ms(ev_twohop);
            ms_tuples = pairs_ms(ev_tuples);
            ms_tc = pairs_ms(ev_tc);
        }
        // planning scratch a replay does not need
        skey.release();
        tk.release();
        tv.release();
        item_off.release();
        ikey.release();
        t1b.release();
        t2b.release();
    }

    // Read the counters after an execution (synchronises the stream).
    void collect() {
        SBC_CUDA(cudaMemcpyAsync(&hc, cnt.ptr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
        SBC_CUDA(cudaStreamSynchronize(s));
        if (hc.err & CERR_OVERFLOW) fail(SBC_E_OVERFLOW, "balanced biclique count exceeds 128 bits");
        if (hc.err & CERR_MASK)
            fail(SBC_E_CUDA, "self-check failed: a candidate mask disagrees with its 2-hop "
                             "counters (flags 0x%x)", hc.err);
        if (hc.err & CERR_TIMEOUT)
            fail(SBC_E_TIMEOUT, "a bounded wait of the tensor-core pair kernel ran out (flags 0x%x)",
                 hc.err);
        if (hc.err & (CERR_RESERVE | CERR_HASH))
            fail(SBC_E_CUDA, "internal error in the 2-hop kernel (flags 0x%x)", hc.err);
        res.count.lo = hc.total[0];
        res.count.hi = hc.total[1];
        const unsigned long long *tt = spec.paper ? hc.tuples_paper : hc.tuples_ours;
        res.anchor_tuples.lo = tt[0];
        res.anchor_tuples.hi = tt[1];
        res.candidates = hc.candidates;
        res.wedges = hc.wedges;
        res.work_items = (uint64_t)n_items;
        res.tested = hc.tested;
        res.typed = hc.leaves;
        res.popc_words = hc.popc_words;
        res.tc_anchors = tc_anchors;
        res.tc_tiles = tc_tiles;
        res.tc_kblocks = tc_kblocks;
        res.twohop_reads = hc.tw_reads;
        res.twohop_split = hc.tw_split;
        const double cyc = (double)(hc.tw_cyc[0] + hc.tw_cyc[1] + hc.tw_cyc[2] + hc.tw_cyc[3]);
        for (int i = 0; i < 4; i++) {
            res.twohop_anchors[i] = hc.tw_anchors[i];
            res.twohop_share[i] = cyc > 0 ? (float)(hc.tw_cyc[i] / cyc) : 0.f;
        }
        res.twohop_tail_ms = std::max(tw_tail_ms, group_tail_ms());
        res.pool_bytes = cum.empty() ? 0 : (uint64_t)cum.back() * 4;
    }
};

CountRun *countrun_create(const Orient &o, int64_t nnz, const CountSpec &spec, cudaStream_t s,
                          EventTimer *tm) {
    if (o.max_deg_x >= (1ll << 21))
        fail(SBC_E_UNSUPPORTED, "anchor-side degree %lld exceeds the 2^21 - 1 limit of the 2-hop counters",
             (long long)o.max_deg_x);
    ensure_kernel_attrs();
    std::unique_ptr<CountRun> run(new CountRun());
    run->o = &o;
    run->nnz = nnz;
    run->nX = o.nX;
    run->spec = spec;
    run->s = s;
    if (nnz > 0 && o.nX > 0) run->plan_and_run(tm);
    return run.release();
}

const CountResult &countrun_result(const CountRun *r) { return r->res; }

void countrun_launch(CountRun *r, cudaStream_t s) {
    if (r->nnz == 0 || r->nX == 0) {
        if (r->spec.per_graph) SBC_CUDA(cudaMemsetAsync(r->spec.per_graph, 0, 16 * (size_t)r->spec.n_graphs, s));
        return;
    }
    cudaStream_t keep = r->s;
    r->s = s;
    if (r->groups.size() > 1) {
        // a multi-group plan re-plans (host reads between groups)
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        SBC_CUDA(cudaStreamIsCapturing(s, &cs));
        if (cs != cudaStreamCaptureStatusNone) {
            r->s = keep;
            fail(SBC_E_UNSUPPORTED, "a count planned in %zu anchor groups cannot be captured",
                 r->groups.size());
        }
        r->plan_and_run(nullptr);
    } else {
        r->launch_count();
    }
    r->s = keep;
}

bool countrun_replayable(const CountRun *r) { return r->groups.size() <= 1; }

void countrun_collect(CountRun *r, cudaStream_t s) {
    if (r->nnz == 0 || r->nX == 0) return;
    cudaStream_t keep = r->s;
    r->s = s;
    r->collect();
    r->s = keep;
}

void countrun_destroy(CountRun *r) { delete r; }

void apply_tune(CountSpec &spec, const sbc_tune_t *t) {
    if (!t) return;
    if (t->small_wedges < 0 || t->small_wedges > SMALL_E_MAX)
        fail(SBC_E_INVAL, "small_wedges must be in [0, %d], got %d", SMALL_E_MAX, t->small_wedges);
    if (t->pos_node_cost < 0 || t->pos_node_cost > (1 << 20))
        fail(SBC_E_INVAL, "pos_node_cost must be in [0, 2^20], got %d", t->pos_node_cost);
    if (t->split_per_warp < 0 || t->split_per_warp > 64)
        fail(SBC_E_INVAL, "split_per_warp must be in [0, 64], got %d", t->split_per_warp);
    if (t->tc_min_words < -1 || t->tc_min_words > 65536)
        fail(SBC_E_INVAL, "tc_min_words must be in [-1, 65536], got %d", t->tc_min_words);
    if (t->small_wedges) spec.small_e = t->small_wedges;
    if (t->pos_node_cost) spec.pos_unit = (unsigned long long)t->pos_node_cost;
    if (t->split_per_warp) spec.split_per_warp = t->split_per_warp;
    if (t->tc_min_words) spec.tc_min_w = t->tc_min_words;
}

// SBC_HASH_SLOTS_CAP (tests only): caps every 2-hop hash table at this many
// slots (rounded down to a multiple of 32, at least 32) so that tables
// overflow and the kernels' CERR_HASH report can be exercised.
uint32_t hash_slots_cap() {
    const char *e = getenv("SBC_HASH_SLOTS_CAP");
    if (!e || !*e) return 0;
    long long v = atoll(e);
    if (v <= 0) return 0;
    if (v > (1 << 20)) v = 1 << 20;
    v &= ~31ll;
    return (uint32_t)(v < 32 ? 32 : v);
}

// Visited wedges up to which the CTA-wide 2-hop kernel hashes an anchor in one
// window (above: bucketed by hash class). SBC_TWOHOP_WINDOW (tests only)
// lowers it, from 32 up, so that small graphs take the bucketed strategy.
uint32_t twohop_window_wedges() {
    const char *e = getenv("SBC_TWOHOP_WINDOW");
    long long v = e && *e ? atoll(e) : 0;
    if (v <= 0 || v > PL_WCAP) return (uint32_t)PL_WCAP;
    return (uint32_t)(v < 32 ? 32 : v);
}

// Candidates an anchor needs for the tensor-core pair step (tuning override
// SBC_TC_MIN_CANDIDATES, at least 2).
uint32_t tc_min_candidates() {
    uint32_t v = kTcMinCandidates;
    if (const char *e = getenv("SBC_TC_MIN_CANDIDATES")) {
        long long x = atoll(e);
        if (x >= 2 && x < (1ll << 31)) v = (uint32_t)x;
    }
    return v;
}

bool debug_checks_env() {
    const char *e = getenv("SBC_DEBUG");
    return e && *e && *e != '0';
}

unsigned long long pos_node_cost_setting() {
    unsigned long long u = kPosNodeCost;
    if (const char *e = getenv("SBC_POS_NODE_COST")) {  // tuning override
        long long v = atoll(e);
        if (v > 0) u = (unsigned long long)v;
    }
    return u;
}

void count_graph(const sbc_graph *gc, int p, int q, const sbc_count_opts *opts,
                 sbc_count_stats *stats, cudaStream_t s) {
    sbc_graph *g = const_cast<sbc_graph *>(gc);
    if (p < 2 || q < 2 || p > 8 || q > 8) fail(SBC_E_INVAL, "p and q must be in [2, 8], got (%d, %d)", p, q);
    int cur = 0;
    SBC_CUDA(cudaGetDevice(&cur));
    if (cur != g->device) fail(SBC_E_INVAL, "graph lives on device %d, current device is %d", g->device, cur);
    int side = opts ? opts->anchor_side : SBC_SIDE_AUTO;
    if (side == SBC_SIDE_AUTO) side = preferred_side(g, p, q);
    if (side != 0 && side != 1) fail(SBC_E_INVAL, "anchor_side must be -1, 0 or 1");
    CountSpec spec;
    spec.k = side == 0 ? p : q;
    spec.l = side == 0 ? q : p;
    spec.paper = opts && (opts->flags & SBC_COUNT_PAPER_TUPLES);
    spec.shard = opts ? opts->shard : 0;
    spec.nshard = opts ? opts->shard_count : 0;
    spec.method = (opts && (opts->flags & SBC_COUNT_CANDIDATE_SIDE)) ? 1
                : (opts && (opts->flags & SBC_COUNT_POSITION_SIDE)) ? 2 : 0;
    spec.pos_unit = pos_node_cost_setting();
    apply_tune(spec, opts ? opts->tune : nullptr);
    spec.per_anchor = opts && opts->per_anchor;
    spec.check = (opts && (opts->flags & SBC_COUNT_CHECK)) || debug_checks_env();
    if (spec.nshard < 0 || (spec.nshard > 0 && (spec.shard < 0 || spec.shard >= spec.nshard)))
        fail(SBC_E_INVAL, "bad shard %d of %d", spec.shard, spec.nshard);
    const int64_t kernels0 = g_launches.load();
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->anchor_side = side;
    }
    const int64_t nX = side == 0 ? g->n_u : g->n_v;
    if (opts && opts->per_anchor && nX > 0) memset(opts->per_anchor, 0, sizeof(sbc_u128) * (size_t)nX);
    if (g->nnz == 0 || nX == 0) return;
    EventTimer tm(stats != nullptr && !thread_arena_active());
    tm.mark(0, s);
    {
        std::lock_guard<std::mutex> lock(g->mu);
        NvtxRange nr("sbc/orientation");
        build_orientation(g, side, s);
    }
    const Orient &o = g->side[side];
    std::unique_ptr<CountRun> run(countrun_create(o, g->nnz, spec, s, tm.on ? &tm : nullptr));
    const CountResult &res = run->res;
    if (spec.per_anchor && run->per.ptr) {
        std::vector<unsigned long long> hp((size_t)2 * nX);
        std::vector<int32_t> vo((size_t)nX);
        SBC_CUDA(cudaMemcpyAsync(hp.data(), run->per.ptr, run->per.bytes(), cudaMemcpyDeviceToHost, s));
        SBC_CUDA(cudaMemcpyAsync(vo.data(), o.vert_of.ptr, (size_t)nX * 4, cudaMemcpyDeviceToHost, s));
        SBC_CUDA(cudaStreamSynchronize(s));
        for (int64_t r = 0; r < nX; r++) {
            opts->per_anchor[vo[r]].lo = hp[2 * r];
            opts->per_anchor[vo[r]].hi = hp[2 * r + 1];
        }
    }
    if (stats) {
        stats->count = res.count;
        stats->anchor_tuples = res.anchor_tuples;
        stats->candidates = res.candidates;
        stats->wedges = res.wedges;
        stats->work_items = res.work_items;
        stats->tuples_tested = res.tested;
        stats->tuples_typed = res.typed;
        stats->popc_words = res.popc_words;
        stats->tc_anchors = res.tc_anchors;
        stats->tc_tiles = res.tc_tiles;
        stats->tc_kblocks = res.tc_kblocks;
        stats->twohop_reads = res.twohop_reads;
        stats->twohop_split_classes = res.twohop_split;
        for (int i = 0; i < 4; i++) {
            stats->twohop_anchors[i] = res.twohop_anchors[i];
            stats->twohop_share[i] = res.twohop_share[i];
        }
        stats->twohop_tail_ms = res.twohop_tail_ms;
        stats->pool_bytes = res.pool_bytes;
        stats->kernels = (int32_t)(g_launches.load() - kernels0);
        if (tm.on) {
            stats->ms_total = tm.ms(0, 4);
            stats->ms_twohop = run->ms_twohop;
            stats->ms_tuples = run->ms_tuples;
            stats->ms_tc = run->ms_tc;
            stats->ms_prepare = stats->ms_total - run->ms_twohop - run->ms_tuples - run->ms_tc;
        }
    }
}

}  // namespace sbc
