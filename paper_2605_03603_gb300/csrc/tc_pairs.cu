// Tensor-core form of the two-partner tuple step (Algorithm 2, Section 4.3,
// the loop over (p-1)-subsets A of C with p - 1 = 2, and the type count of
// Section 4.2) for anchors whose candidate masks are wide.
//
// For an anchor u with candidates 0..nc-1 and useful positions 0..d'-1, let
// S_c = P_c AND NOT D_c (common neighbours where sign(u,v) = sign(c,v)) and
// T_c = P_c AND D_c (where they differ), as 0/1 vectors over the positions.
// For a pair of candidates i < j the four type classes of Section 4.2 are
// (s,s), (s,d), (d,s), (d,d), with sizes <S_i,S_j>, <S_i,T_j>, <T_i,S_j>,
// <T_i,T_j>. Stacking the rows Z = [S_0; T_0; S_1; T_1; ...] (row 2c + 0 is
// S_c, row 2c + 1 is T_c) gives all of them at once as G = Z Z^T, and the
// anchor adds, over row pairs (a, b) with floor(a/2) < floor(b/2),
// binom(G[a][b], l). This is a dense contraction over the positions, so it
// runs on the tensor cores:
//
// * k_zexpand writes Z as fp8 e4m3 bytes (1.0 or 0) in 16 KB blocks of 128
//   rows x 128 positions, each block already in the shared-memory layout of
//   the MMA (K-major, 128-byte swizzle: 16-byte chunk c of row r stored at
//   chunk c ^ (r & 7)), so a block moves to shared memory with one plain
//   bulk copy.
// * k_tcpairs is a persistent kernel over output tiles of 128 x 256 rows of
//   G (only tiles that hold a pair a < b in candidate order). Per CTA: one
//   producer warp issues the bulk copies into a 4-stage ring, one warp issues
//   tcgen05.mma (kind::f8f6f4, M = 128, N = 256, K = 32 per instruction)
//   into one of two TMEM accumulators, and eight epilogue warps read the
//   accumulator with tcgen05.ld, convert each entry to an integer, and add
//   binom(G[a][b], l) (32-bit table lookups when the anchor's positions
//   bound every entry, else a 64-bit table up to 256 and exact 128-bit
//   arithmetic above). The fp32 accumulator holds these integer sums exactly (each is
//   at most d' < 2^21 < 2^24).
//
// Every wait on an mbarrier is bounded by a clock limit; a wait that runs out
// sets the error word, every role stops, copies and MMAs in flight are
// waited for (again bounded), TMEM is freed and the kernel returns.
#include <algorithm>
#include <vector>

#include "sbc_internal.cuh"

namespace sbc {

namespace {

constexpr int TC_THREADS = 320;  // warp 0 producer, warp 1 MMA, warps 2..9 epilogue
constexpr int TC_EPI_WARPS = 8;  // two per TMEM lane group, each on half the columns
constexpr int TC_STAGES = 4;
constexpr uint32_t TC_BLOCK = 16384;           // one Z block: 128 rows x 128 bytes
constexpr uint32_t TC_STAGE = 3 * TC_BLOCK;    // A (128 rows) + B (256 rows)
constexpr size_t TC_SMEM = (size_t)TC_STAGES * TC_STAGE + 1024;  // + alignment slack
constexpr int TC_TMEM_COLS = 512;              // two 128 x 256 fp32 accumulators
constexpr int TC_BINOM = 256;
constexpr long long TC_WAIT_CYCLES = 4000000000ll;  // about 2 s at the SM clock

// kind::f8f6f4 instruction descriptor: D f32, A and B e4m3, both K-major,
// N = 256, M = 128.
constexpr uint32_t TC_IDESC = (1u << 4) | (0u << 7) | (0u << 10) | ((256u >> 3) << 17) |
                              ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of parity `parity` to complete. Returns false
// when the CTA aborts (this wait ran out, or another role's did).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          unsigned *err) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        // try_wait suspends the thread in hardware until the phase completes
        // or a short time limit passes, so this loop needs no sleep of its own
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > TC_WAIT_CYCLES) {
            *abort_flag = 1;
            atomicOr(err, kErrTimeout);
            return false;
        }
    }
}

// One bulk copy of `bytes` (a multiple of 16, both addresses 16-byte
// aligned) from global to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;             // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
    d |= (uint64_t)1 << 46;             // descriptor version
    d |= (uint64_t)2 << 61;             // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(TC_IDESC), "r"(accum));
}
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
          "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
          "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// binom(x, l) exactly for x > TC_BINOM (128-bit multiplicative formula; the
// running value after step i is binom(x - l + i, i), so dividing before
// multiplying by the reduced factor keeps it exact). Sets kErrOverflow when
// the value needs more than 128 bits.
__device__ __noinline__ U128 tc_binom_big(unsigned long long x, int l, unsigned *err) {
    unsigned long long lo = 1, hi = 0;
    for (int i = 1; i <= l; i++) {
        unsigned long long f = x - l + i;
        unsigned long long g = (unsigned long long)i, h = f % g;  // g = gcd(f, i)
        while (h) {
            const unsigned long long t = g % h;
            g = h;
            h = t;
        }
        // divide (hi, lo) by i / g (exact: it divides the running value)
        const unsigned long long dv = (unsigned long long)i / g;
        if (dv > 1) {
            unsigned long long qh = hi / dv, rem = hi % dv;
            unsigned long long a = (rem << 32) | (lo >> 32);
            unsigned long long q1 = a / dv;
            rem = a % dv;
            unsigned long long b = (rem << 32) | (lo & 0xFFFFFFFFull);
            hi = qh;
            lo = (q1 << 32) | (b / dv);
        }
        const unsigned long long m = f / g;
        unsigned long long l0 = lo * m, c = __umul64hi(lo, m);
        unsigned long long h0 = hi * m, hh = __umul64hi(hi, m);
        unsigned long long nh = h0 + c;
        if (hh != 0 || nh < h0) {
            atomicOr(err, kErrOverflow);
            return U128();
        }
        lo = l0;
        hi = nh;
    }
    U128 t;
    t.lo = lo;
    t.hi = hi;
    return t;
}

}  // namespace

// Expand the chunk's candidate masks into Z blocks (see the file comment).
__global__ void __launch_bounds__(512) k_zexpand(TcArgs a) {
    const int r = threadIdx.x & 127, wi = threadIdx.x >> 7;
    // the blocks of a CTA increase, so its anchor index only moves forward
    int ai = -1;
    int64_t next0 = 0;
    TcAnchor A;
    for (int64_t blk = blockIdx.x; blk < a.n_blocks; blk += gridDim.x) {
        while (blk >= next0) {
            A = a.anc[++ai];
            next0 = ai + 1 < a.n_anc ? a.anc[ai + 1].zblk0 : a.n_blocks;
        }
        const int64_t local = blk - A.zblk0;
        const uint32_t rb = (uint32_t)(local / A.KB), kb = (uint32_t)(local % A.KB);
        const uint32_t row = rb * 128 + r, c = row >> 1, w = kb * 4 + wi;
        uint32_t bits = 0;
        if (c < A.nc && w < A.W) {
            const uint32_t *region = a.pool + A.pool_off;
            const uint32_t P = region[(size_t)w * A.rsv + c];
            const uint32_t D = region[(size_t)(A.W + w) * A.rsv + c];
            bits = (row & 1) ? (P & D) : (P & ~D);
        }
        // 32 positions -> 32 bytes of 0x38 (e4m3 1.0) or 0: each nibble is
        // spread to the low bit of 4 bytes and scaled
        uint32_t o[8];
#pragma unroll
        for (int k = 0; k < 8; k++)
            o[k] = ((((bits >> (4 * k)) & 0xFu) * 0x00204081u) & 0x01010101u) * 0x38u;
        unsigned char *dst = a.z + blk * (int64_t)TC_BLOCK + r * 128;
        const int ch0 = 2 * wi, ch1 = 2 * wi + 1;
        *reinterpret_cast<uint4 *>(dst + ((ch0 ^ (r & 7)) << 4)) = make_uint4(o[0], o[1], o[2], o[3]);
        *reinterpret_cast<uint4 *>(dst + ((ch1 ^ (r & 7)) << 4)) = make_uint4(o[4], o[5], o[6], o[7]);
    }
}

namespace {

// Walks the tiles of one CTA (t = blockIdx.x, + gridDim.x, ...): tile t of
// the chunk, its anchor and block coordinates (I rows of 128, J columns of
// 256; column J holds the rows I = 0 .. 2J + 1, the tiles with a pair a < b).
// Anchor and column only move forward, so every step is a few compares
// (the anchor record is loaded once per anchor, not searched per tile).
struct TileCursor {
    int ai = -1;
    int64_t next0 = 0;  // first tile of the next anchor
    TcAnchor A;
    uint32_t I = 0, J = 0;
    __device__ __forceinline__ void seek(const TcArgs &a, int64_t t) {
        while (t >= next0) {
            A = a.anc[++ai];
            next0 = ai + 1 < a.n_anc ? a.anc[ai + 1].tile0 : a.n_tiles;
            J = 0;
        }
        const uint64_t local = (uint64_t)(t - A.tile0);
        while ((uint64_t)(J + 1) * (J + 2) <= local) J++;
        I = (uint32_t)(local - (uint64_t)J * (J + 1));
    }
};

}  // namespace

// binom(x, L) in 64 bits by the multiplicative formula (every partial
// product fits when x <= the host's 64-bit limit for L); the divisors are
// compile-time constants.
template <int L>
__device__ __forceinline__ unsigned long long binom_u64c(unsigned long long x) {
    unsigned long long r = 1;
#pragma unroll
    for (int i = 1; i <= L; i++) r = r * (x - L + i) / (unsigned long long)i;
    return r;
}

// Largest multiple of 32 (at most 2048) with 32 * binom(x, L) < 2^32: for
// anchors of at most this many useful positions every Gram entry indexes a
// 32-bit table and 32 of its binomials sum in 32 bits.
template <int L>
__host__ __device__ constexpr uint32_t tc_fast_max() {
    uint32_t best = 0;
    for (uint32_t x = 32; x <= 2048; x += 32) {
        unsigned long long b = 1;
        for (int i = 1; i <= L; i++) b = b * (x - L + i) / i;
        if (32ull * b >= (1ull << 32)) break;
        best = x;
    }
    return best;
}

template <int L>
__global__ void __launch_bounds__(TC_THREADS, 1) k_tcpairs(TcArgs a) {
    extern __shared__ __align__(16) unsigned char tc_smem_raw[];
    __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES], acc_full[2], acc_empty[2],
        mma_done;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    // binom(x, L) for x <= TC_BINOM, zero below L and at TC_BINOM + 1 (the
    // clamped index of larger entries, which a slower path adds)
    __shared__ unsigned long long s_bt[TC_BINOM + 2];
    // binom(x, L) for x <= FAST in 32 bits (anchors with 32 W <= FAST)
    constexpr uint32_t FAST = tc_fast_max<L>();
    __shared__ uint32_t s_bt32[FAST + 1];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *smem =
        (unsigned char *)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    for (int x = tid; x <= TC_BINOM + 1; x += TC_THREADS)
        s_bt[x] = (x >= L && x <= TC_BINOM) ? binom_u64c<L>(x) : 0ull;
    for (int x = tid; x <= (int)FAST; x += TC_THREADS)
        s_bt32[x] = x >= L ? (uint32_t)binom_u64c<L>(x) : 0u;
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], TC_EPI_WARPS);
        }
        mbar_init(&mma_done, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == 0) {
        // ---- producer: bulk copies of the A block and the two B blocks
        if (lane == 0) {
            uint32_t stage = 0, round = 0;
            int issued[TC_STAGES] = {0, 0, 0, 0};
            uint32_t issued_par[TC_STAGES] = {0, 0, 0, 0};
            TileCursor tr;
            for (int64_t t = blockIdx.x; t < a.n_tiles && !s_abort; t += gridDim.x) {
                tr.seek(a, t);
                const TcAnchor &A = tr.A;
                const unsigned char *zA = a.z + (A.zblk0 + (int64_t)tr.I * A.KB) * TC_BLOCK;
                const unsigned char *zB0 = a.z + (A.zblk0 + (int64_t)(2 * tr.J) * A.KB) * TC_BLOCK;
                const unsigned char *zB1 = zB0 + (int64_t)A.KB * TC_BLOCK;
                for (uint32_t kb = 0; kb < A.KB; kb++) {
                    if (!mbar_wait(&empty[stage], (round & 1) ^ 1, &s_abort, a.err)) break;
                    unsigned char *st = smem + (size_t)stage * TC_STAGE;
                    mbar_expect_tx(&full[stage], TC_STAGE);
                    bulk_g2s(st, zA + (int64_t)kb * TC_BLOCK, TC_BLOCK, &full[stage]);
                    bulk_g2s(st + TC_BLOCK, zB0 + (int64_t)kb * TC_BLOCK, TC_BLOCK, &full[stage]);
                    bulk_g2s(st + 2 * TC_BLOCK, zB1 + (int64_t)kb * TC_BLOCK, TC_BLOCK, &full[stage]);
                    issued[stage] = 1;
                    issued_par[stage] = round & 1;
                    if (++stage == TC_STAGES) {
                        stage = 0;
                        round++;
                    }
                }
            }
            if (s_abort) {
                // let every copy this thread started land before the CTA exits
                for (int s = 0; s < TC_STAGES; s++)
                    if (issued[s]) {
                        const long long t0 = clock64();
                        while (!mbar_try(&full[s], issued_par[s]) && clock64() - t0 < TC_WAIT_CYCLES) {
                        }
                    }
            }
        }
    } else if (warp == 1) {
        // ---- MMA issue
        if (lane == 0) {
            uint32_t stage = 0, round = 0, it = 0;
            const uint32_t sbase = smem_u32(smem);
            TileCursor tr;
            for (int64_t t = blockIdx.x; t < a.n_tiles && !s_abort; t += gridDim.x, it++) {
                tr.seek(a, t);
                const TcAnchor &A = tr.A;
                const uint32_t buf = it & 1;
                if (!mbar_wait(&acc_empty[buf], ((it >> 1) & 1) ^ 1, &s_abort, a.err)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem + buf * 256;
                bool ok = true;
                for (uint32_t kb = 0; kb < A.KB; kb++) {
                    if (!mbar_wait(&full[stage], round & 1, &s_abort, a.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = sbase + stage * TC_STAGE, sb = sa + TC_BLOCK;
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        tc_mma(d_tmem, sw128_desc(sa + 32 * k), sw128_desc(sb + 32 * k),
                               (kb | k) != 0 ? 1u : 0u);
                    tc_commit(&empty[stage]);
                    if (++stage == TC_STAGES) {
                        stage = 0;
                        round++;
                    }
                }
                if (!ok) break;
                tc_commit(&acc_full[buf]);
            }
            // every MMA this thread issued has completed before TMEM is freed
            tc_commit(&mma_done);
            const long long t0 = clock64();
            while (!mbar_try(&mma_done, 0) && clock64() - t0 < TC_WAIT_CYCLES) {
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue: warps 2..9; warp w reads TMEM lanes 32 * (w % 4) ..
        // (the rows of its lane group) and columns 128 * half .. + 128
        const uint32_t g = (uint32_t)(warp & 3), half = (uint32_t)(warp - 2) >> 2;
        uint32_t it = 0;
        TileCursor tr;
        // the warp's sum over its tiles of one anchor, added to the totals
        // when the anchor changes (one set of atomics per anchor, not per tile)
        U128 sum;
        int sum_ai = -1;
        uint32_t sum_r = 0;
        auto flush = [&]() {
            const U128 ws = warp_sum_u128(sum, a.err);
            if (lane == 0 && (ws.lo | ws.hi)) {
                atomic_add_u128(a.total, ws.lo, ws.hi, a.per_graph ? nullptr : a.err);
                if (a.per_anchor) atomic_add_u128(a.per_anchor + 2 * (size_t)sum_r, ws.lo, ws.hi, a.err);
                if (a.per_graph) {
                    int lo = 0, hi = a.n_graphs;  // largest graph with graph_x0 <= r
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (a.graph_x0[mid] <= (int64_t)sum_r) lo = mid; else hi = mid;
                    }
                    atomic_add_u128(a.per_graph + 2 * (size_t)lo, ws.lo, ws.hi, a.err);
                }
            }
            sum = U128();
        };
        // binom(x, L) of entries above the table (rare: larger common sets)
        auto add_big = [&](uint32_t x) {
            if (x <= a.big64) sum.add(binom_u64c<L>(x));
            else if (sum.add(tc_binom_big(x, L, a.err))) atomicOr(a.err, kErrOverflow);
        };
        for (int64_t t = blockIdx.x; t < a.n_tiles; t += gridDim.x, it++) {
            tr.seek(a, t);
            const uint32_t buf = it & 1;
            if (tr.ai != sum_ai) {
                if (sum_ai >= 0) flush();
                sum_ai = tr.ai;
                sum_r = tr.A.r;
            }
            bool ok = true;
            if (lane == 0) ok = mbar_wait(&acc_full[buf], (it >> 1) & 1, &s_abort, a.err);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) break;
            tc_fence_after();
            const uint32_t row = tr.I * 128 + g * 32 + lane;  // row of G
            const uint32_t ca = row >> 1;                       // its candidate
            // columns of this tile (0..255) whose candidate exceeds the row's:
            // all of them off the diagonal, from c0 on it
            const uint32_t c0 = ca + 1 > tr.J * 128 ? (ca + 1 - tr.J * 128) * 2 : 0u;
            const uint32_t cl0 = __shfl_sync(0xffffffffu, c0, 0);  // smallest in the warp
            // entries are at most the anchor's useful positions (<= 32 W)
            const bool fast = 32ull * tr.A.W <= FAST;
            for (uint32_t cb = half * 128; cb < half * 128 + 128; cb += 32) {
                if (cb + 32 <= cl0) continue;  // no lane keeps a column here (warp-uniform)
                uint32_t v[32];
                tmem_ld32(tmem + ((g * 32) << 16) + buf * 256 + cb, v);
                if (fast && cb >= c0) {
                    // The float bits of entry + 2^23 are 0x4B000000 + entry;
                    // the table's address is offset by that constant (32-bit
                    // shared-window arithmetic), and the bits are clamped to
                    // the table's end.
                    const uint32_t tb = smem_u32(s_bt32) - (0x4B000000u << 2);
                    uint32_t part32 = 0;
#pragma unroll
                    for (int j = 0; j < 32; j++) {
                        const uint32_t bits =
                            min(__float_as_uint(__uint_as_float(v[j]) + 8388608.0f), 0x4B000000u + FAST);
                        uint32_t b;
                        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(b) : "r"(tb + (bits << 2)));
                        part32 += b;
                    }
                    sum.add((unsigned long long)part32);
                    continue;
                }
                unsigned long long part = 0;  // < 32 * binom(256, 8) < 2^64
                uint32_t mx = 0;
                if (cb >= c0) {
#pragma unroll
                    for (int j = 0; j < 32; j++) {
                        // the entry is an exact integer below 2^23: adding 2^23
                        // leaves it in the low mantissa bits
                        const uint32_t x =
                            __float_as_uint(__uint_as_float(v[j]) + 8388608.0f) & 0x7FFFFFu;
                        mx = max(mx, x);
                        part += s_bt[min(x, (uint32_t)TC_BINOM + 1)];
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 32; j++) {
                        uint32_t x = __float_as_uint(__uint_as_float(v[j]) + 8388608.0f) & 0x7FFFFFu;
                        x = cb + j >= c0 ? x : 0u;
                        mx = max(mx, x);
                        part += s_bt[min(x, (uint32_t)TC_BINOM + 1)];
                    }
                }
                sum.add(part);
                if (mx > (uint32_t)TC_BINOM) {
#pragma unroll
                    for (int j = 0; j < 32; j++) {
                        const uint32_t x =
                            __float_as_uint(__uint_as_float(v[j]) + 8388608.0f) & 0x7FFFFFu;
                        if (x > (uint32_t)TC_BINOM && cb + j >= c0) add_big(x);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[buf]);
        }
        if (sum_ai >= 0) flush();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

// ------------------------------------------------------------------ host

TcPlan tc_plan(const std::vector<TcInput> &in, int64_t budget_bytes) {
    TcPlan plan;
    std::vector<TcInput> v(in);
    // heaviest per-tile work first, so that the strided tile assignment of
    // the persistent kernel ends with short tiles
    std::sort(v.begin(), v.end(), [](const TcInput &x, const TcInput &y) {
        return x.W != y.W ? x.W > y.W : x.nc > y.nc;
    });
    TcChunk cur;
    int64_t blocks = 0, tiles = 0;
    auto flush = [&]() {
        if (cur.host.empty()) return;
        cur.n_blocks = blocks;
        cur.n_tiles = tiles;
        plan.max_blocks = std::max(plan.max_blocks, blocks);
        plan.chunks.push_back(std::move(cur));
        cur = TcChunk();
        blocks = tiles = 0;
    };
    for (const TcInput &x : v) {
        TcAnchor A;
        A.r = x.r;
        A.nc = x.nc;
        A.W = x.W;
        A.rsv = x.rsv;
        A.RB = 2 * ((x.nc + 127) / 128);
        A.KB = (x.W + 3) / 4;
        A.pool_off = x.pool_off;
        const int64_t nb = (int64_t)A.RB * A.KB;
        if (!cur.host.empty() && (blocks + nb) * (int64_t)TC_BLOCK > budget_bytes) flush();
        A.zblk0 = blocks;
        A.tile0 = tiles;
        const uint64_t h = A.RB / 2;
        tiles += (int64_t)(h * (h + 1));  // sum over J < RB/2 of min(2J + 2, RB)
        plan.kblocks += h * (h + 1) * A.KB;
        blocks += nb;
        cur.host.push_back(A);
        plan.anchors++;
    }
    flush();
    for (const TcChunk &c : plan.chunks) plan.tiles += c.n_tiles;
    return plan;
}

void tc_upload(TcPlan &plan, cudaStream_t s) {
    for (TcChunk &c : plan.chunks) {
        c.dev.alloc(c.host.size(), s);
        SBC_CUDA(cudaMemcpyAsync(c.dev.ptr, c.host.data(), sizeof(TcAnchor) * c.host.size(),
                                 cudaMemcpyHostToDevice, s));
    }
}

void tc_ensure_attrs() {
    static std::mutex mu;
    static bool done[64] = {};
    std::lock_guard<std::mutex> lock(mu);
    int dev = 0;
    SBC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(SBC_E_UNSUPPORTED, "device ordinal %d out of range", dev);
    if (done[dev]) return;
    const void *fns[] = {(const void *)k_tcpairs<2>, (const void *)k_tcpairs<3>,
                         (const void *)k_tcpairs<4>, (const void *)k_tcpairs<5>,
                         (const void *)k_tcpairs<6>, (const void *)k_tcpairs<7>,
                         (const void *)k_tcpairs<8>};
    for (const void *f : fns)
        SBC_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    done[dev] = true;
}

void tc_launch(const TcPlan &plan, TcArgs base, unsigned char *z, cudaStream_t s) {
    const int sms = sm_count();
    for (const TcChunk &c : plan.chunks) {
        TcArgs a = base;
        a.anc = c.dev.ptr;
        a.n_anc = (int)c.host.size();
        a.n_blocks = c.n_blocks;
        a.n_tiles = c.n_tiles;
        a.z = z;
        int ge = (int)std::min<int64_t>(c.n_blocks, (int64_t)sms * 8);
        k_zexpand<<<ge, 512, 0, s>>>(a);
        SBC_LAUNCHED();
        int gt = (int)std::min<int64_t>(c.n_tiles, (int64_t)sms);
        switch (a.l) {
            case 2: k_tcpairs<2><<<gt, TC_THREADS, TC_SMEM, s>>>(a); break;
            case 3: k_tcpairs<3><<<gt, TC_THREADS, TC_SMEM, s>>>(a); break;
            case 4: k_tcpairs<4><<<gt, TC_THREADS, TC_SMEM, s>>>(a); break;
            case 5: k_tcpairs<5><<<gt, TC_THREADS, TC_SMEM, s>>>(a); break;
            case 6: k_tcpairs<6><<<gt, TC_THREADS, TC_SMEM, s>>>(a); break;
            case 7: k_tcpairs<7><<<gt, TC_THREADS, TC_SMEM, s>>>(a); break;
            default: k_tcpairs<8><<<gt, TC_THREADS, TC_SMEM, s>>>(a); break;
        }
        SBC_LAUNCHED();
        g_launches += 2;
    }
}

}  // namespace sbc
