// Internal declarations shared by the CUDA sources of libsbc.
//
// Errors travel as C++ exceptions (SbcError) inside the library and are turned
// into sbc_status codes plus a thread-local message at every C entry point.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <atomic>
#include <mutex>
#include <memory>
#include <vector>
#include <stdexcept>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/sbc.h"

namespace sbc {

struct SbcError : std::runtime_error {
    sbc_status status;
    SbcError(sbc_status s, const std::string &m) : std::runtime_error(m), status(s) {}
};

[[noreturn]] void fail(sbc_status s, const char *fmt, ...);
void set_last_error(const std::string &msg);

#define SBC_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t err_ = (call);                                                       \
        if (err_ != cudaSuccess)                                                         \
            ::sbc::fail(err_ == cudaErrorMemoryAllocation ? SBC_E_NOMEM : SBC_E_CUDA,    \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(err_),        \
                        __FILE__, __LINE__);                                             \
    } while (0)

// Check for a launch error right after a kernel launch.
#define SBC_LAUNCHED() SBC_CUDA(cudaGetLastError())

// A named NVTX range for the lifetime of the object (phases of a count on a
// profiler's timeline; free when no profiler is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// ---------------------------------------------------------------- memory

void *dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void *p, size_t bytes, cudaStream_t s);

// A caller-provided region of device memory that dev_alloc carves from (a
// stack: blocks freed in reverse order are reclaimed) while it is installed on
// the calling thread with set_thread_arena. Only the no-allocation entry point
// installs one.
struct Arena {
    char *base = nullptr;
    size_t size = 0, top = 0, peak = 0;
};
void set_thread_arena(Arena *a);
bool thread_arena_active();

// Owning device buffer (stream-ordered allocation).
template <typename T>
struct DevBuf {
    T *ptr = nullptr;
    size_t n = 0;
    cudaStream_t stream = nullptr;
    DevBuf() = default;
    DevBuf(size_t count, cudaStream_t s) { alloc(count, s); }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : ptr(o.ptr), n(o.n), stream(o.stream) { o.ptr = nullptr; o.n = 0; }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) {
            release();
            ptr = o.ptr; n = o.n; stream = o.stream;
            o.ptr = nullptr; o.n = 0;
        }
        return *this;
    }
    void alloc(size_t count, cudaStream_t s) {
        release();
        stream = s;
        n = count;
        ptr = count ? static_cast<T *>(dev_alloc(count * sizeof(T), s)) : nullptr;
    }
    void release() {
        if (ptr) dev_free(ptr, n * sizeof(T), stream);
        ptr = nullptr;
        n = 0;
    }
    size_t bytes() const { return n * sizeof(T); }
    ~DevBuf() { release(); }
};

// ---------------------------------------------------------------- graph

// Structures for one anchor side X (Algorithm 2's S) of a graph. X-vertices
// are renumbered by their rank in the vertex priority rho of Definition 4
// (ascending degree, ties by ascending id), so "rho(w) > rho(u)" becomes
// "rank(w) > rank(u)".
struct Orient {
    bool built = false;
    int64_t nX = 0, nY = 0;
    DevBuf<int64_t> A_off;   // nX+1: X->Y adjacency, rows in rank order
    DevBuf<uint32_t> A_ent;  // nnz: y | (negative << 31)
    DevBuf<uint32_t> A_pos;  // nnz: index of the mirror entry inside B's list of y
    DevBuf<int64_t> B_off;   // nY+1: Y->X adjacency
    DevBuf<uint32_t> B_ent;  // nnz: rank(x) | (negative << 31), each list ascending by rank
    DevBuf<int32_t> vert_of; // nX: rank -> vertex id
    int64_t max_deg_x = 0, max_deg_y = 0;
    size_t bytes() const {
        return A_off.bytes() + A_ent.bytes() + A_pos.bytes() + B_off.bytes() + B_ent.bytes() +
               vert_of.bytes();
    }
};

}  // namespace sbc

struct sbc_graph {
    int device = 0;
    int64_t n_u = 0, n_v = 0, nnz = 0;
    sbc::DevBuf<int64_t> off;  // n_u+1
    sbc::DevBuf<int32_t> col;  // nnz
    sbc::DevBuf<uint8_t> neg;  // nnz, 1 = negative edge
    sbc::DevBuf<int32_t> deg_u, deg_v;
    int64_t max_deg_u = 0, max_deg_v = 0;
    uint64_t wedges_u = 0, wedges_v = 0;  // 2-paths visited anchoring on U / on V
    sbc::Orient side[2];
    std::mutex mu;
    size_t bytes() const {
        return off.bytes() + col.bytes() + neg.bytes() + deg_u.bytes() + deg_v.bytes() +
               side[0].bytes() + side[1].bytes();
    }
};

namespace sbc {

// Build (once) the oriented structures of side `x` (0 = U, 1 = V).
// Sets *dup when a duplicate (u, v) pair is found.
void build_orientation(sbc_graph *g, int x, cudaStream_t s);

// ---------------------------------------------------------------- primitives

// Exclusive prefix sum of n values; in and out may alias. Returns nothing; the
// total is out[n-1] + in[n-1] and can be requested with total != nullptr
// (device pointer, one element).
void scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total,
                        cudaStream_t s);
void scan_exclusive_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total,
                        cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs by the low `key_bits` bits of
// the key. Sorted data ends in keys/vals; tmp_keys/tmp_vals are n-element
// scratch buffers. `launches` is incremented by the kernels issued.
void radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *tmp_keys, uint32_t *tmp_vals,
                      int64_t n, int key_bits, cudaStream_t s, int *launches = nullptr);

// Number of bits needed to represent v (0 for v == 0).
inline int bits_for(uint64_t v) {
    int b = 0;
    while (v) { b++; v >>= 1; }
    return b;
}

inline int grid_for(int64_t n, int block, int cap = 152 * 32) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// Count of streaming multiprocessors of the current device.
int sm_count();

// Kernel launches issued by the library since load (for reporting).
extern std::atomic<int64_t> g_launches;

// Anchor side of an automatic count (graph.cu): the side with fewer 2-paths
// to visit, except that when p != q and exactly one side gives tuples of 3
// against tuples of 4 or more on the other, that side (whose candidate pairs
// take the tensor-core step) unless it visits more than 64 times the other
// side's 2-paths. 0 = U, 1 = V.
int preferred_side(const sbc_graph *g, int p, int q);

// Upload, validate and prepare a graph (graph.cu).
sbc_graph *create_graph(int64_t n_u, int64_t n_v, int64_t nnz, const void *row_offsets,
                        const int32_t *cols, const void *signs, uint32_t flags, cudaStream_t s);

// Count driver: defined in count.cu.
void count_graph(const sbc_graph *g, int p, int q, const sbc_count_opts *opts,
                 sbc_count_stats *stats, cudaStream_t s);

// One count over an orientation (count.cu): k = tuple size on the anchor
// side, l = size on the other side.
struct CountSpec {
    int k = 0, l = 0;
    bool paper = false;     // also count Algorithm 2's candidate sets
    int method = 0;         // 0 cheaper side per anchor, 1 candidate side, 2 position side
    unsigned long long pos_unit = 0;
    int small_e = 0;         // 2-hop tier threshold in visited wedges (0: default)
    int split_per_warp = 0;  // tuple work items per warp of a full launch (0: default)
    int shard = 0, nshard = 0;
    bool per_anchor = false;
    unsigned long long *per_graph = nullptr;  // device, 2 words per graph (batches)
    const int64_t *graph_x0 = nullptr;        // device, first anchor rank per graph
    int n_graphs = 0;
    bool check = false;     // device self-checks (SBC_COUNT_CHECK or SBC_DEBUG=1)
    int tc_min_w = 0;       // tensor-core pair step from this many mask words (0: default, -1: off)
};
struct CountResult {
    sbc_u128 count{0, 0}, anchor_tuples{0, 0};
    uint64_t candidates = 0, wedges = 0, work_items = 0, tested = 0, typed = 0, popc_words = 0;
    uint64_t tc_anchors = 0, tc_tiles = 0, tc_kblocks = 0;
    uint64_t twohop_reads = 0, twohop_anchors[4] = {0, 0, 0, 0}, pool_bytes = 0, twohop_split = 0;
    float twohop_share[4] = {0, 0, 0, 0}, twohop_tail_ms = 0;
};
struct CountRun;
struct EventTimer;
// Plans and executes the count once (synchronising for sizes).
CountRun *countrun_create(const Orient &o, int64_t nnz, const CountSpec &spec, cudaStream_t s,
                          EventTimer *tm);
const CountResult &countrun_result(const CountRun *r);
// Launches of one execution of a planned count: no allocation, no host
// synchronisation, so they may be captured into a CUDA graph.
void countrun_launch(CountRun *r, cudaStream_t s);
// Reads the counters of the last execution (synchronises s).
void countrun_collect(CountRun *r, cudaStream_t s);
// Batches (batch.cu): plan the unions of `gs` and count them once; with
// capture, record the counting kernels as a CUDA graph for sbc_batch_run.
sbc_batch *batch_create(const sbc_graph *const *gs, size_t n, int p, int q, bool capture,
                        const sbc_tune_t *tune, cudaStream_t s);
const sbc_u128 *batch_first(const sbc_batch *b);
void batch_destroy(sbc_batch *b);

// False when the plan runs in several anchor groups (no graph capture).
bool countrun_replayable(const CountRun *r);
void countrun_destroy(CountRun *r);
unsigned long long pos_node_cost_setting();
// SBC_DEBUG set (and not "0") in the environment: self-checks on every count.
bool debug_checks_env();
// Candidates an anchor needs for the tensor-core pair step.
uint32_t tc_min_candidates();
// SBC_HASH_SLOTS_CAP (tests only): the 2-hop tables' slot cap, 0 for none.
uint32_t hash_slots_cap();
// SBC_TWOHOP_WINDOW (tests only): wedges of a one-window anchor of the CTA-wide
// 2-hop kernel (default and largest: its table's half).
uint32_t twohop_window_wedges();
// Applies launch parameters (NULL or zero fields: defaults) to a count spec;
// SBC_E_INVAL when a field is out of range.
void apply_tune(CountSpec &spec, const sbc_tune_t *t);

// ---------------------------------------------------------------- tensor-core pairs

// Tensor-core form of the two-partner tuple step for wide anchors
// (tc_pairs.cu). One anchor of a chunk:
struct TcAnchor {
    uint32_t r;          // anchor rank
    uint32_t nc, W, rsv; // candidates, mask words, candidate stride of its pool region
    uint32_t RB, KB;     // Z row blocks of 128 (even), position blocks of 128
    int64_t pool_off;    // its pool region (words)
    int64_t zblk0;       // first Z block (16 KB each) in the chunk's arena
    int64_t tile0;       // first output tile in the chunk
};
struct TcInput {
    uint32_t r, nc, W, rsv;
    int64_t pool_off;
};
struct TcChunk {
    std::vector<TcAnchor> host;
    DevBuf<TcAnchor> dev;
    int64_t n_blocks = 0, n_tiles = 0;
};
struct TcPlan {
    std::vector<TcChunk> chunks;
    int64_t max_blocks = 0, tiles = 0, anchors = 0;
    uint64_t kblocks = 0;  // sum over tiles of the anchor's position blocks (MMA K steps of 128)
};
struct TcArgs {
    const TcAnchor *anc = nullptr;
    int n_anc = 0;
    int64_t n_blocks = 0, n_tiles = 0;
    const uint32_t *pool = nullptr;
    unsigned char *z = nullptr;
    int l = 0;
    unsigned long long *total = nullptr, *per_anchor = nullptr, *per_graph = nullptr;
    const int64_t *graph_x0 = nullptr;
    int n_graphs = 0;
    unsigned *err = nullptr;
    unsigned long long big64 = 0;  // largest x with binom(x, l) by the 64-bit formula
};
// Chunks of at most budget_bytes of Z (an anchor larger than that forms a
// chunk of its own).
TcPlan tc_plan(const std::vector<TcInput> &in, int64_t budget_bytes);
void tc_upload(TcPlan &plan, cudaStream_t s);
void tc_ensure_attrs();
// Expansion + pair kernels of every chunk, in stream order (no host sync).
void tc_launch(const TcPlan &plan, TcArgs base, unsigned char *z, cudaStream_t s);
constexpr int64_t kTcBlockBytes = 16384;

}  // namespace sbc

// ---------------------------------------------------------------- device helpers

namespace sbc {

// Error bit of a count whose exact value (or one of its terms) needs more
// than 128 bits.
constexpr unsigned kErrOverflow = 1u;
// Error bit of a bounded device wait that ran out (the kernel stopped early).
constexpr unsigned kErrTimeout = 16u;

// Add the unsigned 128-bit value (lo, hi) into *dst (two 64-bit words) with
// 64-bit atomics: the limb add that wraps carries into the high word. A carry
// out of the high word (the sum left 128 bits) sets kErrOverflow in *err
// (when err is not NULL).
__device__ __forceinline__ void atomic_add_u128(unsigned long long *dst, unsigned long long lo,
                                                unsigned long long hi, unsigned *err) {
    bool ovf = false;
    if (lo) {
        unsigned long long old = atomicAdd(dst, lo);
        if (old + lo < old) {
            hi += 1;
            ovf = hi == 0;
        }
    }
    if (hi) {
        unsigned long long old = atomicAdd(dst + 1, hi);
        ovf |= old + hi < old;
    }
    if (ovf && err) atomicOr(err, kErrOverflow);
}

// A thread's partial sum is flagged once its high word passes this value:
// from below it, the 64-bit adds a thread makes (far fewer than 2^48) cannot
// carry the high word past 2^64, so the only wraps left to detect are the
// 128-bit adds, which check exactly.
constexpr unsigned long long kU128Headroom = 0xFFFF000000000000ull;

struct U128 {
    unsigned long long lo = 0, hi = 0;
    __device__ __forceinline__ void add(unsigned long long v) {
        lo += v;
        hi += (lo < v) ? 1ull : 0ull;
    }
    // Returns true when the sum left 128 bits or passed the headroom mark.
    __device__ __forceinline__ bool add(U128 v) {
        lo += v.lo;
        const unsigned long long c = lo < v.lo ? 1ull : 0ull;
        const unsigned long long h = hi + v.hi;
        bool o = h < hi;
        hi = h + c;
        o |= hi < h;
        return o || hi > kU128Headroom;
    }
};

// Sum of the warp's values (every lane gets it); sets kErrOverflow in *err
// (when not NULL) if a partial sum leaves 128 bits.
__device__ __forceinline__ U128 warp_sum_u128(U128 v, unsigned *err) {
    bool o = false;
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) {
        U128 t;
        t.lo = __shfl_xor_sync(0xffffffffu, v.lo, k);
        t.hi = __shfl_xor_sync(0xffffffffu, v.hi, k);
        o |= v.add(t);
    }
    if (err && __any_sync(0xffffffffu, o) && (threadIdx.x & 31) == 0) atomicOr(err, kErrOverflow);
    return v;
}

}  // namespace sbc
