// Device-wide primitives: exclusive prefix sums and a stable LSD radix sort.
//
// The radix sort orders X-side vertices by degree for the vertex priority of
// Definition 4 (stable, so equal degrees stay in ascending id order) and
// groups edges into the rank-ordered adjacency lists used by Algorithm 2.
#include "sbc_internal.cuh"

namespace sbc {

namespace {

constexpr int SCAN_BLOCK = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of one value per thread across the block; returns the
// exclusive prefix and writes the block total to *total (shared memory).
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T *total) {
    constexpr int NW = SCAN_BLOCK / 32;
    __shared__ T warp_tot[NW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = warp_incl_scan(v);
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T w = lane < NW ? warp_tot[lane] : T(0);
        T wi = warp_incl_scan(w);
        if (lane < NW) warp_tot[lane] = wi - w;
        if (lane == NW - 1) *total = wi;
    }
    __syncthreads();
    T res = warp_tot[warp] + incl - v;
    __syncthreads();
    return res;
}

template <typename T>
__global__ void k_tile_reduce(const T *__restrict__ in, int64_t n, T *__restrict__ partial) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    T s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t idx = base + (int64_t)i * SCAN_BLOCK + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    __shared__ T tot;
    block_excl_scan<T>(s, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// Exclusive scan of each tile, offset by the tile's exclusive prefix.
template <typename T>
__global__ void k_tile_scan(const T *in, T *out, int64_t n, const T *__restrict__ tile_off,
                            T *total) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T v[SCAN_ITEMS];
    T s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t idx = base + i;
        v[i] = idx < n ? in[idx] : T(0);
        s += v[i];
    }
    __shared__ T tot;
    T pre = block_excl_scan<T>(s, &tot);
    T off = tile_off ? tile_off[blockIdx.x] : T(0);
    T run = off + pre;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = off + tot;
}

template <typename T>
void scan_impl(const T *in, T *out, int64_t n, T *total, cudaStream_t s) {
    if (n <= 0) {
        if (total) SBC_CUDA(cudaMemsetAsync(total, 0, sizeof(T), s));
        return;
    }
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 1) {
        k_tile_scan<T><<<1, SCAN_BLOCK, 0, s>>>(in, out, n, nullptr, total);
        SBC_LAUNCHED();
        g_launches++;
        return;
    }
    DevBuf<T> partial(tiles, s);
    k_tile_reduce<T><<<(unsigned)tiles, SCAN_BLOCK, 0, s>>>(in, n, partial.ptr);
    SBC_LAUNCHED();
    g_launches++;
    scan_impl<T>(partial.ptr, partial.ptr, tiles, nullptr, s);
    k_tile_scan<T><<<(unsigned)tiles, SCAN_BLOCK, 0, s>>>(in, out, n, partial.ptr, total);
    SBC_LAUNCHED();
    g_launches++;
}

// ------------------------------------------------------------------ radix sort

constexpr int RS_BLOCK = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_BLOCK * RS_ROUNDS;
constexpr int RS_WARPS = RS_BLOCK / 32;

__global__ void k_radix_hist(const uint32_t *__restrict__ keys, int64_t n, int shift,
                             uint32_t *__restrict__ hist, int64_t ntiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int r = 0; r < RS_ROUNDS; r++) {
        int64_t idx = base + (int64_t)r * RS_BLOCK + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: elements keep their tile order within a digit; tiles are
// placed in order by the digit-major exclusive scan of the histograms.
__global__ void k_radix_scatter(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                                uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                int64_t n, int shift, const uint32_t *__restrict__ offs,
                                int64_t ntiles) {
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcnt[RS_WARPS][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base[tid] = offs[(int64_t)tid * ntiles + blockIdx.x];
    const uint32_t lt_mask = (1u << lane) - 1u;
    int64_t tbase = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; r++) {
        int64_t idx = tbase + (int64_t)r * RS_BLOCK + tid;
        bool valid = idx < n;
        uint32_t k = valid ? kin[idx] : 0u;
        uint32_t v = valid ? vin[idx] : 0u;
        uint32_t d = valid ? ((k >> shift) & 255u) : (256u + lane);
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) wcnt[w][tid] = 0;
        __syncthreads();
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & lt_mask);
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pre = 0;
            for (int w = 0; w < warp; w++) pre += wcnt[w][d];
            uint32_t pos = base[d] + pre + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        uint32_t t = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) t += wcnt[w][tid];
        base[tid] += t;
        __syncthreads();
    }
}

}  // namespace

void scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total,
                        cudaStream_t s) {
    scan_impl<int64_t>(in, out, n, total, s);
}

void scan_exclusive_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total,
                        cudaStream_t s) {
    scan_impl<uint32_t>(in, out, n, total, s);
}

void radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *tmp_keys, uint32_t *tmp_vals,
                      int64_t n, int key_bits, cudaStream_t s, int *launches) {
    if (n <= 1 || key_bits <= 0) return;
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    DevBuf<uint32_t> hist(256 * ntiles, s);
    uint32_t *ka = keys, *va = vals, *kb = tmp_keys, *vb = tmp_vals;
    int passes = (key_bits + 7) / 8;
    for (int p = 0; p < passes; p++) {
        int shift = 8 * p;
        k_radix_hist<<<(unsigned)ntiles, RS_BLOCK, 0, s>>>(ka, n, shift, hist.ptr, ntiles);
        SBC_LAUNCHED();
        scan_exclusive_u32(hist.ptr, hist.ptr, 256 * ntiles, nullptr, s);
        k_radix_scatter<<<(unsigned)ntiles, RS_BLOCK, 0, s>>>(ka, va, kb, vb, n, shift, hist.ptr,
                                                               ntiles);
        SBC_LAUNCHED();
        g_launches += 2;
        if (launches) *launches += 2;
        uint32_t *t = ka; ka = kb; kb = t;
        t = va; va = vb; vb = t;
    }
    if (ka != keys) {
        SBC_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
        SBC_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
}

}  // namespace sbc
