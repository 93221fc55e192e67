// sbc_count_csr_noalloc: counting for callers that cannot allocate device
// memory.
//
// Some callers may not call cudaMalloc: code running where the device
// allocator is off limits (inside a frozen memory budget of a larger
// application, a real-time loop that must not touch the allocator, or a host
// that hands this library a fixed memory plan). This entry point does the
// same work as sbc_count_csr but takes every device buffer it needs from one
// fixed array in device memory, g_noalloc_scratch below, and calls no
// cudaMalloc, cudaMallocAsync, cudaFree or other allocating routine.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds its SBC_NOALLOC_SCRATCH_BYTES until the process exits. In host
// code its name is only a host-side stand-in, so its device address is taken
// with cudaGetSymbolAddress once per device (with that device current), on
// the first call of this entry point on that device; that first call should
// therefore come before any stream capture. All calls share the array and a
// call leaves its contents behind; the counting pipeline clears everything it
// relies on being zero. Calls are serialised by a host mutex; two processes
// (or another user of the same device memory) running calls that overlap on
// the GPU would race on the array.
//
// Inside a call the array is handed out as a stack: a block freed while a
// later block is still live stays reserved until the call returns (every
// call starts again from an empty array). A call that fails after it has
// launched kernels waits for its stream before it returns and releases the
// lock, so no kernel of a failed call can still be writing the array when
// the next call starts.
#include <mutex>

#include "sbc_internal.cuh"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SBC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once).
void *scratch_address() {
    int dev = 0;
    SBC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) sbc::fail(SBC_E_UNSUPPORTED, "device ordinal %d out of range", dev);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            sbc::fail(SBC_E_CUDA, "cudaGetSymbolAddress of the no-allocation scratch failed: %s",
                      cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    return g_noalloc_ptr[dev];
}

// Waits for the call's stream when the call ends (on every path, errors
// included), before the arena and the lock are released.
struct StreamDrain {
    cudaStream_t s;
    ~StreamDrain() { (void)cudaStreamSynchronize(s); }
};

struct ArenaScope {
    sbc::Arena arena;
    explicit ArenaScope(void *base) {
        arena.base = (char *)base;
        arena.size = SBC_NOALLOC_SCRATCH_BYTES;
        sbc::set_thread_arena(&arena);
    }
    ~ArenaScope() { sbc::set_thread_arena(nullptr); }
};

}  // namespace

extern "C" sbc_status sbc_count_csr_noalloc(int64_t n_u, int64_t n_v, int64_t nnz,
                                            const void *row_offsets, const int32_t *cols,
                                            const void *signs, uint32_t flags, int p, int q,
                                            sbc_u128 *out, void *stream) {
    try {
        if (!out) sbc::fail(SBC_E_INVAL, "out is NULL");
        if (p < 2 || q < 2 || p > 8 || q > 8) sbc::fail(SBC_E_INVAL, "p and q must be in [2, 8]");
        if (n_u < 0 || n_v < 0 || nnz < 0 || n_u > SBC_NOALLOC_MAX_VERTICES ||
            n_v > SBC_NOALLOC_MAX_VERTICES || nnz > SBC_NOALLOC_MAX_EDGES)
            sbc::fail(SBC_E_INVAL,
                      "sbc_count_csr_noalloc takes at most %d vertices per side and %d edges "
                      "(got %lld x %lld, %lld edges)",
                      SBC_NOALLOC_MAX_VERTICES, SBC_NOALLOC_MAX_EDGES, (long long)n_u,
                      (long long)n_v, (long long)nnz);
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        ArenaScope scope(scratch_address());
        cudaStream_t s = (cudaStream_t)stream;
        StreamDrain drain{s};
        std::unique_ptr<sbc_graph> g(
            sbc::create_graph(n_u, n_v, nnz, row_offsets, cols, signs, flags, s));
        sbc_count_stats st;
        sbc::count_graph(g.get(), p, q, nullptr, &st, s);
        g.reset();
        *out = st.count;
    } catch (const sbc::SbcError &e) {
        sbc::set_last_error(e.what());
        return e.status;
    } catch (const std::exception &e) {
        sbc::set_last_error(e.what());
        return SBC_E_CUDA;
    }
    return SBC_OK;
}
