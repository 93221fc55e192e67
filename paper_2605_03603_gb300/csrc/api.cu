// C entry points of libsbc: argument checks, exception-to-status conversion,
// the allocator hook. Declarations and contracts are in include/sbc.h.
#include <cstdarg>
#include <cstring>

#include "sbc_internal.cuh"

namespace sbc {

std::atomic<int64_t> g_launches{0};

namespace {
thread_local std::string t_err;
thread_local Arena *t_arena = nullptr;
sbc_alloc_fn g_alloc = nullptr;
sbc_free_fn g_free = nullptr;
void *g_alloc_ctx = nullptr;
}  // namespace

void set_last_error(const std::string &msg) { t_err = msg; }

void fail(sbc_status s, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    throw SbcError(s, buf);
}

void set_thread_arena(Arena *a) { t_arena = a; }
bool thread_arena_active() { return t_arena != nullptr; }

void *dev_alloc(size_t bytes, cudaStream_t s) {
    void *p = nullptr;
    if (t_arena) {
        const size_t need = (bytes + 255) & ~(size_t)255;
        if (t_arena->top + need > t_arena->size)
            fail(SBC_E_NOMEM,
                 "the graph needs more than the %zu bytes of fixed scratch of the "
                 "no-allocation entry point (%zu in use, %zu more requested)",
                 t_arena->size, t_arena->top, need);
        p = t_arena->base + t_arena->top;
        t_arena->top += need;
        if (t_arena->top > t_arena->peak) t_arena->peak = t_arena->top;
        return p;
    }
    if (g_alloc) {
        p = g_alloc(bytes, (void *)s, g_alloc_ctx);
        if (!p) fail(SBC_E_NOMEM, "allocator hook returned NULL for %zu bytes", bytes);
        return p;
    }
    cudaError_t e = cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(SBC_E_NOMEM, "cudaMallocAsync(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    }
    return p;
}

void dev_free(void *p, size_t bytes, cudaStream_t s) {
    if (!p) return;
    if (t_arena) {
        const size_t need = (bytes + 255) & ~(size_t)255;
        if ((char *)p + need == t_arena->base + t_arena->top) t_arena->top -= need;
        return;
    }
    if (g_free) {
        g_free(p, bytes, (void *)s, g_alloc_ctx);
        return;
    }
    cudaFreeAsync(p, s);
}

int sm_count() {
    int dev = 0, n = 0;
    SBC_CUDA(cudaGetDevice(&dev));
    SBC_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    return n;
}

sbc_graph *create_graph(int64_t n_u, int64_t n_v, int64_t nnz, const void *row_offsets,
                        const int32_t *cols, const void *signs, uint32_t flags, cudaStream_t s);

}  // namespace sbc

using namespace sbc;

#define SBC_API_BEGIN try {
#define SBC_API_END                                                  \
    }                                                                \
    catch (const SbcError &e) {                                      \
        set_last_error(e.what());                                    \
        return e.status;                                             \
    }                                                                \
    catch (const std::bad_alloc &) {                                 \
        set_last_error("host allocation failed");                   \
        return SBC_E_NOMEM;                                          \
    }                                                                \
    catch (const std::exception &e) {                                \
        set_last_error(e.what());                                    \
        return SBC_E_CUDA;                                           \
    }                                                                \
    return SBC_OK;

extern "C" {

const char *sbc_last_error(void) { return t_err.c_str(); }

const char *sbc_version(void) { return "sbc 0.1 (sm_103a)"; }

uint64_t sbc_launch_count(void) { return (uint64_t)g_launches.load(); }

sbc_status sbc_set_allocator(sbc_alloc_fn alloc, sbc_free_fn free, void *ctx) {
    SBC_API_BEGIN
    if ((alloc == nullptr) != (free == nullptr))
        fail(SBC_E_INVAL, "alloc and free must both be set or both be NULL");
    g_alloc = alloc;
    g_free = free;
    g_alloc_ctx = ctx;
    SBC_API_END
}

sbc_status sbc_graph_create(sbc_graph **out, int64_t n_u, int64_t n_v, int64_t nnz,
                            const void *row_offsets, const int32_t *cols, const void *signs,
                            uint32_t flags, void *stream) {
    SBC_API_BEGIN
    if (!out) fail(SBC_E_INVAL, "out is NULL");
    *out = nullptr;
    *out = create_graph(n_u, n_v, nnz, row_offsets, cols, signs, flags, (cudaStream_t)stream);
    SBC_API_END
}

sbc_status sbc_graph_destroy(sbc_graph *g) {
    SBC_API_BEGIN
    if (!g) return SBC_OK;
    int cur = 0;
    const int dev = g->device;
    cudaGetDevice(&cur);
    if (cur != dev) cudaSetDevice(dev);
    cudaDeviceSynchronize();
    delete g;
    if (cur != dev) cudaSetDevice(cur);
    SBC_API_END
}

sbc_status sbc_graph_info(const sbc_graph *g, sbc_graph_info_t *out) {
    SBC_API_BEGIN
    if (!g || !out) fail(SBC_E_INVAL, "NULL argument");
    out->n_u = g->n_u;
    out->n_v = g->n_v;
    out->nnz = g->nnz;
    out->max_deg_u = g->max_deg_u;
    out->max_deg_v = g->max_deg_v;
    out->wedges_anchor_u = g->wedges_u;
    out->wedges_anchor_v = g->wedges_v;
    out->device_bytes = g->bytes();
    SBC_API_END
}

sbc_status sbc_count_ex(const sbc_graph *g, int p, int q, const sbc_count_opts *opts,
                        sbc_count_stats *stats, void *stream) {
    SBC_API_BEGIN
    if (!g) fail(SBC_E_INVAL, "graph is NULL");
    count_graph(g, p, q, opts, stats, (cudaStream_t)stream);
    SBC_API_END
}

sbc_status sbc_count(const sbc_graph *g, int p, int q, sbc_u128 *out, void *stream) {
    SBC_API_BEGIN
    if (!g || !out) fail(SBC_E_INVAL, "NULL argument");
    sbc_count_stats st;
    count_graph(g, p, q, nullptr, &st, (cudaStream_t)stream);
    *out = st.count;
    SBC_API_END
}

sbc_status sbc_count_csr(int64_t n_u, int64_t n_v, int64_t nnz, const void *row_offsets,
                         const int32_t *cols, const void *signs, uint32_t flags, int p, int q,
                         sbc_u128 *out, void *stream) {
    SBC_API_BEGIN
    if (!out) fail(SBC_E_INVAL, "out is NULL");
    if (p < 2 || q < 2 || p > 8 || q > 8) fail(SBC_E_INVAL, "p and q must be in [2, 8]");
    std::unique_ptr<sbc_graph> g(
        create_graph(n_u, n_v, nnz, row_offsets, cols, signs, flags, (cudaStream_t)stream));
    sbc_count_stats st;
    count_graph(g.get(), p, q, nullptr, &st, (cudaStream_t)stream);
    *out = st.count;
    SBC_API_END
}

}  // extern "C"
