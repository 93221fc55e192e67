// Batched counting: many independent graphs counted by one pass of the
// counting kernels.
//
// A batch is counted as the disjoint union of its graphs. A biclique is
// connected, so every balanced (p,q)-biclique lies inside one graph, and the
// union's count is the sum of the graphs' counts. Each graph keeps the anchor
// side its cost model prefers; the union concatenates the graphs' oriented
// structures (Algorithm 2's priority order within each graph is unchanged,
// ranks and ids are offset per graph) so that the plan, the 2-hop kernels and
// the tuple kernel each run once, as persistent kernels over the work queue
// of every graph at once. Work items add their partial counts straight into
// their graph's total.
//
// When p != q, graphs anchored on U count (tuple p, other q) and graphs
// anchored on V count (tuple q, other p), so they form two unions.
//
// A batch object keeps the planned counts; sbc_batch_run replays their
// counting kernels from a CUDA graph captured at creation.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sbc_internal.cuh"

namespace sbc {
namespace {

constexpr uint32_t VMASK_B = 0x7FFFFFFFu;

struct GDesc {
    const int64_t *A_off, *B_off;
    const uint32_t *A_ent, *A_pos, *B_ent;
    int64_t nX, nY, nnz, x0, y0, e0;
};

__device__ __forceinline__ int find_graph(const int64_t *start, int n, int64_t i) {
    int lo = 0, hi = n;  // largest g with start[g] <= i
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (start[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// Entries: A (y + y0, sign), A_pos (unchanged), B (rank + x0, sign).
__global__ void k_union_edges(const GDesc *gd, const int64_t *e0s, int n, int64_t nnz,
                              uint32_t *A_ent, uint32_t *A_pos, uint32_t *B_ent) {
    for (int64_t E = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; E < nnz;
         E += (int64_t)gridDim.x * blockDim.x) {
        const int g = find_graph(e0s, n, E);
        const GDesc d = gd[g];
        const int64_t e = E - d.e0;
        const uint32_t a = d.A_ent[e], b = d.B_ent[e];
        A_ent[E] = (uint32_t)((a & VMASK_B) + d.y0) | (a & 0x80000000u);
        A_pos[E] = d.A_pos[e];
        B_ent[E] = (uint32_t)((b & VMASK_B) + d.x0) | (b & 0x80000000u);
    }
}

// Offsets of one side: out[i] = off_g[i - start_g] + e0_g, out[total] = nnz.
__global__ void k_union_offsets(const GDesc *gd, const int64_t *starts, int n, int64_t total,
                                int64_t nnz, int side_b, int64_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= total;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i == total) {
            out[i] = nnz;
            continue;
        }
        const int g = find_graph(starts, n, i);
        const GDesc d = gd[g];
        const int64_t local = i - (side_b ? d.y0 : d.x0);
        out[i] = (side_b ? d.B_off[local] : d.A_off[local]) + d.e0;
    }
}

}  // namespace

// One union of graphs sharing the anchor side's sizes (k, l).
struct BatchGroup {
    std::vector<int> members;  // batch indices
    Orient uni;
    int64_t nnz = 0;
    DevBuf<int64_t> x0;        // first rank of each member, n+1
    DevBuf<unsigned long long> totals;  // 2 words per member
    CountSpec spec;            // defaults plus the batch's launch parameters
    CountRun *run = nullptr;
    ~BatchGroup() {
        if (run) countrun_destroy(run);
    }
};

}  // namespace sbc

struct sbc_batch {
    int device = 0;
    size_t n = 0;
    int p = 0, q = 0;
    std::vector<sbc::BatchGroup *> groups;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture_stream = nullptr;
    std::vector<sbc_u128> first;  // counts of the planning execution
    ~sbc_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (capture_stream) cudaStreamDestroy(capture_stream);
        for (auto *g : groups) delete g;
    }
};

namespace sbc {

namespace {

// Concatenate the members' orientations (member i viewed from sides[i]).
void build_union(const std::vector<const sbc_graph *> &gs, const std::vector<int> &sides,
                 BatchGroup &bg, cudaStream_t s) {
    const int n = (int)bg.members.size();
    std::vector<GDesc> hd(n);
    std::vector<int64_t> xs(n + 1), ys(n + 1), es(n + 1);
    int64_t X = 0, Y = 0, E = 0, mdx = 0, mdy = 0;
    for (int i = 0; i < n; i++) {
        const sbc_graph *g = gs[bg.members[i]];
        const Orient &o = g->side[sides[bg.members[i]]];
        GDesc d;
        d.A_off = o.A_off.ptr;
        d.B_off = o.B_off.ptr;
        d.A_ent = o.A_ent.ptr;
        d.A_pos = o.A_pos.ptr;
        d.B_ent = o.B_ent.ptr;
        d.nX = o.nX;
        d.nY = o.nY;
        d.nnz = g->nnz;
        d.x0 = X;
        d.y0 = Y;
        d.e0 = E;
        hd[i] = d;
        xs[i] = X;
        ys[i] = Y;
        es[i] = E;
        X += o.nX;
        Y += o.nY;
        E += g->nnz;
        mdx = std::max(mdx, o.max_deg_x);
        mdy = std::max(mdy, o.max_deg_y);
    }
    xs[n] = X;
    ys[n] = Y;
    es[n] = E;
    if (X >= (1ll << 31) - 1 || Y >= (1ll << 31) - 1 || E >= (1ll << 31) - 1)
        fail(SBC_E_UNSUPPORTED, "batch too large for 32-bit vertex and edge indices "
                                "(%lld x %lld vertices, %lld edges); split it",
             (long long)X, (long long)Y, (long long)E);
    Orient &u = bg.uni;
    u.nX = X;
    u.nY = Y;
    u.max_deg_x = mdx;
    u.max_deg_y = mdy;
    bg.nnz = E;
    u.A_off.alloc(X + 1, s);
    u.B_off.alloc(Y + 1, s);
    u.A_ent.alloc(E, s);
    u.A_pos.alloc(E, s);
    u.B_ent.alloc(E, s);
    DevBuf<GDesc> dd(n, s);
    DevBuf<int64_t> dxs(n + 1, s), dys(n + 1, s), des(n + 1, s);
    SBC_CUDA(cudaMemcpyAsync(dd.ptr, hd.data(), sizeof(GDesc) * n, cudaMemcpyHostToDevice, s));
    SBC_CUDA(cudaMemcpyAsync(dxs.ptr, xs.data(), 8 * (n + 1), cudaMemcpyHostToDevice, s));
    SBC_CUDA(cudaMemcpyAsync(dys.ptr, ys.data(), 8 * (n + 1), cudaMemcpyHostToDevice, s));
    SBC_CUDA(cudaMemcpyAsync(des.ptr, es.data(), 8 * (n + 1), cudaMemcpyHostToDevice, s));
    const int B = 256;
    if (E > 0) {
        k_union_edges<<<grid_for(E, B), B, 0, s>>>(dd.ptr, des.ptr, n, E, u.A_ent.ptr, u.A_pos.ptr,
                                                   u.B_ent.ptr);
        SBC_LAUNCHED();
        g_launches++;
    }
    k_union_offsets<<<grid_for(X + 1, B), B, 0, s>>>(dd.ptr, dxs.ptr, n, X, E, 0, u.A_off.ptr);
    SBC_LAUNCHED();
    k_union_offsets<<<grid_for(Y + 1, B), B, 0, s>>>(dd.ptr, dys.ptr, n, Y, E, 1, u.B_off.ptr);
    SBC_LAUNCHED();
    g_launches += 2;
    bg.x0.alloc(n + 1, s);
    SBC_CUDA(cudaMemcpyAsync(bg.x0.ptr, xs.data(), 8 * (n + 1), cudaMemcpyHostToDevice, s));
    bg.totals.alloc(2 * (size_t)n, s);
    SBC_CUDA(cudaMemsetAsync(bg.totals.ptr, 0, bg.totals.bytes(), s));
    u.built = true;
    SBC_CUDA(cudaStreamSynchronize(s));  // the host tables and descriptors go out of scope
}

void read_totals(sbc_batch *b, sbc_u128 *out, cudaStream_t s) {
    for (auto *bg : b->groups) {
        std::vector<unsigned long long> h(2 * bg->members.size());
        if (!h.empty())
            SBC_CUDA(cudaMemcpyAsync(h.data(), bg->totals.ptr, 8 * h.size(), cudaMemcpyDeviceToHost, s));
        SBC_CUDA(cudaStreamSynchronize(s));
        for (size_t i = 0; i < bg->members.size(); i++) {
            out[bg->members[i]].lo = h[2 * i];
            out[bg->members[i]].hi = h[2 * i + 1];
        }
    }
}

}  // namespace

sbc_batch *batch_create(const sbc_graph *const *gs_in, size_t n, int p, int q, bool capture,
                        const sbc_tune_t *tune, cudaStream_t s) {
    if (p < 2 || q < 2 || p > 8 || q > 8) fail(SBC_E_INVAL, "p and q must be in [2, 8], got (%d, %d)", p, q);
    if (n > 0 && !gs_in) fail(SBC_E_INVAL, "graphs is NULL");
    std::unique_ptr<sbc_batch> b(new sbc_batch());
    SBC_CUDA(cudaGetDevice(&b->device));
    b->n = n;
    b->p = p;
    b->q = q;
    std::vector<const sbc_graph *> gs(gs_in, gs_in + n);
    std::vector<int> side(n);
    for (size_t i = 0; i < n; i++) {
        if (!gs[i]) fail(SBC_E_INVAL, "graph %zu is NULL", i);
        if (gs[i]->device != b->device)
            fail(SBC_E_INVAL, "graph %zu lives on device %d, current device is %d", i, gs[i]->device,
                 b->device);
        side[i] = preferred_side(gs[i], p, q);
        sbc_graph *g = const_cast<sbc_graph *>(gs[i]);
        std::lock_guard<std::mutex> lock(g->mu);
        build_orientation(g, side[i], s);
    }
    // p == q: one union, each graph on its own preferred side (both count
    // (p, p)); p != q: a union per side, anchored U counts (p, q), V (q, p)
    for (int sd = 0; sd < 2; sd++) {
        std::unique_ptr<BatchGroup> bg(new BatchGroup());
        for (size_t i = 0; i < n; i++)
            if (p == q ? sd == 0 : side[i] == sd) bg->members.push_back((int)i);
        if (bg->members.empty()) continue;
        build_union(gs, side, *bg, s);
        CountSpec spec;
        spec.k = (p == q || sd == 0) ? p : q;
        spec.l = (p == q || sd == 0) ? q : p;
        spec.pos_unit = pos_node_cost_setting();
        apply_tune(spec, tune);
        spec.check = debug_checks_env();
        spec.per_graph = bg->totals.ptr;
        spec.graph_x0 = bg->x0.ptr;
        spec.n_graphs = (int)bg->members.size();
        bg->spec = spec;
        bg->run = countrun_create(bg->uni, bg->nnz, spec, s, nullptr);
        b->groups.push_back(bg.release());
    }
    b->first.assign(n, sbc_u128{0, 0});
    read_totals(b.get(), b->first.data(), s);
    for (auto *bg : b->groups) capture = capture && countrun_replayable(bg->run);
    if (capture) {
        SBC_CUDA(cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking));
        SBC_CUDA(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal));
        try {
            for (auto *bg : b->groups) countrun_launch(bg->run, b->capture_stream);
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(b->capture_stream, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        SBC_CUDA(cudaStreamEndCapture(b->capture_stream, &b->graph));
        SBC_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    }
    return b.release();
}

const sbc_u128 *batch_first(const sbc_batch *b) { return b->first.data(); }

void batch_destroy(sbc_batch *b) { delete b; }

void batch_run(sbc_batch *b, sbc_u128 *out, cudaStream_t s) {
    int cur = 0;
    SBC_CUDA(cudaGetDevice(&cur));
    if (cur != b->device) fail(SBC_E_INVAL, "batch lives on device %d, current device is %d", b->device, cur);
    if (b->exec) {
        SBC_CUDA(cudaGraphLaunch(b->exec, s));
    } else {
        for (auto *bg : b->groups) countrun_launch(bg->run, s);
    }
    for (auto *bg : b->groups) countrun_collect(bg->run, s);
    read_totals(b, out, s);
}

namespace {

bool same_counts(const std::vector<sbc_u128> &a, const std::vector<sbc_u128> &b) {
    if (a.size() != b.size()) return false;
    for (size_t i = 0; i < a.size(); i++)
        if (a[i].lo != b[i].lo || a[i].hi != b[i].hi) return false;
    return true;
}

struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    Events() {
        SBC_CUDA(cudaEventCreate(&a));
        SBC_CUDA(cudaEventCreate(&b));
    }
    ~Events() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

}  // namespace

// Coordinate descent over the launch parameters; every candidate is planned on
// the same unions and its counting kernels are timed.
void autotune(const sbc_graph *const *gs, size_t n, int p, int q, int reps, sbc_tune_t *out,
              cudaStream_t s) {
    if (n == 0) fail(SBC_E_INVAL, "autotune needs at least one graph");
    if (reps < 0 || reps > 1000) fail(SBC_E_INVAL, "reps must be in [0, 1000], got %d", reps);
    if (reps == 0) reps = 3;
    std::unique_ptr<sbc_batch> b(batch_create(gs, n, p, q, false, nullptr, s));
    const std::vector<sbc_u128> want = b->first;
    std::vector<sbc_u128> got(n);
    Events ev;
    auto measure = [&](const sbc_tune_t &t) -> float {
        for (auto *bg : b->groups) {
            countrun_destroy(bg->run);
            bg->run = nullptr;
            CountSpec spec = bg->spec;
            apply_tune(spec, &t);
            bg->run = countrun_create(bg->uni, bg->nnz, spec, s, nullptr);
        }
        read_totals(b.get(), got.data(), s);
        if (!same_counts(got, want))
            fail(SBC_E_CUDA, "internal error: launch parameters (%d, %d, %d) changed a count",
                 t.small_wedges, t.pos_node_cost, t.split_per_warp);
        float best = 3.0e38f;
        for (int r = 0; r < reps; r++) {
            SBC_CUDA(cudaEventRecord(ev.a, s));
            for (auto *bg : b->groups) countrun_launch(bg->run, s);
            SBC_CUDA(cudaEventRecord(ev.b, s));
            SBC_CUDA(cudaEventSynchronize(ev.b));
            float ms = 0;
            SBC_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
            best = std::min(best, ms);
        }
        for (auto *bg : b->groups) countrun_collect(bg->run, s);
        read_totals(b.get(), got.data(), s);
        if (!same_counts(got, want))
            fail(SBC_E_CUDA, "internal error: a replay with launch parameters (%d, %d, %d) "
                             "changed a count", t.small_wedges, t.pos_node_cost, t.split_per_warp);
        return best;
    };
    sbc_tune_t cur{0, 0, 0, 0, 0.0f};
    cur.ms = measure(cur);
    const int splits[] = {1, 2, 4, 8, 16};
    const int smalls[] = {32, 64, 128, 256, 512};
    const int costs[] = {2, 4, 6, 10, 16, 64, 1 << 20};
    auto sweep = [&](int32_t sbc_tune_t::*field, const int *vals, int nv) {
        sbc_tune_t best = cur;
        for (int i = 0; i < nv; i++) {
            sbc_tune_t t = cur;
            t.*field = vals[i];
            t.ms = measure(t);
            if (t.ms < best.ms) best = t;
        }
        cur = best;
    };
    sweep(&sbc_tune_t::split_per_warp, splits, 5);
    sweep(&sbc_tune_t::small_wedges, smalls, 5);
    sweep(&sbc_tune_t::pos_node_cost, costs, 7);
    const int tcs[] = {-1, 3, 5, 9, 17};
    sweep(&sbc_tune_t::tc_min_words, tcs, 5);
    *out = cur;
}

}  // namespace sbc

using namespace sbc;

#define SBC_BATCH_TRY try {
#define SBC_BATCH_END                         \
    }                                         \
    catch (const SbcError &e) {               \
        set_last_error(e.what());             \
        return e.status;                      \
    }                                         \
    catch (const std::exception &e) {         \
        set_last_error(e.what());             \
        return SBC_E_CUDA;                    \
    }                                         \
    return SBC_OK;

extern "C" {

sbc_status sbc_batch_create(const sbc_graph *const *graphs, size_t n, int p, int q,
                            sbc_batch **out, void *stream) {
    SBC_BATCH_TRY
    if (!out) fail(SBC_E_INVAL, "out is NULL");
    *out = nullptr;
    *out = batch_create(graphs, n, p, q, true, nullptr, (cudaStream_t)stream);
    SBC_BATCH_END
}

sbc_status sbc_batch_create_ex(const sbc_graph *const *graphs, size_t n, int p, int q,
                               const sbc_tune_t *tune, sbc_batch **out, void *stream) {
    SBC_BATCH_TRY
    if (!out) fail(SBC_E_INVAL, "out is NULL");
    *out = nullptr;
    *out = batch_create(graphs, n, p, q, true, tune, (cudaStream_t)stream);
    SBC_BATCH_END
}

sbc_status sbc_autotune(const sbc_graph *const *graphs, size_t n, int p, int q, int32_t reps,
                        sbc_tune_t *out, void *stream) {
    SBC_BATCH_TRY
    if (!out) fail(SBC_E_INVAL, "out is NULL");
    autotune(graphs, n, p, q, reps, out, (cudaStream_t)stream);
    SBC_BATCH_END
}

namespace sbc {
namespace {

// Cache key of a tuning: the GPU (name and SM count) and the shape of the
// batch (p, q, and the powers of two just above its graph count and total
// edges), so batches of the same kind on the same GPU share one entry.
std::string tune_key(const sbc_graph *const *gs, size_t n, int p, int q) {
    int dev = 0, sms = 0;
    SBC_CUDA(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    SBC_CUDA(cudaGetDeviceProperties(&prop, dev));
    SBC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    uint64_t edges = 0;
    for (size_t i = 0; i < n; i++) edges += gs[i] ? (uint64_t)gs[i]->nnz : 0;
    std::string name(prop.name);
    for (char &c : name)
        if (c == ' ' || c == '\t' || c == '|') c = '_';
    char buf[256];
    snprintf(buf, sizeof(buf), "%s|%d|%d,%d|g%d|e%d", name.c_str(), sms, p, q, bits_for(n),
             bits_for(edges));
    return buf;
}

// Looks `key` up in the cache file (one line per entry: key, then the four
// launch parameters and the time); the last matching line wins.
bool tune_lookup(const char *path, const std::string &key, sbc_tune_t *out) {
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[512], k[300];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        sbc_tune_t t{};
        if (sscanf(line, "%299s %d %d %d %d %f", k, &t.small_wedges, &t.pos_node_cost,
                   &t.split_per_warp, &t.tc_min_words, &t.ms) == 6 &&
            key == k) {
            *out = t;
            found = true;
        }
    }
    fclose(f);
    return found;
}

void tune_store(const char *path, const std::string &key, const sbc_tune_t &t) {
    FILE *f = fopen(path, "a");
    if (!f) fail(SBC_E_INVAL, "cannot open the tuning cache %s for appending", path);
    fprintf(f, "%s %d %d %d %d %.4f\n", key.c_str(), t.small_wedges, t.pos_node_cost,
            t.split_per_warp, t.tc_min_words, t.ms);
    fclose(f);
}

}  // namespace
}  // namespace sbc

sbc_status sbc_autotune_cached(const sbc_graph *const *graphs, size_t n, int p, int q,
                               int32_t reps, const char *cache_path, sbc_tune_t *out,
                               int32_t *from_cache, void *stream) {
    SBC_BATCH_TRY
    if (!out || !cache_path || !*cache_path) fail(SBC_E_INVAL, "out and cache_path are required");
    if (n == 0 || !graphs) fail(SBC_E_INVAL, "autotune needs at least one graph");
    for (size_t i = 0; i < n; i++)
        if (!graphs[i]) fail(SBC_E_INVAL, "graph %zu is NULL", i);
    if (p < 2 || q < 2 || p > 8 || q > 8) fail(SBC_E_INVAL, "p and q must be in [2, 8]");
    const std::string key = tune_key(graphs, n, p, q);
    if (from_cache) *from_cache = 0;
    sbc_tune_t t{};
    if (tune_lookup(cache_path, key, &t)) {
        CountSpec chk;
        apply_tune(chk, &t);  // the stored fields must be valid launch parameters
        *out = t;
        if (from_cache) *from_cache = 1;
    } else {
        autotune(graphs, n, p, q, reps, out, (cudaStream_t)stream);
        tune_store(cache_path, key, *out);
    }
    SBC_BATCH_END
}

sbc_status sbc_batch_run(sbc_batch *b, sbc_u128 *out, void *stream) {
    SBC_BATCH_TRY
    if (!b || (!out && b->n)) fail(SBC_E_INVAL, "NULL argument");
    batch_run(b, out, (cudaStream_t)stream);
    SBC_BATCH_END
}

sbc_status sbc_batch_destroy(sbc_batch *b) {
    SBC_BATCH_TRY
    if (!b) return SBC_OK;
    cudaDeviceSynchronize();
    delete b;
    SBC_BATCH_END
}

sbc_status sbc_count_batch(const sbc_graph *const *graphs, size_t n, int p, int q, sbc_u128 *out,
                           void *stream) {
    SBC_BATCH_TRY
    if (!out && n) fail(SBC_E_INVAL, "out is NULL");
    std::unique_ptr<sbc_batch> b(batch_create(graphs, n, p, q, false, nullptr, (cudaStream_t)stream));
    for (size_t i = 0; i < n; i++) out[i] = b->first[i];
    SBC_BATCH_END
}

}  // extern "C"
