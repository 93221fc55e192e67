// Counts kept exact under edge insertions, deletions and sign changes (the
// dynamic setting the paper leaves to future work, Section 6).
//
// An update of edge (u, v) changes the count by the balanced (p,q)-bicliques
// that contain (u, v). Such a biclique is L = {u} + L', R = {v} + R' with
// L' a (p-1)-subset of Gamma(v) - {u}, R' a (q-1)-subset of Gamma(u) - {v},
// L x R complete. It is balanced (Section 3: no butterfly with an odd number
// of negative edges) exactly when every butterfly (u, w, v, x), w in L',
// x in R', is: a butterfly (u, w, x, x') is the product of (u, w, v, x) and
// (u, w, v, x'), and a butterfly (w, w', x, x') the product of (u, w, x, x')
// and (u, w', x, x'). So the contribution of (u, v) is the number of complete
// (p-1, q-1) bipartite subgraphs of the local graph H(u, v) on
// Gamma(v) - {u} and Gamma(u) - {v} whose edges are the (w, x) in E with
// sign(u,v) sign(u,x) sign(w,v) sign(w,x) = +1, i.e. the balanced
// (p-1, q-1) count of H with every sign positive, which the counting kernels
// compute. p and q must be at least 3 so that p-1 and q-1 are valid sizes.
//
// The adjacency is kept on the host (sorted lists per vertex, the mutable
// state of the graph); H is assembled on the host from Gamma(w) and Gamma(u)
// for every w in Gamma(v) (a merge, or binary searches into Gamma(u) when
// Gamma(w) is much shorter), then uploaded and counted on the GPU.
#include <algorithm>
#include <memory>
#include <utility>
#include <vector>

#include "sbc_internal.cuh"

namespace sbc {

namespace {

typedef std::vector<std::pair<int32_t, int8_t>> AdjList;  // (neighbour, sign), by neighbour

struct Csr {
    int64_t n_l = 0, n_r = 0;
    std::vector<int64_t> off;
    std::vector<int32_t> col;
};

int8_t sign_in(const AdjList &a, int32_t x) {
    auto it = std::lower_bound(a.begin(), a.end(), std::make_pair(x, (int8_t)-128));
    return it != a.end() && it->first == x ? it->second : 0;
}

// H(u, v) for an edge of sign s_uv: rows Gamma(v) - {u} in the order of
// adj_v[v], columns Gamma(u) - {v} in the order of adj_u[u].
Csr local_graph(const std::vector<AdjList> &adj_u, const std::vector<AdjList> &adj_v, int32_t u,
                int32_t v, int8_t s_uv) {
    const AdjList &Nu = adj_u[u], &Nv = adj_v[v];
    Csr h;
    std::vector<int32_t> col_of(Nu.size());  // column index of Nu[i] (-1 for v)
    for (size_t i = 0; i < Nu.size(); i++) {
        col_of[i] = Nu[i].first == v ? -1 : (int32_t)h.n_r;
        if (Nu[i].first != v) h.n_r++;
    }
    h.off.push_back(0);
    for (const auto &wv : Nv) {
        const int32_t w = wv.first;
        if (w == u) continue;
        const int8_t s_wv = wv.second;
        const AdjList &Nw = adj_u[w];
        auto keep = [&](size_t i, int8_t s_wx) {
            if (col_of[i] >= 0 && s_uv * Nu[i].second * s_wv * s_wx == 1) h.col.push_back(col_of[i]);
        };
        if (8 * Nw.size() < Nu.size()) {
            // Gamma(w) much shorter: look each of its vertices up in Gamma(u)
            for (const auto &xs : Nw) {
                auto it = std::lower_bound(Nu.begin(), Nu.end(), std::make_pair(xs.first, (int8_t)-128));
                if (it != Nu.end() && it->first == xs.first) keep((size_t)(it - Nu.begin()), xs.second);
            }
        } else {
            size_t i = 0, j = 0;  // merge Gamma(u) with Gamma(w), both by V id
            while (i < Nu.size() && j < Nw.size()) {
                if (Nu[i].first < Nw[j].first) {
                    i++;
                } else if (Nw[j].first < Nu[i].first) {
                    j++;
                } else {
                    keep(i, Nw[j].second);
                    i++;
                    j++;
                }
            }
        }
        h.off.push_back((int64_t)h.col.size());
        h.n_l++;
    }
    return h;
}

// Balanced (p-1, q-1) count of H with every sign positive.
U128 local_count(const Csr &h, int p, int q, cudaStream_t s) {
    U128 r;
    if (h.col.empty() || h.n_l < p - 1 || h.n_r < q - 1) return r;
    std::vector<int8_t> plus(h.col.size(), 1);
    std::unique_ptr<sbc_graph> g(create_graph(h.n_l, h.n_r, (int64_t)h.col.size(), h.off.data(),
                                              h.col.data(), plus.data(), SBC_OFFS_I64, s));
    sbc_count_stats st;
    count_graph(g.get(), p - 1, q - 1, nullptr, &st, s);
    r.lo = st.count.lo;
    r.hi = st.count.hi;
    return r;
}

typedef unsigned __int128 u128_t;
u128_t wide(const U128 &a) { return ((u128_t)a.hi << 64) | a.lo; }
U128 narrow(u128_t x) {
    U128 r;
    r.lo = (unsigned long long)x;
    r.hi = (unsigned long long)(x >> 64);
    return r;
}

bool add_u128(U128 &a, const U128 &b) {  // false on overflow
    const u128_t s = wide(a) + wide(b);
    if (s < wide(a)) return false;
    a = narrow(s);
    return true;
}

bool sub_u128(U128 &a, const U128 &b) {  // false when b > a
    if (wide(b) > wide(a)) return false;
    a = narrow(wide(a) - wide(b));
    return true;
}

void check_vertices(int64_t n_u, int64_t n_v, int64_t u, int64_t v) {
    if (u < 0 || u >= n_u || v < 0 || v >= n_v)
        fail(SBC_E_INVAL, "edge (%lld, %lld) outside the graph's %lld x %lld vertices", (long long)u,
             (long long)v, (long long)n_u, (long long)n_v);
}

// Sorted adjacency of both sides from a host CSR with int8 signs.
void build_adjacency(int64_t n_u, int64_t n_v, int64_t nnz, const int64_t *off, const int32_t *col,
                     const int8_t *sgn, std::vector<AdjList> &adj_u, std::vector<AdjList> &adj_v) {
    if (n_u < 0 || n_v < 0 || n_u >= (1ll << 31) || n_v >= (1ll << 31))
        fail(SBC_E_INVAL, "vertex counts out of range");
    if ((n_u > 0 || nnz > 0) && (!off || (nnz > 0 && (!col || !sgn))))
        fail(SBC_E_INVAL, "NULL CSR array");
    if (nnz < 0 || (n_u == 0 && nnz != 0) || (n_u > 0 && (off[0] != 0 || off[n_u] != nnz)))
        fail(SBC_E_GRAPH, "offsets do not span the edges");
    adj_u.assign((size_t)n_u, AdjList());
    adj_v.assign((size_t)n_v, AdjList());
    for (int64_t x = 0; x < n_u; x++) {
        if (off[x + 1] < off[x]) fail(SBC_E_GRAPH, "offsets decrease at row %lld", (long long)x);
        for (int64_t e = off[x]; e < off[x + 1]; e++) {
            if (col[e] < 0 || col[e] >= n_v) fail(SBC_E_GRAPH, "column id out of range at edge %lld", (long long)e);
            if (sgn[e] != 1 && sgn[e] != -1) fail(SBC_E_GRAPH, "sign not +1 / -1 at edge %lld", (long long)e);
            adj_u[x].push_back({col[e], sgn[e]});
            adj_v[col[e]].push_back({(int32_t)x, sgn[e]});
        }
        std::sort(adj_u[x].begin(), adj_u[x].end());
        for (size_t i = 1; i < adj_u[x].size(); i++)
            if (adj_u[x][i].first == adj_u[x][i - 1].first)
                fail(SBC_E_GRAPH, "duplicate edge (%lld, %d)", (long long)x, adj_u[x][i].first);
    }
    for (auto &a : adj_v) std::sort(a.begin(), a.end());
}

}  // namespace

}  // namespace sbc

using namespace sbc;

struct sbc_dyn {
    int64_t n_u = 0, n_v = 0, nnz = 0;
    int p = 0, q = 0;
    std::vector<AdjList> adj_u, adj_v;
    U128 count;
};

#define SBC_DYN_TRY try {
#define SBC_DYN_END                           \
    }                                         \
    catch (const SbcError &e) {               \
        set_last_error(e.what());             \
        return e.status;                      \
    }                                         \
    catch (const std::bad_alloc &) {          \
        set_last_error("host allocation failed"); \
        return SBC_E_NOMEM;                   \
    }                                         \
    catch (const std::exception &e) {         \
        set_last_error(e.what());             \
        return SBC_E_CUDA;                    \
    }                                         \
    return SBC_OK;

extern "C" {

sbc_status sbc_dyn_create(sbc_dyn **out, int64_t n_u, int64_t n_v, int64_t nnz,
                          const int64_t *row_offsets, const int32_t *cols, const int8_t *signs,
                          int p, int q, void *stream) {
    SBC_DYN_TRY
    if (!out) fail(SBC_E_INVAL, "out is NULL");
    *out = nullptr;
    if (p < 3 || q < 3 || p > 8 || q > 8) fail(SBC_E_INVAL, "p and q must be in [3, 8]");
    std::unique_ptr<sbc_dyn> d(new sbc_dyn());
    d->n_u = n_u;
    d->n_v = n_v;
    d->nnz = nnz;
    d->p = p;
    d->q = q;
    build_adjacency(n_u, n_v, nnz, row_offsets, cols, signs, d->adj_u, d->adj_v);
    std::unique_ptr<sbc_graph> g(create_graph(n_u, n_v, nnz, row_offsets, cols, signs, SBC_OFFS_I64,
                                              (cudaStream_t)stream));
    sbc_count_stats st;
    count_graph(g.get(), p, q, nullptr, &st, (cudaStream_t)stream);
    d->count.lo = st.count.lo;
    d->count.hi = st.count.hi;
    *out = d.release();
    SBC_DYN_END
}

sbc_status sbc_dyn_update(sbc_dyn *d, int op, int64_t u, int64_t v, int8_t sign, sbc_u128 *count,
                          void *stream) {
    SBC_DYN_TRY
    if (!d) fail(SBC_E_INVAL, "handle is NULL");
    check_vertices(d->n_u, d->n_v, u, v);
    const cudaStream_t s = (cudaStream_t)stream;
    AdjList &Nu = d->adj_u[u], &Nv = d->adj_v[v];
    const int8_t cur = sign_in(Nu, (int32_t)v);
    U128 next = d->count;
    if (op == SBC_DYN_INSERT) {
        if (cur) fail(SBC_E_INVAL, "edge (%lld, %lld) already present", (long long)u, (long long)v);
        if (sign != 1 && sign != -1) fail(SBC_E_INVAL, "sign must be +1 or -1");
        const U128 add = local_count(local_graph(d->adj_u, d->adj_v, (int32_t)u, (int32_t)v, sign), d->p, d->q, s);
        if (!add_u128(next, add)) fail(SBC_E_OVERFLOW, "balanced biclique count exceeds 128 bits");
        Nu.insert(std::lower_bound(Nu.begin(), Nu.end(), std::make_pair((int32_t)v, (int8_t)-128)),
                  {(int32_t)v, sign});
        Nv.insert(std::lower_bound(Nv.begin(), Nv.end(), std::make_pair((int32_t)u, (int8_t)-128)),
                  {(int32_t)u, sign});
        d->nnz++;
    } else if (op == SBC_DYN_DELETE) {
        if (!cur) fail(SBC_E_INVAL, "edge (%lld, %lld) not present", (long long)u, (long long)v);
        const U128 sub = local_count(local_graph(d->adj_u, d->adj_v, (int32_t)u, (int32_t)v, cur), d->p, d->q, s);
        if (!sub_u128(next, sub)) fail(SBC_E_CUDA, "internal error: count below an edge's share");
        Nu.erase(std::lower_bound(Nu.begin(), Nu.end(), std::make_pair((int32_t)v, (int8_t)-128)));
        Nv.erase(std::lower_bound(Nv.begin(), Nv.end(), std::make_pair((int32_t)u, (int8_t)-128)));
        d->nnz--;
    } else if (op == SBC_DYN_SET_SIGN) {
        if (!cur) fail(SBC_E_INVAL, "edge (%lld, %lld) not present", (long long)u, (long long)v);
        if (sign != 1 && sign != -1) fail(SBC_E_INVAL, "sign must be +1 or -1");
        if (sign != cur) {
            const U128 sub = local_count(local_graph(d->adj_u, d->adj_v, (int32_t)u, (int32_t)v, cur), d->p, d->q, s);
            const U128 add = local_count(local_graph(d->adj_u, d->adj_v, (int32_t)u, (int32_t)v, sign), d->p, d->q, s);
            if (!sub_u128(next, sub)) fail(SBC_E_CUDA, "internal error: count below an edge's share");
            if (!add_u128(next, add)) fail(SBC_E_OVERFLOW, "balanced biclique count exceeds 128 bits");
            std::lower_bound(Nu.begin(), Nu.end(), std::make_pair((int32_t)v, (int8_t)-128))->second = sign;
            std::lower_bound(Nv.begin(), Nv.end(), std::make_pair((int32_t)u, (int8_t)-128))->second = sign;
        }
    } else {
        fail(SBC_E_INVAL, "unknown update %d", op);
    }
    d->count = next;
    if (count) {
        count->lo = next.lo;
        count->hi = next.hi;
    }
    SBC_DYN_END
}

sbc_status sbc_dyn_count(const sbc_dyn *d, sbc_u128 *count, int64_t *nnz) {
    SBC_DYN_TRY
    if (!d || !count) fail(SBC_E_INVAL, "NULL argument");
    count->lo = d->count.lo;
    count->hi = d->count.hi;
    if (nnz) *nnz = d->nnz;
    SBC_DYN_END
}

sbc_status sbc_dyn_destroy(sbc_dyn *d) {
    delete d;
    return SBC_OK;
}

sbc_status sbc_edge_local_graph(int64_t n_u, int64_t n_v, int64_t nnz, const int64_t *row_offsets,
                                const int32_t *cols, const int8_t *signs, int64_t u, int64_t v,
                                int8_t sign, int64_t *n_l, int64_t *n_r, int64_t *h_nnz,
                                int64_t *h_offsets, int32_t *h_cols, int64_t capacity) {
    SBC_DYN_TRY
    if (!n_l || !n_r || !h_nnz) fail(SBC_E_INVAL, "NULL argument");
    if (sign != 1 && sign != -1) fail(SBC_E_INVAL, "sign must be +1 or -1");
    check_vertices(n_u, n_v, u, v);
    std::vector<AdjList> adj_u, adj_v;
    build_adjacency(n_u, n_v, nnz, row_offsets, cols, signs, adj_u, adj_v);
    const Csr h = local_graph(adj_u, adj_v, (int32_t)u, (int32_t)v, sign);
    *n_l = h.n_l;
    *n_r = h.n_r;
    *h_nnz = (int64_t)h.col.size();
    if (h_offsets) {
        if (capacity < (int64_t)h.col.size()) fail(SBC_E_INVAL, "capacity below the local graph's edges");
        std::copy(h.off.begin(), h.off.end(), h_offsets);
        if (h_cols) std::copy(h.col.begin(), h.col.end(), h_cols);
    }
    SBC_DYN_END
}

}  // extern "C"
