// Device-side graph construction.
//
// Input model (Section 3): a signed bipartite graph G = (U, V, E), every edge
// carrying a sign. The caller hands a CSR over U; this file validates it,
// computes degrees on both sides, and builds for an anchor side X the
// structures Algorithm 2 walks:
//   A: X -> Y adjacency with X renumbered by the vertex priority rho of
//      Definition 4 (ascending degree, ties by ascending id);
//   B: Y -> X adjacency, each list ascending in rank, so that the partners w
//      of an anchor u with rho(w) > rho(u) in the list of v are the suffix
//      after u's own entry (Algorithm 2, "for each w in Gamma(v) with
//      rho(w) > rho(u)");
//   A_pos: for each A entry (u, v), the index of the mirror entry in B's list
//      of v, which locates that suffix without a search.
// Edge signs travel as bit 31 of each adjacency entry (1 = negative).
#include "sbc_internal.cuh"

namespace sbc {

namespace {

enum : uint32_t {
    ERR_OFF0 = 1u << 0,      // row_offsets[0] != 0
    ERR_OFFMONO = 1u << 1,   // decreasing offsets
    ERR_OFFEND = 1u << 2,    // row_offsets[n_u] != nnz
    ERR_COL = 1u << 3,       // column id out of range
    ERR_SIGN = 1u << 4,      // sign not +1 / -1
    ERR_DUP = 1u << 5,       // duplicate (u, v)
};

__global__ void k_offsets_to_i64(const void *in, int is64, int64_t n1, int64_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n1;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = is64 ? ((const int64_t *)in)[i] : (int64_t)((const int32_t *)in)[i];
}

__global__ void k_check_offsets(const int64_t *off, int64_t n_u, int64_t nnz, uint32_t *err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_u;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (off[i + 1] < off[i]) atomicOr(err, ERR_OFFMONO);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (off[0] != 0) atomicOr(err, ERR_OFF0);
        if (off[n_u] != nnz) atomicOr(err, ERR_OFFEND);
    }
}

// Signs from int8 +-1 (sign_bits == 0) or packed bits; column range check;
// V-side degree histogram.
__global__ void k_edges(const int32_t *col, const void *signs, int sign_bits, int64_t nnz,
                        int64_t n_v, uint8_t *neg, int32_t *deg_v, uint32_t *err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        uint8_t ng;
        if (sign_bits) {
            ng = (((const uint8_t *)signs)[e >> 3] >> (e & 7)) & 1u;
        } else {
            int8_t s = ((const int8_t *)signs)[e];
            if (s != 1 && s != -1) atomicOr(err, ERR_SIGN);
            ng = s < 0;
        }
        neg[e] = ng;
        int32_t c = col[e];
        if (c < 0 || c >= n_v) {
            atomicOr(err, ERR_COL);
        } else {
            atomicAdd(&deg_v[c], 1);
        }
    }
}

// Degrees of U, and per side: maximum degree and sum of binom(deg, 2).
__global__ void k_deg_u(const int64_t *off, int64_t n_u, int32_t *deg_u) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_u;
         i += (int64_t)gridDim.x * blockDim.x)
        deg_u[i] = (int32_t)(off[i + 1] - off[i]);
}

__global__ void k_deg_stats(const int32_t *deg, int64_t n, unsigned long long *out /* [2]: pairs, max */) {
    unsigned long long pairs = 0, mx = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long d = (unsigned long long)deg[i];
        pairs += d * (d - (d ? 1 : 0)) / 2;
        mx = d > mx ? d : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
        unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = t > mx ? t : mx;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], pairs);
        atomicMax(&out[1], mx);
    }
}

// Row id of every edge (warp per row).
__global__ void k_edge_rows(const int64_t *off, int64_t n_u, uint32_t *erow) {
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < n_u; u += nwarps)
        for (int64_t e = off[u] + lane; e < off[u + 1]; e += 32) erow[e] = (uint32_t)u;
}

__global__ void k_iota_deg(const int32_t *deg, int64_t n, uint32_t *keys, uint32_t *vals) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        keys[i] = (uint32_t)deg[i];
        vals[i] = (uint32_t)i;
    }
}

// vert_of (rank -> vertex) is the sorted value array; invert it and gather the
// degrees in rank order (n+1 entries, last 0, for the offset scan).
__global__ void k_rank_tables(const uint32_t *sorted_vertex, const int32_t *deg, int64_t n,
                              int32_t *vert_of, uint32_t *rank_of, int64_t *deg_by_rank) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= n;
         r += (int64_t)gridDim.x * blockDim.x) {
        if (r == n) {
            deg_by_rank[n] = 0;
            continue;
        }
        uint32_t x = sorted_vertex[r];
        vert_of[r] = (int32_t)x;
        rank_of[x] = (uint32_t)r;
        deg_by_rank[r] = deg[x];
    }
}

// keys = rank of the X end of every edge, vals = edge index.
__global__ void k_edge_rank_keys(const int32_t *col, const uint32_t *erow, const uint32_t *rank_of,
                                 int x_is_v, int64_t nnz, uint32_t *keys, uint32_t *vals) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        uint32_t x = x_is_v ? (uint32_t)col[e] : erow[e];
        keys[e] = rank_of[x];
        vals[e] = (uint32_t)e;
    }
}

// A entries in rank-major order; keys for the B sort (Y id) and its values
// (A index).
__global__ void k_fill_A(const uint32_t *edge_of_a, const int32_t *col, const uint32_t *erow,
                         const uint8_t *neg, int x_is_v, int64_t nnz, uint32_t *A_ent,
                         uint32_t *bkeys, uint32_t *bvals) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t e = edge_of_a[i];
        uint32_t y = x_is_v ? erow[e] : (uint32_t)col[e];
        A_ent[i] = y | ((uint32_t)neg[e] << 31);
        bkeys[i] = y;
        bvals[i] = (uint32_t)i;
    }
}

// B entries (rank of the X end + sign), mirror positions, duplicate check.
__global__ void k_fill_B(const uint32_t *a_of_b, const uint32_t *y_of_b, const uint32_t *a_rank,
                         const uint32_t *A_ent, const int64_t *B_off, int64_t nnz, uint32_t *B_ent,
                         uint32_t *A_pos, uint32_t *err) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nnz;
         b += (int64_t)gridDim.x * blockDim.x) {
        uint32_t i = a_of_b[b];
        uint32_t y = y_of_b[b];
        uint32_t r = a_rank[i];
        B_ent[b] = r | (A_ent[i] & 0x80000000u);
        int64_t start = B_off[y];
        A_pos[i] = (uint32_t)(b - start);
        if (b > start && a_rank[a_of_b[b - 1]] == r) atomicOr(err, ERR_DUP);
    }
}

std::string graph_error_text(uint32_t e) {
    std::string s;
    if (e & ERR_OFF0) s += " row_offsets[0] != 0;";
    if (e & ERR_OFFMONO) s += " row_offsets decrease;";
    if (e & ERR_OFFEND) s += " row_offsets[n_u] != nnz;";
    if (e & ERR_COL) s += " column id out of [0, n_v);";
    if (e & ERR_SIGN) s += " sign not +1/-1;";
    if (e & ERR_DUP) s += " duplicate edge (u, v);";
    return s;
}

uint32_t read_err(uint32_t *d_err, cudaStream_t s) {
    uint32_t h = 0;
    SBC_CUDA(cudaMemcpyAsync(&h, d_err, sizeof(h), cudaMemcpyDeviceToHost, s));
    SBC_CUDA(cudaStreamSynchronize(s));
    return h;
}

}  // namespace

void build_orientation(sbc_graph *g, int x, cudaStream_t s) {
    Orient &o = g->side[x];
    if (o.built) return;
    const int64_t nnz = g->nnz;
    const int x_is_v = x == 1;
    o.nX = x_is_v ? g->n_v : g->n_u;
    o.nY = x_is_v ? g->n_u : g->n_v;
    o.max_deg_x = x_is_v ? g->max_deg_v : g->max_deg_u;
    o.max_deg_y = x_is_v ? g->max_deg_u : g->max_deg_v;
    const int32_t *degX = x_is_v ? g->deg_v.ptr : g->deg_u.ptr;
    const int32_t *degY = x_is_v ? g->deg_u.ptr : g->deg_v.ptr;
    const int B = 256;

    o.A_off.alloc(o.nX + 1, s);
    o.B_off.alloc(o.nY + 1, s);
    o.vert_of.alloc(o.nX, s);
    o.A_ent.alloc(nnz, s);
    o.A_pos.alloc(nnz, s);
    o.B_ent.alloc(nnz, s);

    DevBuf<uint32_t> err(1, s);
    SBC_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(uint32_t), s));

    // rank: stable sort of X vertices by degree (Definition 4)
    {
        int64_t n = o.nX;
        DevBuf<uint32_t> k(n, s), v(n, s), tk(n, s), tv(n, s);
        DevBuf<uint32_t> rank_of(n, s);
        DevBuf<int64_t> deg_by_rank(n + 1, s);
        if (n > 0) {
            k_iota_deg<<<grid_for(n, B), B, 0, s>>>(degX, n, k.ptr, v.ptr);
            SBC_LAUNCHED();
            g_launches++;
            radix_sort_pairs(k.ptr, v.ptr, tk.ptr, tv.ptr, n, bits_for((uint64_t)o.max_deg_x), s);
        }
        k_rank_tables<<<grid_for(n + 1, B), B, 0, s>>>(v.ptr, degX, n, o.vert_of.ptr, rank_of.ptr,
                                                       deg_by_rank.ptr);
        SBC_LAUNCHED();
        g_launches++;
        scan_exclusive_i64(deg_by_rank.ptr, o.A_off.ptr, n + 1, nullptr, s);

        // Y offsets: degrees of Y in id order
        DevBuf<int64_t> degy(o.nY + 1, s);
        if (o.nY > 0) {
            k_offsets_to_i64<<<grid_for(o.nY, B), B, 0, s>>>(degY, 0, o.nY, degy.ptr);
            SBC_LAUNCHED();
            g_launches++;
        }
        SBC_CUDA(cudaMemsetAsync(degy.ptr + o.nY, 0, sizeof(int64_t), s));
        scan_exclusive_i64(degy.ptr, o.B_off.ptr, o.nY + 1, nullptr, s);

        if (nnz > 0) {
            DevBuf<uint32_t> erow(nnz, s);
            k_edge_rows<<<grid_for(g->n_u * 32, B), B, 0, s>>>(g->off.ptr, g->n_u, erow.ptr);
            SBC_LAUNCHED();
            g_launches++;
            // A order: edges stably sorted by the rank of their X end
            DevBuf<uint32_t> ak(nnz, s), av(nnz, s), t1(nnz, s), t2(nnz, s);
            k_edge_rank_keys<<<grid_for(nnz, B), B, 0, s>>>(g->col.ptr, erow.ptr, rank_of.ptr,
                                                            x_is_v, nnz, ak.ptr, av.ptr);
            SBC_LAUNCHED();
            g_launches++;
            radix_sort_pairs(ak.ptr, av.ptr, t1.ptr, t2.ptr, nnz, bits_for((uint64_t)(n - 1)), s);
            // B order: A entries stably sorted by Y id (rank order kept within a list)
            DevBuf<uint32_t> bk(nnz, s), bv(nnz, s);
            k_fill_A<<<grid_for(nnz, B), B, 0, s>>>(av.ptr, g->col.ptr, erow.ptr, g->neg.ptr,
                                                    x_is_v, nnz, o.A_ent.ptr, bk.ptr, bv.ptr);
            SBC_LAUNCHED();
            g_launches++;
            radix_sort_pairs(bk.ptr, bv.ptr, t1.ptr, t2.ptr, nnz, bits_for((uint64_t)(o.nY - 1)), s);
            k_fill_B<<<grid_for(nnz, B), B, 0, s>>>(bv.ptr, bk.ptr, ak.ptr, o.A_ent.ptr,
                                                    o.B_off.ptr, nnz, o.B_ent.ptr, o.A_pos.ptr,
                                                    err.ptr);
            SBC_LAUNCHED();
            g_launches++;
        }
    }
    uint32_t e = read_err(err.ptr, s);
    if (e) fail(SBC_E_GRAPH, "invalid graph:%s", graph_error_text(e).c_str());
    o.built = true;
}

}  // namespace sbc




namespace sbc {

// Upload, validate and prepare a graph; builds the orientation of the side
// the cost model prefers (which also checks for duplicate edges).
sbc_graph *create_graph(int64_t n_u, int64_t n_v, int64_t nnz, const void *row_offsets,
                        const int32_t *cols, const void *signs, uint32_t flags, cudaStream_t s) {
    NvtxRange nr("sbc/create_graph");
    if (n_u < 0 || n_v < 0 || nnz < 0) fail(SBC_E_INVAL, "negative size");
    if (n_u >= (1ll << 31) - 1 || n_v >= (1ll << 31) - 1 || nnz >= (1ll << 31) - 1)
        fail(SBC_E_UNSUPPORTED, "sizes must be below 2^31 - 1");
    if (!row_offsets) fail(SBC_E_INVAL, "row_offsets is NULL");
    if (nnz > 0 && (!cols || !signs)) fail(SBC_E_INVAL, "cols or signs is NULL");
    const bool dev = flags & SBC_DEVICE_PTRS;
    const bool off64 = flags & SBC_OFFS_I64;
    const bool bits = flags & SBC_SIGN_BITS;
    const int B = 256;

    std::unique_ptr<sbc_graph> g(new sbc_graph());
    SBC_CUDA(cudaGetDevice(&g->device));
    g->n_u = n_u;
    g->n_v = n_v;
    g->nnz = nnz;
    g->off.alloc(n_u + 1, s);
    g->col.alloc(nnz, s);
    g->neg.alloc(nnz, s);
    g->deg_u.alloc(n_u, s);
    g->deg_v.alloc(n_v, s);

    const size_t off_bytes = (size_t)(n_u + 1) * (off64 ? 8 : 4);
    const size_t sign_bytes = bits ? (size_t)((nnz + 7) / 8) : (size_t)nnz;
    DevBuf<uint8_t> off_in, sign_in;
    const void *d_off = row_offsets;
    const void *d_sign = signs;
    if (!dev) {
        off_in.alloc(off_bytes, s);
        SBC_CUDA(cudaMemcpyAsync(off_in.ptr, row_offsets, off_bytes, cudaMemcpyHostToDevice, s));
        d_off = off_in.ptr;
        if (nnz > 0) {
            SBC_CUDA(cudaMemcpyAsync(g->col.ptr, cols, (size_t)nnz * 4, cudaMemcpyHostToDevice, s));
            sign_in.alloc(sign_bytes, s);
            SBC_CUDA(cudaMemcpyAsync(sign_in.ptr, signs, sign_bytes, cudaMemcpyHostToDevice, s));
            d_sign = sign_in.ptr;
        }
    } else if (nnz > 0) {
        SBC_CUDA(cudaMemcpyAsync(g->col.ptr, cols, (size_t)nnz * 4, cudaMemcpyDeviceToDevice, s));
    }

    DevBuf<uint32_t> err(1, s);
    DevBuf<unsigned long long> st(4, s);
    SBC_CUDA(cudaMemsetAsync(err.ptr, 0, 4, s));
    SBC_CUDA(cudaMemsetAsync(st.ptr, 0, 32, s));
    if (n_v > 0) SBC_CUDA(cudaMemsetAsync(g->deg_v.ptr, 0, (size_t)n_v * 4, s));
    k_offsets_to_i64<<<grid_for(n_u + 1, B), B, 0, s>>>(d_off, off64, n_u + 1, g->off.ptr);
    SBC_LAUNCHED();
    k_check_offsets<<<grid_for(n_u, B), B, 0, s>>>(g->off.ptr, n_u, nnz, err.ptr);
    SBC_LAUNCHED();
    g_launches += 2;
    if (uint32_t e = read_err(err.ptr, s)) fail(SBC_E_GRAPH, "invalid graph:%s", graph_error_text(e).c_str());
    if (nnz > 0) {
        k_edges<<<grid_for(nnz, B), B, 0, s>>>(g->col.ptr, d_sign, bits, nnz, n_v, g->neg.ptr,
                                               g->deg_v.ptr, err.ptr);
        SBC_LAUNCHED();
        g_launches++;
    }
    if (n_u > 0) {
        k_deg_u<<<grid_for(n_u, B), B, 0, s>>>(g->off.ptr, n_u, g->deg_u.ptr);
        SBC_LAUNCHED();
        k_deg_stats<<<grid_for(n_u, B), B, 0, s>>>(g->deg_u.ptr, n_u, st.ptr);
        SBC_LAUNCHED();
        g_launches += 2;
    }
    if (n_v > 0) {
        k_deg_stats<<<grid_for(n_v, B), B, 0, s>>>(g->deg_v.ptr, n_v, st.ptr + 2);
        SBC_LAUNCHED();
        g_launches++;
    }
    unsigned long long hst[4];
    SBC_CUDA(cudaMemcpyAsync(hst, st.ptr, sizeof(hst), cudaMemcpyDeviceToHost, s));
    if (uint32_t e = read_err(err.ptr, s)) fail(SBC_E_GRAPH, "invalid graph:%s", graph_error_text(e).c_str());
    g->wedges_v = hst[0];  // anchoring on V visits 2-paths through U
    g->max_deg_u = (int64_t)hst[1];
    g->wedges_u = hst[2];  // anchoring on U visits 2-paths through V
    g->max_deg_v = (int64_t)hst[3];
    off_in.release();
    sign_in.release();
    // the preferred side's orientation also checks for duplicate edges
    int side = g->wedges_u <= g->wedges_v ? 0 : 1;
    build_orientation(g.get(), side, s);
    SBC_CUDA(cudaStreamSynchronize(s));
    return g.release();
}

int preferred_side(const sbc_graph *g, int p, int q) {
    const int by_wedges = g->wedges_u <= g->wedges_v ? 0 : 1;
    // anchoring on U gives tuples of p, on V of q
    const bool u3 = p == 3 && q >= 4, v3 = q == 3 && p >= 4;
    if (!u3 && !v3) return by_wedges;
    const int side3 = u3 ? 0 : 1;
    const uint64_t w3 = side3 == 0 ? g->wedges_u : g->wedges_v;
    const uint64_t wo = side3 == 0 ? g->wedges_v : g->wedges_u;
    return w3 / 64 <= wo ? side3 : by_wedges;
}

}  // namespace sbc
