// Grid intake, triangle geometry, singular-pair lists and P1 mass matrices
// (paper Sec. 2.4: P1 Lagrange functions on a conforming triangular grid;
//  Sec. 3.1: mass matrix M_ij = <phi_j, theta_i>).
//
// Host side (integer bookkeeping at intake, O(T log T)): validation, the
// consistency of the orientation, the lists of edge- and vertex-adjacent triangle
// pairs with their Sauter-Schwab vertex placement, and the CSR pattern of M.
// Device side: the per-triangle geometry records and all floating-point values.
#include "bem_internal.cuh"

#include <algorithm>
#include <cmath>
#include <map>
#include <unordered_map>

namespace bem {

namespace {

__global__ void k_geometry(const double* __restrict__ xyz, const int32_t* __restrict__ tri, int64_t nt,
                           TriRule R, TriRec* __restrict__ out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double v[3][3];
    for (int a = 0; a < 3; ++a) {
        int32_t id = tri[3 * t + a];
        for (int d = 0; d < 3; ++d) v[a][d] = xyz[3 * (int64_t)id + d];
    }
    double e1[3], e2[3], cr[3];
    for (int d = 0; d < 3; ++d) {
        e1[d] = v[1][d] - v[0][d];
        e2[d] = v[2][d] - v[0][d];
    }
    cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
    cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
    cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
    double J = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    double iJ = 1.0 / J;
    TriRec r;
    for (int d = 0; d < 3; ++d) r.n[d] = cr[d] * iJ;
    r.J = J;
    for (int p = 0; p < 6; ++p) {
        double s = R.s[p], tt = R.t[p];
        for (int d = 0; d < 3; ++d) r.q[p][d] = v[0][d] + s * e1[d] + tt * e2[d];
        double wJ = R.w[p] * J;
        r.wl[p][0] = wJ * (1.0 - s - tt);
        r.wl[p][1] = wJ * s;
        r.wl[p][2] = wJ * tt;
    }
    // surface curl of the shape function of vertex i: (v_{i+1} - v_{i+2}) / J
    for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d) r.curl[a][d] = (v[(a + 1) % 3][d] - v[(a + 2) % 3][d]) * iJ;
    out[t] = r;
}

__global__ void k_mass_values(const TriRec* __restrict__ rec, const int32_t* __restrict__ slot, int64_t nt,
                              double* __restrict__ val) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    // element mass matrix (|tau| / 12) [[2,1,1],[1,2,1],[1,1,2]] with |tau| = J / 2
    double J = rec[t].J;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            atomicAdd(&val[slot[9 * t + 3 * a + b]], (a == b ? 2.0 : 1.0) * J / 24.0);
}

__global__ void k_diag_inverse(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const double* __restrict__ val, int64_t n, double* __restrict__ dinv) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
        if (col[e] == i) dinv[i] = 1.0 / val[e];
}

__global__ void k_geometry32(const double* __restrict__ xyz, const int32_t* __restrict__ tri,
                             const int32_t* __restrict__ order, const TriRec* __restrict__ rec, int64_t nt,
                             TriRec32* __restrict__ out) {
    int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (pos >= nt) return;
    const int64_t t = order[pos];
    double c[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) {
        const int32_t id = tri[3 * t + a];
        for (int d = 0; d < 3; ++d) c[d] += xyz[3 * (int64_t)id + d];
    }
    const TriRec& R = rec[t];
    TriRec32 r;
    for (int d = 0; d < 3; ++d) {
        c[d] /= 3.0;
        r.ch[d] = (float)c[d];
        r.cl[d] = (float)(c[d] - (double)r.ch[d]);
        r.n[d] = (float)R.n[d];
    }
    for (int p = 0; p < 6; ++p)
        for (int d = 0; d < 3; ++d) {
            r.u[p][d] = (float)(R.q[p][d] - c[d]);
            r.wl[p][d] = (float)R.wl[p][d];
        }
    for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d) r.curl[a][d] = (float)R.curl[a][d];
    r.pad[0] = r.pad[1] = 0.f;
    out[pos] = r;
}

// Morton code of a point in the unit cube (21 bits per axis)
uint64_t morton3(double x, double y, double z) {
    auto spread = [](uint64_t v) {
        v &= 0x1fffffull;
        v = (v | (v << 32)) & 0x1f00000000ffffull;
        v = (v | (v << 16)) & 0x1f0000ff0000ffull;
        v = (v | (v << 8)) & 0x100f00f00f00f00full;
        v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
        v = (v | (v << 2)) & 0x1249249249249249ull;
        return v;
    };
    auto q = [](double u) { return (uint64_t)(std::min(std::max(u, 0.0), 1.0) * 2097151.0); };
    return spread(q(x)) | (spread(q(y)) << 1) | (spread(q(z)) << 2);
}

struct Tiles {
    std::vector<int32_t> tstart, vstart, vert;
    std::vector<uint32_t> slots;  // per position
    int64_t total_vertices = 0;
};

// Greedy tiles over a triangle order: a tile takes triangles while it has fewer than
// TILE_TRI of them and at most TILE_NV distinct vertices.
Tiles make_tiles(const std::vector<int32_t>& tri, const std::vector<int32_t>& order) {
    Tiles T;
    const int64_t nt = (int64_t)order.size();
    T.slots.resize(nt);
    std::vector<int32_t> cur;
    int64_t start = 0;
    auto close = [&](int64_t end) {
        T.tstart.push_back((int32_t)start);
        T.vstart.push_back((int32_t)T.vert.size());
        std::vector<int32_t> vs(cur);
        std::sort(vs.begin(), vs.end());
        for (int64_t p = start; p < end; ++p) {
            uint32_t pk = 0;
            for (int a = 0; a < 3; ++a) {
                const int32_t v = tri[3 * (int64_t)order[p] + a];
                const uint32_t sl = (uint32_t)(std::lower_bound(vs.begin(), vs.end(), v) - vs.begin());
                pk |= sl << (8 * a);
            }
            T.slots[p] = pk;
        }
        T.vert.insert(T.vert.end(), vs.begin(), vs.end());
        T.total_vertices += (int64_t)vs.size();
        cur.clear();
        start = end;
    };
    for (int64_t p = 0; p < nt; ++p) {
        const int32_t* tv = &tri[3 * (int64_t)order[p]];
        int add = 0;
        for (int a = 0; a < 3; ++a)
            if (std::find(cur.begin(), cur.end(), tv[a]) == cur.end() &&
                std::find(tv, tv + a, tv[a]) == tv + a)
                ++add;
        if (p > start && (p - start >= TILE_TRI || (int)cur.size() + add > TILE_NV)) close(p);
        for (int a = 0; a < 3; ++a)
            if (std::find(cur.begin(), cur.end(), tv[a]) == cur.end()) cur.push_back(tv[a]);
    }
    close(nt);
    T.tstart.push_back((int32_t)nt);
    T.vstart.push_back((int32_t)T.vert.size());
    return T;
}

}  // namespace

bem_status grid_build_rec32(const bem_grid* g, cudaStream_t s) {
    BEM_LAUNCH(k_geometry32, (unsigned)((g->nt + 127) / 128), 128, 0, s, g->xyz.as<double>(), g->tri.as<int32_t>(),
               g->t_order.as<int32_t>(), g->rec.as<TriRec>(), g->nt, g->rec32.as<TriRec32>());
    return BEM_OK;
}

bem_status grid_build_geometry(bem_grid* g) {
    cudaStream_t s = g->ctx->stream;
    const int64_t nt = g->nt, nv = g->nv;
    // ---- singular pair lists (host) ------------------------------------------------
    std::vector<std::vector<int32_t>> vt(nv);
    for (int64_t t = 0; t < nt; ++t)
        for (int a = 0; a < 3; ++a) vt[g->h_tri[3 * t + a]].push_back((int32_t)t);
    std::vector<SingPair> edges, verts;
    std::vector<int32_t> nb;
    for (int64_t t = 0; t < nt; ++t) {
        nb.clear();
        for (int a = 0; a < 3; ++a)
            for (int32_t s2 : vt[g->h_tri[3 * t + a]])
                if (s2 > t) nb.push_back(s2);
        std::sort(nb.begin(), nb.end());
        nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
        const int32_t* A = &g->h_tri[3 * t];
        for (int32_t s2 : nb) {
            const int32_t* B = &g->h_tri[3 * (int64_t)s2];
            int shared[3], ns = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    if (A[a] == B[b]) shared[ns++] = A[a];
            auto loc = [](const int32_t* T, int v) { return T[0] == v ? 0 : (T[1] == v ? 1 : 2); };
            SingPair P{};
            P.t = (int32_t)t;
            P.s = s2;
            if (ns == 2) {
                int p = std::min(shared[0], shared[1]), q = std::max(shared[0], shared[1]);
                int la = loc(A, p), lb = loc(A, q);
                P.pt[0] = la; P.pt[1] = lb; P.pt[2] = 3 - la - lb;
                la = loc(B, p); lb = loc(B, q);
                P.ps[0] = la; P.ps[1] = lb; P.ps[2] = 3 - la - lb;
                P.kind = 1;
                edges.push_back(P);
            } else if (ns == 1) {
                int la = loc(A, shared[0]);
                P.pt[0] = la; P.pt[1] = (la + 1) % 3; P.pt[2] = (la + 2) % 3;
                la = loc(B, shared[0]);
                P.ps[0] = la; P.ps[1] = (la + 1) % 3; P.ps[2] = (la + 2) % 3;
                P.kind = 2;
                verts.push_back(P);
            } else {
                set_error("internal: triangles with three shared vertices are duplicates");
                return BEM_E_INVALID_ARG;
            }
        }
    }
    g->n_edge = (int64_t)edges.size();
    g->n_vertex = (int64_t)verts.size();
    std::vector<SingPair> all(edges);
    all.insert(all.end(), verts.begin(), verts.end());
    if (!all.empty()) {
        BEM_TRY(g->sing.alloc(all.size() * sizeof(SingPair), s));
        BEM_CUDA_TRY(cudaMemcpyAsync(g->sing.p, all.data(), all.size() * sizeof(SingPair),
                                     cudaMemcpyHostToDevice, s));
    }
    // ---- mass-matrix CSR pattern (host) --------------------------------------------
    std::vector<std::vector<int32_t>> adj(nv);
    for (int64_t v = 0; v < nv; ++v) {
        adj[v].push_back((int32_t)v);
        for (int32_t t : vt[v])
            for (int a = 0; a < 3; ++a) adj[v].push_back(g->h_tri[3 * (int64_t)t + a]);
        std::sort(adj[v].begin(), adj[v].end());
        adj[v].erase(std::unique(adj[v].begin(), adj[v].end()), adj[v].end());
    }
    std::vector<int32_t> rowptr(nv + 1, 0), col;
    for (int64_t v = 0; v < nv; ++v) {
        rowptr[v + 1] = rowptr[v] + (int32_t)adj[v].size();
        col.insert(col.end(), adj[v].begin(), adj[v].end());
    }
    std::vector<int32_t> slot(9 * nt);
    for (int64_t t = 0; t < nt; ++t)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                int32_t i = g->h_tri[3 * t + a], j = g->h_tri[3 * t + b];
                auto it = std::lower_bound(col.begin() + rowptr[i], col.begin() + rowptr[i + 1], j);
                slot[9 * t + 3 * a + b] = (int32_t)(it - col.begin());
            }
    g->m_nnz = (int64_t)col.size();
    g->m_maxrow = 0;
    for (int64_t v = 0; v < nv; ++v) g->m_maxrow = std::max(g->m_maxrow, rowptr[v + 1] - rowptr[v]);
    BEM_TRY(g->m_rowptr.alloc(rowptr.size() * 4, s));
    BEM_TRY(g->m_col.alloc(col.size() * 4, s));
    BEM_TRY(g->m_slot.alloc(slot.size() * 4, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(g->m_rowptr.p, rowptr.data(), rowptr.size() * 4, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(g->m_col.p, col.data(), col.size() * 4, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(g->m_slot.p, slot.data(), slot.size() * 4, cudaMemcpyHostToDevice, s));
    // ---- tiles for the mixed-precision assembly (host) -------------------------------
    // the better of the given order and a Morton order of the centroids (fewer tile vertices)
    std::vector<int32_t> natural(nt), morton(nt);
    for (int64_t t = 0; t < nt; ++t) natural[t] = morton[t] = (int32_t)t;
    {
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int64_t v = 0; v < nv; ++v)
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], g->h_xyz[3 * v + d]);
                hi[d] = std::max(hi[d], g->h_xyz[3 * v + d]);
            }
        std::vector<uint64_t> code(nt);
        for (int64_t t = 0; t < nt; ++t) {
            double c[3] = {0, 0, 0};
            for (int a = 0; a < 3; ++a)
                for (int d = 0; d < 3; ++d) c[d] += g->h_xyz[3 * (int64_t)g->h_tri[3 * t + a] + d] / 3.0;
            double u[3];
            for (int d = 0; d < 3; ++d) u[d] = hi[d] > lo[d] ? (c[d] - lo[d]) / (hi[d] - lo[d]) : 0.0;
            code[t] = morton3(u[0], u[1], u[2]);
        }
        std::stable_sort(morton.begin(), morton.end(), [&](int32_t a, int32_t b) { return code[a] < code[b]; });
    }
    Tiles tn = make_tiles(g->h_tri, natural), tm = make_tiles(g->h_tri, morton);
    const bool use_morton = tm.total_vertices < tn.total_vertices;
    const Tiles& TL = use_morton ? tm : tn;
    const std::vector<int32_t>& order = use_morton ? morton : natural;
    g->ntile = (int64_t)TL.tstart.size() - 1;
    std::vector<int32_t> tverts(3 * nt);
    for (int64_t p = 0; p < nt; ++p)
        for (int a = 0; a < 3; ++a) tverts[3 * p + a] = g->h_tri[3 * (int64_t)order[p] + a];
    BEM_TRY(g->t_order.alloc(nt * 4, s));
    BEM_TRY(g->t_verts.alloc(nt * 12, s));
    BEM_TRY(g->t_slots.alloc(nt * 4, s));
    BEM_TRY(g->tile_tstart.alloc(TL.tstart.size() * 4, s));
    BEM_TRY(g->tile_vstart.alloc(TL.vstart.size() * 4, s));
    BEM_TRY(g->tile_vert.alloc(TL.vert.size() * 4, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(g->t_order.p, order.data(), nt * 4, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(g->t_verts.p, tverts.data(), nt * 12, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(g->t_slots.p, TL.slots.data(), nt * 4, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(g->tile_tstart.p, TL.tstart.data(), TL.tstart.size() * 4, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(g->tile_vstart.p, TL.vstart.data(), TL.vstart.size() * 4, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(g->tile_vert.p, TL.vert.data(), TL.vert.size() * 4, cudaMemcpyHostToDevice, s));
    // ---- geometry records (device) -------------------------------------------------
    BEM_TRY(g->rec.alloc(nt * sizeof(TriRec), s));
    BEM_LAUNCH(k_geometry, (unsigned)((nt + 127) / 128), 128, 0, s, g->xyz.as<double>(), g->tri.as<int32_t>(), nt,
                                                          tri_rule_degree4(), g->rec.as<TriRec>());
    BEM_TRY(g->rec32.alloc(nt * sizeof(TriRec32), s));
    BEM_TRY(grid_build_rec32(g, s));
    // the host vectors above must outlive the asynchronous copies
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    return BEM_OK;
}

bem_status mass_values(const bem_grid* g, double* d_val, cudaStream_t s) {
    BEM_CUDA_TRY(cudaMemsetAsync(d_val, 0, g->m_nnz * sizeof(double), s));
    BEM_LAUNCH(k_mass_values, (unsigned)((g->nt + 127) / 128), 128, 0, s, g->rec.as<TriRec>(), g->m_slot.as<int32_t>(),
                                                                 g->nt, d_val);
    BEM_CHECK_LAUNCH();
    return BEM_OK;
}

bem_status mass_inverse_diag(const bem_grid* g, const double* d_val, double* d_dinv, cudaStream_t s) {
    BEM_LAUNCH(k_diag_inverse, (unsigned)((g->nv + 127) / 128), 128, 0, s, g->m_rowptr.as<int32_t>(), g->m_col.as<int32_t>(),
                                                                  d_val, g->nv, d_dinv);
    BEM_CHECK_LAUNCH();
    return BEM_OK;
}

}  // namespace bem
