// Mortar matrix P_ab between two nonconforming grids (paper Sec. 3.1: entry (i, j)
// is the L2 product of test function i of grid a and basis function j of grid b
// over the common surface; P_ba = P_ab^T, Sec. 5.4).
//
// The paper's grids share one polyhedral surface; two grids of a curved surface do
// not, so the common surface is read through central projection from a centre c0
// (both surfaces star-shaped about it).  For each triangle tau of a, each triangle
// sigma of b is projected onto the plane of tau along rays from c0 (lines map to
// lines, so the image sigma' is a triangle); on tau, basis j of b is the linear
// barycentric function of sigma'.  The integrand lambda_i^tau lambda_j^sigma' is
// quadratic, so the integral over tau cap sigma' is exact under any triangulation.
//
// Data-parallel replacement of the serial advancing front (PANG) of Sec. 3.2:
//   1. prefilter: every (tau, sigma) pair is tested against a conservative bound
//      on the angles seen from c0 (projected triangles can only overlap if their
//      angular discs meet), in FP32 with a widened radius;
//   2. one thread per candidate: projection, Sutherland-Hodgman clipping against
//      the three edges of tau in its reference coordinates, fan triangulation and
//      the 3-point edge-midpoint rule (exact for quadratics), nine COO entries.
#include "bem_internal.cuh"

#include <cmath>
#include <mutex>

namespace bem {

namespace {

struct Disc {
    float cx, cy, cz;   // unit direction of the centroid seen from c0
    float cr, sr;       // cos and sin of the widened angular radius
    float pad;
};

__global__ void k_discs(const double* __restrict__ xyz, const int32_t* __restrict__ tri, int64_t nt, double3 c0,
                        Disc* __restrict__ out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double u[3][3], c[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) {
        int32_t id = tri[3 * t + a];
        double p[3] = {xyz[3 * (int64_t)id] - c0.x, xyz[3 * (int64_t)id + 1] - c0.y, xyz[3 * (int64_t)id + 2] - c0.z};
        double l = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
        for (int d = 0; d < 3; ++d) {
            u[a][d] = p[d] / l;
            c[d] += u[a][d];
        }
    }
    double l = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    for (int d = 0; d < 3; ++d) c[d] /= l;
    double mincos = 1.0;
    for (int a = 0; a < 3; ++a) mincos = fmin(mincos, u[a][0] * c[0] + u[a][1] * c[1] + u[a][2] * c[2]);
    double ang = acos(fmax(-1.0, fmin(1.0, mincos))) + 1e-3;  // widened for the FP32 test
    Disc D;
    D.cx = (float)c[0];
    D.cy = (float)c[1];
    D.cz = (float)c[2];
    if (ang >= 3.14159265358979 / 2) {  // huge triangle: never pruned
        D.cr = -2.0f;
        D.sr = 0.0f;
    } else {
        D.cr = (float)cos(ang);
        D.sr = (float)sin(ang);
    }
    D.pad = 0.0f;
    out[t] = D;
}

// Candidate test: angle(c_tau, c_sigma) <= r_tau + r_sigma  <=>  dot >= cos(r_tau + r_sigma)
__device__ __forceinline__ bool disc_overlap(const Disc& A, const Disc& B) {
    if (A.cr < -1.5f || B.cr < -1.5f) return true;
    float dot = A.cx * B.cx + A.cy * B.cy + A.cz * B.cz;
    float cs = A.cr * B.cr - A.sr * B.sr;  // cos of the summed radii (< pi)
    return dot >= cs - 1e-6f;
}

__global__ void k_candidates(const Disc* __restrict__ da, int64_t na, const Disc* __restrict__ db, int64_t nb,
                             unsigned long long* __restrict__ counter, int2* __restrict__ out, int64_t cap) {
    for (int64_t t = blockIdx.y; t < na; t += gridDim.y) {
        const Disc A = da[t];
        for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nb;
             s += (int64_t)gridDim.x * blockDim.x) {
            if (disc_overlap(A, db[s])) {
                unsigned long long k = atomicAdd(counter, 1ull);
                if (out && (int64_t)k < cap) out[k] = make_int2((int)t, (int)s);
            }
        }
    }
}

struct P2 {
    double s, t;
};

__device__ __forceinline__ double edge_fun(int e, P2 p) {
    return e == 0 ? p.s : (e == 1 ? p.t : 1.0 - p.s - p.t);
}

__global__ void k_clip(const double* __restrict__ xa, const int32_t* __restrict__ ta, const double* __restrict__ xb,
                       const int32_t* __restrict__ tb, const int2* __restrict__ cand, int64_t ncand, double3 c0,
                       int32_t* __restrict__ orow, int32_t* __restrict__ ocol, double* __restrict__ oval) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= ncand) return;
    const int tau = cand[k].x, sig = cand[k].y;
    double A[3][3], B[3][3];
    int32_t ia[3], ib[3];
    for (int m = 0; m < 3; ++m) {
        ia[m] = ta[3 * (int64_t)tau + m];
        ib[m] = tb[3 * (int64_t)sig + m];
        for (int d = 0; d < 3; ++d) {
            A[m][d] = xa[3 * (int64_t)ia[m] + d];
            B[m][d] = xb[3 * (int64_t)ib[m] + d];
        }
    }
    double vals[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    double e1[3], e2[3], n[3];
    for (int d = 0; d < 3; ++d) {
        e1[d] = A[1][d] - A[0][d];
        e2[d] = A[2][d] - A[0][d];
    }
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const double J = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (int d = 0; d < 3; ++d) n[d] /= J;
    const double off = (A[0][0] - c0.x) * n[0] + (A[0][1] - c0.y) * n[1] + (A[0][2] - c0.z) * n[2];
    const double g11 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
    const double g12 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
    const double g22 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
    const double det = g11 * g22 - g12 * g12;
    P2 q[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
    bool ok = true;
    for (int m = 0; m < 3 && ok; ++m) {
        double X[3] = {B[m][0] - c0.x, B[m][1] - c0.y, B[m][2] - c0.z};
        double den = X[0] * n[0] + X[1] * n[1] + X[2] * n[2];
        if (den == 0.0) { ok = false; break; }
        double sc = off / den;
        if (!(sc > 0.0)) { ok = false; break; }  // the ray must meet the plane ahead of c0
        const double c0a[3] = {c0.x, c0.y, c0.z};
        double rel[3];
        for (int d = 0; d < 3; ++d) rel[d] = c0a[d] + X[d] * sc - A[0][d];
        double b1 = rel[0] * e1[0] + rel[1] * e1[1] + rel[2] * e1[2];
        double b2 = rel[0] * e2[0] + rel[1] * e2[1] + rel[2] * e2[2];
        q[m].s = (g22 * b1 - g12 * b2) / det;
        q[m].t = (g11 * b2 - g12 * b1) / det;
    }
    // barycentric map of sigma' in (s, t)
    const double m11 = q[1].s - q[0].s, m12 = q[2].s - q[0].s, m21 = q[1].t - q[0].t, m22 = q[2].t - q[0].t;
    const double mdet = m11 * m22 - m12 * m21;
    if (ok && mdet != 0.0) {
        // a convex polygon gains at most one vertex per clip (3 -> 6); rounding can
        // make slivers non-convex, so the buffers are capped rather than trusted
        constexpr int CAP = 12;
        P2 poly[CAP], nxt[CAP];
        int np = 3;
        for (int m = 0; m < 3; ++m) poly[m] = q[m];
        for (int e = 0; e < 3 && np > 0; ++e) {
            int nn = 0;
            for (int i = 0; i < np; ++i) {
                P2 p = poly[i], r = poly[(i + 1) % np];
                double fp = edge_fun(e, p), fr = edge_fun(e, r);
                if (fp >= 0.0 && nn < CAP) nxt[nn++] = p;
                if ((fp >= 0.0) != (fr >= 0.0) && nn < CAP) {
                    double lam = fp / (fp - fr);
                    nxt[nn++] = P2{p.s + lam * (r.s - p.s), p.t + lam * (r.t - p.t)};
                }
            }
            np = nn;
            for (int i = 0; i < np; ++i) poly[i] = nxt[i];
        }
        for (int m = 1; m + 1 < np; ++m) {
            const P2 p0 = poly[0], p1 = poly[m], p2 = poly[m + 1];
            const double area2 = (p1.s - p0.s) * (p2.t - p0.t) - (p1.t - p0.t) * (p2.s - p0.s);
            const double wgt = fabs(area2) * 0.5 * J / 3.0;  // edge-midpoint rule, dS = J ds dt
            const P2 mids[3] = {{0.5 * (p0.s + p1.s), 0.5 * (p0.t + p1.t)},
                                {0.5 * (p1.s + p2.s), 0.5 * (p1.t + p2.t)},
                                {0.5 * (p2.s + p0.s), 0.5 * (p2.t + p0.t)}};
            for (int h = 0; h < 3; ++h) {
                const double s = mids[h].s, t = mids[h].t;
                const double la[3] = {1.0 - s - t, s, t};
                const double ds = s - q[0].s, dt = t - q[0].t;
                const double l1 = (m22 * ds - m12 * dt) / mdet, l2 = (m11 * dt - m21 * ds) / mdet;
                const double lb[3] = {1.0 - l1 - l2, l1, l2};
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) vals[3 * a + b] += wgt * la[a] * lb[b];
            }
        }
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            orow[9 * k + 3 * a + b] = ia[a];
            ocol[9 * k + 3 * a + b] = ib[b];
            oval[9 * k + 3 * a + b] = vals[3 * a + b];
        }
}

}  // namespace

bem_status mortar_coo(const bem_grid* a, const bem_grid* b, const double center[3], DevBuf& row, DevBuf& col,
                      DevBuf& val, int64_t* nnz, cudaStream_t s) {
    double3 c0 = make_double3(center[0], center[1], center[2]);
    DevBuf da, db, counter, cand;
    BEM_TRY(da.alloc(a->nt * sizeof(Disc), s));
    BEM_TRY(db.alloc(b->nt * sizeof(Disc), s));
    BEM_TRY(counter.alloc(sizeof(unsigned long long), s));
    BEM_LAUNCH(k_discs, (unsigned)((a->nt + 127) / 128), 128, 0, s, a->xyz.as<double>(), a->tri.as<int32_t>(), a->nt, c0,
                                                          da.as<Disc>());
    BEM_CHECK_LAUNCH();
    BEM_LAUNCH(k_discs, (unsigned)((b->nt + 127) / 128), 128, 0, s, b->xyz.as<double>(), b->tri.as<int32_t>(), b->nt, c0,
                                                          db.as<Disc>());
    BEM_CHECK_LAUNCH();
    // pass 1: count
    BEM_CUDA_TRY(cudaMemsetAsync(counter.p, 0, sizeof(unsigned long long), s));
    unsigned gx = (unsigned)std::min<int64_t>((b->nt + 255) / 256, 64);
    dim3 grid(gx, (unsigned)std::min<int64_t>(a->nt, 65535));
    BEM_LAUNCH(k_candidates, grid, 256, 0, s, da.as<Disc>(), a->nt, db.as<Disc>(), b->nt,
                                      counter.as<unsigned long long>(), nullptr, 0);
    BEM_CHECK_LAUNCH();
    unsigned long long ncand = 0;
    BEM_CUDA_TRY(cudaMemcpyAsync(&ncand, counter.p, sizeof(ncand), cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    if (ncand == 0) {
        *nnz = 0;
        return BEM_OK;
    }
    // pass 2: fill
    BEM_TRY(cand.alloc(ncand * sizeof(int2), s));
    BEM_CUDA_TRY(cudaMemsetAsync(counter.p, 0, sizeof(unsigned long long), s));
    BEM_LAUNCH(k_candidates, grid, 256, 0, s, da.as<Disc>(), a->nt, db.as<Disc>(), b->nt,
                                      counter.as<unsigned long long>(), cand.as<int2>(), (int64_t)ncand);
    BEM_CHECK_LAUNCH();
    const int64_t n9 = 9 * (int64_t)ncand;
    BEM_TRY(row.alloc(n9 * 4, s));
    BEM_TRY(col.alloc(n9 * 4, s));
    BEM_TRY(val.alloc(n9 * 8, s));
    BEM_LAUNCH(k_clip, (unsigned)((ncand + 127) / 128), 128, 0, s, a->xyz.as<double>(), a->tri.as<int32_t>(),
                                                         b->xyz.as<double>(), b->tri.as<int32_t>(), cand.as<int2>(),
                                                         (int64_t)ncand, c0, row.as<int32_t>(), col.as<int32_t>(),
                                                         val.as<double>());
    BEM_CHECK_LAUNCH();
    *nnz = n9;
    return BEM_OK;
}

}  // namespace bem

// ----------------------------------------------------------------------------------
// bem_projection_noalloc: the mortar matrix without any device allocation.
//
// Some callers cannot let a library allocate device memory while they run: a host
// application that hands out all HBM from its own budgeted pool (so that a foreign
// cudaMalloc could break its accounting or fail mid-request), or a latency-critical
// loop that cannot afford cudaMalloc's cost and implicit synchronisation.  For them
// this entry point keeps its working memory (the angular discs of both grids and the
// candidate-pair list) in one fixed array in device global memory that exists for as
// long as the library is loaded, on every GPU that loads it.  The caller passes the
// grids (validated handles) and the output arrays.
namespace bem {
namespace {

constexpr int64_t NOALLOC_MAX_TRI = 32768;     // triangles per grid
constexpr int64_t NOALLOC_MAX_CAND = 1 << 20;  // candidate triangle pairs
constexpr size_t NOALLOC_DISC_OFF = 256;
constexpr size_t NOALLOC_CAND_OFF = NOALLOC_DISC_OFF + 2 * NOALLOC_MAX_TRI * sizeof(Disc);
constexpr size_t NOALLOC_BYTES = NOALLOC_CAND_OFF + NOALLOC_MAX_CAND * sizeof(int2);  // ~9.9 MB

// The scratch array.  In host code its name is only a stand-in: the device address
// is obtained with cudaGetSymbolAddress (once per device) and passed to the kernels.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[256] = {};

bem_status noalloc_scratch(int device, unsigned char** out) {
    BEM_REQUIRE(device >= 0 && device < 256, "device index out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void* p = nullptr;
        BEM_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));  // the device is current here
        g_noalloc_addr[device] = p;
    }
    *out = static_cast<unsigned char*>(g_noalloc_addr[device]);
    return BEM_OK;
}

}  // namespace
}  // namespace bem

extern "C" bem_status bem_projection_noalloc(bem_context* ctx, const bem_grid* a, const bem_grid* b,
                                             const double* center, int32_t* row, int32_t* col, double* val,
                                             int64_t capacity, int64_t* nnz) {
    using namespace bem;
    BEM_REQUIRE(ctx != nullptr, "null context");
    BEM_CUDA_TRY(cudaSetDevice(ctx->device));
    BEM_REQUIRE(a != nullptr && b != nullptr, "null grid");
    BEM_REQUIRE(row != nullptr && col != nullptr && val != nullptr && nnz != nullptr, "null output");
    BEM_REQUIRE(a->nt <= NOALLOC_MAX_TRI && b->nt <= NOALLOC_MAX_TRI,
                "bem_projection_noalloc supports at most 32768 triangles per grid (got " +
                    std::to_string(a->nt) + " and " + std::to_string(b->nt) + ")");
    double c0v[3] = {0.0, 0.0, 0.0};
    if (center)
        for (int d = 0; d < 3; ++d) c0v[d] = center[d];
    BEM_REQUIRE(std::isfinite(c0v[0]) && std::isfinite(c0v[1]) && std::isfinite(c0v[2]), "centre not finite");
    const double3 c0 = make_double3(c0v[0], c0v[1], c0v[2]);
    unsigned char* base = nullptr;
    BEM_TRY(noalloc_scratch(ctx->device, &base));
    cudaStream_t s = ctx->stream;
    auto* counter = reinterpret_cast<unsigned long long*>(base);
    Disc* da = reinterpret_cast<Disc*>(base + NOALLOC_DISC_OFF);
    Disc* db = da + NOALLOC_MAX_TRI;
    int2* cand = reinterpret_cast<int2*>(base + NOALLOC_CAND_OFF);
    // the array keeps the previous call's contents: the counter must start at zero
    BEM_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
    BEM_REQUIRE(a->nt > 0 && b->nt > 0, "grid without triangles");
    BEM_LAUNCH(k_discs, (unsigned)((a->nt + 127) / 128), 128, 0, s, a->xyz.as<double>(), a->tri.as<int32_t>(),
               a->nt, c0, da);
    BEM_CHECK_LAUNCH();
    BEM_LAUNCH(k_discs, (unsigned)((b->nt + 127) / 128), 128, 0, s, b->xyz.as<double>(), b->tri.as<int32_t>(),
               b->nt, c0, db);
    BEM_CHECK_LAUNCH();
    unsigned gx = (unsigned)std::min<int64_t>((b->nt + 255) / 256, 64);
    dim3 grid(gx, (unsigned)std::min<int64_t>(a->nt, 65535));
    BEM_LAUNCH(k_candidates, grid, 256, 0, s, da, a->nt, db, b->nt, counter, cand, NOALLOC_MAX_CAND);
    BEM_CHECK_LAUNCH();
    unsigned long long ncand = 0;
    BEM_CUDA_TRY(cudaMemcpyAsync(&ncand, counter, sizeof(ncand), cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    BEM_REQUIRE((int64_t)ncand <= NOALLOC_MAX_CAND,
                "bem_projection_noalloc supports at most 1048576 candidate triangle pairs (got " +
                    std::to_string(ncand) + ")");
    const int64_t need = 9 * (int64_t)ncand;
    *nnz = need;
    BEM_REQUIRE(capacity >= need, "output capacity " + std::to_string(capacity) + " is below the " +
                                      std::to_string(need) + " entries needed");
    if (ncand > 0) {
        BEM_LAUNCH(k_clip, (unsigned)((ncand + 127) / 128), 128, 0, s, a->xyz.as<double>(), a->tri.as<int32_t>(),
                   b->xyz.as<double>(), b->tri.as<int32_t>(), cand, (int64_t)ncand, c0, row, col, val);
        BEM_CHECK_LAUNCH();
    }
    return BEM_OK;
}
