// Transmission solve on the device (paper Sec. 2.2 unknowns and transmission
// conditions, eq. mtf:discrete, Sec. 3.3 mass-matrix preconditioning, Sec. 5.1
// unrestarted GMRES), for R plane waves at once.
//
// Unknown vector x = [v_e (N_e), w_e (N_e), v_i (N_i), w_i (N_i)], complex128; a
// block of R right-hand sides is stored as R such vectors back to back.
// Weak-form MTF (derived signs, s = +1; printed signs, s = -1):
//   z1 = -K_e v_e + V_e w_e - (s/2) P_ei v_i
//   z2 =  D_e v_e + T_e w_e - (s/2)(rho_e/rho_i) P_ei w_i
//   z3 = (s/2) P_ie v_e - K_i v_i + V_i w_i
//   z4 = (s/2)(rho_i/rho_e) P_ie w_e + D_i v_i + T_i w_i
// with P_ie = P_int,ext (mortar, COO) and P_ei = P_ie^T.  The strong form applies
// M_e^-1 to z1, z2 and M_i^-1 to z3, z4.
//
// Batching: the R right-hand sides share every operator application (the dense
// blocks are read once per iteration for all R columns), and R independent GMRES
// processes advance in lockstep; a column that has converged keeps its iteration
// count and is not disturbed by the further steps of the others.
//
// Mass inverse: Chebyshev iteration on the Jacobi-scaled mass matrix.  For P1
// triangles every element matrix scaled by its diagonal has eigenvalues {2, 1/2, 1/2}
// (whatever the triangle's shape), so D^-1 M has its spectrum in [1/2, 2] and the
// Chebyshev error contracts by (sqrt(4) - 1)/(sqrt(4) + 1) = 1/3 per step with no
// inner products: 34 steps reach 2 * 3^-34 ~ 1e-16.
//
// GMRES: Arnoldi with classical Gram-Schmidt applied twice (CGS2), complex Givens
// rotations and the residual estimates kept on the device; the host reads R scalars
// per iteration to stop.  x0 = 0, stop when |g_{j+1}| <= tol * ||S b||.
#include "bem_internal.cuh"
#include "ddf.cuh"

#include <algorithm>
#include <cmath>
#include <complex>
#include <functional>
#include <mutex>
#include <vector>

namespace bem {

namespace {

constexpr int CHEB_STEPS = 34;        // error <= 2 * 3^-34 ~ 1e-16: FP64 applications
constexpr int CHEB_STEPS_INNER = 17;  // error <= 2 * 3^-17 ~ 1.6e-8: inner solves with FP32 products
constexpr int CHEB_STEPS_DD = 24;     // error <= 2 * 3^-24 ~ 7e-12: inner solves with double-float products
// The mass inverse of the multiple-traces system is a left preconditioner only (S A x =
// S b, with no inverse inside A), so any fixed approximation S' of it gives the same
// solution when both sides use it.  The FP32 inner solves of the refinement take
// S' = 6 Chebyshev steps (error <= 2 * 3^-6 ~ 3e-3: the preconditioned spectrum moves
// by that much, ~1 % more iterations at the sphere pairs of levels 2-3 than with the
// exact inverse) on both their operator and their right-hand side S'(b - A x); the
// refinement's convergence test keeps the FP64 inverse.
constexpr int CHEB_STEPS_PRE = 6;
constexpr double CHEB_ALPHA = 0.5, CHEB_BETA = 2.0;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ double2 warp_sum2(double2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}


unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------- right-hand sides
// f_j = <u_inc, theta_j>, g_j = <du_inc/dn, theta_j> on the exterior grid,
// u_inc = amp exp(i k x.d), du_inc/dn = i k (d.n) u_inc (paper eq. planewave);
// blockIdx.y = right-hand side.
// dirs [R][3], amps [R] (device); blockIdx.y = right-hand side
__global__ void k_plane_wave(const TriRec* __restrict__ rec, const int32_t* __restrict__ tri, int64_t nt,
                             double kr, double ki, const double* __restrict__ dirs, const double2* __restrict__ amps,
                             int64_t Ne, double2* __restrict__ f, double2* __restrict__ g) {
    const int r = blockIdx.y;
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const double3 d = make_double3(dirs[3 * r], dirs[3 * r + 1], dirs[3 * r + 2]);
    const double2 amp = amps[r];
    const TriRec& R = rec[t];
    const double dn = d.x * R.n[0] + d.y * R.n[1] + d.z * R.n[2];
    double2 fa[3] = {}, ga[3] = {};
    for (int p = 0; p < 6; ++p) {
        double xd = d.x * R.q[p][0] + d.y * R.q[p][1] + d.z * R.q[p][2];
        double sn, cs;
        sincos(kr * xd, &sn, &cs);
        double mag = (ki != 0.0) ? exp(-ki * xd) : 1.0;
        double2 u = cmul(amp, make_double2(mag * cs, mag * sn));
        double2 du = cmul(make_double2(-ki * dn, kr * dn), u);  // i k (d.n) u
        for (int a = 0; a < 3; ++a) {
            fa[a].x += R.wl[p][a] * u.x;
            fa[a].y += R.wl[p][a] * u.y;
            ga[a].x += R.wl[p][a] * du.x;
            ga[a].y += R.wl[p][a] * du.y;
        }
    }
    for (int a = 0; a < 3; ++a) {
        const int64_t v = r * Ne + tri[3 * t + a];
        atomicAdd(&f[v].x, fa[a].x);
        atomicAdd(&f[v].y, fa[a].y);
        atomicAdd(&g[v].x, ga[a].x);
        atomicAdd(&g[v].y, ga[a].y);
    }
}

// The same data for point sources (the incident-field kind BEM_INC_POINT_SOURCE):
// u_inc = amp exp(i k r) / (4 pi r) with r = |x - s|, du_inc/dn = u_inc (i k - 1/r) ((x - s).n) / r.
// src [R][3], amps [R] (device); blockIdx.y = right-hand side
__global__ void k_point_source(const TriRec* __restrict__ rec, const int32_t* __restrict__ tri, int64_t nt,
                               double kr, double ki, const double* __restrict__ src,
                               const double2* __restrict__ amps, int64_t Ne, double2* __restrict__ f,
                               double2* __restrict__ g) {
    const int r = blockIdx.y;
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const double3 c = make_double3(src[3 * r], src[3 * r + 1], src[3 * r + 2]);
    const double2 amp = amps[r];
    const TriRec& R = rec[t];
    double2 fa[3] = {}, ga[3] = {};
    for (int p = 0; p < 6; ++p) {
        const double dx = R.q[p][0] - c.x, dy = R.q[p][1] - c.y, dz = R.q[p][2] - c.z;
        const double rr = sqrt(dx * dx + dy * dy + dz * dz);
        const double ri = 1.0 / rr;
        double sn, cs;
        sincos(kr * rr, &sn, &cs);
        const double mag = ((ki != 0.0) ? exp(-ki * rr) : 1.0) * ri * 0.07957747154594767;  // 1 / (4 pi r)
        const double2 u = cmul(amp, make_double2(mag * cs, mag * sn));
        const double dn = (dx * R.n[0] + dy * R.n[1] + dz * R.n[2]) * ri;
        const double2 du = cmul(make_double2((-ki - ri) * dn, kr * dn), u);  // (i k - 1/r) (x - s).n / r u
        for (int a = 0; a < 3; ++a) {
            fa[a].x += R.wl[p][a] * u.x;
            fa[a].y += R.wl[p][a] * u.y;
            ga[a].x += R.wl[p][a] * du.x;
            ga[a].y += R.wl[p][a] * du.y;
        }
    }
    for (int a = 0; a < 3; ++a) {
        const int64_t v = r * Ne + tri[3 * t + a];
        atomicAdd(&f[v].x, fa[a].x);
        atomicAdd(&f[v].y, fa[a].y);
        atomicAdd(&g[v].x, ga[a].x);
        atomicAdd(&g[v].y, ga[a].y);
    }
}

// b = [-f, -g, 0, 0] per right-hand side
__global__ void k_rhs_pack(const double2* __restrict__ f, const double2* __restrict__ g, int64_t Ne, int64_t n,
                           double2* __restrict__ b) {
    const int r = blockIdx.y;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    double2 v = make_double2(0.0, 0.0);
    if (e < Ne) v = make_double2(-f[r * Ne + e].x, -f[r * Ne + e].y);
    else if (e < 2 * Ne) v = make_double2(-g[r * Ne + e - Ne].x, -g[r * Ne + e - Ne].y);
    b[r * n + e] = v;
}

// ---------------------------------------------------------------- dense MTF blocks
template <class MT>
struct Blocks {
    const MT* A1[4];       // first matrix of each block row (K_e, D_e, K_i, D_i)
    const MT* A2[4];       // second matrix (V_e, T_e, V_i, T_i)
    double c1[4], c2[4];   // real coefficients
    int64_t rows[4];       // N of each block row
    int64_t base[4];       // offset of block row b in the vector
    int64_t x1[4], x2[4];  // offsets of the vectors multiplying A1, A2
};

__global__ void k_to_c64(const double2* __restrict__ x, int64_t n, float2* __restrict__ y) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) y[e] = make_float2((float)x[e].x, (float)x[e].y);
}

// x split into FP32 high and low parts, (Re hi, Im hi, Re lo, Im lo): x = hi + lo to
// about 2^-48 relative
__global__ void k_split_x(const double2* __restrict__ x, int64_t n, float4* __restrict__ xs) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double2 v = x[e];
    const float hr = (float)v.x, hi = (float)v.y;
    xs[e] = make_float4(hr, hi, (float)(v.x - (double)hr), (float)(v.y - (double)hi));
}

// ---------------------------------------------------------------- mortar transfer
// P_ie (rows: interior vertices, columns: exterior vertices) and P_ei = P_ie^T in
// CSR form, built once per solve from the COO list of the clipping kernel: zero
// entries are dropped and the duplicates of one (row, column) -- one per clipped
// triangle pair -- are summed in a fixed order (sorted by value), so that the
// product does not depend on the order in which the clipping kernel wrote them.
__global__ void k_csr_count(const int32_t* __restrict__ key, const double* __restrict__ val, int64_t nnz,
                            int32_t* __restrict__ cnt) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < nnz && val[e] != 0.0) atomicAdd(&cnt[key[e]], 1);
}

// exclusive prefix sum of cnt[0, n) into out[0, n]; out[n] = total (one block of 1024 threads)
__global__ void __launch_bounds__(1024) k_scan(const int32_t* __restrict__ cnt, int64_t n, int32_t* __restrict__ out) {
    __shared__ int32_t part[1024];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const int32_t v = i < n ? cnt[i] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {  // inclusive scan in shared memory
            const int32_t t = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
            __syncthreads();
            part[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < n) out[i] = carry + part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += part[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = carry;
}

__global__ void k_csr_scatter(const int32_t* __restrict__ key, const int32_t* __restrict__ other,
                              const double* __restrict__ val, int64_t nnz, const int32_t* __restrict__ start,
                              int32_t* __restrict__ fill, int32_t* __restrict__ oc, double* __restrict__ ov) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nnz || val[e] == 0.0) return;
    const int32_t k = key[e];
    const int32_t p = start[k] + atomicAdd(&fill[k], 1);
    oc[p] = other[e];
    ov[p] = val[e];
}

// Entries of one row sorted in shared memory (12 bytes each: 48 KB); longer rows are
// sorted in place in global memory by the same network.
constexpr int CSR_MERGE_SMEM = 4096;

__device__ __forceinline__ bool csr_less(int32_t ca, double va, int32_t cb, double vb) {
    return ca < cb || (ca == cb && va < vb);
}

// One block per row: sort the row's entries by (column, value), then sum equal columns
// in that order and compact in place (the order, hence the sums, do not depend on the
// order in which the entries were produced).  Bitonic network with every comparator
// ascending (the first step of each stage pairs i with its mirror i ^ (size - 1)), so
// the row length need not be a power of two: slots past its end act as +infinity and
// are never touched.
__global__ void __launch_bounds__(256) k_csr_merge(const int32_t* __restrict__ start, int64_t rows,
                                                   int32_t* __restrict__ oc, double* __restrict__ ov,
                                                   int32_t* __restrict__ mcnt) {
    __shared__ int32_t s_c[CSR_MERGE_SMEM];
    __shared__ double s_v[CSR_MERGE_SMEM];
    const int64_t k = blockIdx.x;
    if (k >= rows) return;
    const int32_t b = start[k], len = start[k + 1] - b;
    const bool in_smem = len <= CSR_MERGE_SMEM;
    int32_t* C = in_smem ? s_c : oc + b;
    double* V = in_smem ? s_v : ov + b;
    if (in_smem)
        for (int32_t i = threadIdx.x; i < len; i += blockDim.x) {
            s_c[i] = oc[b + i];
            s_v[i] = ov[b + i];
        }
    __syncthreads();
    int32_t p2 = 1;
    while (p2 < len) p2 <<= 1;
    for (int32_t size = 2; size <= p2; size <<= 1) {
        for (int32_t j = size >> 1; j > 0; j >>= 1) {
            for (int32_t i = threadIdx.x; i < p2; i += blockDim.x) {
                const int32_t partner = j == (size >> 1) ? (i ^ (size - 1)) : (i ^ j);
                if (partner > i && partner < len && csr_less(C[partner], V[partner], C[i], V[i])) {
                    const int32_t tc = C[i];
                    const double tv = V[i];
                    C[i] = C[partner];
                    V[i] = V[partner];
                    C[partner] = tc;
                    V[partner] = tv;
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {  // the write position never passes the read position
        int32_t w = 0;
        for (int32_t i = 0; i < len;) {
            const int32_t c = C[i];
            double sum = 0.0;
            while (i < len && C[i] == c) sum += V[i++];
            oc[b + w] = c;
            ov[b + w] = sum;
            ++w;
        }
        mcnt[k] = w;
    }
}

__global__ void k_csr_compact(const int32_t* __restrict__ start, const int32_t* __restrict__ rp, int64_t rows,
                              const int32_t* __restrict__ oc, const double* __restrict__ ov, int32_t* __restrict__ ci,
                              double* __restrict__ v) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= rows) return;
    const int32_t src = start[k], dst = rp[k], len = rp[k + 1] - rp[k];
    for (int32_t i = 0; i < len; ++i) {
        ci[dst + i] = oc[src + i];
        v[dst + i] = ov[src + i];
    }
}

struct TransferCsr {
    const int32_t *prp, *pci;  // P_ie: rows = interior vertices
    const double* pv;
    const int32_t *trp, *tci;  // P_ei = P_ie^T: rows = exterior vertices
    const double* tv;
    int64_t Ne, Ni, n;
    double ca, cb, cc, cd;  // z1 += ca P_ei v_i, z2 += cb P_ei w_i, z3 += cc P_ie v_e, z4 += cd P_ie w_e
};

// one thread per row of z (blockIdx.y = right-hand side); no atomics
__global__ void k_transfer(TransferCsr T, const double2* __restrict__ xb, double2* __restrict__ zb) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= T.n) return;
    const double2* x = xb + blockIdx.y * T.n;
    double2* z = zb + blockIdx.y * T.n;
    const bool ext = g < 2 * T.Ne;
    const int32_t* rp = ext ? T.trp : T.prp;
    const int32_t* ci = ext ? T.tci : T.pci;
    const double* v = ext ? T.tv : T.pv;
    int64_t row, src;
    double c;
    if (g < T.Ne) { row = g; src = 2 * T.Ne; c = T.ca; }
    else if (g < 2 * T.Ne) { row = g - T.Ne; src = 2 * T.Ne + T.Ni; c = T.cb; }
    else if (g < 2 * T.Ne + T.Ni) { row = g - 2 * T.Ne; src = 0; c = T.cc; }
    else { row = g - 2 * T.Ne - T.Ni; src = T.Ne; c = T.cd; }
    double sr = 0.0, si = 0.0;
    for (int32_t e = rp[row]; e < rp[row + 1]; ++e) {
        const double p = v[e];
        const double2 xx = x[src + ci[e]];
        sr = fma(p, xx.x, sr);
        si = fma(p, xx.y, si);
    }
    double2 zz = z[g];
    zz.x = fma(c, sr, zz.x);
    zz.y = fma(c, si, zz.y);
    z[g] = zz;
}

// One mortar matrix (CSR, `rows` rows, columns on a grid of `cols` vertices) applied to
// two vectors of a column: z[b rows + i] = c_b (P x_b)_i for b = 0, 1, with x_b at
// x0 or x1 (both of column stride nx; z of stride nz, blockIdx.y = right-hand side);
// `add` accumulates into z instead.  One thread per row of z, no atomics.
__global__ void k_csr_pair(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const double* __restrict__ v, int64_t rows, const double2* __restrict__ x0,
                           const double2* __restrict__ x1, int64_t nx, double2* __restrict__ zb, int64_t nz,
                           double c0, double c1, int add) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= 2 * rows) return;
    const int b = g >= rows ? 1 : 0;
    const int64_t i = g - b * rows;
    const double2* x = (b ? x1 : x0) + blockIdx.y * nx;
    double sr = 0.0, si = 0.0;
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
        const double p = v[e];
        const double2 xx = x[ci[e]];
        sr = fma(p, xx.x, sr);
        si = fma(p, xx.y, si);
    }
    const double c = b ? c1 : c0;
    double2* zp = zb + blockIdx.y * nz + g;
    double2 zz = add ? *zp : make_double2(0.0, 0.0);
    zz.x = fma(c, sr, zz.x);
    zz.y = fma(c, si, zz.y);
    *zp = zz;
}

// y = C s over pairs of vectors of one grid (R columns of stride `stride`, two halves of
// N entries): for half b, y_b = sum_k C[6 b + k] s_k with s = (x_0, x_1, u_0, u_1, w_0, w_1)
// the halves of x, u and w.  Real coefficients; y must not be one of the inputs.
struct PairCoef {
    double c[12];
};

__global__ void k_pair_lin(double2* __restrict__ y, const double2* x, const double2* u, const double2* w, int64_t N,
                           int64_t stride, PairCoef C) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= 2 * N) return;
    const int b = g >= N ? 1 : 0;
    const int64_t i = g - b * N, off = blockIdx.y * stride;
    const double2 s[6] = {x[off + i], x[off + N + i], u[off + i], u[off + N + i], w[off + i], w[off + N + i]};
    double2 r = make_double2(0.0, 0.0);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double c = C.c[6 * b + k];
        r.x = fma(c, s[k].x, r.x);
        r.y = fma(c, s[k].y, r.y);
    }
    y[off + g] = r;
}

// ---------------------------------------------------------------- open screens
// A CSR matrix on one vector per column: z = c P x (x of stride nx, z of stride nz,
// blockIdx.y = right-hand side), one thread per row
__global__ void k_csr_apply(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const double* __restrict__ v, int64_t rows, const double2* __restrict__ x, int64_t nx,
                            double2* __restrict__ z, int64_t nz, double c) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rows) return;
    const double2* xc = x + blockIdx.y * nx;
    double sr = 0.0, si = 0.0;
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
        const double p = v[e];
        const double2 xx = xc[ci[e]];
        sr = fma(p, xx.x, sr);
        si = fma(p, xx.y, si);
    }
    z[blockIdx.y * nz + i] = make_double2(c * sr, c * si);
}

// y[i] = 0 at the screen's boundary nodes (keep[i] == 0), R columns of stride n
__global__ void k_mask_rows(double2* __restrict__ y, const uint8_t* __restrict__ keep, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && !keep[i]) y[blockIdx.y * n + i] = make_double2(0.0, 0.0);
}

// The ELL mass matrix of the functions that vanish on the boundary, padded to the full
// node set: boundary rows become identity rows, couplings to boundary columns are
// dropped; the Jacobi diagonal of a boundary row is 1.
__global__ void k_mask_mass_ell(int32_t* __restrict__ ci, double* __restrict__ v, double* __restrict__ dinv, int W,
                                int64_t N, const uint8_t* __restrict__ keep) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (!keep[i]) {
        for (int k = 0; k < W; ++k) {
            ci[(int64_t)k * N + i] = (int32_t)i;
            v[(int64_t)k * N + i] = k == 0 ? 1.0 : 0.0;
        }
        dinv[i] = 1.0;
        return;
    }
    for (int k = 0; k < W; ++k) {
        const int32_t c = ci[(int64_t)k * N + i];
        if (!keep[c]) v[(int64_t)k * N + i] = 0.0;
    }
}

// ---------------------------------------------------------------- mass inverse
// Mass matrices of the two grids in ELL form (column-major [W][N]: entry k of row i
// at k * N + i; rows shorter than W padded with (i, 0)), so that all column indices
// and values of a row are loaded at once, independent of each other.
struct MassPair {
    const int32_t* ci[2];
    const double *v[2], *dinv[2];
    const float *vf[2] = {nullptr, nullptr}, *dinvf[2] = {nullptr, nullptr};  // FP32 copies (optional)
    int W[2];
    int64_t Ne, Ni, n;
};

struct MassRow {
    const int32_t* ci;
    const double *v, *dinv;
    int W;
    int64_t N, i, base;
};

__device__ __forceinline__ MassRow mass_row(const MassPair& M, int64_t g) {
    MassRow m;
    const bool ext = g < 2 * M.Ne;
    m.ci = ext ? M.ci[0] : M.ci[1];
    m.v = ext ? M.v[0] : M.v[1];
    m.dinv = ext ? M.dinv[0] : M.dinv[1];
    m.W = ext ? M.W[0] : M.W[1];
    m.N = ext ? M.Ne : M.Ni;
    if (g < M.Ne) { m.i = g; m.base = 0; }
    else if (g < 2 * M.Ne) { m.i = g - M.Ne; m.base = M.Ne; }
    else if (g < 2 * M.Ne + M.Ni) { m.i = g - 2 * M.Ne; m.base = 2 * M.Ne; }
    else { m.i = g - 2 * M.Ne - M.Ni; m.base = 2 * M.Ne + M.Ni; }
    return m;
}

// (M d)_i over the ELL row of m, d the vector block of that grid
__device__ __forceinline__ double2 mass_apply_row(const MassRow& m, const double2* __restrict__ d) {
    double2 md = make_double2(0, 0);
    for (int k = 0; k < m.W; ++k) {
        const double v = m.v[(int64_t)k * m.N + m.i];
        const double2 dd = d[m.ci[(int64_t)k * m.N + m.i]];
        md.x += v * dd.x;
        md.y += v * dd.y;
    }
    return md;
}

// FP32 copy of FP64 values
__global__ void k_narrow(const double* __restrict__ a, int64_t n, float* __restrict__ b) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// ELL copy of one grid's mass CSR (one thread per row)
__global__ void k_mass_ell(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const double* __restrict__ val, int64_t N, int W, int32_t* __restrict__ ci,
                           double* __restrict__ v) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int32_t b = rp[i], len = rp[i + 1] - b;
    for (int k = 0; k < W; ++k) {
        ci[(int64_t)k * N + i] = k < len ? col[b + k] : (int32_t)i;
        v[(int64_t)k * N + i] = k < len ? val[b + k] : 0.0;
    }
}

// y = 0, r = z, d = D^-1 r / theta  (blockIdx.y = right-hand side)
__global__ void k_cheb_init(MassPair M, const double2* __restrict__ z, double2* __restrict__ y,
                            double2* __restrict__ r, double2* __restrict__ d, double inv_theta) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= M.n) return;
    const int64_t off = blockIdx.y * M.n;
    const MassRow m = mass_row(M, g);
    const double2 zz = z[off + g];
    const double s = m.dinv[m.i] * inv_theta;
    y[off + g] = make_double2(0, 0);
    r[off + g] = zz;
    d[off + g] = make_double2(s * zz.x, s * zz.y);
}

// The same iteration in FP32 (the 17-step inverse of the inner solves that use FP32
// products: its rounding, ~2e-7, matches theirs): r, d and the running sum y as float2
// (y in the second half of the dA workspace), the result widened to FP64 by the last step.
// The FP32 vectors are interleaved by column (entry (g, c) of R columns at g R + c): the
// threads of a warp take consecutive columns of a row, so that the row's mass entries
// are loaded once per warp and the gathers of its neighbours are contiguous.  z and the
// result keep the column-major layout of the other kernels.  Thread t = g R + c; n R
// stays below 2^31 (checked by the caller).
__global__ void k_cheb_init32(MassPair M, int R, const double2* __restrict__ z, float2* __restrict__ r,
                              float2* __restrict__ d, float inv_theta) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if ((int64_t)t >= M.n * R) return;
    const uint32_t g = t / (uint32_t)R, c = t - g * (uint32_t)R;
    const MassRow m = mass_row(M, g);
    const double2 zz = z[(int64_t)c * M.n + g];
    const float2 rz = make_float2((float)zz.x, (float)zz.y);
    const float sc = (m.base < 2 * M.Ne ? M.dinvf[0] : M.dinvf[1])[m.i] * inv_theta;
    r[t] = rz;
    d[t] = make_float2(sc * rz.x, sc * rz.y);
}

__global__ void k_cheb_step32(MassPair M, int R, const float2* __restrict__ dk, float2* __restrict__ dn,
                              float2* __restrict__ y, float2* __restrict__ r, float c1, float c2, int first,
                              double2* __restrict__ yout) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if ((int64_t)t >= M.n * R) return;
    const uint32_t g = t / (uint32_t)R, c = t - g * (uint32_t)R;
    const MassRow m = mass_row(M, g);
    const bool ext = m.base < 2 * M.Ne;
    const float* __restrict__ vf = ext ? M.vf[0] : M.vf[1];
    const float2* __restrict__ d = dk + m.base * R + c;
    float2 md = make_float2(0.f, 0.f);
    for (int k = 0; k < m.W; ++k) {
        const float v = vf[(int64_t)k * m.N + m.i];
        const float2 dd = d[(int64_t)m.ci[(int64_t)k * m.N + m.i] * R];
        md.x = fmaf(v, dd.x, md.x);
        md.y = fmaf(v, dd.y, md.y);
    }
    const float2 d0 = dk[t];
    float2 yy = d0;
    if (!first) {
        const float2 yp = y[t];
        yy.x += yp.x;
        yy.y += yp.y;
    }
    float2 rr = r[t];
    rr.x -= md.x;
    rr.y -= md.y;
    if (yout) yout[(int64_t)c * M.n + g] = make_double2((double)yy.x, (double)yy.y);
    else y[t] = yy;
    r[t] = rr;
    const float sc = c2 * (ext ? M.dinvf[0] : M.dinvf[1])[m.i];
    dn[t] = make_float2(fmaf(c1, d0.x, sc * rr.x), fmaf(c1, d0.y, sc * rr.y));
}

// y += d_k; r -= M d_k; d_{k+1} = c1 d_k + c2 D^-1 r
__global__ void k_cheb_step(MassPair M, const double2* __restrict__ dk, double2* __restrict__ dn,
                            double2* __restrict__ y, double2* __restrict__ r, double c1, double c2) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= M.n) return;
    const int64_t off = blockIdx.y * M.n;
    const MassRow m = mass_row(M, g);
    const double2 md = mass_apply_row(m, dk + off + m.base);
    const double2 d0 = dk[off + g];
    double2 yy = y[off + g], rr = r[off + g];
    yy.x += d0.x;
    yy.y += d0.y;
    rr.x -= md.x;
    rr.y -= md.y;
    y[off + g] = yy;
    r[off + g] = rr;
    const double s = c2 * m.dinv[m.i];
    dn[off + g] = make_double2(c1 * d0.x + s * rr.x, c1 * d0.y + s * rr.y);
}

// Grid-wide barrier of a cooperative launch (all blocks resident): a generation counter
// that the last block to arrive advances.  Waits are bounded: a block that waits about
// a second, or sees another block's failure, records it in *err and returns false, and
// the kernel then returns (its results are not used: the host checks *err).
struct GridBarrier {
    unsigned int count, gen;
};

__device__ bool grid_sync(GridBarrier* b, int* err) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned int* vgen = &b->gen;
        volatile int* verr = err;
        const unsigned int g = *vgen;
        __threadfence();
        if (atomicAdd(&b->count, 1u) + 1u == gridDim.x) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            unsigned int spins = 0;
            while (*vgen == g) {
                if (*verr) {
                    ok = 0;
                    break;
                }
                if (++spins > (1u << 21)) {
                    atomicExch(err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Barrier rounds only (the self-test of the bounded wait)
__global__ void k_barrier_probe(GridBarrier* bar, int* err, int rounds) {
    for (int k = 0; k < rounds; ++k)
        if (!grid_sync(bar, err)) return;
}

// The whole Chebyshev iteration of mass_solve in one cooperative launch: the
// arithmetic of k_cheb_init and k_cheb_step, item by item (item = row of one column),
// with a grid barrier between steps (a step reads its neighbours' d_k).
__global__ void __launch_bounds__(256) k_cheb_fused(MassPair M, const double2* __restrict__ z,
                                                    double2* __restrict__ y, double2* __restrict__ r, double2* dA,
                                                    double2* dB, int R, int steps, double inv_theta, double sigma,
                                                    double delta, GridBarrier* bar, int* err) {
    const int64_t n = M.n, items = (int64_t)R * n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t first = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t e = first; e < items; e += stride) {
        const int64_t off = (e / n) * n, g = e - off;
        const MassRow m = mass_row(M, g);
        const double2 zz = z[off + g];
        const double sc = m.dinv[m.i] * inv_theta;
        y[off + g] = make_double2(0, 0);
        r[off + g] = zz;
        dA[off + g] = make_double2(sc * zz.x, sc * zz.y);
    }
    double rho = 1.0 / sigma;
    double2 *dk = dA, *dn = dB;
    for (int k = 0; k < steps; ++k) {
        if (!grid_sync(bar, err)) return;
        const double rho_n = 1.0 / (2.0 * sigma - rho);
        const double c1 = rho_n * rho, c2 = 2.0 * rho_n / delta;
        for (int64_t e = first; e < items; e += stride) {
            const int64_t off = (e / n) * n, g = e - off;
            const MassRow m = mass_row(M, g);
            const double2 md = mass_apply_row(m, dk + off + m.base);
            const double2 d0 = dk[off + g];
            double2 yy = y[off + g], rr = r[off + g];
            yy.x += d0.x;
            yy.y += d0.y;
            rr.x -= md.x;
            rr.y -= md.y;
            y[off + g] = yy;
            r[off + g] = rr;
            const double sc = c2 * m.dinv[m.i];
            dn[off + g] = make_double2(c1 * d0.x + sc * rr.x, c1 * d0.y + sc * rr.y);
        }
        rho = rho_n;
        double2* t = dk;
        dk = dn;
        dn = t;
    }
}

// ---------------------------------------------------------------- GMRES kernels
// Krylov basis: vector i of right-hand side r at V + (i * R + r) * n.
// Hessenberg of r: column-major, H + r * ldh * ldh, column j at + j * ldh.
// The vectors are FP64; the inner products and basis updates run in double-float
// arithmetic on the FP32 pipe (ddf.cuh: 2^-48 relative per product, errors collected
// in a second word), which is several times faster than GB300's FP64 pipe.
// Inner products conj(V_{i,r}) . w_r for i < m: the rows are cut into `nblk`
// contiguous chunks; warp w of block (chunk, y, r) takes the DOT_VPW basis vectors
// i = (8 y + w) DOT_VPW + u over its chunk (w split once per row for all of them),
// reduces within the warp and writes partial[((r * m) + i) * nblk + chunk].
constexpr int DOT_ROWS = 256;         // target rows per chunk
constexpr int DOT_MAX_BLOCKS = 1216;  // 8 per SM
constexpr int DOT_VPW = 4;            // basis vectors per warp
constexpr int DOT_VPB = 8 * DOT_VPW;  // basis vectors per block

int dot_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(DOT_MAX_BLOCKS, (n + DOT_ROWS - 1) / DOT_ROWS)); }

__global__ void __launch_bounds__(256) k_dots_partial(const double2* __restrict__ Vb, int64_t n, int R, int m,
                                                      const double2* __restrict__ w, int nblk,
                                                      double2* __restrict__ partial) {
    const int r = blockIdx.z, b = blockIdx.x;
    const int lane = threadIdx.x & 31;
    const int i0 = (blockIdx.y * 8 + (threadIdx.x >> 5)) * DOT_VPW;
    if (i0 >= m) return;
    const int nv = min(DOT_VPW, m - i0);
    const int64_t chunk = (n + nblk - 1) / nblk;
    const int64_t e0 = b * chunk, e1 = min(n, e0 + chunk);
    const double2* __restrict__ wr = w + (int64_t)r * n;
    float4 S[DOT_VPW];
#pragma unroll
    for (int u = 0; u < DOT_VPW; ++u) S[u] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 2
    for (int64_t e = e0 + lane; e < e1; e += 32) {
        const float4 c = ddf::split2(wr[e]);
#pragma unroll
        for (int u = 0; u < DOT_VPW; ++u)
            if (u < nv) ddf::cmac<true>(S[u], ddf::split2(Vb[((int64_t)(i0 + u) * R + r) * n + e]), c);
    }
#pragma unroll
    for (int u = 0; u < DOT_VPW; ++u) {
        if (u >= nv) break;
        float4 t = S[u];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float4 q;
            q.x = __shfl_xor_sync(0xffffffffu, t.x, o);
            q.y = __shfl_xor_sync(0xffffffffu, t.y, o);
            q.z = __shfl_xor_sync(0xffffffffu, t.z, o);
            q.w = __shfl_xor_sync(0xffffffffu, t.w, o);
            ddf::add(t, q);
        }
        if (lane == 0) partial[((int64_t)r * m + i0 + u) * nblk + b] = ddf::value(t);
    }
}

// out[r * ostride + i] = sum_b partial[r][i][b]  (+= when accumulate)
__global__ void k_dots_final(const double2* __restrict__ partial, int m, int nblk, double2* __restrict__ out,
                             int64_t ostride, int accumulate) {
    const int i = blockIdx.x, r = blockIdx.y;
    double2 s = make_double2(0, 0);
    for (int b = threadIdx.x; b < nblk; b += 32) {
        const double2 p = partial[((int64_t)r * m + i) * nblk + b];
        s.x += p.x;
        s.y += p.y;
    }
    s = warp_sum2(s);
    if (threadIdx.x == 0) {
        double2* o = out + r * ostride + i;
        if (accumulate) { o->x += s.x; o->y += s.y; }
        else *o = s;
    }
}

// w_r -= sum_{i<m} h_r[i] V_{i,r}   or (overwrite) x_r = sum_{i<m_r} y_r[i] V_{i,r}.
// A block takes 32 rows; its 8 warps take the basis vectors i = warp (mod 8), and the 8
// partial sums of a row are added in a fixed order: many more threads than rows for the
// latency-bound late iterations.  HS: the coefficients are split once per block into
// shared memory (m of them), else per use.
constexpr int COMBINE_HS_MAX = 2048;

template <bool HS>
__global__ void __launch_bounds__(256) k_combine(const double2* __restrict__ Vb, int64_t n, int R, int m,
                                                 const int* __restrict__ mr, const double2* __restrict__ h,
                                                 int64_t hstride, double2* __restrict__ w, int overwrite) {
    extern __shared__ float4 hs[];
    const int r = blockIdx.y;
    const int lr = threadIdx.x & 31, sl = threadIdx.x >> 5;
    const int64_t e = blockIdx.x * 32ll + lr;
    const int mm = mr ? mr[r] : m;
    const double2* __restrict__ hr = h + r * hstride;
    if (HS) {
        for (int i = threadIdx.x; i < mm; i += blockDim.x) hs[i] = ddf::split2(hr[i]);
        __syncthreads();
    }
    float4 S = make_float4(0.f, 0.f, 0.f, 0.f);
    if (e < n) {
#pragma unroll 4
        for (int i = sl; i < mm; i += 8) {
            const float4 hv = HS ? hs[i] : ddf::split2(hr[i]);
            ddf::cmac<false>(S, hv, ddf::split2(Vb[((int64_t)i * R + r) * n + e]));
        }
    }
    __shared__ float4 part[8][32];
    part[sl][lr] = S;
    __syncthreads();
    if (sl == 0 && e < n) {
        float4 t = part[0][lr];
#pragma unroll
        for (int k = 1; k < 8; ++k) ddf::add(t, part[k][lr]);
        const double2 tv = ddf::value(t);
        double2* wr = w + (int64_t)r * n;
        if (overwrite) wr[e] = tv;
        else {
            const double2 q = wr[e];
            wr[e] = make_double2(q.x - tv.x, q.y - tv.y);
        }
    }
}

// the basis update / combination above, with the coefficients in shared memory when
// their count is known on the host and small enough
bem_status launch_combine(dim3 grid, const double2* Vb, int64_t n, int R, int m, const int* mr, const double2* h,
                          int64_t hstride, double2* w, int overwrite, cudaStream_t s) {
    if (!mr && m <= COMBINE_HS_MAX)
        BEM_LAUNCH(k_combine<true>, grid, 256, (size_t)m * sizeof(float4), s, Vb, n, R, m, mr, h, hstride, w,
                   overwrite);
    else BEM_LAUNCH(k_combine<false>, grid, 256, 0, s, Vb, n, R, m, mr, h, hstride, w, overwrite);
    return BEM_OK;
}

__global__ void k_add_cols(double2* __restrict__ a, int64_t astride, const double2* __restrict__ b,
                           int64_t bstride, int m) {
    const int r = blockIdx.y;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        a[r * astride + i].x += b[r * bstride + i].x;
        a[r * astride + i].y += b[r * bstride + i].y;
    }
}

// the norm and its reciprocal once per block (FP64 square roots and divisions run on
// GB300's narrow FP64 pipe: one per thread cost more than the whole copy)
__device__ __forceinline__ double2 block_norm_inv(const double2* __restrict__ nrm2, int r) {
    __shared__ double2 ni;
    if (threadIdx.x == 0) {
        const double nr = sqrt(fmax(nrm2[r].x, 0.0));
        ni = make_double2(nr, nr > 0.0 ? 1.0 / nr : 0.0);
    }
    __syncthreads();
    return ni;
}

// v_r = w_r / |w_r| (|w_r|^2 = real part of nrm2[r]); writes |w_r| to dst[r * dstride]
__global__ void k_normalize(const double2* __restrict__ w, int64_t n, const double2* __restrict__ nrm2,
                            double2* __restrict__ v, int64_t vstride, double2* __restrict__ dst, int64_t dstride) {
    const int r = blockIdx.y;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const double2 ni = block_norm_inv(nrm2, r);
    if (e == 0 && dst) dst[r * dstride] = make_double2(ni.x, 0.0);
    if (e >= n) return;
    const double inv = ni.y;
    v[r * vstride + e] = make_double2(w[(int64_t)r * n + e].x * inv, w[(int64_t)r * n + e].y * inv);
}

// ---- complex64 Krylov basis (mixed precision, several right-hand sides)
// The inner solves of a batch run on FP32 or tensor-core products (~1e-7) and are
// refined against the FP64 residual, so their basis is stored in complex64 and
// orthogonalised in FP32 arithmetic: half the bytes of the basis passes, which for a
// batch are most of an iteration's memory traffic.  CGS2 keeps the FP32 basis
// orthogonal to O(2^-24).  The working vector w stays FP64; the current basis vector
// is also kept widened to FP64 (exactly the stored value) as the operator's input.
constexpr int DOT32_VPW = 8;              // basis vectors per warp
constexpr int DOT32_VPB = 8 * DOT32_VPW;  // basis vectors per block

// conj(V_{i,r}) . w_r partial sums over row chunks, as k_dots_partial: FP32 products
// and sums within a chunk, partial[((r * m) + i) * nblk + chunk] in FP64
__global__ void __launch_bounds__(256) k_dots_partial32(const float2* __restrict__ Vb, int64_t n, int R, int m,
                                                        const double2* __restrict__ w, int nblk,
                                                        double2* __restrict__ partial) {
    const int r = blockIdx.z, b = blockIdx.x;
    const int lane = threadIdx.x & 31;
    const int i0 = (blockIdx.y * 8 + (threadIdx.x >> 5)) * DOT32_VPW;
    if (i0 >= m) return;
    const int nv = min(DOT32_VPW, m - i0);
    const int64_t chunk = (n + nblk - 1) / nblk;
    const int64_t e0 = b * chunk, e1 = min(n, e0 + chunk);
    const double2* __restrict__ wr = w + (int64_t)r * n;
    float2 S[DOT32_VPW];
#pragma unroll
    for (int u = 0; u < DOT32_VPW; ++u) S[u] = make_float2(0.f, 0.f);
#pragma unroll 2
    for (int64_t e = e0 + lane; e < e1; e += 32) {
        const double2 wd = wr[e];
        const float wx = (float)wd.x, wy = (float)wd.y;
#pragma unroll
        for (int u = 0; u < DOT32_VPW; ++u)
            if (u < nv) {
                const float2 v = Vb[((int64_t)(i0 + u) * R + r) * n + e];
                S[u].x = fmaf(v.x, wx, fmaf(v.y, wy, S[u].x));
                S[u].y = fmaf(v.x, wy, fmaf(-v.y, wx, S[u].y));
            }
    }
#pragma unroll
    for (int u = 0; u < DOT32_VPW; ++u) {
        if (u >= nv) break;
        float2 t = S[u];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
            t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
        }
        if (lane == 0) partial[((int64_t)r * m + i0 + u) * nblk + b] = make_double2(t.x, t.y);
    }
}

// w_r -= sum_{i<m} h_r[i] V_{i,r}  or (overwrite) x_r = sum_{i<m_r} y_r[i] V_{i,r}, as
// k_combine with the sums in FP32 (fixed order) and the update of w in FP64
template <bool HS>
__global__ void __launch_bounds__(256) k_combine32(const float2* __restrict__ Vb, int64_t n, int R, int m,
                                                   const int* __restrict__ mr, const double2* __restrict__ h,
                                                   int64_t hstride, double2* __restrict__ w, int overwrite) {
    extern __shared__ float2 hs2[];
    const int r = blockIdx.y;
    const int lr = threadIdx.x & 31, sl = threadIdx.x >> 5;
    const int64_t e = blockIdx.x * 32ll + lr;
    const int mm = mr ? mr[r] : m;
    const double2* __restrict__ hr = h + r * hstride;
    if (HS) {
        for (int i = threadIdx.x; i < mm; i += blockDim.x) hs2[i] = make_float2((float)hr[i].x, (float)hr[i].y);
        __syncthreads();
    }
    float2 S = make_float2(0.f, 0.f);
    if (e < n) {
#pragma unroll 4
        for (int i = sl; i < mm; i += 8) {
            const float2 hv = HS ? hs2[i] : make_float2((float)hr[i].x, (float)hr[i].y);
            const float2 v = Vb[((int64_t)i * R + r) * n + e];
            S.x = fmaf(hv.x, v.x, fmaf(-hv.y, v.y, S.x));
            S.y = fmaf(hv.x, v.y, fmaf(hv.y, v.x, S.y));
        }
    }
    __shared__ float2 part[8][32];
    part[sl][lr] = S;
    __syncthreads();
    if (sl == 0 && e < n) {
        float2 t = part[0][lr];
#pragma unroll
        for (int k = 1; k < 8; ++k) {
            t.x += part[k][lr].x;
            t.y += part[k][lr].y;
        }
        double2* wr = w + (int64_t)r * n;
        if (overwrite) wr[e] = make_double2(t.x, t.y);
        else {
            const double2 q = wr[e];
            wr[e] = make_double2(q.x - (double)t.x, q.y - (double)t.y);
        }
    }
}

bem_status launch_combine32(dim3 grid, const float2* Vb, int64_t n, int R, int m, const int* mr, const double2* h,
                            int64_t hstride, double2* w, int overwrite, cudaStream_t s) {
    if (!mr && m <= COMBINE_HS_MAX)
        BEM_LAUNCH(k_combine32<true>, grid, 256, (size_t)m * sizeof(float2), s, Vb, n, R, m, mr, h, hstride, w,
                   overwrite);
    else BEM_LAUNCH(k_combine32<false>, grid, 256, 0, s, Vb, n, R, m, mr, h, hstride, w, overwrite);
    return BEM_OK;
}

// CGS2's first update and second projection in one pass over the basis: w_r -= sum_{i<m}
// h_r[i] V_{i,r} over the block's CD_ROWS rows (as k_combine32: FP32 sums in a fixed
// order, the update in FP64), then the inner products of the updated rows with the same
// m basis vectors (as k_dots_partial32), partial[((r * m) + i) * nchunk + block].  The
// second read of the block's basis rows comes from L1/L2, so the basis crosses HBM three
// times per iteration instead of four.  m <= COMBINE_HS_MAX (coefficients in shared memory).
constexpr int CD_ROWS = 128;  // rows per block, 4 per lane

__global__ void __launch_bounds__(256) k_combine_dots32(const float2* __restrict__ Vb, int64_t n, int R, int m,
                                                        const double2* __restrict__ h, int64_t hstride,
                                                        double2* __restrict__ w, int nchunk,
                                                        double2* __restrict__ partial) {
    extern __shared__ float2 hs2[];
    __shared__ float2 part[8][CD_ROWS];
    __shared__ float2 w1s[CD_ROWS];
    const int r = blockIdx.y, b = blockIdx.x;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int64_t e0 = (int64_t)b * CD_ROWS;
    const double2* __restrict__ hr = h + r * hstride;
    for (int i = threadIdx.x; i < m; i += blockDim.x) hs2[i] = make_float2((float)hr[i].x, (float)hr[i].y);
    __syncthreads();
    float2 S[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) S[q] = make_float2(0.f, 0.f);
    for (int i = wp; i < m; i += 8) {
        const float2 hv = hs2[i];
        const float2* __restrict__ vi = Vb + ((int64_t)i * R + r) * n;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t e = e0 + lane + 32 * q;
            if (e < n) {
                const float2 v = vi[e];
                S[q].x = fmaf(hv.x, v.x, fmaf(-hv.y, v.y, S[q].x));
                S[q].y = fmaf(hv.x, v.y, fmaf(hv.y, v.x, S[q].y));
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) part[wp][lane + 32 * q] = S[q];
    __syncthreads();
    if (threadIdx.x < CD_ROWS) {
        const int t = threadIdx.x;
        const int64_t e = e0 + t;
        float2 acc = part[0][t];
#pragma unroll
        for (int k = 1; k < 8; ++k) {
            acc.x += part[k][t].x;
            acc.y += part[k][t].y;
        }
        float2 wf = make_float2(0.f, 0.f);
        if (e < n) {
            double2* wr = w + (int64_t)r * n;
            const double2 q = wr[e];
            const double2 u = make_double2(q.x - (double)acc.x, q.y - (double)acc.y);
            wr[e] = u;
            wf = make_float2((float)u.x, (float)u.y);
        }
        w1s[t] = wf;
    }
    __syncthreads();
    for (int i = wp; i < m; i += 8) {
        const float2* __restrict__ vi = Vb + ((int64_t)i * R + r) * n;
        float2 t = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t e = e0 + lane + 32 * q;
            if (e < n) {
                const float2 v = vi[e];
                const float2 c = w1s[lane + 32 * q];
                t.x = fmaf(v.x, c.x, fmaf(v.y, c.y, t.x));
                t.y = fmaf(v.x, c.y, fmaf(-v.y, c.x, t.y));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
            t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
        }
        if (lane == 0) partial[((int64_t)r * m + i) * nchunk + b] = make_double2(t.x, t.y);
    }
}

// v_r = w_r / |w_r| into the complex64 basis, and the stored value widened into
// vcur (columns of length n, stride n); |w_r| to dst[r * dstride]
__global__ void k_normalize32(const double2* __restrict__ w, int64_t n, const double2* __restrict__ nrm2,
                              float2* __restrict__ v, double2* __restrict__ vcur, double2* __restrict__ dst,
                              int64_t dstride) {
    const int r = blockIdx.y;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const double2 ni = block_norm_inv(nrm2, r);
    if (e == 0 && dst) dst[r * dstride] = make_double2(ni.x, 0.0);
    if (e >= n) return;
    const double inv = ni.y;
    const double2 q = w[(int64_t)r * n + e];
    const float2 f = make_float2((float)(q.x * inv), (float)(q.y * inv));
    v[(int64_t)r * n + e] = f;
    vcur[(int64_t)r * n + e] = make_double2(f.x, f.y);
}

// y = a - b;  x += d (whole blocks)
__global__ void k_sub(const double2* __restrict__ a, const double2* __restrict__ b, int64_t n,
                      double2* __restrict__ y) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) y[e] = make_double2(a[e].x - b[e].x, a[e].y - b[e].y);
}

__global__ void k_acc(double2* __restrict__ x, const double2* __restrict__ d, int64_t n) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) {
        x[e].x += d[e].x;
        x[e].y += d[e].y;
    }
}

// ------------------------------------------------------------------ host side
// ELL form of one grid's mass matrix (values of this solve)
struct MassEll {
    DevBuf ci, v, vf;  // vf: FP32 copy of the values (FP32 Chebyshev iterations)
    int W = 0;
    bem_status build(const bem_grid* g, const double* val, cudaStream_t s) {
        W = std::max(1, (int)g->m_maxrow);
        BEM_TRY(ci.alloc((size_t)W * g->nv * 4, s));
        BEM_TRY(v.alloc((size_t)W * g->nv * 8, s));
        BEM_LAUNCH(k_mass_ell, blocks_for(g->nv, 128), 128, 0, s, g->m_rowptr.as<int32_t>(), g->m_col.as<int32_t>(),
                   val, g->nv, W, ci.as<int32_t>(), v.as<double>());
        BEM_TRY(vf.alloc((size_t)W * g->nv * 4, s));
        BEM_LAUNCH(k_narrow, blocks_for((int64_t)W * g->nv, 256), 256, 0, s, v.as<double>(), (int64_t)W * g->nv,
                   vf.as<float>());
        return BEM_OK;
    }
};

// Fixed launch sequences of an iteration (the same kernels with the same arguments and
// buffers every time it runs) replayed as CUDA graphs: the sequence is captured on its
// first run under a key that fixes all of its arguments, and each later run with that
// key is one graph launch.  Used for the Chebyshev mass inverses (18 to 35 short
// kernels per application).  Profiling that times every kernel, a disabled cache, or a
// stream that cannot be captured runs the sequence kernel by kernel instead (same
// kernels, same results).
struct GraphKey {
    const void *a, *b, *c;
    int64_t i, j;
    bool operator==(const GraphKey& o) const { return a == o.a && b == o.b && c == o.c && i == o.i && j == o.j; }
};

struct GraphCache {
    struct Entry {
        GraphKey key;
        cudaGraphExec_t exec;
        uint64_t kernels;
    };
    std::vector<Entry> entries;
    bool enabled = true;
    explicit GraphCache(bool on) : enabled(on) {}
    GraphCache(const GraphCache&) = delete;
    GraphCache& operator=(const GraphCache&) = delete;
    ~GraphCache() {
        for (Entry& e : entries) cudaGraphExecDestroy(e.exec);
    }
    template <class F>
    bem_status run(const GraphKey& key, cudaStream_t s, F&& body) {
        if (!enabled || s == nullptr || prof_times_every_kernel()) return body();
        for (const Entry& e : entries)
            if (e.key == key) {
                BEM_CUDA_TRY(cudaGraphLaunch(e.exec, s));
                count_launch(e.kernels);
                return BEM_OK;
            }
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            enabled = false;
            return body();
        }
        g_capturing = 1;
        const bem_status st = body();
        g_capturing = 0;
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(s, &g);
        cudaGraphExec_t ex = nullptr;
        size_t nodes = 0;
        bool ok = st == BEM_OK && ce == cudaSuccess && g != nullptr &&
                  cudaGraphGetNodes(g, nullptr, &nodes) == cudaSuccess;
        uint64_t kernels = 0;  // kernel nodes (memset nodes are not launches)
        if (ok) {
            std::vector<cudaGraphNode_t> list(nodes);
            ok = cudaGraphGetNodes(g, list.data(), &nodes) == cudaSuccess;
            for (size_t i = 0; ok && i < nodes; ++i) {
                cudaGraphNodeType t;
                ok = cudaGraphNodeGetType(list[i], &t) == cudaSuccess;
                if (ok && t == cudaGraphNodeTypeKernel) ++kernels;
            }
        }
        ok = ok && cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        if (!ok) {
            // capture refused (this stream, or a launch that cannot be captured): from now on
            // launch the sequences directly; a real error shows again when they run
            cudaGetLastError();
            enabled = false;
            return body();
        }
        entries.push_back({key, ex, kernels});
        BEM_CUDA_TRY(cudaGraphLaunch(ex, s));
        count_launch(kernels);
        return BEM_OK;
    }
};

struct MassOp {
    MassPair M{};
    double2 *r = nullptr, *dA = nullptr, *dB = nullptr;  // workspaces [R * n]
    GraphCache* graphs = nullptr;                        // replay the step sequence as a graph
    GridBarrier* bar = nullptr;  // set: the iteration runs as one cooperative launch
    int* err = nullptr;          // its barrier's failure flag (checked by the solve)
};

// Blocks of k_cheb_fused that fit on the current device at once (0: no cooperative launch)
int cheb_fused_capacity() {
    static std::mutex mu;
    static int cap[64];
    static bool known[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 0;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!known[dev]) {
        int sms = 0, coop = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cheb_fused, 256, 0) != cudaSuccess) {
            cudaGetLastError();
            cap[dev] = 0;
        } else {
            cap[dev] = coop ? sms * per_sm : 0;
        }
        known[dev] = true;
    }
    return cap[dev];
}

// Barrier and failure flag shared by the fused mass inverses of one solve (its launches
// run one after another on one stream)
struct ChebSync {
    DevBuf buf;
    bem_status init(cudaStream_t s) {
        BEM_TRY(buf.alloc(64, s));
        BEM_CUDA_TRY(cudaMemsetAsync(buf.p, 0, 64, s));
        return BEM_OK;
    }
    GridBarrier* bar() { return buf.as<GridBarrier>(); }
    int* err() { return reinterpret_cast<int*>(static_cast<char*>(buf.p) + 32); }
    void attach(MassOp& op) {
        op.bar = bar();
        op.err = err();
    }
    // a barrier wait that timed out in any of the solve's mass inverses
    bem_status check() {
        int h = 0;
        BEM_CUDA_TRY(cudaMemcpy(&h, err(), sizeof(int), cudaMemcpyDeviceToHost));
        if (h) {
            set_error("mass inverse: a grid barrier wait timed out");
            return BEM_E_INTERNAL;
        }
        return BEM_OK;
    }
};

// M^-1 on the four blocks of R columns, Chebyshev on the Jacobi-scaled mass matrices
bem_status mass_solve(const MassOp& op, const double2* z, double2* y, int R, cudaStream_t s, int steps) {
    if (op.graphs && !g_capturing) {
        MassOp eager = op;
        eager.graphs = nullptr;
        return op.graphs->run(GraphKey{op.r, z, y, R, steps}, s,
                              [&]() { return mass_solve(eager, z, y, R, s, steps); });
    }
    const int64_t n = op.M.n;
    const double theta = 0.5 * (CHEB_BETA + CHEB_ALPHA), delta = 0.5 * (CHEB_BETA - CHEB_ALPHA);
    const double sigma = theta / delta;
    const int cap = op.bar ? cheb_fused_capacity() : 0;
    if (cap > 0) {
        // one cooperative launch for the whole iteration (steps + 1 launches otherwise):
        // one item per thread where half the resident blocks suffice (so that a second
        // such launch from another stream would still fit beside it)
        const int64_t items = (int64_t)R * n;
        const int G = (int)std::max<int64_t>(1, std::min<int64_t>(std::max(1, cap / 2), (items + 255) / 256));
        BEM_CUDA_TRY(cudaMemsetAsync(op.bar, 0, sizeof(GridBarrier), s));
        MassPair M = op.M;
        const double2* zp = z;
        double2 *yp = y, *rp = op.r, *ap = op.dA, *bp = op.dB;
        int Rv = R, sv = steps;
        double inv_theta = 1.0 / theta, sg = sigma, dl = delta;
        GridBarrier* bar = op.bar;
        int* err = op.err;
        void* args[] = {&M, &zp, &yp, &rp, &ap, &bp, &Rv, &sv, &inv_theta, &sg, &dl, &bar, &err};
        const int slot = g_capturing ? -1 : prof_begin("k_cheb_fused", s);
        const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_cheb_fused, dim3(G), dim3(256), args, 0, s);
        prof_end(slot, s);
        BEM_CUDA_TRY(e);
        if (!g_capturing) count_launch();
        return BEM_OK;
    }
    // small blocks by default: a step is FP64 work of a few rows per thread, spread over
    // every SM
    const int nb = tune_get(TUNE_CHEB, R, n, TuneChoice{64, 0, 0.0}).block;
    const dim3 grid(blocks_for(n, nb), R);
    if (steps <= CHEB_STEPS_INNER && op.M.vf[0] && op.M.vf[1] && steps >= 1 && (int64_t)R * n < (1ll << 31)) {
        // FP32 iteration, vectors interleaved by column: r in op.r, d in the first halves
        // of dA / dB, y in the second half of dA
        float2* r32 = reinterpret_cast<float2*>(op.r);
        float2* da = reinterpret_cast<float2*>(op.dA);
        float2* db = reinterpret_cast<float2*>(op.dB);
        float2* y32 = da + (int64_t)R * n;
        const dim3 g1(blocks_for((int64_t)R * n, nb));
        BEM_LAUNCH(k_cheb_init32, g1, nb, 0, s, op.M, R, z, r32, da, (float)(1.0 / theta));
        double rho = 1.0 / sigma;
        float2 *dk = da, *dn = db;
        for (int k = 0; k < steps; ++k) {
            const double rho_n = 1.0 / (2.0 * sigma - rho);
            BEM_LAUNCH(k_cheb_step32, g1, nb, 0, s, op.M, R, dk, dn, y32, r32, (float)(rho_n * rho),
                       (float)(2.0 * rho_n / delta), k == 0 ? 1 : 0, k == steps - 1 ? y : nullptr);
            rho = rho_n;
            std::swap(dk, dn);
        }
        return BEM_OK;
    }
    BEM_LAUNCH(k_cheb_init, grid, nb, 0, s, op.M, z, y, op.r, op.dA, 1.0 / theta);
    double rho = 1.0 / sigma;
    double2 *dk = op.dA, *dn = op.dB;
    for (int k = 0; k < steps; ++k) {
        const double rho_n = 1.0 / (2.0 * sigma - rho);
        BEM_LAUNCH(k_cheb_step, grid, nb, 0, s, op.M, dk, dn, y, op.r, rho_n * rho, 2.0 * rho_n / delta);
        rho = rho_n;
        std::swap(dk, dn);
    }
    return BEM_OK;
}

struct CsrBuf {
    DevBuf rp, ci, v;
};

// CSR of the COO list (key, other, val) with `rows` rows keyed by `key`
bem_status build_csr(const int32_t* key, const int32_t* other, const double* val, int64_t nnz, int64_t rows,
                     CsrBuf& out, cudaStream_t s) {
    DevBuf cnt, start, fill, oc, ov;
    const size_t cap = (size_t)std::max<int64_t>(nnz, 1);
    BEM_TRY(cnt.alloc(rows * 4, s));
    BEM_TRY(start.alloc((rows + 1) * 4, s));
    BEM_TRY(fill.alloc(rows * 4, s));
    BEM_TRY(oc.alloc(cap * 4, s));
    BEM_TRY(ov.alloc(cap * 8, s));
    BEM_TRY(out.rp.alloc((rows + 1) * 4, s));
    BEM_TRY(out.ci.alloc(cap * 4, s));
    BEM_TRY(out.v.alloc(cap * 8, s));
    BEM_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, rows * 4, s));
    BEM_CUDA_TRY(cudaMemsetAsync(fill.p, 0, rows * 4, s));
    if (nnz > 0) BEM_LAUNCH(k_csr_count, blocks_for(nnz, 256), 256, 0, s, key, val, nnz, cnt.as<int32_t>());
    BEM_LAUNCH(k_scan, 1, 1024, 0, s, cnt.as<int32_t>(), rows, start.as<int32_t>());
    if (nnz > 0)
        BEM_LAUNCH(k_csr_scatter, blocks_for(nnz, 256), 256, 0, s, key, other, val, nnz, start.as<int32_t>(),
                   fill.as<int32_t>(), oc.as<int32_t>(), ov.as<double>());
    if (rows > 0)
        BEM_LAUNCH(k_csr_merge, (unsigned)rows, 256, 0, s, start.as<int32_t>(), rows, oc.as<int32_t>(), ov.as<double>(),
               cnt.as<int32_t>());
    BEM_LAUNCH(k_scan, 1, 1024, 0, s, cnt.as<int32_t>(), rows, out.rp.as<int32_t>());
    BEM_LAUNCH(k_csr_compact, blocks_for(rows, 128), 128, 0, s, start.as<int32_t>(), out.rp.as<int32_t>(), rows,
               oc.as<int32_t>(), ov.as<double>(), out.ci.as<int32_t>(), out.v.as<double>());
    return BEM_OK;
}

bem_status transfer_add(const TransferCsr& t, int R, const double2* x, double2* z, cudaStream_t s) {
    BEM_LAUNCH(k_transfer, dim3(blocks_for(t.n, 64), R), 64, 0, s, t, x, z);
    return BEM_OK;
}

// compiled widths of the multi-column kernels; a batch of R columns runs at the
// next width and the padding columns read and write spare, in-bounds slots

using Apply = std::function<bem_status(const double2* in, double2* out, int R)>;
using StopCheck = std::function<bem_status()>;

// iterations a host check of the residual trails the launches by (the GPU keeps
// this many iterations queued; at most this many are computed past convergence)
constexpr int GMRES_LAG = 2;

// relative inner tolerances of the mixed mode's refinement when
// bem_solve_opts.ir_inner_tol is 0: one right-hand side (double-float products above
// the switch point: one inner solve reaches the target) and batches (FP32 or
// tensor-core products throughout: the true inner residual stalls near their
// accuracy while the recurrence estimate runs on, so the first inner solve stops
// early and a second one starts from the FP64 residual)
constexpr double IR_INNER_TOL_SINGLE = 1e-8;
constexpr double IR_INNER_TOL_BATCH = 1e-5;

// Tolerance of an inner solve whose right-hand side has norm rin (in the inner
// preconditioner's norm) while the outer residual has norm rn against the target
// tol_abs: a reduction by inner_rel, or by what the last pass needs with a margin of 2
// (so that the outer residual, measured with the exact mass inverse, lands below the
// target even where the two norms differ slightly).
double inner_tolerance(double rin, double rn, double tol_abs, double inner_rel) {
    const double last = rn > 0.0 ? 0.5 * tol_abs / rn : 1.0;
    return rin * std::max(inner_rel, last);
}
constexpr int GMRES_SLOTS = GMRES_LAG + 2;

using cplx = std::complex<double>;

// Arnoldi state on the device (basis, Hessenberg columns, reductions) and the small
// least-squares problem on the host: each new Hessenberg column is copied to pinned
// memory and the Givens QR, the residual estimate and the final back substitution
// are done there (O(j) sequential FP64 work per iteration, microseconds on a CPU core,
// but a long dependent chain for one GPU thread).
struct GmresWork {
    int maxit = 0, R = 0, RW = 0, nblk = 0;
    int64_t n = 0, ldh = 0, gstride = 0;
    bool f32 = false;  // complex64 basis + FP32 orthogonalisation (vcur: the current vector in FP64)
    DevBuf Vb, H, partial, hbuf, y, w, nrm, mr, vcur;
    double2* h_nrm = nullptr;  // pinned, [R]
    double2* h_col = nullptr;  // pinned, [GMRES_SLOTS][R][maxit + 2]: copied Hessenberg columns
    double2* h_y = nullptr;    // pinned, [R][gstride]: least-squares solutions
    int* h_mr = nullptr;       // pinned, [R]
    double* h_wave = nullptr;  // pinned, [5 R]: plane-wave amplitudes (R complex) then directions (3 R)
    cudaEvent_t ev[GMRES_SLOTS] = {};
    cudaStream_t stream = nullptr;
    ~GmresWork() {
        // an early return (cancel, deadline, error) may leave copies into pinned memory queued
        if (stream) cudaStreamSynchronize(stream);
        if (h_nrm) cudaFreeHost(h_nrm);
        if (h_col) cudaFreeHost(h_col);
        if (h_y) cudaFreeHost(h_y);
        if (h_mr) cudaFreeHost(h_mr);
        if (h_wave) cudaFreeHost(h_wave);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
    bem_status init(int maxit_, int64_t n_, int R_, int spare, cudaStream_t s, bool f32_ = false) {
        maxit = maxit_;
        n = n_;
        R = R_;
        stream = s;
        RW = R_ + spare;
        f32 = f32_;
        nblk = dot_blocks(n_);
        ldh = maxit + 1;
        gstride = maxit + 2;
        if (f32) {
            // (maxit + 1) complex64 basis blocks of R columns; the operator reads vcur,
            // whose RW - R spare columns stay zero for the width-padded kernels
            const size_t vb = (size_t)(maxit + 1) * R * n * 8;
            BEM_TRY(Vb.alloc(vb, s));
            BEM_CUDA_TRY(cudaMemsetAsync(Vb.p, 0, vb, s));
            BEM_TRY(vcur.alloc((size_t)RW * n * 16, s));
            BEM_CUDA_TRY(cudaMemsetAsync(vcur.p, 0, vcur.bytes, s));
        } else {
            // (maxit + 1) basis blocks of R columns, plus RW - R spare columns read by the
            // width-padded operator kernels past the last block
            const size_t vb = ((size_t)(maxit + 1) * R + (RW - R)) * n * 16;
            BEM_TRY(Vb.alloc(vb, s));
            BEM_CUDA_TRY(cudaMemsetAsync(Vb.p, 0, vb, s));
        }
        BEM_TRY(H.alloc((size_t)R * ldh * ldh * 16, s));
        // inner-product partials: nblk chunks, or the fused kernel's CD_ROWS-row chunks
        const int64_t nchunk = std::max<int64_t>(nblk, f32 ? (n + CD_ROWS - 1) / CD_ROWS : 0);
        BEM_TRY(partial.alloc((size_t)R * (maxit + 1) * nchunk * 16, s));
        BEM_TRY(hbuf.alloc((size_t)R * gstride * 16, s));
        BEM_TRY(y.alloc((size_t)R * gstride * 16, s));
        BEM_TRY(w.alloc((size_t)R * n * 16, s));
        BEM_TRY(nrm.alloc(R * 16, s));
        BEM_TRY(mr.alloc(R * 4, s));
        BEM_CUDA_TRY(cudaMallocHost(&h_nrm, (size_t)R * 16));
        BEM_CUDA_TRY(cudaMallocHost(&h_col, (size_t)GMRES_SLOTS * R * gstride * 16));
        BEM_CUDA_TRY(cudaMallocHost(&h_y, (size_t)R * gstride * 16));
        BEM_CUDA_TRY(cudaMallocHost(&h_mr, (size_t)R * 4));
        BEM_CUDA_TRY(cudaMallocHost(&h_wave, (size_t)5 * R * 8));
        for (cudaEvent_t& e : ev) BEM_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        return BEM_OK;
    }
    // squared norms of the R columns of v (stored back to back) into nrm[r].x
    bem_status sq_norms(const double2* v, cudaStream_t s) {
        // with basis width 1 and m = 1, "basis vector 0" of column r is v + r * n
        BEM_LAUNCH(k_dots_partial, dim3(nblk, 1, R), 256, 0, s, v, n, 1, 1, v, nblk, partial.as<double2>());
        BEM_LAUNCH(k_dots_final, dim3(1, R), 32, 0, s, partial.as<double2>(), 1, nblk, nrm.as<double2>(), 1, 0);
        return BEM_OK;
    }
};

// 2-norms of R columns stored back to back -> host
bem_status norms(GmresWork& W, const double2* v, int R, double* out, cudaStream_t s) {
    BEM_TRY(W.sq_norms(v, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(W.h_nrm, W.nrm.p, R * 16, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    for (int r = 0; r < R; ++r) out[r] = std::sqrt(std::max(W.h_nrm[r].x, 0.0));
    return BEM_OK;
}

// Givens QR of one right-hand side's Hessenberg matrix, one column at a time
struct HostQR {
    std::vector<std::vector<cplx>> Rc;  // Rc[j][0..j]: column j of the triangular factor
    std::vector<double> cs;
    std::vector<cplx> sn, g;
    void reset(double beta) {
        Rc.clear();
        cs.clear();
        sn.clear();
        g.assign(1, cplx(beta, 0.0));
    }
    // column j (entries 0..j+1); returns |g_{j+1}|, the residual estimate
    double add_column(const double2* col, int j) {
        std::vector<cplx> h(j + 2);
        for (int i = 0; i < j + 2; ++i) h[i] = cplx(col[i].x, col[i].y);
        for (int i = 0; i < j; ++i) {  // h[i] = c h[i] + s h[i+1];  h[i+1] = -conj(s) h[i] + c h[i+1]
            const cplx a = h[i], b = h[i + 1];
            h[i] = cs[i] * a + sn[i] * b;
            h[i + 1] = -std::conj(sn[i]) * a + cs[i] * b;
        }
        const cplx a = h[j], b = h[j + 1];
        const double aa = std::abs(a), bb = std::abs(b);
        double c;
        cplx sv, rr;
        if (aa == 0.0) {
            c = 0.0;
            sv = cplx(1.0, 0.0);
            rr = b;
        } else {
            const double t = std::hypot(aa, bb);
            const cplx ph = a / aa;
            c = aa / t;
            sv = ph * std::conj(b) / t;
            rr = ph * t;
        }
        cs.push_back(c);
        sn.push_back(sv);
        h[j] = rr;
        h.resize(j + 1);
        Rc.push_back(std::move(h));
        const cplx gj = g[j];
        g.push_back(-std::conj(sv) * gj);
        g[j] = c * gj;
        return std::abs(g[j + 1]);
    }
    // y = R(0:m,0:m)^-1 g(0:m)
    void solve(int m, double2* y) const {
        std::vector<cplx> w(g.begin(), g.begin() + m);
        for (int c = m - 1; c >= 0; --c) {
            const cplx d = Rc[c][c];
            const cplx yc = std::norm(d) > 0.0 ? w[c] / d : cplx(0.0, 0.0);
            y[c] = make_double2(yc.real(), yc.imag());
            for (int i = 0; i < c; ++i) w[i] -= Rc[c][i] * yc;
        }
    }
};

// Unrestarted GMRES from x0 = 0 on apply(x) = rhs for R columns in lockstep; column
// r stops counting once its residual estimate is <= tol_abs[r].  The Hessenberg
// column of iteration j is copied to pinned memory and processed GMRES_LAG
// iterations later, so the host never waits for the GPU to drain; iterations
// launched past convergence do not touch the columns the solution uses.  Writes x
// (R columns); returns per-column iterations and final estimates.
bem_status gmres_run(GmresWork& W, int R, const Apply& apply, const double2* rhs, const double* beta,
                     const double* tol_abs, double2* x, int* iters_out, double* res_out, cudaStream_t s,
                     const StopCheck& stop, double* progress = nullptr) {
    const int64_t n = W.n, ldh = W.ldh, gs = W.gstride;
    double2* Vp = W.Vb.as<double2>();
    const dim3 eb(blocks_for(n, 256), R);
    const dim3 ecb(blocks_for(n, 32), R);  // k_combine: 32 rows per block
    BEM_CUDA_TRY(cudaMemsetAsync(W.H.p, 0, (size_t)R * ldh * ldh * 16, s));
    std::vector<HostQR> qr(R);
    std::vector<int> it(R, 0);
    std::vector<char> done(R, 0);
    int ndone = 0;
    for (int r = 0; r < R; ++r) {
        qr[r].reset(beta[r]);
        res_out[r] = beta[r];
        if (!(beta[r] > tol_abs[r])) {
            done[r] = 1;
            ++ndone;
        }
    }
    if (progress) *progress = 1.0;
    int launched = 0, checked = 0;
    auto check_one = [&]() -> bem_status {  // iteration `checked`, whose copy is enqueued
        const int slot = checked % GMRES_SLOTS;
        BEM_CUDA_TRY(cudaEventSynchronize(W.ev[slot]));
        for (int r = 0; r < R; ++r) {
            if (done[r]) continue;
            const double est = qr[r].add_column(W.h_col + ((size_t)slot * R + r) * gs, checked);
            it[r] = checked + 1;
            res_out[r] = est;
            if (!(est > tol_abs[r])) {
                done[r] = 1;
                ++ndone;
            }
        }
        if (progress) {  // largest relative estimate over the columns still iterating
            double worst = 0.0;
            for (int r = 0; r < R; ++r)
                if (!done[r] && beta[r] > 0.0) worst = std::max(worst, res_out[r] / beta[r]);
            *progress = worst;
        }
        ++checked;
        return BEM_OK;
    };
    float2* Vp32 = W.Vb.as<float2>();  // the complex64 basis (W.f32)
    // v_{j} = w / |w| into basis block j (and vcur), |w| to dst
    auto normalize_into = [&](const double2* wv, int j, double2* dst, int64_t dstride) -> bem_status {
        if (W.f32)
            BEM_LAUNCH(k_normalize32, eb, 256, 0, s, wv, n, W.nrm.as<double2>(), Vp32 + (int64_t)j * R * n,
                       W.vcur.as<double2>(), dst, dstride);
        else
            BEM_LAUNCH(k_normalize, eb, 256, 0, s, wv, n, W.nrm.as<double2>(), Vp + (int64_t)j * R * n, n, dst,
                       dstride);
        return BEM_OK;
    };
    if (ndone < R) {
        BEM_TRY(W.sq_norms(rhs, s));  // V_0 = rhs / beta
        BEM_TRY(normalize_into(rhs, 0, nullptr, 0));
        for (int j = 0; j < W.maxit && ndone < R; ++j) {
            const double2* vj = W.f32 ? W.vcur.as<double2>() : Vp + (int64_t)j * R * n;
            BEM_TRY(apply(vj, W.w.as<double2>(), R));
            double2* Hj = W.H.as<double2>() + (int64_t)j * ldh;  // + r * ldh * ldh per column
            if (W.f32 && j + 1 <= COMBINE_HS_MAX) {
                // CGS2 with the first update and the second projection fused
                const unsigned gy = (unsigned)((j + 1 + DOT32_VPB - 1) / DOT32_VPB);
                const int nch = (int)((n + CD_ROWS - 1) / CD_ROWS);
                BEM_LAUNCH(k_dots_partial32, dim3(W.nblk, gy, R), 256, 0, s, Vp32, n, R, j + 1, W.w.as<double2>(),
                           W.nblk, W.partial.as<double2>());
                BEM_LAUNCH(k_dots_final, dim3(j + 1, R), 32, 0, s, W.partial.as<double2>(), j + 1, W.nblk, Hj,
                           ldh * ldh, 0);
                BEM_LAUNCH(k_combine_dots32, dim3(nch, R), 256, (size_t)(j + 1) * sizeof(float2), s, Vp32, n, R,
                           j + 1, Hj, ldh * ldh, W.w.as<double2>(), nch, W.partial.as<double2>());
                BEM_LAUNCH(k_dots_final, dim3(j + 1, R), 32, 0, s, W.partial.as<double2>(), j + 1, nch,
                           W.hbuf.as<double2>(), gs, 0);
                BEM_TRY(launch_combine32(ecb, Vp32, n, R, j + 1, nullptr, W.hbuf.as<double2>(), gs, W.w.as<double2>(),
                                         0, s));
            } else {
                for (int pass = 0; pass < 2; ++pass) {  // CGS2
                    double2* h = pass == 0 ? Hj : W.hbuf.as<double2>();
                    const int64_t hst = pass == 0 ? ldh * ldh : gs;
                    if (W.f32) {
                        const unsigned gy = (unsigned)((j + 1 + DOT32_VPB - 1) / DOT32_VPB);
                        BEM_LAUNCH(k_dots_partial32, dim3(W.nblk, gy, R), 256, 0, s, Vp32, n, R, j + 1,
                                   W.w.as<double2>(), W.nblk, W.partial.as<double2>());
                    } else {
                        const unsigned gy = (unsigned)((j + 1 + DOT_VPB - 1) / DOT_VPB);
                        BEM_LAUNCH(k_dots_partial, dim3(W.nblk, gy, R), 256, 0, s, Vp, n, R, j + 1,
                                   W.w.as<double2>(), W.nblk, W.partial.as<double2>());
                    }
                    BEM_LAUNCH(k_dots_final, dim3(j + 1, R), 32, 0, s, W.partial.as<double2>(), j + 1, W.nblk, h,
                               hst, 0);
                    if (W.f32)
                        BEM_TRY(launch_combine32(ecb, Vp32, n, R, j + 1, nullptr, h, hst, W.w.as<double2>(), 0, s));
                    else BEM_TRY(launch_combine(ecb, Vp, n, R, j + 1, nullptr, h, hst, W.w.as<double2>(), 0, s));
                }
            }
            BEM_LAUNCH(k_add_cols, dim3(1, R), 256, 0, s, Hj, ldh * ldh, W.hbuf.as<double2>(), gs, j + 1);
            BEM_TRY(W.sq_norms(W.w.as<double2>(), s));
            BEM_TRY(normalize_into(W.w.as<double2>(), j + 1, Hj + j + 1, ldh * ldh));
            const int slot = j % GMRES_SLOTS;
            BEM_CUDA_TRY(cudaMemcpy2DAsync(W.h_col + (size_t)slot * R * gs, gs * 16, Hj, ldh * ldh * 16,
                                           (size_t)(j + 2) * 16, R, cudaMemcpyDeviceToHost, s));
            BEM_CUDA_TRY(cudaEventRecord(W.ev[slot], s));
            launched = j + 1;
            while (checked < launched - GMRES_LAG && ndone < R) BEM_TRY(check_one());
            if (stop) BEM_TRY(stop());
        }
        while (checked < launched && ndone < R) BEM_TRY(check_one());
    }
    for (int r = 0; r < R; ++r) {
        W.h_mr[r] = it[r];
        qr[r].solve(it[r], W.h_y + (size_t)r * gs);
    }
    BEM_CUDA_TRY(cudaMemcpyAsync(W.mr.p, W.h_mr, R * 4, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(W.y.p, W.h_y, (size_t)R * gs * 16, cudaMemcpyHostToDevice, s));
    if (W.f32) BEM_TRY(launch_combine32(ecb, Vp32, n, R, 0, W.mr.as<int>(), W.y.as<double2>(), gs, x, 1, s));
    else BEM_TRY(launch_combine(ecb, Vp, n, R, 0, W.mr.as<int>(), W.y.as<double2>(), gs, x, 1, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));  // pinned h_y / h_mr are reused by the next run
    for (int r = 0; r < R; ++r) iters_out[r] = it[r];
    return BEM_OK;
}

struct EventTimer {
    cudaEvent_t a = nullptr, b = nullptr;
    EventTimer() {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~EventTimer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
    float ms() {
        float t = 0.f;
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&t, a, b);
        return t;
    }
};

// Single-trace systems (Sec. 2.2): the Calderon operator of the unknowns' grid A,
// [[-K_A, V_A], [D_A, T_A]] times sA, on (v_A, w_A) ("own"), and the density-scaled
// Calderon operator of the other grid B, [[-K_B, cv V_B], [cd D_B, T_B]] times sB, on
// the two vectors mapped to B ("hat"); the unused block rows 2, 3 are empty (no rows,
// based at the end of the vector).  m1 = (K_e, D_e, K_i, D_i), m2 = (V_e, T_e, V_i, T_i);
// oA, oB = 0 for the exterior grid's operators, 2 for the interior grid's.
template <class BT, class MT>
void fill_blocks_single(BT& Bo, BT& Bh, MT* const m1[4], MT* const m2[4], int oA, int oB, int64_t NA, int64_t NB,
                        double sA, double sB, double cv, double cd) {
    for (int b = 0; b < 4; ++b) {
        const int u = b < 2 ? b : 1;
        Bo.A1[b] = m1[oA + u]; Bo.A2[b] = m2[oA + u];
        Bo.c1[b] = u == 0 ? -sA : sA; Bo.c2[b] = sA;
        Bo.rows[b] = b < 2 ? NA : 0;
        Bo.base[b] = b < 2 ? b * NA : 2 * NA;
        Bo.x1[b] = 0; Bo.x2[b] = b < 2 ? NA : 0;
        Bh.A1[b] = m1[oB + u]; Bh.A2[b] = m2[oB + u];
        Bh.c1[b] = u == 0 ? -sB : cd * sB;
        Bh.c2[b] = u == 0 ? cv * sB : sB;
        Bh.rows[b] = b < 2 ? NB : 0;
        Bh.base[b] = b < 2 ? b * NB : 2 * NB;
        Bh.x1[b] = 0; Bh.x2[b] = b < 2 ? NB : 0;
    }
}

template <class BT, class MT>
void fill_blocks(BT& B, MT* const m1[4], MT* const m2[4], int64_t Ne, int64_t Ni) {
    const double c1[4] = {-1.0, 1.0, -1.0, 1.0};
    const int64_t rows[4] = {Ne, Ne, Ni, Ni};
    const int64_t base[4] = {0, Ne, 2 * Ne, 2 * Ne + Ni};
    const int64_t x1[4] = {0, 0, 2 * Ne, 2 * Ne};
    const int64_t x2[4] = {Ne, Ne, 2 * Ne + Ni, 2 * Ne + Ni};
    for (int b = 0; b < 4; ++b) {
        B.A1[b] = m1[b]; B.A2[b] = m2[b]; B.c1[b] = c1[b]; B.c2[b] = 1.0;
        B.rows[b] = rows[b]; B.base[b] = base[b]; B.x1[b] = x1[b]; B.x2[b] = x2[b];
    }
}

// seeded uniform values in [lo, hi) (a 64-bit mixing hash of the index)
__global__ void k_fill_uniform(float* __restrict__ a, int64_t count, uint64_t seed, float lo, float hi) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    uint64_t h = (uint64_t)i * 0x9E3779B97F4A7C15ull + seed;
    h ^= h >> 30;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 27;
    h *= 0x94D049BB133111EBull;
    h ^= h >> 31;
    a[i] = lo + (hi - lo) * (float)((h >> 40) * (1.0 / 16777216.0));
}

__global__ void k_widen(const float2* __restrict__ x, int64_t count, double2* __restrict__ y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) y[i] = make_double2(x[i].x, x[i].y);
}

}  // namespace

// One grid's operators in the tiled storage (V, D upper tile triangles, K full; T = K^T
// is never stored), complex64 (mixed) or complex128.
struct GridOps {
    DevBuf V, K, D;
    int64_t N = 0;
    size_t esz = 16;
    // assemble the requested operators of grid g at wavenumber k
    bem_status assemble(const bem_grid* g, bem_c128 k, bool mixed, int n_singular, cudaStream_t s,
                        bool want_v = true, bool want_k = true, bool want_d = true) {
        N = g->nv;
        esz = mixed ? 8 : 16;
        const OpLayouts L = op_layouts_tiled();
        if (want_v) BEM_TRY(V.alloc(op_entries(OP_SYM, N) * esz, s));
        if (want_k) BEM_TRY(K.alloc(op_entries(OP_FULL, N) * esz, s));
        if (want_d) BEM_TRY(D.alloc(op_entries(OP_SYM, N) * esz, s));
        if (mixed) {
            for (DevBuf* b : {&V, &K, &D})
                if (b->p) BEM_CUDA_TRY(cudaMemsetAsync(b->p, 0, b->bytes, s));
            BEM_TRY(assemble_regular_fp32(g, k.re, k.im, V.as<float2>(), K.as<float2>(), nullptr, D.as<float2>(), L,
                                          s));
            BEM_TRY(assemble_singular_into_c64(g, k.re, k.im, n_singular, V.as<float2>(), K.as<float2>(), nullptr,
                                               D.as<float2>(), L, s));
        } else {
            BEM_TRY(assemble_operators_fp64(g, k.re, k.im, n_singular, V.as<double2>(), K.as<double2>(), nullptr,
                                            D.as<double2>(), L, s));
        }
        return BEM_OK;
    }
    // zeroed buffers for V, K, D of an N-vertex grid (assembled by the caller)
    bem_status alloc(int64_t n_vertices, size_t entry_bytes, cudaStream_t s) {
        N = n_vertices;
        esz = entry_bytes;
        BEM_TRY(V.alloc(op_entries(OP_SYM, N) * esz, s));
        BEM_TRY(K.alloc(op_entries(OP_FULL, N) * esz, s));
        BEM_TRY(D.alloc(op_entries(OP_SYM, N) * esz, s));
        for (DevBuf* b : {&V, &K, &D}) BEM_CUDA_TRY(cudaMemsetAsync(b->p, 0, b->bytes, s));
        return BEM_OK;
    }
    // a set y1 = cK K xa + cV V xb, y2 = cD D xc + cT K^T xd of product P
    void add(TileProd& P, double cK, double cV, double cD, double cT, int64_t xa, int64_t xb, int64_t xc, int64_t xd,
             int64_t y1, int64_t y2) const {
        tile_prod_add(P, K.p, V.p, D.p, N, cK, cV, cD, cT, xa, xb, xc, xd, y1, y2);
    }
    // dense row-major copies [V, K, T, D] (for the tensor-core products)
    bem_status dense_copies(DevBuf* out, cudaStream_t s) const {
        const int esz_i = (int)esz;
        for (int m = 0; m < 4; ++m) BEM_TRY(out[m].alloc((size_t)N * N * esz, s));
        BEM_TRY(tiles_to_dense(V.p, OP_SYM, false, N, esz_i, out[0].p, s));
        BEM_TRY(tiles_to_dense(K.p, OP_FULL, false, N, esz_i, out[1].p, s));
        BEM_TRY(tiles_to_dense(K.p, OP_FULL, true, N, esz_i, out[2].p, s));
        BEM_TRY(tiles_to_dense(D.p, OP_SYM, false, N, esz_i, out[3].p, s));
        return BEM_OK;
    }
};

// the tile products' error flag (an mbarrier wait that gave up)
bem_status check_tile_flag(const DevBuf& flag) {
    int h = 0;
    BEM_CUDA_TRY(cudaMemcpy(&h, flag.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        set_error("tile product: an mbarrier wait timed out");
        return BEM_E_INTERNAL;
    }
    return BEM_OK;
}


// The tensor-core product against the FP32 CUDA-core product on seeded random
// blocks whose entries have positive real parts (little cancellation, so the
// relative difference measures the products' rounding and not the data).
// The grid barrier's bounded wait: two cooperative blocks whose barrier count starts
// past the grid size, so that it never completes; both must give up and flag it.
// Returns the flag (1) times 1000 plus the elapsed seconds.
bem_status selftest_barrier(double* result, cudaStream_t s) {
    DevBuf b;
    BEM_TRY(b.alloc(64, s));
    BEM_CUDA_TRY(cudaMemsetAsync(b.p, 0, 64, s));
    const unsigned int start = 7;  // > gridDim.x: the last arrival is never seen
    BEM_CUDA_TRY(cudaMemcpyAsync(b.p, &start, sizeof(start), cudaMemcpyHostToDevice, s));
    GridBarrier* bar = b.as<GridBarrier>();
    int* err = reinterpret_cast<int*>(static_cast<char*>(b.p) + 32);
    int rounds = 3;
    void* args[] = {&bar, &err, &rounds};
    const double t0 = now_seconds();
    BEM_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_barrier_probe, dim3(2), dim3(64), args, 0, s));
    count_launch();
    int h = 0;
    BEM_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    *result = 1000.0 * h + (now_seconds() - t0);
    return BEM_OK;
}

bem_status selftest_tc(int R, double* rel_err, cudaStream_t s, int kind) {
    const bool fp16 = kind >= 2;
    const int64_t Ne = 300, Ni = 170, n = 2 * Ne + 2 * Ni;
    const int RW = R + 7;
    DevBuf tl[2][3], dn[2][4], xf, x, z1, z2, work, err, part, tperr;
    BEM_TRY(random_tiled_ops(Ne, 8, 1000, tl[0], dn[0], s));
    BEM_TRY(random_tiled_ops(Ni, 8, 2000, tl[1], dn[1], s));
    BEM_TRY(xf.alloc((size_t)RW * n * 8, s));
    BEM_LAUNCH(k_fill_uniform, blocks_for(2 * RW * n, 256), 256, 0, s, xf.as<float>(), 2 * RW * n, 3000ull, 0.5f, 1.0f);
    BEM_TRY(x.alloc((size_t)RW * n * 16, s));
    BEM_LAUNCH(k_widen, blocks_for(RW * n, 256), 256, 0, s, xf.as<float2>(), RW * n, x.as<double2>());
    BEM_TRY(z1.alloc((size_t)RW * n * 16, s));
    BEM_TRY(z2.alloc((size_t)RW * n * 16, s));
    // the tensor-core product on the dense copies
    Blocks<float2> B{};
    const float2* m1[4] = {dn[0][1].as<float2>(), dn[0][3].as<float2>(), dn[1][1].as<float2>(), dn[1][3].as<float2>()};
    const float2* m2[4] = {dn[0][0].as<float2>(), dn[0][2].as<float2>(), dn[1][0].as<float2>(), dn[1][2].as<float2>()};
    fill_blocks(B, m1, m2, Ne, Ni);
    BEM_TRY(err.alloc(sizeof(int), s));
    BEM_CUDA_TRY(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    Tc16Ops t16;
    if (fp16) {
        BEM_TRY(tc16_build(B.A1, B.A2, B.rows, t16, s, kind == 3));
        BEM_TRY(work.alloc(tc16_workspace_bytes(B.rows, tc_padded_columns(R)), s));
        BEM_TRY(mtf_product_tc16(t16, B.c1, B.c2, B.base, B.x1, B.x2, n, R, x.as<double2>(), z1.as<double2>(),
                                 work.p, work.bytes, err.as<int>(), s));
    } else {
        BEM_TRY(work.alloc(tc_workspace_bytes(B.rows, tc_padded_columns(R)), s));
        BEM_TRY(mtf_product_tc(B.A1, B.A2, B.c1, B.c2, B.rows, B.base, B.x1, B.x2, n, R, x.as<double2>(),
                               z1.as<double2>(), work.p, work.bytes, err.as<int>(), s));
    }
    // the FP32 tile product of the same operators
    TileProd P;
    tile_prod_add(P, tl[0][1].p, tl[0][0].p, tl[0][2].p, Ne, -1.0, 1.0, 1.0, 1.0, 0, Ne, 0, Ne, 0, Ne);
    tile_prod_add(P, tl[1][1].p, tl[1][0].p, tl[1][2].p, Ni, -1.0, 1.0, 1.0, 1.0, 2 * Ne, 2 * Ne + Ni, 2 * Ne,
                  2 * Ne + Ni, 2 * Ne, 2 * Ne + Ni);
    BEM_TRY(tile_prod_finish(P, n, 8, s));
    BEM_TRY(part.alloc(tile_part_bytes(P, TP_F32, 8), s));
    BEM_TRY(tperr.alloc(sizeof(int), s));
    BEM_CUDA_TRY(cudaMemsetAsync(tperr.p, 0, sizeof(int), s));
    for (int c0 = 0; c0 < R; c0 += 8)
        BEM_TRY(tile_product(P, TP_F32, std::min(8, R - c0), xf.as<float2>() + c0 * n, z2.as<double2>() + c0 * n,
                             part.p, tperr.as<int>(), s));
    std::vector<double2> h1((size_t)R * n), h2((size_t)R * n);
    int h_err = 0;
    BEM_CUDA_TRY(cudaMemcpyAsync(h1.data(), z1.p, h1.size() * 16, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(h2.data(), z2.p, h2.size() * 16, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_err) {
        set_error("tensor-core product: an mbarrier wait timed out");
        return BEM_E_INTERNAL;
    }
    BEM_TRY(check_tile_flag(tperr));
    double num = 0.0, den = 0.0;
    for (size_t i = 0; i < h1.size(); ++i) {
        const double dx = h1[i].x - h2[i].x, dy = h1[i].y - h2[i].y;
        num += dx * dx + dy * dy;
        den += h2[i].x * h2[i].x + h2[i].y * h2[i].y;
    }
    *rel_err = den > 0.0 ? std::sqrt(num / den) : 0.0;
    return BEM_OK;
}

// Autotuner: times the candidate launch shapes of the iteration's kernels for the given
// grids' sizes (the grids' own mass matrices; seeded random operators for the
// tensor-core product, whose timing does not depend on the values) and records the
// fastest per (kernel, width, size class):
//   Chebyshev mass steps for 1 and 8 columns: 64, 128 or 256 threads;
//   tensor-core product of n_rhs > 8 columns (batches of up to 64): 1 or 2 K splits.
// (The dense single- and few-column products are persistent tile-product launches, one
// CTA per SM, with nothing to tune.)  The GPU is first kept busy for a while (clocks
// up), each candidate runs once untimed, then the candidates are timed round-robin
// `reps` times, four launches back to back between CUDA events (so that a drift of the
// clocks affects all alike), and the median counts; the kernel's built-in shape is kept
// unless another is faster by more than 2 %.
bem_status autotune_impl(bem_context* ctx, const bem_grid* ge, const bem_grid* gi, int n_rhs, int reps) {
    cudaStream_t s = ctx->stream;
    const int64_t Ne = ge->nv, Ni = gi->nv, n = 2 * Ne + 2 * Ni;
    const int RT = 64 + 7;
    DevBuf tl[2][3], dn[2][4], xf, x, z, part, tperr;
    const bool tc = n_rhs > 8;
    BEM_TRY(random_tiled_ops(Ne, 8, 5000, tl[0], tc ? dn[0] : nullptr, s));
    BEM_TRY(random_tiled_ops(Ni, 8, 6000, tl[1], tc ? dn[1] : nullptr, s));
    BEM_TRY(xf.alloc((size_t)RT * n * 8, s));
    BEM_LAUNCH(k_fill_uniform, blocks_for(2 * RT * n, 256), 256, 0, s, xf.as<float>(), 2 * RT * n, 6000ull, -1.0f, 1.0f);
    BEM_TRY(x.alloc((size_t)RT * n * 16, s));
    BEM_LAUNCH(k_widen, blocks_for(RT * n, 256), 256, 0, s, xf.as<float2>(), RT * n, x.as<double2>());
    BEM_TRY(z.alloc((size_t)RT * n * 16, s));
    TileProd P;  // the multiple-traces product of the random operators (warm-up)
    tile_prod_add(P, tl[0][1].p, tl[0][0].p, tl[0][2].p, Ne, -1.0, 1.0, 1.0, 1.0, 0, Ne, 0, Ne, 0, Ne);
    tile_prod_add(P, tl[1][1].p, tl[1][0].p, tl[1][2].p, Ni, -1.0, 1.0, 1.0, 1.0, 2 * Ne, 2 * Ne + Ni, 2 * Ne,
                  2 * Ne + Ni, 2 * Ne, 2 * Ne + Ni);
    BEM_TRY(tile_prod_finish(P, n, 8, s));
    BEM_TRY(part.alloc(tile_part_bytes(P, TP_F32, 1), s));
    BEM_TRY(tperr.alloc(sizeof(int), s));
    BEM_CUDA_TRY(cudaMemsetAsync(tperr.p, 0, sizeof(int), s));
    Blocks<float2> B{};
    if (tc) {
        const float2* m1[4] = {dn[0][1].as<float2>(), dn[0][3].as<float2>(), dn[1][1].as<float2>(),
                               dn[1][3].as<float2>()};
        const float2* m2[4] = {dn[0][0].as<float2>(), dn[0][2].as<float2>(), dn[1][0].as<float2>(),
                               dn[1][2].as<float2>()};
        fill_blocks(B, m1, m2, Ne, Ni);
    }
    EventTimer ev;
    // times of the candidates (index 0: the built-in shape), round-robin; returns the
    // index chosen and its median time
    auto pick = [&](int count, const std::function<bem_status(int)>& run, double* best_ms) -> int {
        std::vector<std::vector<float>> t(count);
        for (int c = 0; c < count; ++c)
            if (run(c) != BEM_OK) return -1;
        // each sample: 4 launches back to back (the steady state of an iteration, not a
        // launch after an idle GPU), per launch
        for (int r = 0; r < reps; ++r)
            for (int c = 0; c < count; ++c) {
                if (cudaEventRecord(ev.a, s) != cudaSuccess) return -1;
                for (int k = 0; k < 4; ++k)
                    if (run(c) != BEM_OK) return -1;
                if (cudaEventRecord(ev.b, s) != cudaSuccess) return -1;
                t[c].push_back(ev.ms() / 4.0f);
            }
        std::vector<double> med(count);
        for (int c = 0; c < count; ++c) {
            std::sort(t[c].begin(), t[c].end());
            med[c] = t[c][reps / 2];
        }
        int best = 0;
        for (int c = 1; c < count; ++c)
            if (med[c] < med[best]) best = c;
        if (med[best] > 0.98 * med[0]) best = 0;
        *best_ms = med[best];
        return best;
    };
    auto tune_failed = []() {
        set_error("autotune: a candidate launch failed");
        return BEM_E_CUDA;
    };
    // keep the GPU busy for ~0.3 s before measuring
    {
        const auto t0 = now_seconds();
        while (now_seconds() - t0 < 0.3) {
            for (int k = 0; k < 8; ++k)
                BEM_TRY(tile_product(P, TP_F32, 1, xf.p, z.as<double2>(), part.p, tperr.as<int>(), s));
            BEM_CUDA_TRY(cudaStreamSynchronize(s));
        }
        BEM_TRY(check_tile_flag(tperr));
    }
    // Chebyshev mass steps on the grids' own mass matrices (MTF layout: both grids)
    {
        DevBuf mve, mvi, dve, dvi, wr, wa, wb, y;
        BEM_TRY(mve.alloc(ge->m_nnz * 8, s));
        BEM_TRY(mvi.alloc(gi->m_nnz * 8, s));
        BEM_TRY(dve.alloc(Ne * 8, s));
        BEM_TRY(dvi.alloc(Ni * 8, s));
        BEM_TRY(mass_values(ge, mve.as<double>(), s));
        BEM_TRY(mass_values(gi, mvi.as<double>(), s));
        BEM_TRY(mass_inverse_diag(ge, mve.as<double>(), dve.as<double>(), s));
        BEM_TRY(mass_inverse_diag(gi, mvi.as<double>(), dvi.as<double>(), s));
        MassEll ell_e, ell_i;
        BEM_TRY(ell_e.build(ge, mve.as<double>(), s));
        BEM_TRY(ell_i.build(gi, mvi.as<double>(), s));
        for (DevBuf* b : {&wr, &wa, &wb, &y}) BEM_TRY(b->alloc((size_t)8 * n * 16, s));
        MassOp op;
        op.M.ci[0] = ell_e.ci.as<int32_t>(); op.M.v[0] = ell_e.v.as<double>(); op.M.W[0] = ell_e.W;
        op.M.dinv[0] = dve.as<double>();
        op.M.ci[1] = ell_i.ci.as<int32_t>(); op.M.v[1] = ell_i.v.as<double>(); op.M.W[1] = ell_i.W;
        op.M.dinv[1] = dvi.as<double>();
        op.M.Ne = Ne; op.M.Ni = Ni; op.M.n = n;
        op.r = wr.as<double2>(); op.dA = wa.as<double2>(); op.dB = wb.as<double2>();
        for (int R : {1, 8}) {
            const int blocks[3] = {64, 128, 256};
            double ms = 0.0;
            const int b = pick(3, [&](int c) {
                tune_put(TUNE_CHEB, R, n, TuneChoice{blocks[c], 0, 0.0});
                return mass_solve(op, x.as<double2>(), y.as<double2>(), R, s, CHEB_STEPS);
            }, &ms);
            if (b < 0) return tune_failed();
            tune_put(TUNE_CHEB, R, n, TuneChoice{blocks[b], 0, ms});
        }
    }
    // tensor-core product
    if (tc) {
        const int R = std::min(n_rhs, 64);
        const int RP = tc_padded_columns(R);
        DevBuf work, err;
        BEM_TRY(work.alloc(tc_workspace_bytes(B.rows, RP), s));
        BEM_TRY(err.alloc(sizeof(int), s));
        BEM_CUDA_TRY(cudaMemsetAsync(err.p, 0, sizeof(int), s));
        int sms = 0, dev = 0;
        BEM_CUDA_TRY(cudaGetDevice(&dev));
        BEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        int64_t tiles = 0;
        for (int b = 0; b < 4; ++b) tiles += (B.rows[b] + 127) / 128;
        const int dflt = tiles < sms ? 2 : 1;
        const int ks[2] = {dflt, 3 - dflt};
        double ms = 0.0;
        const int b = pick(2, [&](int c) {
            tune_put(TUNE_GEMM_TC, RP, n, TuneChoice{0, ks[c], 0.0});
            return mtf_product_tc(B.A1, B.A2, B.c1, B.c2, B.rows, B.base, B.x1, B.x2, n, R, x.as<double2>(),
                                  z.as<double2>(), work.p, work.bytes, err.as<int>(), s);
        }, &ms);
        if (b < 0) return tune_failed();
        tune_put(TUNE_GEMM_TC, RP, n, TuneChoice{0, ks[b], ms});
        int h_err = 0;
        BEM_CUDA_TRY(cudaMemcpy(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost));
        if (h_err) {
            set_error("tensor-core product: an mbarrier wait timed out");
            return BEM_E_INTERNAL;
        }
    }
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    return BEM_OK;
}

// f, g [R][N] of right-hand sides r0 .. r0 + R - 1 of an incident field on grid g (plane
// waves, point sources, or the caller's data copied in); wave is a device buffer of at
// least 5 RB doubles, h_wave its pinned host staging (amplitudes, then directions or
// source positions); inputs_on_device tells where the caller's f, g live.
bem_status incident_data(const bem_incident* inc, int r0, int R, int RB, const bem_grid* g, bem_c128 k,
                         double* h_wave, DevBuf& wave, double2* f, double2* gv, bool inputs_on_device,
                         cudaStream_t s) {
    const int64_t N = g->nv;
    if (inc->kind == BEM_INC_USER_TRACES) {
        const cudaMemcpyKind kind = inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if (inc->f) BEM_CUDA_TRY(cudaMemcpyAsync(f, inc->f + (int64_t)r0 * N, (size_t)R * N * 16, kind, s));
        else BEM_CUDA_TRY(cudaMemsetAsync(f, 0, (size_t)R * N * 16, s));
        BEM_CUDA_TRY(cudaMemcpyAsync(gv, inc->g + (int64_t)r0 * N, (size_t)R * N * 16, kind, s));
        return BEM_OK;
    }
    const double* pos = inc->kind == BEM_INC_POINT_SOURCE ? inc->sources : inc->dirs;
    // amplitudes first (2 R doubles: 16-byte aligned complex values), then 3 R coordinates
    for (int r = 0; r < R; ++r) {
        h_wave[2 * r] = inc->amps ? inc->amps[r0 + r].re : 1.0;
        h_wave[2 * r + 1] = inc->amps ? inc->amps[r0 + r].im : 0.0;
        for (int d = 0; d < 3; ++d) h_wave[2 * RB + 3 * r + d] = pos[3 * (r0 + r) + d];
    }
    BEM_CUDA_TRY(cudaMemcpyAsync(wave.p, h_wave, (size_t)5 * RB * 8, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(cudaMemsetAsync(f, 0, (size_t)R * N * 16, s));
    BEM_CUDA_TRY(cudaMemsetAsync(gv, 0, (size_t)R * N * 16, s));
    if (inc->kind == BEM_INC_POINT_SOURCE)
        BEM_LAUNCH(k_point_source, dim3(blocks_for(g->nt, 128), R), 128, 0, s, g->rec.as<TriRec>(),
                   g->tri.as<int32_t>(), g->nt, k.re, k.im, wave.as<double>() + 2 * RB, wave.as<double2>(), N, f, gv);
    else
        BEM_LAUNCH(k_plane_wave, dim3(blocks_for(g->nt, 128), R), 128, 0, s, g->rec.as<TriRec>(),
                   g->tri.as<int32_t>(), g->nt, k.re, k.im, wave.as<double>() + 2 * RB, wave.as<double2>(), N, f, gv);
    return BEM_OK;
}

bem_status solve_transmission_impl(bem_context* ctx, const bem_grid* ge, const bem_grid* gi, bem_c128 k_int,
                                   bem_c128 k_ext, double rho_ratio, const bem_incident* inc,
                                   const bem_solve_opts* o, bem_c128* v_ext, bem_c128* w_ext, bem_c128* v_int,
                                   bem_c128* w_int, int on_device, bem_solve_report* rep) {
    cudaStream_t s = ctx->stream;
    // unknowns per right-hand side: (v_e, w_e, v_i, w_i) for the multiple-traces system;
    // for a single-trace system the two potentials of one grid A (the exterior grid for
    // the exterior variants, the interior grid for the interior ones), whose products
    // also apply the other grid B's operators to vectors of nB = 2 N_B entries (the two
    // potentials mapped by M_B^-1 P_BA)
    const int form = o->formulation;
    const bool st = form != BEM_FORM_MTF;
    const bool hc = form >= BEM_FORM_HC_EXT_NEU;  // high-contrast systems (Sec. 2.3)
    const bool hc_neu = form == BEM_FORM_HC_EXT_NEU || form == BEM_FORM_HC_INT_NEU;
    const bool st_int = form == BEM_FORM_PMCHWT_INT || form == BEM_FORM_MULLER_INT || form == BEM_FORM_HC_INT_NEU ||
                        form == BEM_FORM_HC_INT_DIR;
    const bool muller = form == BEM_FORM_MULLER || form == BEM_FORM_MULLER_INT;
    const int64_t Ne = ge->nv, Ni = gi->nv;
    const int64_t NA = st_int ? Ni : Ne, NB = st_int ? Ne : Ni, nB = 2 * NB;
    const int64_t n = st ? 2 * NA : 2 * Ne + 2 * Ni;
    const bool mixed = o->precision == BEM_PREC_MIXED;
    const StopCheck stop = [ctx]() -> bem_status {
        if (ctx->cancel && ctx->cancel->load(std::memory_order_relaxed)) {
            set_error("request cancelled");
            return BEM_E_CANCELLED;
        }
        if (ctx->deadline > 0.0 && now_seconds() > ctx->deadline) {
            set_error("request exceeded its time limit");
            return BEM_E_TIMEOUT;
        }
        return BEM_OK;
    };
    BEM_TRY(stop());
    EventTimer t_asm, t_mor, t_sol;
    GraphCache graphs(o->cuda_graphs != 0);
    // ---- operators on both grids --------------------------------------------------
    // tiled storage: V and D as their upper tile triangles, K in full, no T (= K^T)
    const size_t esz = mixed ? 8 : 16;
    const OpLayouts TL = op_layouts_tiled();
    GridOps ops[2];  // exterior, interior
    cudaEventRecord(t_asm.a, s);
    BEM_TRY(ops[0].assemble(ge, k_ext, mixed, o->n_singular, s));
    BEM_TRY(ops[1].assemble(gi, k_int, mixed, o->n_singular, s));
    cudaEventRecord(t_asm.b, s);
    // ---- mass and mortar (FP64) ----------------------------------------------------
    cudaEventRecord(t_mor.a, s);
    DevBuf mve, mvi, dve, dvi, prow, pcol, pval;
    BEM_TRY(mve.alloc(ge->m_nnz * 8, s));
    BEM_TRY(mvi.alloc(gi->m_nnz * 8, s));
    BEM_TRY(dve.alloc(Ne * 8, s));
    BEM_TRY(dvi.alloc(Ni * 8, s));
    BEM_TRY(mass_values(ge, mve.as<double>(), s));
    BEM_TRY(mass_values(gi, mvi.as<double>(), s));
    BEM_TRY(mass_inverse_diag(ge, mve.as<double>(), dve.as<double>(), s));
    BEM_TRY(mass_inverse_diag(gi, mvi.as<double>(), dvi.as<double>(), s));
    int64_t pnnz = 0;
    BEM_TRY(mortar_coo(gi, ge, o->center, prow, pcol, pval, &pnnz, s));
    CsrBuf csr_p, csr_t;  // P_ie and P_ei
    BEM_TRY(build_csr(prow.as<int32_t>(), pcol.as<int32_t>(), pval.as<double>(), pnnz, Ni, csr_p, s));
    BEM_TRY(build_csr(pcol.as<int32_t>(), prow.as<int32_t>(), pval.as<double>(), pnnz, Ne, csr_t, s));
    cudaEventRecord(t_mor.b, s);
    // ---- workspaces for batches of RB right-hand sides ---------------------------------
    const bool use_tc = mixed && o->tensor_cores != 0;
    const int rmax = o->batch_columns > 0 ? o->batch_columns : (use_tc ? 64 : 8);
    const int RB = std::min<int>(rmax, inc->n_rhs);
    // CUDA-core products take the columns in groups of w <= 8 at width gemm_width(w),
    // reading and writing up to 7 spare (in-bounds) columns past the batch
    const int RW = RB + 7;
    const bool tc_batches = use_tc && RB > 8 && !hc;  // high-contrast products: CUDA cores
    // Single-column inner solves of the refinement with dd_switch < 1: the products run
    // in double-float arithmetic while the inner residual is above dd_switch of its
    // right-hand side and in FP32 after it.  GMRES tolerates product errors that grow as
    // the residual falls (the residual gap is a sum of each product's error times its
    // coefficient in the solution, and those coefficients shrink with the residual), so
    // a 1e-7 FP32 product after the switch leaves the inner solve accurate to ~1e-9 and
    // the refinement converges in one pass.  The default (dd_switch = 1) runs FP32
    // products throughout and refines in two passes instead, which costs fewer
    // double-float products than the one pass saves.
    const bool dd_single = mixed && RB == 1;
    double inner_progress = 1.0;
    auto dd_now = [&]() { return dd_single && inner_progress > o->dd_switch; };
    // inner solves on FP32 (or tensor-core) products throughout: batches, and single
    // columns with dd_switch >= 1.  They keep a complex64 basis and stop the first inner
    // solve early (IR_INNER_TOL_BATCH) unless ir_inner_tol is given.
    const bool fp32_inner = mixed && (!dd_single || o->dd_switch >= 1.0);
    const size_t colb = (size_t)n * 16;
    DevBuf wz, wr, wa, wb, x32, tcw, tcerr, xsplit;
    BEM_TRY(wz.alloc(RW * colb, s));
    BEM_TRY(wr.alloc(RB * colb, s));
    BEM_TRY(wa.alloc(RB * colb, s));
    BEM_TRY(wb.alloc(RB * colb, s));
    MassOp mop;
    MassEll ell_e, ell_i;
    BEM_TRY(ell_e.build(ge, mve.as<double>(), s));
    BEM_TRY(ell_i.build(gi, mvi.as<double>(), s));
    mop.M.ci[0] = ell_e.ci.as<int32_t>(); mop.M.v[0] = ell_e.v.as<double>(); mop.M.W[0] = ell_e.W;
    mop.M.dinv[0] = dve.as<double>();
    mop.M.ci[1] = ell_i.ci.as<int32_t>(); mop.M.v[1] = ell_i.v.as<double>(); mop.M.W[1] = ell_i.W;
    mop.M.dinv[1] = dvi.as<double>();
    DevBuf dvef, dvif;  // FP32 copies for the FP32 inner mass inverses
    if (mixed) {
        BEM_TRY(dvef.alloc((size_t)Ne * 4, s));
        BEM_TRY(dvif.alloc((size_t)Ni * 4, s));
        BEM_LAUNCH(k_narrow, blocks_for(Ne, 256), 256, 0, s, dve.as<double>(), Ne, dvef.as<float>());
        BEM_LAUNCH(k_narrow, blocks_for(Ni, 256), 256, 0, s, dvi.as<double>(), Ni, dvif.as<float>());
        mop.M.vf[0] = ell_e.vf.as<float>(); mop.M.vf[1] = ell_i.vf.as<float>();
        mop.M.dinvf[0] = dvef.as<float>(); mop.M.dinvf[1] = dvif.as<float>();
    }
    // a MassPair with no rows on one grid is the mass inverse of the other grid alone
    // (vectors of its two potentials): single-trace systems use M_A^-1 (mop) and M_B^-1 (mopB)
    mop.M.Ne = st_int ? 0 : Ne; mop.M.Ni = st && !st_int ? 0 : Ni; mop.M.n = n;
    mop.r = wr.as<double2>(); mop.dA = wa.as<double2>(); mop.dB = wb.as<double2>();
    mop.graphs = &graphs;
    ChebSync csync;
    BEM_TRY(csync.init(s));
    if (ctx->exclusive) csync.attach(mop);
    // single-trace: the grid-B vectors of a product (tb1: M_B^-1 P_BA x, then M_B^-1 of the
    // grid-B product; tb2, tb3: input and output of the grid-B product, which reads and
    // writes up to 7 spare columns)
    MassOp mopB;
    DevBuf wrb, wab, wbb, tb1, tb2, tb3, x32b;
    if (st) {
        const size_t colB = (size_t)nB * 16;
        BEM_TRY(wrb.alloc(RB * colB, s));
        BEM_TRY(wab.alloc(RB * colB, s));
        BEM_TRY(wbb.alloc(RB * colB, s));
        BEM_TRY(tb1.alloc(RB * colB, s));
        BEM_TRY(tb2.alloc(RW * colB, s));
        BEM_TRY(tb3.alloc(RW * colB, s));
        BEM_CUDA_TRY(cudaMemsetAsync(tb2.p, 0, tb2.bytes, s));
        mopB.M = mop.M;
        mopB.M.Ne = st_int ? Ne : 0; mopB.M.Ni = st_int ? 0 : Ni; mopB.M.n = nB;
        mopB.r = wrb.as<double2>(); mopB.dA = wab.as<double2>(); mopB.dB = wbb.as<double2>();
        mopB.graphs = &graphs;
        if (ctx->exclusive) csync.attach(mopB);
    }
    // P_BA (rows on grid B) and P_AB = P_BA^T: P_ie and P_ei for the exterior variants
    const CsrBuf& csr_ba = st_int ? csr_t : csr_p;
    const CsrBuf& csr_ab = st_int ? csr_p : csr_t;
    // density scaling of grid B's Calderon operator, r = rho_i / rho_e: (cv V, cd D) =
    // (r V_i, D_i / r) mapped to the exterior grid, (V_e / r, r D_e) to the interior grid;
    // Mueller: exterior A_e - hat, interior hat - A_i (identity added after M_A^-1)
    const double cv = st_int ? 1.0 / rho_ratio : rho_ratio, cd = st_int ? rho_ratio : 1.0 / rho_ratio;
    const double sA = form == BEM_FORM_MULLER_INT ? -1.0 : 1.0, sB = form == BEM_FORM_MULLER ? -1.0 : 1.0;
    const int oA = st_int ? 2 : 0, oB = st_int ? 0 : 2;
    // high-contrast: coefficients of the grid-B row (X1 t_0, X2 t_1), r = rho_i / rho_e:
    // exterior Neumann -T_i, -D_i / r; interior Neumann T_e, r D_e; exterior Dirichlet
    // -r V_i, K_i; interior Dirichlet V_e / r, -K_e
    const double hc_c1 = form == BEM_FORM_HC_EXT_NEU ? -1.0 : form == BEM_FORM_HC_INT_NEU ? 1.0
                       : form == BEM_FORM_HC_EXT_DIR ? -rho_ratio : 1.0 / rho_ratio;
    const double hc_c2 = form == BEM_FORM_HC_EXT_NEU ? -1.0 / rho_ratio : form == BEM_FORM_HC_INT_NEU ? rho_ratio
                       : form == BEM_FORM_HC_EXT_DIR ? 1.0 : -1.0;
    TransferCsr top;
    const double sgn = o->mtf_variant == BEM_MTF_PRINTED ? -1.0 : 1.0;
    top.prp = csr_p.rp.as<int32_t>(); top.pci = csr_p.ci.as<int32_t>(); top.pv = csr_p.v.as<double>();
    top.trp = csr_t.rp.as<int32_t>(); top.tci = csr_t.ci.as<int32_t>(); top.tv = csr_t.v.as<double>();
    top.Ne = Ne; top.Ni = Ni; top.n = n;
    top.ca = -0.5 * sgn;
    top.cb = -0.5 * sgn / rho_ratio;
    top.cc = 0.5 * sgn;
    top.cd = 0.5 * sgn * rho_ratio;
    double2* z = wz.as<double2>();
    // ---- the dense products as tile products (tile_product.cu) ------------------------
    //   P0: the multiple-traces blocks of both grids, or the own-grid rows of a
    //       single-trace / high-contrast system (vectors of n);
    //   Ph: the other grid's rows (vectors of nB); Pr, Pq: the high-contrast data and
    //       output rows (vectors of nB and n).
    TileProd P0, Ph, Pr, Pq;
    const GridOps& gA = ops[st_int ? 1 : 0];
    const GridOps& gB = ops[st_int ? 0 : 1];
    if (hc) {
        if (hc_neu) {  // own rows (T_A mu; V_A mu), mu = x_1; hat row c1 T_B t_0 + c2 D_B t_1
            gA.add(P0, 0.0, 1.0, 0.0, 1.0, 0, NA, 0, NA, NA, 0);
            gB.add(Ph, 0.0, 0.0, hc_c2, hc_c1, 0, 0, NB, 0, -1, 0);
        } else {       // own rows (K_A nu; D_A nu), nu = x_0; hat row c1 V_B t_0 + c2 K_B t_1
            gA.add(P0, 1.0, 0.0, 1.0, 0.0, 0, 0, 0, 0, 0, NA);
            gB.add(Ph, hc_c2, hc_c1, 0.0, 0.0, NB, 0, 0, 0, 0, -1);
        }
        const double r = rho_ratio;
        switch (form) {
            case BEM_FORM_HC_EXT_NEU:  // (1/r) D_i t_0;  -V_e x_1
                gB.add(Pr, 0.0, 0.0, 1.0 / r, 0.0, 0, 0, 0, 0, -1, 0);
                gA.add(Pq, 0.0, -1.0, 0.0, 0.0, 0, NA, 0, 0, 0, -1);
                break;
            case BEM_FORM_HC_EXT_DIR:  // r V_i t_0;  -D_e x_0
                gB.add(Pr, 0.0, r, 0.0, 0.0, 0, 0, 0, 0, 0, -1);
                gA.add(Pq, 0.0, 0.0, -1.0, 0.0, 0, 0, 0, 0, -1, 0);
                break;
            case BEM_FORM_HC_INT_NEU:  // D_e t_0 + T_e t_1;  V_i x_1
                gB.add(Pr, 0.0, 0.0, 1.0, 1.0, 0, 0, 0, NB, -1, 0);
                gA.add(Pq, 0.0, 1.0, 0.0, 0.0, 0, NA, 0, 0, 0, -1);
                break;
            default:  // interior Dirichlet: V_e t_1 - K_e t_0;  D_i x_0
                gB.add(Pr, -1.0, 1.0, 0.0, 0.0, 0, NB, 0, 0, 0, -1);
                gA.add(Pq, 0.0, 0.0, 1.0, 0.0, 0, 0, 0, 0, -1, 0);
                break;
        }
        BEM_TRY(tile_prod_finish(Pr, nB, (int)esz, s));
        BEM_TRY(tile_prod_finish(Pq, n, (int)esz, s));
    } else if (st) {  // own: sA [[-K_A, V_A], [D_A, T_A]]; hat: sB [[-K_B, cv V_B], [cd D_B, T_B]]
        gA.add(P0, -sA, sA, sA, sA, 0, NA, 0, NA, 0, NA);
        gB.add(Ph, -sB, cv * sB, cd * sB, sB, 0, NB, 0, NB, 0, NB);
    } else {  // [[-K_e, V_e], [D_e, T_e]] on (v_e, w_e) and the same on the interior grid
        ops[0].add(P0, -1.0, 1.0, 1.0, 1.0, 0, Ne, 0, Ne, 0, Ne);
        ops[1].add(P0, -1.0, 1.0, 1.0, 1.0, 2 * Ne, 2 * Ne + Ni, 2 * Ne, 2 * Ne + Ni, 2 * Ne, 2 * Ne + Ni);
    }
    BEM_TRY(tile_prod_finish(P0, n, (int)esz, s));
    if (st) BEM_TRY(tile_prod_finish(Ph, nB, (int)esz, s));
    // workspaces: complex64 copies of the inputs (FP32 products), double-float splits of
    // 8 columns (FP64-accurate products), partial sums of 8 columns, error flag
    const int64_t nmax = st ? std::max(n, nB) : n;
    DevBuf part, tperr;
    BEM_TRY(xsplit.alloc((size_t)8 * nmax * 16, s));
    {
        size_t pb = 0;
        for (const TileProd* q : {&P0, &Ph, &Pr, &Pq})
            if (!q->sets.empty()) pb = std::max(pb, tile_part_bytes(*q, TP_DD, std::min(RB, 8)));
        BEM_TRY(part.alloc(pb, s));
    }
    BEM_TRY(tperr.alloc(sizeof(int), s));
    BEM_CUDA_TRY(cudaMemsetAsync(tperr.p, 0, sizeof(int), s));
    // tensor-core batches read dense row-major blocks: dense copies of the operators
    DevBuf dense[8];  // Ve, Ke, Te, De, Vi, Ki, Ti, Di
    Blocks<float2> B32{}, Bh32{};
    const bool tc16 = o->tensor_cores >= 2;  // FP16 (2) or BF16 (3) two-term split, TMA-fed
    Tc16Ops t16, t16h;                       // its operator copies of B32 and Bh32
    if (mixed) {
        BEM_TRY(x32.alloc((size_t)RW * n * 8, s));
        BEM_CUDA_TRY(cudaMemsetAsync(x32.p, 0, x32.bytes, s));
        if (st) {
            BEM_TRY(x32b.alloc((size_t)RW * nB * 8, s));
            BEM_CUDA_TRY(cudaMemsetAsync(x32b.p, 0, x32b.bytes, s));
        }
        if (tc_batches) {
            for (int g = 0; g < 2; ++g) BEM_TRY(ops[g].dense_copies(&dense[4 * g], s));
            const float2* m1[4] = {dense[1].as<float2>(), dense[3].as<float2>(), dense[5].as<float2>(),
                                   dense[7].as<float2>()};
            const float2* m2[4] = {dense[0].as<float2>(), dense[2].as<float2>(), dense[4].as<float2>(),
                                   dense[6].as<float2>()};
            if (st) fill_blocks_single(B32, Bh32, m1, m2, oA, oB, NA, NB, sA, sB, cv, cd);
            else fill_blocks(B32, m1, m2, Ne, Ni);
            const int RP = tc_padded_columns(RB);
            if (tc16) {
                // the split copies replace the dense complex64 copies
                BEM_TRY(tc16_build(B32.A1, B32.A2, B32.rows, t16, s, o->tensor_cores == 3));
                if (st) BEM_TRY(tc16_build(Bh32.A1, Bh32.A2, Bh32.rows, t16h, s, o->tensor_cores == 3));
                for (DevBuf& d : dense) d.release();  // stream-ordered: after the split kernels
                BEM_TRY(tcw.alloc(std::max(tc16_workspace_bytes(B32.rows, RP),
                                           st ? tc16_workspace_bytes(Bh32.rows, RP) : 0),
                                  s));
            } else {
                BEM_TRY(tcw.alloc(
                    std::max(tc_workspace_bytes(B32.rows, RP), st ? tc_workspace_bytes(Bh32.rows, RP) : 0), s));
            }
            BEM_TRY(tcerr.alloc(sizeof(int), s));
            BEM_CUDA_TRY(cudaMemsetAsync(tcerr.p, 0, sizeof(int), s));
        }
    }
    // zo = product P of nn rows applied to R columns xin in the working arithmetic: FP32
    // on complex64 (mixed; xw receives the complex64 copy of xin), double-float for the
    // single-column products of the mixed mode above the dd_switch, double-float on
    // complex128 (FP64 mode), tensor cores for mixed batches of more than 8 columns (tcb:
    // the dense view of the same blocks)
    auto gemm_work_on = [&](const TileProd& P, const Blocks<float2>* tcb, int64_t nn, float2* xw, const double2* xin,
                            double2* zo, int R) -> bem_status {
        if (mixed && tc_batches && R > 8) {
            if (tc16)
                return mtf_product_tc16(tcb == &Bh32 ? t16h : t16, tcb->c1, tcb->c2, tcb->base, tcb->x1, tcb->x2, nn,
                                        R, xin, zo, tcw.p, tcw.bytes, tcerr.as<int>(), s);
            return mtf_product_tc(tcb->A1, tcb->A2, tcb->c1, tcb->c2, tcb->rows, tcb->base, tcb->x1, tcb->x2, nn, R,
                                  xin, zo, tcw.p, tcw.bytes, tcerr.as<int>(), s);
        }
        const bool dd = !mixed || (R == 1 && dd_now());
        if (mixed && !dd)
            BEM_LAUNCH(k_to_c64, blocks_for((int64_t)R * nn, 256), 256, 0, s, xin, (int64_t)R * nn, xw);
        for (int c0 = 0; c0 < R; c0 += 8) {
            const int w = std::min(8, R - c0);
            double2* zc = zo + (int64_t)c0 * nn;
            if (dd) {
                BEM_LAUNCH(k_split_x, blocks_for((int64_t)w * nn, 256), 256, 0, s, xin + (int64_t)c0 * nn,
                           (int64_t)w * nn, xsplit.as<float4>());
                BEM_TRY(tile_product(P, TP_DD, w, xsplit.p, zc, part.p, tperr.as<int>(), s));
            } else {
                BEM_TRY(tile_product(P, TP_F32, w, xw + (int64_t)c0 * nn, zc, part.p, tperr.as<int>(), s));
            }
        }
        return BEM_OK;
    };
    // the same with FP64-accurate arithmetic on the stored matrices (double-float)
    auto gemm_fp64_on = [&](const TileProd& P, int64_t nn, const double2* xin, double2* zo, int R) -> bem_status {
        for (int c0 = 0; c0 < R; c0 += 8) {
            const int w = std::min(8, R - c0);
            BEM_LAUNCH(k_split_x, blocks_for((int64_t)w * nn, 256), 256, 0, s, xin + (int64_t)c0 * nn, (int64_t)w * nn,
                       xsplit.as<float4>());
            BEM_TRY(tile_product(P, TP_DD, w, xsplit.p, zo + (int64_t)c0 * nn, part.p, tperr.as<int>(), s));
        }
        return BEM_OK;
    };
    // single-trace product z = sA A_A x + sB P_AB M_B^-1 A_B^rho M_B^-1 P_BA x (the hat
    // transformation applied factor by factor), then y = M_A^-1 z, plus x for Mueller
    auto apply_single = [&](bool fp64, const double2* xin, double2* yout, int R, int steps) -> bem_status {
        auto prod = [&](const TileProd& P, const Blocks<float2>* tcb, int64_t nn, float2* xw, const double2* xi,
                        double2* zo) -> bem_status {
            return fp64 ? gemm_fp64_on(P, nn, xi, zo, R) : gemm_work_on(P, tcb, nn, xw, xi, zo, R);
        };
        BEM_TRY(prod(P0, &B32, n, x32.as<float2>(), xin, z));
        BEM_LAUNCH(k_csr_pair, dim3(blocks_for(nB, 64), R), 64, 0, s, csr_ba.rp.as<int32_t>(),
                   csr_ba.ci.as<int32_t>(), csr_ba.v.as<double>(), NB, xin, xin + NA, n, tb1.as<double2>(), nB, 1.0,
                   1.0, 0);
        BEM_TRY(mass_solve(mopB, tb1.as<double2>(), tb2.as<double2>(), R, s, steps));
        BEM_TRY(prod(Ph, &Bh32, nB, x32b.as<float2>(), tb2.as<double2>(), tb3.as<double2>()));
        BEM_TRY(mass_solve(mopB, tb3.as<double2>(), tb1.as<double2>(), R, s, steps));
        BEM_LAUNCH(k_csr_pair, dim3(blocks_for(n, 64), R), 64, 0, s, csr_ab.rp.as<int32_t>(), csr_ab.ci.as<int32_t>(),
                   csr_ab.v.as<double>(), NA, tb1.as<double2>(), tb1.as<double2>() + NB, nB, z, n, 1.0, 1.0, 1);
        BEM_TRY(mass_solve(mop, z, yout, R, s, steps));
        if (muller)
            BEM_LAUNCH(k_acc, blocks_for((int64_t)R * n, 256), 256, 0, s, yout, xin, (int64_t)R * n);
        return BEM_OK;
    };
    // high-contrast product (Sec. 2.3; the strong form of the system, left-multiplied by
    // M_A^-1), for x = (x_0, x_1) on grid A:
    //   z = own rows (T_A x_1; V_A x_1) or (K_A x_0; D_A x_0);  w = M_A^-1 z
    //   t = M_B^-1 P_BA (x_0; w_1) [Neumann] or (w_1; x_1) [Dirichlet]
    //   h = M_B^-1 (c1 X1 t_0 + c2 X2 t_1);  u = M_A^-1 P_AB h into half 0 [Neumann] or 1
    //   y = the formulation's combination of x, u and w (hc_y)
    DevBuf hw, hz2, hu, hfp, hmf;
    if (hc) {
        BEM_TRY(hw.alloc(RB * colb, s));
        BEM_TRY(hz2.alloc(RB * colb, s));
        BEM_TRY(hu.alloc(RB * colb, s));
        BEM_TRY(hfp.alloc((size_t)RB * 2 * Ne * 16, s));  // -(f; g), exterior grid
        BEM_TRY(hmf.alloc((size_t)RB * 2 * Ne * 16, s));  // M_e^-1 of it (exterior variants)
    }
    PairCoef hc_y{};
    {
        // sources (x_0, x_1, u_0, u_1, w_0, w_1) of y_0 (first six) and y_1
        const double en[12] = {0.5, 0, 1, 0, 0, 0, 1, 0.5, 0, 0, -1, 0};   // exterior Neumann
        const double in[12] = {0.5, 0, 1, 0, 0, 0, -1, 0.5, 0, 0, 1, 0};   // interior Neumann
        const double ed[12] = {0.5, 1, 0, 0, 1, 0, 0, 0.5, 0, 1, 0, 0};    // exterior Dirichlet
        const double id[12] = {0.5, -1, 0, 0, -1, 0, 0, 0.5, 0, 1, 0, 0};  // interior Dirichlet
        const double* c = form == BEM_FORM_HC_EXT_NEU ? en : form == BEM_FORM_HC_INT_NEU ? in
                        : form == BEM_FORM_HC_EXT_DIR ? ed : id;
        for (int k = 0; k < 12; ++k) hc_y.c[k] = c[k];
    }
    auto pair_lin = [&](double2* y, const double2* x, const double2* u, const double2* w, int64_t N, int R,
                        const PairCoef& C) -> bem_status {
        BEM_LAUNCH(k_pair_lin, dim3(blocks_for(2 * N, 256), R), 256, 0, s, y, x, u, w, N, 2 * N, C);
        return BEM_OK;
    };
    auto csr_pair = [&](const CsrBuf& P, int64_t rows, const double2* x0, const double2* x1, int64_t nx, double2* zo,
                        int64_t nz, double c0, double c1, int R) -> bem_status {
        BEM_LAUNCH(k_csr_pair, dim3(blocks_for(2 * rows, 64), R), 64, 0, s, P.rp.as<int32_t>(), P.ci.as<int32_t>(),
                   P.v.as<double>(), rows, x0, x1, nx, zo, nz, c0, c1, 0);
        return BEM_OK;
    };
    auto apply_hc = [&](bool fp64, const double2* xin, double2* yout, int R, int steps) -> bem_status {
        auto prod = [&](const TileProd& P, const Blocks<float2>* tcb, int64_t nn, float2* xw, const double2* xi,
                        double2* zo) -> bem_status {
            return fp64 ? gemm_fp64_on(P, nn, xi, zo, R) : gemm_work_on(P, tcb, nn, xw, xi, zo, R);
        };
        double2* w = hw.as<double2>();
        BEM_TRY(prod(P0, &B32, n, x32.as<float2>(), xin, z));
        BEM_TRY(mass_solve(mop, z, w, R, s, steps));
        if (hc_neu) BEM_TRY(csr_pair(csr_ba, NB, xin, w + NA, n, tb1.as<double2>(), nB, 1.0, 1.0, R));
        else BEM_TRY(csr_pair(csr_ba, NB, w + NA, xin + NA, n, tb1.as<double2>(), nB, 1.0, 1.0, R));
        BEM_TRY(mass_solve(mopB, tb1.as<double2>(), tb2.as<double2>(), R, s, steps));
        BEM_TRY(prod(Ph, &Bh32, nB, x32b.as<float2>(), tb2.as<double2>(), tb3.as<double2>()));
        BEM_TRY(mass_solve(mopB, tb3.as<double2>(), tb1.as<double2>(), R, s, steps));
        // tb1 = (M_B^-1 h; 0): P_AB of its first half into half 0 (Neumann) or 1 (Dirichlet)
        const double2* t0 = tb1.as<double2>();
        const double2* t1 = tb1.as<double2>() + NB;
        if (hc_neu) BEM_TRY(csr_pair(csr_ab, NA, t0, t1, nB, hz2.as<double2>(), n, 1.0, 0.0, R));
        else BEM_TRY(csr_pair(csr_ab, NA, t1, t0, nB, hz2.as<double2>(), n, 0.0, 1.0, R));
        BEM_TRY(mass_solve(mop, hz2.as<double2>(), hu.as<double2>(), R, s, steps));
        return pair_lin(yout, xin, hu.as<double2>(), w, NA, R, hc_y);
    };
    // S A x in the working precision, and with FP64 arithmetic on the stored matrices
    // the multiple-traces system's FP32 inner solves precondition with S' (CHEB_STEPS_PRE)
    const bool pre_inner = fp32_inner && !hc && !st;
    Apply apply_work = [&](const double2* xin, double2* yout, int R) -> bem_status {
        const int steps = !mixed                 ? CHEB_STEPS
                          : (R == 1 && dd_now()) ? CHEB_STEPS_DD
                          : pre_inner            ? CHEB_STEPS_PRE
                                                 : CHEB_STEPS_INNER;
        if (hc) return apply_hc(false, xin, yout, R, steps);
        if (st) return apply_single(false, xin, yout, R, steps);
        BEM_TRY(gemm_work_on(P0, &B32, n, x32.as<float2>(), xin, z, R));
        BEM_TRY(transfer_add(top, R, xin, z, s));
        return mass_solve(mop, z, yout, R, s, steps);
    };
    // A x of the multiple-traces system with FP64 arithmetic, before the mass inverse
    auto raw_fp64 = [&](const double2* xin, double2* zout, int R) -> bem_status {
        BEM_TRY(gemm_fp64_on(P0, n, xin, zout, R));
        return transfer_add(top, R, xin, zout, s);
    };
    Apply apply_fp64 = [&](const double2* xin, double2* yout, int R) -> bem_status {
        if (hc) return apply_hc(true, xin, yout, R, CHEB_STEPS);
        if (st) return apply_single(true, xin, yout, R, CHEB_STEPS);
        BEM_TRY(raw_fp64(xin, z, R));
        return mass_solve(mop, z, yout, R, s, CHEB_STEPS);
    };
    // ---- GMRES ------------------------------------------------------------------------
    const int maxit = (int)std::min<int64_t>(o->gmres_maxiter, n);
    GmresWork W;
    // inner solves on FP32 or tensor-core products throughout keep a complex64 basis;
    // single right-hand sides with a double-float phase keep the FP64 basis
    BEM_TRY(W.init(maxit, n, RB, RW - RB, s, fp32_inner));
    DevBuf fvec, gvec, bvec, sb, xsol, dvec, rvec, tmp, wave;
    BEM_TRY(wave.alloc((size_t)5 * RB * 8, s));
    BEM_TRY(fvec.alloc((size_t)RB * Ne * 16, s));
    BEM_TRY(gvec.alloc((size_t)RB * Ne * 16, s));
    BEM_TRY(bvec.alloc(RB * colb, s));
    BEM_TRY(sb.alloc(RB * colb, s));
    BEM_TRY(xsol.alloc(RW * colb, s));  // read with RW columns by the FP64 residual
    BEM_CUDA_TRY(cudaMemsetAsync(xsol.p, 0, RW * colb, s));
    BEM_TRY(dvec.alloc(RB * colb, s));
    BEM_TRY(rvec.alloc(RB * colb, s));
    BEM_TRY(tmp.alloc(RB * colb, s));
    DevBuf rin;  // S'(b - A x): the inner right-hand side when pre_inner
    if (pre_inner) BEM_TRY(rin.alloc(RB * colb, s));
    bem_status result = BEM_OK;
    int total_inner = 0, outer_used = 0;
    double worst_res = 0.0;
    bool all_conv = true;
    cudaEventRecord(t_sol.a, s);
    for (int r0 = 0; r0 < inc->n_rhs; r0 += RB) {
        const int R = std::min(RB, inc->n_rhs - r0);
        BEM_TRY(incident_data(inc, r0, R, RB, ge, k_ext, W.h_wave, wave, fvec.as<double2>(), gvec.as<double2>(),
                              on_device != 0, s));
        if (hc) {
            // high-contrast data (weak form), from F = -(f; g):
            //   exterior Neumann ((1/r) D^_i M_e^-1 f; g), Dirichlet (f; r V^_i M_e^-1 g);
            //   interior Neumann (r P_ie M_e^-1 (D_e M_e^-1 f + g/2 + T_e M_e^-1 g); 0),
            //   Dirichlet (0; P_ie M_e^-1 (V_e M_e^-1 g + f/2 - K_e M_e^-1 f))
            const MassOp& E = st_int ? mopB : mop;  // the exterior grid's pair
            double2* F = hfp.as<double2>();
            double2* mF = st_int ? tb2.as<double2>() : hmf.as<double2>();
            BEM_LAUNCH(k_rhs_pack, dim3(blocks_for(2 * Ne, 256), R), 256, 0, s, fvec.as<double2>(),
                       gvec.as<double2>(), Ne, 2 * Ne, F);
            BEM_TRY(mass_solve(E, F, mF, R, s, CHEB_STEPS));
            if (!st_int) {
                const double2* src = hc_neu ? mF : mF + Ne;
                BEM_TRY(csr_pair(csr_p, Ni, src, src, 2 * Ne, tb1.as<double2>(), nB, 1.0, 0.0, R));
                BEM_TRY(mass_solve(mopB, tb1.as<double2>(), tb2.as<double2>(), R, s, CHEB_STEPS));
                BEM_TRY(gemm_fp64_on(Pr, nB, tb2.as<double2>(), tb3.as<double2>(), R));
                BEM_TRY(mass_solve(mopB, tb3.as<double2>(), tb1.as<double2>(), R, s, CHEB_STEPS));
                BEM_TRY(csr_pair(csr_t, Ne, tb1.as<double2>(), tb1.as<double2>(), nB, hz2.as<double2>(), n, 1.0, 0.0,
                                 R));
                PairCoef C{};  // sources (x = hat part, u = F): negated, F = -(f; g)
                if (hc_neu) { C.c[0] = -1.0; C.c[6 + 3] = -1.0; }
                else { C.c[2] = -1.0; C.c[6 + 0] = -1.0; }
                BEM_TRY(pair_lin(bvec.as<double2>(), hz2.as<double2>(), F, F, Ne, R, C));
            } else {
                BEM_TRY(gemm_fp64_on(Pr, nB, mF, tb3.as<double2>(), R));
                PairCoef C{};  // (x = product, u = F): x_0 + F_1 / 2 (Neumann) or x_0 + F_0 / 2
                C.c[0] = 1.0;
                C.c[hc_neu ? 3 : 2] = 0.5;
                BEM_TRY(pair_lin(tb1.as<double2>(), tb3.as<double2>(), F, F, Ne, R, C));
                BEM_TRY(mass_solve(mopB, tb1.as<double2>(), tb2.as<double2>(), R, s, CHEB_STEPS));
                const double2* t0 = tb2.as<double2>();
                const double2* t1 = tb2.as<double2>() + Ne;
                if (hc_neu) BEM_TRY(csr_pair(csr_p, Ni, t0, t1, nB, bvec.as<double2>(), n, -rho_ratio, 0.0, R));
                else BEM_TRY(csr_pair(csr_p, Ni, t1, t0, nB, bvec.as<double2>(), n, 0.0, -1.0, R));
            }
        } else if (st_int) {
            // interior variants: [P_ie M_e^-1 f; (rho_i / rho_e) P_ie M_e^-1 g]
            BEM_LAUNCH(k_rhs_pack, dim3(blocks_for(nB, 256), R), 256, 0, s, fvec.as<double2>(), gvec.as<double2>(),
                       Ne, nB, tb1.as<double2>());
            BEM_TRY(mass_solve(mopB, tb1.as<double2>(), tb2.as<double2>(), R, s, CHEB_STEPS));
            BEM_LAUNCH(k_csr_pair, dim3(blocks_for(n, 64), R), 64, 0, s, csr_ab.rp.as<int32_t>(),
                       csr_ab.ci.as<int32_t>(), csr_ab.v.as<double>(), NA, tb2.as<double2>(), tb2.as<double2>() + NB,
                       nB, bvec.as<double2>(), n, -1.0, -rho_ratio, 0);
        } else {
            BEM_LAUNCH(k_rhs_pack, dim3(blocks_for(n, 256), R), 256, 0, s, fvec.as<double2>(), gvec.as<double2>(),
                       Ne, n, bvec.as<double2>());
        }
        BEM_TRY(mass_solve(mop, bvec.as<double2>(), sb.as<double2>(), R, s, CHEB_STEPS));
        std::vector<double> beta(R), tol_abs(R), rn(R), est(R), inner_tol(R);
        std::vector<int> its(R), total(R, 0);
        BEM_TRY(norms(W, sb.as<double2>(), R, beta.data(), s));
        for (int r = 0; r < R; ++r) tol_abs[r] = o->gmres_tol * beta[r];
        if (!mixed) {
            BEM_TRY(gmres_run(W, R, apply_work, sb.as<double2>(), beta.data(), tol_abs.data(), xsol.as<double2>(),
                              its.data(), est.data(), s, stop));
            for (int r = 0; r < R; ++r) {
                rn[r] = est[r];
                total[r] = its[r];
            }
            outer_used = 1;
        } else {
            // iterative refinement: FP64 residual of the stored system, FP32-matvec GMRES corrections
            BEM_CUDA_TRY(cudaMemsetAsync(xsol.p, 0, (size_t)R * colb, s));
            BEM_CUDA_TRY(cudaMemcpyAsync(rvec.p, sb.p, (size_t)R * colb, cudaMemcpyDeviceToDevice, s));
            rn = beta;
            // inner right-hand side and its norms: S r itself, or S' r with the inner
            // solves' own preconditioner (the raw residual r = b at x = 0)
            std::vector<double> rinn(R);
            double2* inner_rhs = rvec.as<double2>();
            if (pre_inner) {
                BEM_TRY(mass_solve(mop, bvec.as<double2>(), rin.as<double2>(), R, s, CHEB_STEPS_PRE));
                BEM_TRY(norms(W, rin.as<double2>(), R, rinn.data(), s));
                inner_rhs = rin.as<double2>();
            } else {
                rinn = rn;
            }
            int outer = 0;
            const int max_outer = 12;
            auto pending = [&](int r) {
                return beta[r] > 0.0 && rn[r] > tol_abs[r] && total[r] < o->gmres_maxiter;
            };
            auto any_pending = [&] {
                for (int r = 0; r < R; ++r)
                    if (pending(r)) return true;
                return false;
            };
            const double inner_rel =
                o->ir_inner_tol > 0.0 ? o->ir_inner_tol : fp32_inner ? IR_INNER_TOL_BATCH : IR_INNER_TOL_SINGLE;
            while (any_pending() && outer < max_outer) {
                // a column that is finished (or out of iterations) gets tolerance |r|,
                // so that its inner GMRES takes no step and its correction is zero
                for (int r = 0; r < R; ++r)
                    inner_tol[r] = pending(r) ? inner_tolerance(rinn[r], rn[r], tol_abs[r], inner_rel) : rinn[r];
                BEM_TRY(gmres_run(W, R, apply_work, inner_rhs, rinn.data(), inner_tol.data(), dvec.as<double2>(),
                                  its.data(), est.data(), s, stop, &inner_progress));
                int moved = 0;
                for (int r = 0; r < R; ++r) {
                    total[r] += its[r];
                    moved += its[r];
                }
                BEM_LAUNCH(k_acc, blocks_for((int64_t)R * n, 256), 256, 0, s, xsol.as<double2>(), dvec.as<double2>(),
                           (int64_t)R * n);
                if (pre_inner) {
                    // r = b - A x in FP64 (into dvec, free until the next inner solve); S r for
                    // the convergence test, S' r for the next inner solve
                    BEM_TRY(raw_fp64(xsol.as<double2>(), z, R));
                    BEM_LAUNCH(k_sub, blocks_for((int64_t)R * n, 256), 256, 0, s, bvec.as<double2>(), z,
                               (int64_t)R * n, dvec.as<double2>());
                    BEM_TRY(mass_solve(mop, dvec.as<double2>(), rvec.as<double2>(), R, s, CHEB_STEPS));
                    BEM_TRY(mass_solve(mop, dvec.as<double2>(), rin.as<double2>(), R, s, CHEB_STEPS_PRE));
                    BEM_TRY(norms(W, rvec.as<double2>(), R, rn.data(), s));
                    BEM_TRY(norms(W, rin.as<double2>(), R, rinn.data(), s));
                } else {
                    BEM_TRY(apply_fp64(xsol.as<double2>(), tmp.as<double2>(), R));
                    BEM_LAUNCH(k_sub, blocks_for((int64_t)R * n, 256), 256, 0, s, sb.as<double2>(), tmp.as<double2>(),
                               (int64_t)R * n, rvec.as<double2>());
                    BEM_TRY(norms(W, rvec.as<double2>(), R, rn.data(), s));
                    rinn = rn;
                }
                ++outer;
                if (moved == 0) break;
            }
            outer_used = std::max(outer_used, outer);
        }
        for (int r = 0; r < R; ++r) {
            const double rel = beta[r] > 0.0 ? rn[r] / beta[r] : 0.0;
            const bool conv = beta[r] == 0.0 || rel <= o->gmres_tol;
            all_conv = all_conv && conv;
            worst_res = std::max(worst_res, rel);
            total_inner += total[r];
            if (!conv) result = BEM_E_NOT_CONVERGED;
        }
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        const double2* trace_src = xsol.as<double2>();
        if (hc) {
            // the unknowns' grid traces from the representation formula:
            //   exterior Neumann (M_e^-1 (f + V_e mu) negated; -a), Dirichlet (-b; -M_e^-1 (g + D_e nu)),
            //   interior Neumann (M_i^-1 V_i mu; a), Dirichlet (b; M_i^-1 D_i nu)
            BEM_TRY(gemm_fp64_on(Pq, n, xsol.as<double2>(), z, R));
            const double2* zin = z;
            if (!st_int) {
                PairCoef C{};  // z_0 + F_0 (Neumann) or z_0 + F_1, F = -(f; g)
                C.c[0] = 1.0;
                C.c[hc_neu ? 2 : 3] = 1.0;
                BEM_TRY(pair_lin(hz2.as<double2>(), z, hfp.as<double2>(), hfp.as<double2>(), NA, R, C));
                zin = hz2.as<double2>();
            }
            BEM_TRY(mass_solve(mop, zin, hu.as<double2>(), R, s, CHEB_STEPS));
            PairCoef C{};  // sources (x = unknowns, u = M_A^-1 part)
            switch (form) {
                case BEM_FORM_HC_EXT_NEU: C.c[2] = 1.0; C.c[6 + 0] = -1.0; break;
                case BEM_FORM_HC_EXT_DIR: C.c[1] = -1.0; C.c[6 + 2] = 1.0; break;
                case BEM_FORM_HC_INT_NEU: C.c[2] = 1.0; C.c[6 + 0] = 1.0; break;
                default: C.c[1] = 1.0; C.c[6 + 2] = 1.0; break;
            }
            BEM_TRY(pair_lin(hw.as<double2>(), xsol.as<double2>(), hu.as<double2>(), hu.as<double2>(), NA, R, C));
            trace_src = hw.as<double2>();
        }
        if (st) {
            // the other grid's potentials from the transmission conditions tested on it:
            // v_i = -M_i^-1 P_ie v_e, w_i = -(rho_i / rho_e) M_i^-1 P_ie w_e (exterior
            // variants); v_e = -M_e^-1 P_ei v_i, w_e = -(rho_e / rho_i) M_e^-1 P_ei w_i
            BEM_LAUNCH(k_csr_pair, dim3(blocks_for(nB, 64), R), 64, 0, s, csr_ba.rp.as<int32_t>(),
                       csr_ba.ci.as<int32_t>(), csr_ba.v.as<double>(), NB, trace_src, trace_src + NA, n,
                       tb1.as<double2>(), nB, -1.0, st_int ? -1.0 / rho_ratio : -rho_ratio, 0);
            BEM_TRY(mass_solve(mopB, tb1.as<double2>(), tb2.as<double2>(), R, s, CHEB_STEPS));
        }
        for (int r = 0; r < R; ++r) {
            const double2* X = trace_src + (int64_t)r * n;
            const double2* XB = st ? tb2.as<double2>() + (int64_t)r * nB : nullptr;
            const double2* XE = !st ? X : st_int ? XB : X;
            const double2* XI = !st ? X + 2 * Ne : st_int ? X : XB;
            const int64_t rr = r0 + r;
            BEM_CUDA_TRY(cudaMemcpyAsync(v_ext + rr * Ne, XE, Ne * 16, kind, s));
            BEM_CUDA_TRY(cudaMemcpyAsync(w_ext + rr * Ne, XE + Ne, Ne * 16, kind, s));
            BEM_CUDA_TRY(cudaMemcpyAsync(v_int + rr * Ni, XI, Ni * 16, kind, s));
            BEM_CUDA_TRY(cudaMemcpyAsync(w_int + rr * Ni, XI + Ni, Ni * 16, kind, s));
        }
        BEM_CUDA_TRY(cudaStreamSynchronize(s));
    }
    cudaEventRecord(t_sol.b, s);
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    if (tc_batches) {
        int h_err = 0;
        BEM_CUDA_TRY(cudaMemcpy(&h_err, tcerr.p, sizeof(int), cudaMemcpyDeviceToHost));
        if (h_err) {
            set_error("tensor-core product: an mbarrier wait timed out");
            return BEM_E_INTERNAL;
        }
    }
    BEM_TRY(check_tile_flag(tperr));
    BEM_TRY(csync.check());
    if (result == BEM_E_NOT_CONVERGED)
        set_error("GMRES did not reach the tolerance within gmres_maxiter iterations; outputs hold the last iterate");
    if (rep) {
        rep->iterations = total_inner;
        rep->converged = all_conv ? 1 : 0;
        rep->residual = worst_res;
        rep->t_assembly_ms = t_asm.ms();
        rep->t_mortar_ms = t_mor.ms();
        rep->t_solve_ms = t_sol.ms();
        rep->mtf_variant = o->mtf_variant;
        rep->outer_iterations = outer_used;
    }
    return result;
}

// ================================================================ many instances
// Independent transmission problems of uneven sizes (different grids, wavenumbers,
// density ratios), one plane wave each, solved together: their vectors are
// concatenated, every row-indexed kernel looks up the instance of its row, and each
// step of the lockstep GMRES / refinement is one launch for all instances, each with
// its own Krylov process and stopping test.  The regular-pair assembly of all their
// grids is one persistent launch.  Mixed-precision mode.

namespace {

struct InstDesc {
    int64_t off, n;    // the instance's vector occupies [off, off + n) of the concatenation
    MassPair M;        // mass matrices of its two grids
    TransferCsr T;     // mortar transfer
};

__global__ void k_transfer_many(const InstDesc* __restrict__ D, const int32_t* __restrict__ row_inst, int64_t total,
                                const double2* __restrict__ xall, double2* __restrict__ zall) {
    const int64_t gw = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gw >= total) return;
    const InstDesc& d = D[row_inst[gw]];
    const TransferCsr& T = d.T;
    const int64_t g = gw - d.off;
    const double2* x = xall + d.off;
    const bool ext = g < 2 * T.Ne;
    const int32_t* rp = ext ? T.trp : T.prp;
    const int32_t* ci = ext ? T.tci : T.pci;
    const double* v = ext ? T.tv : T.pv;
    int64_t row, src;
    double c;
    if (g < T.Ne) { row = g; src = 2 * T.Ne; c = T.ca; }
    else if (g < 2 * T.Ne) { row = g - T.Ne; src = 2 * T.Ne + T.Ni; c = T.cb; }
    else if (g < 2 * T.Ne + T.Ni) { row = g - 2 * T.Ne; src = 0; c = T.cc; }
    else { row = g - 2 * T.Ne - T.Ni; src = T.Ne; c = T.cd; }
    double sr = 0.0, si = 0.0;
    for (int32_t e = rp[row]; e < rp[row + 1]; ++e) {
        const double p = v[e];
        const double2 xx = x[src + ci[e]];
        sr = fma(p, xx.x, sr);
        si = fma(p, xx.y, si);
    }
    double2 zz = zall[gw];
    zz.x = fma(c, sr, zz.x);
    zz.y = fma(c, si, zz.y);
    zall[gw] = zz;
}

__global__ void k_cheb_init_many(const InstDesc* __restrict__ D, const int32_t* __restrict__ row_inst,
                                 int64_t total, const double2* __restrict__ z, double2* __restrict__ y,
                                 double2* __restrict__ r, double2* __restrict__ d0, double inv_theta) {
    const int64_t gw = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gw >= total) return;
    const InstDesc& d = D[row_inst[gw]];
    const MassRow m = mass_row(d.M, gw - d.off);
    const double2 zz = z[gw];
    const double sc = m.dinv[m.i] * inv_theta;
    y[gw] = make_double2(0, 0);
    r[gw] = zz;
    d0[gw] = make_double2(sc * zz.x, sc * zz.y);
}

__global__ void k_cheb_step_many(const InstDesc* __restrict__ D, const int32_t* __restrict__ row_inst,
                                 int64_t total, const double2* __restrict__ dk, double2* __restrict__ dn,
                                 double2* __restrict__ y, double2* __restrict__ r, double c1, double c2) {
    const int64_t gw = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gw >= total) return;
    const InstDesc& d = D[row_inst[gw]];
    const MassRow m = mass_row(d.M, gw - d.off);
    const double2 md = mass_apply_row(m, dk + d.off + m.base);
    const double2 d0 = dk[gw];
    double2 yy = y[gw], rr = r[gw];
    yy.x += d0.x;
    yy.y += d0.y;
    rr.x -= md.x;
    rr.y -= md.y;
    y[gw] = yy;
    r[gw] = rr;
    const double sc = c2 * m.dinv[m.i];
    dn[gw] = make_double2(c1 * d0.x + sc * rr.x, c1 * d0.y + sc * rr.y);
}

// the FP32 iteration of k_cheb_init32 / k_cheb_step32 over the concatenation
__global__ void k_cheb_init32_many(const InstDesc* __restrict__ D, const int32_t* __restrict__ row_inst,
                                   int64_t total, const double2* __restrict__ z, float2* __restrict__ r,
                                   float2* __restrict__ d0, float inv_theta) {
    const int64_t gw = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gw >= total) return;
    const InstDesc& d = D[row_inst[gw]];
    const MassRow m = mass_row(d.M, gw - d.off);
    const double2 zz = z[gw];
    const float2 rz = make_float2((float)zz.x, (float)zz.y);
    const float sc = (m.base < 2 * d.M.Ne ? d.M.dinvf[0] : d.M.dinvf[1])[m.i] * inv_theta;
    r[gw] = rz;
    d0[gw] = make_float2(sc * rz.x, sc * rz.y);
}

__global__ void k_cheb_step32_many(const InstDesc* __restrict__ D, const int32_t* __restrict__ row_inst,
                                   int64_t total, const float2* __restrict__ dk, float2* __restrict__ dn,
                                   float2* __restrict__ y, float2* __restrict__ r, float c1, float c2, int first,
                                   double2* __restrict__ yout) {
    const int64_t gw = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gw >= total) return;
    const InstDesc& d = D[row_inst[gw]];
    const MassRow m = mass_row(d.M, gw - d.off);
    const bool ext = m.base < 2 * d.M.Ne;
    const float* __restrict__ vf = ext ? d.M.vf[0] : d.M.vf[1];
    const float2* __restrict__ dd = dk + d.off + m.base;
    float2 md = make_float2(0.f, 0.f);
    for (int k = 0; k < m.W; ++k) {
        const float v = vf[(int64_t)k * m.N + m.i];
        const float2 x = dd[m.ci[(int64_t)k * m.N + m.i]];
        md.x = fmaf(v, x.x, md.x);
        md.y = fmaf(v, x.y, md.y);
    }
    const float2 d0 = dk[gw];
    float2 yy = d0;
    if (!first) {
        const float2 yp = y[gw];
        yy.x += yp.x;
        yy.y += yp.y;
    }
    float2 rr = r[gw];
    rr.x -= md.x;
    rr.y -= md.y;
    if (yout) yout[gw] = make_double2((double)yy.x, (double)yy.y);
    else y[gw] = yy;
    r[gw] = rr;
    const float sc = c2 * (ext ? d.M.dinvf[0] : d.M.dinvf[1])[m.i];
    dn[gw] = make_float2(fmaf(c1, d0.x, sc * rr.x), fmaf(c1, d0.y, sc * rr.y));
}

// inner products over chunks that never straddle two instances: chunk c covers
// rows [cs[c], ce[c]) of instance ci[c]; partial[i * nchunks + c]
__global__ void __launch_bounds__(256) k_dots_partial_many(const double2* __restrict__ Vb, int64_t total, int m,
                                                           const double2* __restrict__ w,
                                                           const int64_t* __restrict__ cs,
                                                           const int64_t* __restrict__ ce, int nchunks,
                                                           double2* __restrict__ partial) {
    // double-float, DOT_VPW basis vectors per warp, as k_dots_partial
    const int c = blockIdx.x;
    const int lane = threadIdx.x & 31;
    const int i0 = (blockIdx.y * 8 + (threadIdx.x >> 5)) * DOT_VPW;
    if (i0 >= m) return;
    const int nv = min(DOT_VPW, m - i0);
    const int64_t e1 = ce[c];
    float4 S[DOT_VPW];
#pragma unroll
    for (int u = 0; u < DOT_VPW; ++u) S[u] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 2
    for (int64_t e = cs[c] + lane; e < e1; e += 32) {
        const float4 b = ddf::split2(w[e]);
#pragma unroll
        for (int u = 0; u < DOT_VPW; ++u)
            if (u < nv) ddf::cmac<true>(S[u], ddf::split2(Vb[(int64_t)(i0 + u) * total + e]), b);
    }
#pragma unroll
    for (int u = 0; u < DOT_VPW; ++u) {
        if (u >= nv) break;
        float4 t = S[u];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float4 q;
            q.x = __shfl_xor_sync(0xffffffffu, t.x, o);
            q.y = __shfl_xor_sync(0xffffffffu, t.y, o);
            q.z = __shfl_xor_sync(0xffffffffu, t.z, o);
            q.w = __shfl_xor_sync(0xffffffffu, t.w, o);
            ddf::add(t, q);
        }
        if (lane == 0) partial[(int64_t)(i0 + u) * nchunks + c] = ddf::value(t);
    }
}

// out[r * ostride + i] = sum of the chunks of instance r (grid (m, instances))
__global__ void k_dots_final_many(const double2* __restrict__ partial, int nchunks, const int* __restrict__ cb,
                                  double2* __restrict__ out, int64_t ostride) {
    const int i = blockIdx.x, r = blockIdx.y;
    double2 s = make_double2(0, 0);
    for (int c = cb[r] + threadIdx.x; c < cb[r + 1]; c += 32) {
        const double2 p = partial[(int64_t)i * nchunks + c];
        s.x += p.x;
        s.y += p.y;
    }
    s = warp_sum2(s);
    if (threadIdx.x == 0) out[r * ostride + i] = s;
}

__global__ void __launch_bounds__(256) k_combine_many(const double2* __restrict__ Vb, int64_t total, int m,
                                                      const int* __restrict__ mr, const int32_t* __restrict__ row_inst,
                                                      const double2* __restrict__ h, int64_t hstride,
                                                      double2* __restrict__ w, int overwrite) {
    // double-float, as k_combine (each row's instance picks its coefficients)
    const int lr = threadIdx.x & 31, sl = threadIdx.x >> 5;
    const int64_t e = blockIdx.x * 32ll + lr;
    float4 S = make_float4(0.f, 0.f, 0.f, 0.f);
    if (e < total) {
        const int r = row_inst[e];
        const int mm = mr ? mr[r] : m;
        const double2* __restrict__ hr = h + r * hstride;
#pragma unroll 4
        for (int i = sl; i < mm; i += 8)
            ddf::cmac<false>(S, ddf::split2(hr[i]), ddf::split2(Vb[(int64_t)i * total + e]));
    }
    __shared__ float4 part[8][32];
    part[sl][lr] = S;
    __syncthreads();
    if (sl == 0 && e < total) {
        float4 t = part[0][lr];
#pragma unroll
        for (int k = 1; k < 8; ++k) ddf::add(t, part[k][lr]);
        const double2 tv = ddf::value(t);
        if (overwrite) w[e] = tv;
        else w[e] = make_double2(w[e].x - tv.x, w[e].y - tv.y);
    }
}

// v = w / |w| per instance; the first row of each instance writes |w| to dst[r * dstride]
__global__ void k_normalize_many(const InstDesc* __restrict__ D, const int32_t* __restrict__ row_inst,
                                 const double2* __restrict__ w, int64_t total, const double2* __restrict__ nrm2,
                                 double2* __restrict__ v, double2* __restrict__ dst, int64_t dstride) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int r = row_inst[e];
    const double nr = sqrt(fmax(nrm2[r].x, 0.0));
    if (dst && e == D[r].off) dst[r * dstride] = make_double2(nr, 0.0);
    const double inv = nr > 0.0 ? 1.0 / nr : 0.0;
    v[e] = make_double2(w[e].x * inv, w[e].y * inv);
}

// b = [-f, -g, 0, 0] of instance r from its plane-wave data f, g (N_ext each)
__global__ void k_rhs_pack_one(const double2* __restrict__ f, const double2* __restrict__ g, int64_t Ne, int64_t n,
                               double2* __restrict__ b) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    double2 v = make_double2(0.0, 0.0);
    if (e < Ne) v = make_double2(-f[e].x, -f[e].y);
    else if (e < 2 * Ne) v = make_double2(-g[e - Ne].x, -g[e - Ne].y);
    b[e] = v;
}

// device layout of many instances and the workspaces of their lockstep solve
struct ManyLayout {
    int count = 0, nchunks = 0;
    int64_t total = 0;
    std::vector<int64_t> off, len;
    DevBuf desc, row_inst, cs, ce, cb;
};

struct ManyGmres {
    int maxit = 0, count = 0;
    int64_t total = 0, ldh = 0, gstride = 0;
    DevBuf Vb, H, partial, hbuf, y, w, nrm, mr;
    double2* h_nrm = nullptr;
    double2* h_col = nullptr;
    double2* h_y = nullptr;
    int* h_mr = nullptr;
    cudaEvent_t ev[GMRES_SLOTS] = {};
    cudaStream_t stream = nullptr;
    ~ManyGmres() {
        if (stream) cudaStreamSynchronize(stream);
        if (h_nrm) cudaFreeHost(h_nrm);
        if (h_col) cudaFreeHost(h_col);
        if (h_y) cudaFreeHost(h_y);
        if (h_mr) cudaFreeHost(h_mr);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
    bem_status init(int maxit_, const ManyLayout& L, cudaStream_t s) {
        maxit = maxit_;
        count = L.count;
        total = L.total;
        stream = s;
        ldh = maxit + 1;
        gstride = maxit + 2;
        BEM_TRY(Vb.alloc((size_t)(maxit + 1) * total * 16, s));
        BEM_TRY(H.alloc((size_t)count * ldh * ldh * 16, s));
        BEM_TRY(partial.alloc((size_t)(maxit + 1) * L.nchunks * 16, s));
        BEM_TRY(hbuf.alloc((size_t)count * gstride * 16, s));
        BEM_TRY(y.alloc((size_t)count * gstride * 16, s));
        BEM_TRY(w.alloc((size_t)total * 16, s));
        BEM_TRY(nrm.alloc((size_t)count * 16, s));
        BEM_TRY(mr.alloc((size_t)count * 4, s));
        BEM_CUDA_TRY(cudaMallocHost(&h_nrm, (size_t)count * 16));
        BEM_CUDA_TRY(cudaMallocHost(&h_col, (size_t)GMRES_SLOTS * count * gstride * 16));
        BEM_CUDA_TRY(cudaMallocHost(&h_y, (size_t)count * gstride * 16));
        BEM_CUDA_TRY(cudaMallocHost(&h_mr, (size_t)count * 4));
        for (cudaEvent_t& e : ev) BEM_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        return BEM_OK;
    }
};

bem_status many_sq_norms(const ManyLayout& L, ManyGmres& W, const double2* v, cudaStream_t s) {
    BEM_LAUNCH(k_dots_partial_many, dim3(L.nchunks, 1), 256, 0, s, v, L.total, 1, v, L.cs.as<int64_t>(),
               L.ce.as<int64_t>(), L.nchunks, W.partial.as<double2>());
    BEM_LAUNCH(k_dots_final_many, dim3(1, L.count), 32, 0, s, W.partial.as<double2>(), L.nchunks, L.cb.as<int>(),
               W.nrm.as<double2>(), 1);
    return BEM_OK;
}

bem_status many_norms(const ManyLayout& L, ManyGmres& W, const double2* v, double* out, cudaStream_t s) {
    BEM_TRY(many_sq_norms(L, W, v, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(W.h_nrm, W.nrm.p, (size_t)L.count * 16, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    for (int r = 0; r < L.count; ++r) out[r] = std::sqrt(std::max(W.h_nrm[r].x, 0.0));
    return BEM_OK;
}

using ApplyMany = std::function<bem_status(const double2* in, double2* out)>;

// the lockstep GMRES of gmres_run, one Krylov process per instance
bem_status gmres_run_many(const ManyLayout& L, ManyGmres& W, const ApplyMany& apply, const double2* rhs,
                          const double* beta, const double* tol_abs, double2* x, int* iters_out, double* res_out,
                          const HaltCheck& halted, cudaStream_t s) {
    const int C = L.count;
    const int64_t T = L.total, ldh = W.ldh, gs = W.gstride;
    double2* Vp = W.Vb.as<double2>();
    const unsigned eb = blocks_for(T, 256), ecb = blocks_for(T, 32);
    BEM_CUDA_TRY(cudaMemsetAsync(W.H.p, 0, (size_t)C * ldh * ldh * 16, s));
    std::vector<HostQR> qr(C);
    std::vector<int> it(C, 0);
    std::vector<char> done(C, 0);
    int ndone = 0;
    for (int r = 0; r < C; ++r) {
        qr[r].reset(beta[r]);
        res_out[r] = beta[r];
        if (!(beta[r] > tol_abs[r]) || halted(r) != BEM_OK) {
            done[r] = 1;
            ++ndone;
        }
    }
    int launched = 0, checked = 0;
    auto check_one = [&]() -> bem_status {
        const int slot = checked % GMRES_SLOTS;
        BEM_CUDA_TRY(cudaEventSynchronize(W.ev[slot]));
        for (int r = 0; r < C; ++r) {
            if (done[r]) continue;
            const double est = qr[r].add_column(W.h_col + ((size_t)slot * C + r) * gs, checked);
            it[r] = checked + 1;
            res_out[r] = est;
            if (!(est > tol_abs[r]) || halted(r) != BEM_OK) {
                done[r] = 1;
                ++ndone;
            }
        }
        ++checked;
        return BEM_OK;
    };
    const InstDesc* D = L.desc.as<InstDesc>();
    const int32_t* RI = L.row_inst.as<int32_t>();
    if (ndone < C) {
        BEM_TRY(many_sq_norms(L, W, rhs, s));
        BEM_LAUNCH(k_normalize_many, eb, 256, 0, s, D, RI, rhs, T, W.nrm.as<double2>(), Vp, nullptr, 0);
        for (int j = 0; j < W.maxit && ndone < C; ++j) {
            const double2* vj = Vp + (int64_t)j * T;
            BEM_TRY(apply(vj, W.w.as<double2>()));
            double2* Hj = W.H.as<double2>() + (int64_t)j * ldh;
            const unsigned gy = (unsigned)((j + 1 + DOT_VPB - 1) / DOT_VPB);
            for (int pass = 0; pass < 2; ++pass) {
                double2* h = pass == 0 ? Hj : W.hbuf.as<double2>();
                const int64_t hst = pass == 0 ? ldh * ldh : gs;
                BEM_LAUNCH(k_dots_partial_many, dim3(L.nchunks, gy), 256, 0, s, Vp, T, j + 1, W.w.as<double2>(),
                           L.cs.as<int64_t>(), L.ce.as<int64_t>(), L.nchunks, W.partial.as<double2>());
                BEM_LAUNCH(k_dots_final_many, dim3(j + 1, C), 32, 0, s, W.partial.as<double2>(), L.nchunks,
                           L.cb.as<int>(), h, hst);
                BEM_LAUNCH(k_combine_many, ecb, 256, 0, s, Vp, T, j + 1, nullptr, RI, h, hst, W.w.as<double2>(), 0);
            }
            BEM_LAUNCH(k_add_cols, dim3(1, C), 256, 0, s, Hj, ldh * ldh, W.hbuf.as<double2>(), gs, j + 1);
            BEM_TRY(many_sq_norms(L, W, W.w.as<double2>(), s));
            BEM_LAUNCH(k_normalize_many, eb, 256, 0, s, D, RI, W.w.as<double2>(), T, W.nrm.as<double2>(),
                       Vp + (int64_t)(j + 1) * T, Hj + j + 1, ldh * ldh);
            const int slot = j % GMRES_SLOTS;
            BEM_CUDA_TRY(cudaMemcpy2DAsync(W.h_col + (size_t)slot * C * gs, gs * 16, Hj, ldh * ldh * 16,
                                           (size_t)(j + 2) * 16, C, cudaMemcpyDeviceToHost, s));
            BEM_CUDA_TRY(cudaEventRecord(W.ev[slot], s));
            launched = j + 1;
            while (checked < launched - GMRES_LAG && ndone < C) BEM_TRY(check_one());
        }
        while (checked < launched && ndone < C) BEM_TRY(check_one());
    }
    for (int r = 0; r < C; ++r) {
        W.h_mr[r] = it[r];
        qr[r].solve(it[r], W.h_y + (size_t)r * gs);
    }
    BEM_CUDA_TRY(cudaMemcpyAsync(W.mr.p, W.h_mr, (size_t)C * 4, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(W.y.p, W.h_y, (size_t)C * gs * 16, cudaMemcpyHostToDevice, s));
    BEM_LAUNCH(k_combine_many, ecb, 256, 0, s, Vp, T, 0, W.mr.as<int>(), RI, W.y.as<double2>(), gs, x, 1);
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    for (int r = 0; r < C; ++r) iters_out[r] = it[r];
    return BEM_OK;
}

// operators, masses and mortar of one distinct problem (grids and wavenumbers), shared by
// the instances that differ only in their wave or density ratio (owned buffers)
struct ProblemData {
    GridOps ops[2];  // exterior, interior
    DevBuf mve, mvi, dve, dvi, dvef, dvif, prow, pcol, pval;
    CsrBuf csr_p, csr_t;
    MassEll ell_e, ell_i;
};

}  // namespace

bem_status solve_many_impl(bem_context* ctx, int count, const bem_instance* inst, const bem_solve_opts* o,
                           int on_device, bem_solve_report* reps, const HaltCheck* halt, int32_t* status_out) {
    cudaStream_t s = ctx->stream;
    // distinct problems: instances with the same grids and wavenumbers share one
    std::vector<int> prob(count);
    std::vector<int> first;  // an instance of each problem
    for (int i = 0; i < count; ++i) {
        int p = 0;
        for (; p < (int)first.size(); ++p) {
            const bem_instance& q = inst[first[p]];
            if (q.ext == inst[i].ext && q.intr == inst[i].intr && q.k_ext.re == inst[i].k_ext.re &&
                q.k_ext.im == inst[i].k_ext.im && q.k_int.re == inst[i].k_int.re && q.k_int.im == inst[i].k_int.im)
                break;
        }
        if (p == (int)first.size()) first.push_back(i);
        prob[i] = p;
    }
    const int nprob = (int)first.size();
    std::vector<ProblemData> data(nprob);
    // per-instance halting (cancellation, deadlines), remembered once it happens
    std::vector<bem_status> halted(count, BEM_OK);
    const HaltCheck halted_check = [&](int r) -> bem_status {
        if (halted[r] == BEM_OK && halt) halted[r] = (*halt)(r);
        return halted[r];
    };
    EventTimer t_asm, t_mor, t_sol;
    // ---- operators: one persistent launch for the regular pairs of all grids, then the
    // singular pairs grid by grid
    cudaEventRecord(t_asm.a, s);
    std::vector<const bem_grid*> grids;
    std::vector<double> kre, kim;
    std::vector<float2*> PV, PK, PT, PD;
    const OpLayouts TL = op_layouts_tiled();
    for (int p = 0; p < nprob; ++p) {
        const bem_instance& q = inst[first[p]];
        for (int side = 0; side < 2; ++side) {
            const bem_grid* g = side == 0 ? q.ext : q.intr;
            GridOps& go = data[p].ops[side];
            BEM_TRY(go.alloc(g->nv, 8, s));
            grids.push_back(g);
            const bem_c128 k = side == 0 ? q.k_ext : q.k_int;
            kre.push_back(k.re);
            kim.push_back(k.im);
            PV.push_back(go.V.as<float2>());
            PK.push_back(go.K.as<float2>());
            PT.push_back(nullptr);
            PD.push_back(go.D.as<float2>());
        }
    }
    BEM_TRY(assemble_regular_fp32_many((int)grids.size(), grids.data(), kre.data(), kim.data(), PV.data(), PK.data(),
                                       PT.data(), PD.data(), TL, s));
    for (size_t g = 0; g < grids.size(); ++g)
        BEM_TRY(assemble_singular_into_c64(grids[g], kre[g], kim[g], o->n_singular, PV[g], PK[g], PT[g], PD[g], TL,
                                           s));
    cudaEventRecord(t_asm.b, s);
    // ---- masses and mortar, problem by problem
    cudaEventRecord(t_mor.a, s);
    for (int p = 0; p < nprob; ++p) {
        const bem_grid *ge = inst[first[p]].ext, *gi = inst[first[p]].intr;
        ProblemData& d = data[p];
        BEM_TRY(d.mve.alloc(ge->m_nnz * 8, s));
        BEM_TRY(d.mvi.alloc(gi->m_nnz * 8, s));
        BEM_TRY(d.dve.alloc(ge->nv * 8, s));
        BEM_TRY(d.dvi.alloc(gi->nv * 8, s));
        BEM_TRY(mass_values(ge, d.mve.as<double>(), s));
        BEM_TRY(mass_values(gi, d.mvi.as<double>(), s));
        BEM_TRY(mass_inverse_diag(ge, d.mve.as<double>(), d.dve.as<double>(), s));
        BEM_TRY(mass_inverse_diag(gi, d.mvi.as<double>(), d.dvi.as<double>(), s));
        int64_t pnnz = 0;
        BEM_TRY(mortar_coo(gi, ge, o->center, d.prow, d.pcol, d.pval, &pnnz, s));
        BEM_TRY(build_csr(d.prow.as<int32_t>(), d.pcol.as<int32_t>(), d.pval.as<double>(), pnnz, gi->nv, d.csr_p, s));
        BEM_TRY(build_csr(d.pcol.as<int32_t>(), d.prow.as<int32_t>(), d.pval.as<double>(), pnnz, ge->nv, d.csr_t, s));
    }
    cudaEventRecord(t_mor.b, s);
    // ---- concatenated layout and instance descriptors
    ManyLayout L;
    L.count = count;
    TileProd PM;  // the dense products of all instances, one tile-product launch
    std::vector<InstDesc> desc(count);
    std::vector<int32_t> rinst;
    std::vector<int64_t> cs, ce;
    std::vector<int> cb(count + 1, 0);
    const double sgn = o->mtf_variant == BEM_MTF_PRINTED ? -1.0 : 1.0;
    for (int i = 0; i < count; ++i) {
        const int64_t Ne = inst[i].ext->nv, Ni = inst[i].intr->nv, n = 2 * Ne + 2 * Ni;
        const double rho = inst[i].rho_int_over_rho_ext;
        ProblemData& d = data[prob[i]];
        InstDesc& D = desc[i];
        D.off = L.total;
        D.n = n;
        // the instance's multiple-traces blocks, at its offset in the concatenation
        const int64_t o0 = D.off;
        d.ops[0].add(PM, -1.0, 1.0, 1.0, 1.0, o0, o0 + Ne, o0, o0 + Ne, o0, o0 + Ne);
        d.ops[1].add(PM, -1.0, 1.0, 1.0, 1.0, o0 + 2 * Ne, o0 + 2 * Ne + Ni, o0 + 2 * Ne, o0 + 2 * Ne + Ni,
                     o0 + 2 * Ne, o0 + 2 * Ne + Ni);
        if (first[prob[i]] == i) {
            BEM_TRY(d.ell_e.build(inst[i].ext, d.mve.as<double>(), s));
            BEM_TRY(d.ell_i.build(inst[i].intr, d.mvi.as<double>(), s));
            BEM_TRY(d.dvef.alloc((size_t)Ne * 4, s));
            BEM_TRY(d.dvif.alloc((size_t)Ni * 4, s));
            BEM_LAUNCH(k_narrow, blocks_for(Ne, 256), 256, 0, s, d.dve.as<double>(), Ne, d.dvef.as<float>());
            BEM_LAUNCH(k_narrow, blocks_for(Ni, 256), 256, 0, s, d.dvi.as<double>(), Ni, d.dvif.as<float>());
        }
        D.M.ci[0] = d.ell_e.ci.as<int32_t>(); D.M.v[0] = d.ell_e.v.as<double>(); D.M.W[0] = d.ell_e.W;
        D.M.dinv[0] = d.dve.as<double>();
        D.M.ci[1] = d.ell_i.ci.as<int32_t>(); D.M.v[1] = d.ell_i.v.as<double>(); D.M.W[1] = d.ell_i.W;
        D.M.dinv[1] = d.dvi.as<double>();
        D.M.vf[0] = d.ell_e.vf.as<float>(); D.M.vf[1] = d.ell_i.vf.as<float>();
        D.M.dinvf[0] = d.dvef.as<float>(); D.M.dinvf[1] = d.dvif.as<float>();
        D.M.Ne = Ne; D.M.Ni = Ni; D.M.n = n;
        D.T.prp = d.csr_p.rp.as<int32_t>(); D.T.pci = d.csr_p.ci.as<int32_t>(); D.T.pv = d.csr_p.v.as<double>();
        D.T.trp = d.csr_t.rp.as<int32_t>(); D.T.tci = d.csr_t.ci.as<int32_t>(); D.T.tv = d.csr_t.v.as<double>();
        D.T.Ne = Ne; D.T.Ni = Ni; D.T.n = n;
        D.T.ca = -0.5 * sgn;
        D.T.cb = -0.5 * sgn / rho;
        D.T.cc = 0.5 * sgn;
        D.T.cd = 0.5 * sgn * rho;
        L.off.push_back(L.total);
        L.len.push_back(n);
        rinst.insert(rinst.end(), (size_t)n, i);
        cb[i] = (int)cs.size();
        for (int64_t c0 = 0; c0 < n; c0 += DOT_ROWS) {
            cs.push_back(L.total + c0);
            ce.push_back(L.total + std::min<int64_t>(n, c0 + DOT_ROWS));
        }
        L.total += n;
    }
    cb[count] = (int)cs.size();
    L.nchunks = (int)cs.size();
    const int64_t T = L.total;
    BEM_TRY(L.desc.alloc(desc.size() * sizeof(InstDesc), s));
    BEM_TRY(L.row_inst.alloc(rinst.size() * 4, s));
    BEM_TRY(L.cs.alloc(cs.size() * 8, s));
    BEM_TRY(L.ce.alloc(ce.size() * 8, s));
    BEM_TRY(L.cb.alloc(cb.size() * 4, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(L.desc.p, desc.data(), desc.size() * sizeof(InstDesc), cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(L.row_inst.p, rinst.data(), rinst.size() * 4, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(L.cs.p, cs.data(), cs.size() * 8, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(L.ce.p, ce.data(), ce.size() * 8, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(L.cb.p, cb.data(), cb.size() * 4, cudaMemcpyHostToDevice, s));
    const InstDesc* Dd = L.desc.as<InstDesc>();
    const int32_t* RI = L.row_inst.as<int32_t>();
    // ---- workspaces
    DevBuf z, wr, wa, wb, x32, bvec, sb, xsol, dvec, rvec, tmp, fg, xsplit, part, tperr;
    for (DevBuf* b : {&z, &wr, &wa, &wb, &bvec, &sb, &xsol, &dvec, &rvec, &tmp}) BEM_TRY(b->alloc((size_t)T * 16, s));
    BEM_TRY(x32.alloc((size_t)T * 8, s));
    BEM_TRY(xsplit.alloc((size_t)T * 16, s));
    BEM_TRY(tile_prod_finish(PM, T, 8, s));
    BEM_TRY(part.alloc(tile_part_bytes(PM, TP_DD, 1), s));
    BEM_TRY(tperr.alloc(sizeof(int), s));
    BEM_CUDA_TRY(cudaMemsetAsync(tperr.p, 0, sizeof(int), s));
    const double theta = 0.5 * (CHEB_BETA + CHEB_ALPHA), delta = 0.5 * (CHEB_BETA - CHEB_ALPHA);
    const double sigma = theta / delta;
    GraphCache graphs(o->cuda_graphs != 0);
    std::function<bem_status(const double2*, double2*, int)> mass_many_eager;
    auto mass_many = [&](const double2* zin, double2* yout, int steps) -> bem_status {
        return graphs.run(GraphKey{wr.p, zin, yout, 0, steps}, s, [&]() { return mass_many_eager(zin, yout, steps); });
    };
    mass_many_eager = [&](const double2* zin, double2* yout, int steps) -> bem_status {
        const unsigned g64 = blocks_for(T, 64);
        if (steps <= CHEB_STEPS_INNER) {  // FP32 iteration (inner solves with FP32 products)
            float2* r32 = reinterpret_cast<float2*>(wr.p);
            float2* da = reinterpret_cast<float2*>(wa.p);
            float2* db = reinterpret_cast<float2*>(wb.p);
            float2* y32 = da + T;
            BEM_LAUNCH(k_cheb_init32_many, g64, 64, 0, s, Dd, RI, T, zin, r32, da, (float)(1.0 / theta));
            double rho = 1.0 / sigma;
            float2 *dk = da, *dn = db;
            for (int k = 0; k < steps; ++k) {
                const double rho_n = 1.0 / (2.0 * sigma - rho);
                BEM_LAUNCH(k_cheb_step32_many, g64, 64, 0, s, Dd, RI, T, dk, dn, y32, r32, (float)(rho_n * rho),
                           (float)(2.0 * rho_n / delta), k == 0 ? 1 : 0, k == steps - 1 ? yout : nullptr);
                rho = rho_n;
                std::swap(dk, dn);
            }
            return BEM_OK;
        }
        BEM_LAUNCH(k_cheb_init_many, g64, 64, 0, s, Dd, RI, T, zin, yout, wr.as<double2>(), wa.as<double2>(),
                   1.0 / theta);
        double rho = 1.0 / sigma;
        double2 *dk = wa.as<double2>(), *dn = wb.as<double2>();
        for (int k = 0; k < steps; ++k) {
            const double rho_n = 1.0 / (2.0 * sigma - rho);
            BEM_LAUNCH(k_cheb_step_many, g64, 64, 0, s, Dd, RI, T, dk, dn, yout, wr.as<double2>(), rho_n * rho,
                       2.0 * rho_n / delta);
            rho = rho_n;
            std::swap(dk, dn);
        }
        return BEM_OK;
    };
    // FP32 products throughout (dd_switch >= 1): the inner solves precondition with
    // S' (CHEB_STEPS_PRE) on both sides, as the single-problem solver's
    const bool pre_inner = o->dd_switch >= 1.0;
    ApplyMany apply_f32 = [&](const double2* xin, double2* yout) -> bem_status {
        BEM_LAUNCH(k_to_c64, blocks_for(T, 256), 256, 0, s, xin, T, x32.as<float2>());
        BEM_TRY(tile_product(PM, TP_F32, 1, x32.p, z.as<double2>(), part.p, tperr.as<int>(), s));
        BEM_LAUNCH(k_transfer_many, blocks_for(T, 64), 64, 0, s, Dd, RI, T, xin, z.as<double2>());
        return mass_many(z.as<double2>(), yout, pre_inner ? CHEB_STEPS_PRE : CHEB_STEPS_INNER);
    };
    // A x with double-float products, before the mass inverse
    auto raw_fp64 = [&](const double2* xin, double2* zout) -> bem_status {
        BEM_LAUNCH(k_split_x, blocks_for(T, 256), 256, 0, s, xin, T, xsplit.as<float4>());
        BEM_TRY(tile_product(PM, TP_DD, 1, xsplit.p, zout, part.p, tperr.as<int>(), s));
        BEM_LAUNCH(k_transfer_many, blocks_for(T, 64), 64, 0, s, Dd, RI, T, xin, zout);
        return BEM_OK;
    };
    ApplyMany apply_fp64 = [&](const double2* xin, double2* yout) -> bem_status {
        BEM_TRY(raw_fp64(xin, z.as<double2>()));
        return mass_many(z.as<double2>(), yout, CHEB_STEPS);
    };
    // ---- right-hand sides
    cudaEventRecord(t_sol.a, s);
    int64_t maxNe = 0;
    for (int i = 0; i < count; ++i) maxNe = std::max<int64_t>(maxNe, inst[i].ext->nv);
    BEM_TRY(fg.alloc((size_t)2 * maxNe * 16, s));
    DevBuf wave;
    BEM_TRY(wave.alloc((size_t)5 * count * 8, s));
    std::vector<double> hw(5 * (size_t)count);
    for (int i = 0; i < count; ++i) {
        hw[2 * i] = inst[i].amp.re;
        hw[2 * i + 1] = inst[i].amp.im;
        for (int dd = 0; dd < 3; ++dd) hw[2 * count + 3 * i + dd] = inst[i].dir[dd];
    }
    BEM_CUDA_TRY(cudaMemcpyAsync(wave.p, hw.data(), hw.size() * 8, cudaMemcpyHostToDevice, s));
    for (int i = 0; i < count; ++i) {
        const bem_grid* ge = inst[i].ext;
        const int64_t Ne = ge->nv;
        BEM_CUDA_TRY(cudaMemsetAsync(fg.p, 0, (size_t)2 * Ne * 16, s));
        double2* f = fg.as<double2>();
        double2* g = f + Ne;
        BEM_LAUNCH(k_plane_wave, dim3(blocks_for(ge->nt, 128), 1), 128, 0, s, ge->rec.as<TriRec>(),
                   ge->tri.as<int32_t>(), ge->nt, inst[i].k_ext.re, inst[i].k_ext.im,
                   wave.as<double>() + 2 * count + 3 * i, wave.as<double2>() + i, Ne, f, g);
        BEM_LAUNCH(k_rhs_pack_one, blocks_for(L.len[i], 256), 256, 0, s, f, g, Ne, L.len[i],
                   bvec.as<double2>() + L.off[i]);
    }
    BEM_TRY(mass_many(bvec.as<double2>(), sb.as<double2>(), CHEB_STEPS));
    const int maxit = (int)std::min<int64_t>(o->gmres_maxiter, T);
    ManyGmres W;
    BEM_TRY(W.init(maxit, L, s));
    std::vector<double> beta(count), tol_abs(count), rn(count), est(count), inner_tol(count);
    std::vector<int> its(count), total(count, 0);
    BEM_TRY(many_norms(L, W, sb.as<double2>(), beta.data(), s));
    for (int r = 0; r < count; ++r) tol_abs[r] = o->gmres_tol * beta[r];
    // ---- iterative refinement, all instances in lockstep
    const double inner_rel =
        o->ir_inner_tol > 0.0 ? o->ir_inner_tol : o->dd_switch >= 1.0 ? IR_INNER_TOL_BATCH : IR_INNER_TOL_SINGLE;
    BEM_CUDA_TRY(cudaMemsetAsync(xsol.p, 0, (size_t)T * 16, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(rvec.p, sb.p, (size_t)T * 16, cudaMemcpyDeviceToDevice, s));
    rn = beta;
    // the inner right-hand side S r, or S' r (pre_inner; r = b at x = 0), and its norms
    std::vector<double> rinn(rn);
    DevBuf rin;
    double2* inner_rhs = rvec.as<double2>();
    if (pre_inner) {
        BEM_TRY(rin.alloc((size_t)T * 16, s));
        BEM_TRY(mass_many(bvec.as<double2>(), rin.as<double2>(), CHEB_STEPS_PRE));
        BEM_TRY(many_norms(L, W, rin.as<double2>(), rinn.data(), s));
        inner_rhs = rin.as<double2>();
    }
    auto pending = [&](int r) {
        return beta[r] > 0.0 && rn[r] > tol_abs[r] && total[r] < o->gmres_maxiter && halted_check(r) == BEM_OK;
    };
    // inner products: double-float while the residual estimate of some running instance
    // is above dd_switch of its inner right-hand side (the estimates trail the launches by
    // a few iterations), FP32 after, as in the single-problem solver
    ApplyMany apply_work = [&](const double2* xin, double2* yout) -> bem_status {
        bool dd = false;
        for (int r = 0; r < count && !dd && !pre_inner; ++r)
            dd = halted[r] == BEM_OK && est[r] > inner_tol[r] && est[r] > o->dd_switch * rn[r];
        return dd ? apply_fp64(xin, yout) : apply_f32(xin, yout);
    };
    int outer = 0;
    for (; outer < 12; ++outer) {
        bool any = false;
        for (int r = 0; r < count; ++r) {
            inner_tol[r] = pending(r) ? inner_tolerance(rinn[r], rn[r], tol_abs[r], inner_rel) : rinn[r];
            any = any || pending(r);
        }
        if (!any) break;
        BEM_TRY(gmres_run_many(L, W, apply_work, inner_rhs, rinn.data(), inner_tol.data(), dvec.as<double2>(),
                               its.data(), est.data(), halted_check, s));
        int moved = 0;
        for (int r = 0; r < count; ++r) {
            total[r] += its[r];
            moved += its[r];
        }
        BEM_LAUNCH(k_acc, blocks_for(T, 256), 256, 0, s, xsol.as<double2>(), dvec.as<double2>(), T);
        if (pre_inner) {
            // r = b - A x (into dvec, free until the next inner solve); S r for the test,
            // S' r for the next inner solve
            BEM_TRY(raw_fp64(xsol.as<double2>(), tmp.as<double2>()));
            BEM_LAUNCH(k_sub, blocks_for(T, 256), 256, 0, s, bvec.as<double2>(), tmp.as<double2>(), T,
                       dvec.as<double2>());
            BEM_TRY(mass_many(dvec.as<double2>(), rvec.as<double2>(), CHEB_STEPS));
            BEM_TRY(mass_many(dvec.as<double2>(), rin.as<double2>(), CHEB_STEPS_PRE));
            BEM_TRY(many_norms(L, W, rvec.as<double2>(), rn.data(), s));
            BEM_TRY(many_norms(L, W, rin.as<double2>(), rinn.data(), s));
        } else {
            BEM_TRY(apply_fp64(xsol.as<double2>(), tmp.as<double2>()));
            BEM_LAUNCH(k_sub, blocks_for(T, 256), 256, 0, s, sb.as<double2>(), tmp.as<double2>(), T,
                       rvec.as<double2>());
            BEM_TRY(many_norms(L, W, rvec.as<double2>(), rn.data(), s));
            rinn = rn;
        }
        if (moved == 0) {
            ++outer;
            break;
        }
    }
    // ---- outputs
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int i = 0; i < count; ++i) {
        const int64_t Ne = inst[i].ext->nv, Ni = inst[i].intr->nv;
        const double2* X = xsol.as<double2>() + L.off[i];
        BEM_CUDA_TRY(cudaMemcpyAsync(inst[i].v_ext, X, Ne * 16, kind, s));
        BEM_CUDA_TRY(cudaMemcpyAsync(inst[i].w_ext, X + Ne, Ne * 16, kind, s));
        BEM_CUDA_TRY(cudaMemcpyAsync(inst[i].v_int, X + 2 * Ne, Ni * 16, kind, s));
        BEM_CUDA_TRY(cudaMemcpyAsync(inst[i].w_int, X + 2 * Ne + Ni, Ni * 16, kind, s));
    }
    cudaEventRecord(t_sol.b, s);
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    BEM_TRY(check_tile_flag(tperr));
    bem_status result = BEM_OK;
    const float ms_asm = t_asm.ms(), ms_mor = t_mor.ms(), ms_sol = t_sol.ms();
    for (int r = 0; r < count; ++r) {
        const double rel = beta[r] > 0.0 ? rn[r] / beta[r] : 0.0;
        const bool conv = beta[r] == 0.0 || rel <= o->gmres_tol;
        if (status_out) status_out[r] = halted[r] != BEM_OK ? halted[r] : conv ? BEM_OK : BEM_E_NOT_CONVERGED;
        if (!conv && halted[r] == BEM_OK) result = BEM_E_NOT_CONVERGED;
        if (reps) {
            reps[r].iterations = total[r];
            reps[r].converged = conv ? 1 : 0;
            reps[r].residual = rel;
            reps[r].t_assembly_ms = ms_asm;
            reps[r].t_mortar_ms = ms_mor;
            reps[r].t_solve_ms = ms_sol;
            reps[r].mtf_variant = o->mtf_variant;
            reps[r].outer_iterations = outer;
        }
    }
    if (result == BEM_E_NOT_CONVERGED)
        set_error("GMRES did not reach the tolerance within gmres_maxiter iterations for some instance");
    return result;
}

// ================================================================ Neumann screen
// Sec. 4.2 (eq. neumannscreen) and the screen of Sec. 5.7: D phi = gamma_N u_inc on an
// open screen, phi in the P1 functions of the screen's interior nodes (padded to all
// nodes with zeros at the boundary).  precond = BEM_SCREEN_MASS: M^-1 D; BEM_SCREEN_OO:
// M^-1 V^_c M^-1 D with V^_c = P_cf^T M_c^-1 V_c M_c^-1 P_cf the single layer of the
// coarse grid c through the mortar (paper: Z_e^-1 Z_i V_i Z_i^-1 Z_e D_e), left-applied
// to both sides.  M is the fine grid's mass matrix restricted to the interior nodes.
bem_status solve_screen_impl(bem_context* ctx, const bem_grid* gf, const bem_grid* gc, bem_c128 k,
                             const bem_incident* inc, const bem_solve_opts* o, int precond, bem_c128* phi,
                             int on_device, bem_solve_report* rep) {
    cudaStream_t s = ctx->stream;
    const bool oo = precond == BEM_SCREEN_OO;
    const bool mixed = o->precision == BEM_PREC_MIXED;
    const int64_t N = gf->nv, Nc = oo ? gc->nv : 0;
    const StopCheck stop = [ctx]() -> bem_status {
        if (ctx->cancel && ctx->cancel->load(std::memory_order_relaxed)) {
            set_error("request cancelled");
            return BEM_E_CANCELLED;
        }
        if (ctx->deadline > 0.0 && now_seconds() > ctx->deadline) {
            set_error("request exceeded its time limit");
            return BEM_E_TIMEOUT;
        }
        return BEM_OK;
    };
    EventTimer t_asm, t_mor, t_sol;
    GraphCache graphs(o->cuda_graphs != 0);
    // ---- boundary nodes (edges of one triangle) on the host
    std::vector<uint8_t> keep(N, 1);
    {
        std::vector<std::pair<int32_t, int32_t>> edges;
        edges.reserve(3 * gf->nt);
        for (int64_t t = 0; t < gf->nt; ++t)
            for (int a = 0; a < 3; ++a) {
                int32_t p = gf->h_tri[3 * t + a], q = gf->h_tri[3 * t + (a + 1) % 3];
                edges.emplace_back(std::min(p, q), std::max(p, q));
            }
        std::sort(edges.begin(), edges.end());
        for (size_t i = 0; i < edges.size();) {
            size_t j = i;
            while (j < edges.size() && edges[j] == edges[i]) ++j;
            if (j - i == 1) keep[edges[i].first] = keep[edges[i].second] = 0;
            i = j;
        }
    }
    DevBuf dkeep;
    BEM_TRY(dkeep.alloc((size_t)N, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(dkeep.p, keep.data(), (size_t)N, cudaMemcpyHostToDevice, s));
    const uint8_t* K8 = dkeep.as<uint8_t>();
    // ---- operators: D on the screen, V on the coarse grid (tiled storage)
    const size_t esz = mixed ? 8 : 16;
    const bool same = oo && gc == gf;  // conforming: V of the screen itself, from the same assembly pass
    GridOps opF, opC;
    cudaEventRecord(t_asm.a, s);
    BEM_TRY(opF.assemble(gf, k, mixed, o->n_singular, s, same, false, true));
    if (oo && !same) BEM_TRY(opC.assemble(gc, k, mixed, o->n_singular, s, true, false, false));
    cudaEventRecord(t_asm.b, s);
    const GridOps& opV = same ? opF : opC;
    // ---- mass matrices (the screen's restricted to its interior nodes) and mortar
    cudaEventRecord(t_mor.a, s);
    DevBuf mvf, dvf, mvc, dvc, prow, pcol, pval;
    BEM_TRY(mvf.alloc(gf->m_nnz * 8, s));
    BEM_TRY(dvf.alloc(N * 8, s));
    BEM_TRY(mass_values(gf, mvf.as<double>(), s));
    BEM_TRY(mass_inverse_diag(gf, mvf.as<double>(), dvf.as<double>(), s));
    MassEll ell_f, ell_c;
    BEM_TRY(ell_f.build(gf, mvf.as<double>(), s));
    BEM_LAUNCH(k_mask_mass_ell, blocks_for(N, 128), 128, 0, s, ell_f.ci.as<int32_t>(), ell_f.v.as<double>(),
               dvf.as<double>(), ell_f.W, N, K8);
    CsrBuf csr_cf, csr_fc;  // P_cf (rows: coarse nodes) and P_fc
    if (oo) {
        BEM_TRY(mvc.alloc(gc->m_nnz * 8, s));
        BEM_TRY(dvc.alloc(Nc * 8, s));
        BEM_TRY(mass_values(gc, mvc.as<double>(), s));
        BEM_TRY(mass_inverse_diag(gc, mvc.as<double>(), dvc.as<double>(), s));
        BEM_TRY(ell_c.build(gc, mvc.as<double>(), s));
        // central projection from a point off the screen's plane (identity on coplanar grids)
        double cen[3] = {0.0, 0.0, 0.0}, nrm[3] = {0.0, 0.0, 0.0};
        for (int64_t i = 0; i < N; ++i)
            for (int d = 0; d < 3; ++d) cen[d] += gf->h_xyz[3 * i + d] / (double)N;
        {
            const int32_t* t = gf->h_tri.data();
            const double* x = gf->h_xyz.data();
            double e1[3], e2[3];
            for (int d = 0; d < 3; ++d) {
                e1[d] = x[3 * t[1] + d] - x[3 * t[0] + d];
                e2[d] = x[3 * t[2] + d] - x[3 * t[0] + d];
            }
            nrm[0] = e1[1] * e2[2] - e1[2] * e2[1];
            nrm[1] = e1[2] * e2[0] - e1[0] * e2[2];
            nrm[2] = e1[0] * e2[1] - e1[1] * e2[0];
            const double l = std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
            for (int d = 0; d < 3; ++d) cen[d] += nrm[d] / l;
        }
        int64_t pnnz = 0;
        BEM_TRY(mortar_coo(gc, gf, cen, prow, pcol, pval, &pnnz, s));
        BEM_TRY(build_csr(prow.as<int32_t>(), pcol.as<int32_t>(), pval.as<double>(), pnnz, Nc, csr_cf, s));
        BEM_TRY(build_csr(pcol.as<int32_t>(), prow.as<int32_t>(), pval.as<double>(), pnnz, N, csr_fc, s));
    }
    cudaEventRecord(t_mor.b, s);
    // ---- workspaces
    const int RB = std::min<int>(o->batch_columns > 0 ? std::min(o->batch_columns, 8) : 8, inc->n_rhs);
    const int RW = RB + 7;
    const size_t colf = (size_t)N * 16, colc = (size_t)std::max<int64_t>(Nc, 1) * 16;
    DevBuf z, w, u, wr, wa, wb, x32, xsplit, c1, c2, c3, x32c, wrc, wac, wbc;
    BEM_TRY(z.alloc(RW * colf, s));
    for (DevBuf* b : {&w, &u, &wr, &wa, &wb}) BEM_TRY(b->alloc(RB * colf, s));
    if (mixed) {
        BEM_TRY(x32.alloc((size_t)RW * N * 8, s));
        BEM_CUDA_TRY(cudaMemsetAsync(x32.p, 0, x32.bytes, s));
    }
    const bool dd_single = mixed && RB == 1;
    double inner_progress = 1.0;
    auto dd_now = [&]() { return dd_single && inner_progress > o->dd_switch; };
    DevBuf part, tperr;
    BEM_TRY(xsplit.alloc((size_t)8 * std::max(N, Nc) * 16, s));
    // one-matrix products: D phi on the screen (y2 = D x) and V c on the coarse grid (y1 = V x)
    TileProd PD, PV;
    opF.add(PD, 0.0, 0.0, 1.0, 0.0, 0, 0, 0, 0, -1, 0);
    BEM_TRY(tile_prod_finish(PD, N, (int)esz, s));
    size_t pbytes = tile_part_bytes(PD, TP_DD, std::min(RB, 8));
    if (oo) {
        opV.add(PV, 0.0, 1.0, 0.0, 0.0, 0, 0, 0, 0, 0, -1);
        BEM_TRY(tile_prod_finish(PV, Nc, (int)esz, s));
        pbytes = std::max(pbytes, tile_part_bytes(PV, TP_DD, std::min(RB, 8)));
    }
    BEM_TRY(part.alloc(pbytes, s));
    BEM_TRY(tperr.alloc(sizeof(int), s));
    BEM_CUDA_TRY(cudaMemsetAsync(tperr.p, 0, sizeof(int), s));
    MassOp mf;
    mf.M.ci[0] = ell_f.ci.as<int32_t>(); mf.M.v[0] = ell_f.v.as<double>(); mf.M.W[0] = ell_f.W;
    mf.M.dinv[0] = dvf.as<double>();
    mf.M.ci[1] = mf.M.ci[0]; mf.M.v[1] = mf.M.v[0]; mf.M.W[1] = mf.M.W[0]; mf.M.dinv[1] = mf.M.dinv[0];
    mf.M.Ne = N; mf.M.Ni = 0; mf.M.n = N;  // one vector of the screen per column
    mf.r = wr.as<double2>(); mf.dA = wa.as<double2>(); mf.dB = wb.as<double2>();
    mf.graphs = &graphs;
    ChebSync csync;
    BEM_TRY(csync.init(s));
    if (ctx->exclusive) csync.attach(mf);
    MassOp mc;
    if (oo) {
        for (DevBuf* b : {&c1, &wrc, &wac, &wbc}) BEM_TRY(b->alloc(RB * colc, s));
        for (DevBuf* b : {&c2, &c3}) BEM_TRY(b->alloc(RW * colc, s));
        BEM_CUDA_TRY(cudaMemsetAsync(c2.p, 0, c2.bytes, s));
        if (mixed) {
            BEM_TRY(x32c.alloc((size_t)RW * Nc * 8, s));
            BEM_CUDA_TRY(cudaMemsetAsync(x32c.p, 0, x32c.bytes, s));
        }
        mc.M.ci[0] = ell_c.ci.as<int32_t>(); mc.M.v[0] = ell_c.v.as<double>(); mc.M.W[0] = ell_c.W;
        mc.M.dinv[0] = dvc.as<double>();
        mc.M.ci[1] = mc.M.ci[0]; mc.M.v[1] = mc.M.v[0]; mc.M.W[1] = mc.M.W[0]; mc.M.dinv[1] = mc.M.dinv[0];
        mc.M.Ne = Nc; mc.M.Ni = 0; mc.M.n = Nc;
        mc.r = wrc.as<double2>(); mc.dA = wac.as<double2>(); mc.dB = wbc.as<double2>();
        mc.graphs = &graphs;
        if (ctx->exclusive) csync.attach(mc);
    }
    // zo = one-matrix product P on nn rows: FP32 (mixed), double-float (FP64 mode, FP64
    // residuals of the refinement, single-column products above the dd_switch)
    auto product = [&](bool fp64, const TileProd& P, int64_t nn, float2* xw, const double2* xin, double2* zo,
                       int R) -> bem_status {
        const bool dd = !mixed || fp64 || (R == 1 && dd_now());
        if (!dd) BEM_LAUNCH(k_to_c64, blocks_for((int64_t)R * nn, 256), 256, 0, s, xin, (int64_t)R * nn, xw);
        for (int c0 = 0; c0 < R; c0 += 8) {
            const int w = std::min(8, R - c0);
            double2* zc = zo + (int64_t)c0 * nn;
            if (dd) {
                BEM_LAUNCH(k_split_x, blocks_for((int64_t)w * nn, 256), 256, 0, s, xin + (int64_t)c0 * nn,
                           (int64_t)w * nn, xsplit.as<float4>());
                BEM_TRY(tile_product(P, TP_DD, w, xsplit.p, zc, part.p, tperr.as<int>(), s));
            } else {
                BEM_TRY(tile_product(P, TP_F32, w, xw + (int64_t)c0 * nn, zc, part.p, tperr.as<int>(), s));
            }
        }
        return BEM_OK;
    };
    // y = M^-1 V^_c M^-1 v (OO) or M^-1 v, for v on the screen (boundary entries ignored)
    auto precondition = [&](bool fp64, const double2* v, double2* y, int R, int steps) -> bem_status {
        BEM_LAUNCH(k_mask_rows, dim3(blocks_for(N, 256), R), 256, 0, s, const_cast<double2*>(v), K8, N);
        if (!oo) return mass_solve(mf, v, y, R, s, steps);
        BEM_TRY(mass_solve(mf, v, u.as<double2>(), R, s, steps));
        BEM_LAUNCH(k_csr_apply, dim3(blocks_for(Nc, 128), R), 128, 0, s, csr_cf.rp.as<int32_t>(),
                   csr_cf.ci.as<int32_t>(), csr_cf.v.as<double>(), Nc, u.as<double2>(), N, c1.as<double2>(), Nc, 1.0);
        BEM_TRY(mass_solve(mc, c1.as<double2>(), c2.as<double2>(), R, s, steps));
        BEM_TRY(product(fp64, PV, Nc, x32c.as<float2>(), c2.as<double2>(), c3.as<double2>(), R));
        BEM_TRY(mass_solve(mc, c3.as<double2>(), c1.as<double2>(), R, s, steps));
        BEM_LAUNCH(k_csr_apply, dim3(blocks_for(N, 128), R), 128, 0, s, csr_fc.rp.as<int32_t>(),
                   csr_fc.ci.as<int32_t>(), csr_fc.v.as<double>(), N, c1.as<double2>(), Nc, u.as<double2>(), N, 1.0);
        BEM_LAUNCH(k_mask_rows, dim3(blocks_for(N, 256), R), 256, 0, s, u.as<double2>(), K8, N);
        return mass_solve(mf, u.as<double2>(), y, R, s, steps);
    };
    auto apply_on = [&](bool fp64, const double2* xin, double2* yout, int R, int steps) -> bem_status {
        BEM_TRY(product(fp64, PD, N, x32.as<float2>(), xin, z.as<double2>(), R));
        return precondition(fp64, z.as<double2>(), yout, R, steps);
    };
    Apply apply_work = [&](const double2* xin, double2* yout, int R) -> bem_status {
        const int steps = !mixed ? CHEB_STEPS : (R == 1 && dd_now()) ? CHEB_STEPS_DD : CHEB_STEPS_INNER;
        return apply_on(false, xin, yout, R, steps);
    };
    Apply apply_fp64 = [&](const double2* xin, double2* yout, int R) -> bem_status {
        return apply_on(true, xin, yout, R, CHEB_STEPS);
    };
    // ---- right-hand sides and GMRES (with refinement in the mixed mode)
    const int maxit = (int)std::min<int64_t>(o->gmres_maxiter, N);
    GmresWork W;
    BEM_TRY(W.init(maxit, N, RB, RW - RB, s));
    DevBuf fvec, gvec, sb, xsol, dvec, rvec, tmp, wave;
    BEM_TRY(wave.alloc((size_t)5 * RB * 8, s));
    BEM_TRY(fvec.alloc(RB * colf, s));
    BEM_TRY(gvec.alloc(RB * colf, s));
    BEM_TRY(sb.alloc(RB * colf, s));
    BEM_TRY(xsol.alloc(RW * colf, s));
    BEM_CUDA_TRY(cudaMemsetAsync(xsol.p, 0, RW * colf, s));
    for (DevBuf* b : {&dvec, &rvec, &tmp}) BEM_TRY(b->alloc(RB * colf, s));
    bem_status result = BEM_OK;
    int total_inner = 0, outer_used = 0;
    double worst_res = 0.0;
    bool all_conv = true;
    cudaEventRecord(t_sol.a, s);
    for (int r0 = 0; r0 < inc->n_rhs; r0 += RB) {
        const int R = std::min(RB, inc->n_rhs - r0);
        BEM_TRY(incident_data(inc, r0, R, RB, gf, k, W.h_wave, wave, fvec.as<double2>(), gvec.as<double2>(),
                              on_device != 0, s));
        // g_i = <gamma_N u_inc, theta_i>: the preconditioned right-hand side
        BEM_TRY(precondition(true, gvec.as<double2>(), sb.as<double2>(), R, CHEB_STEPS));
        std::vector<double> beta(R), tol_abs(R), rn(R), est(R), inner_tol(R);
        std::vector<int> its(R), total(R, 0);
        BEM_TRY(norms(W, sb.as<double2>(), R, beta.data(), s));
        for (int r = 0; r < R; ++r) tol_abs[r] = o->gmres_tol * beta[r];
        if (!mixed) {
            BEM_TRY(gmres_run(W, R, apply_work, sb.as<double2>(), beta.data(), tol_abs.data(), xsol.as<double2>(),
                              its.data(), est.data(), s, stop));
            for (int r = 0; r < R; ++r) {
                rn[r] = est[r];
                total[r] = its[r];
            }
            outer_used = 1;
        } else {
            BEM_CUDA_TRY(cudaMemsetAsync(xsol.p, 0, (size_t)R * colf, s));
            BEM_CUDA_TRY(cudaMemcpyAsync(rvec.p, sb.p, (size_t)R * colf, cudaMemcpyDeviceToDevice, s));
            rn = beta;
            int outer = 0;
            auto pending = [&](int r) {
                return beta[r] > 0.0 && rn[r] > tol_abs[r] && total[r] < o->gmres_maxiter;
            };
            auto any_pending = [&] {
                for (int r = 0; r < R; ++r)
                    if (pending(r)) return true;
                return false;
            };
            const double inner_rel =
                o->ir_inner_tol > 0.0                          ? o->ir_inner_tol
                : (!dd_single || o->dd_switch >= 1.0) ? IR_INNER_TOL_BATCH
                                                      : IR_INNER_TOL_SINGLE;
            while (any_pending() && outer < 12) {
                for (int r = 0; r < R; ++r)
                    inner_tol[r] = pending(r) ? inner_tolerance(rn[r], rn[r], tol_abs[r], inner_rel) : rn[r];
                BEM_TRY(gmres_run(W, R, apply_work, rvec.as<double2>(), rn.data(), inner_tol.data(), dvec.as<double2>(),
                                  its.data(), est.data(), s, stop, &inner_progress));
                int moved = 0;
                for (int r = 0; r < R; ++r) {
                    total[r] += its[r];
                    moved += its[r];
                }
                BEM_LAUNCH(k_acc, blocks_for((int64_t)R * N, 256), 256, 0, s, xsol.as<double2>(), dvec.as<double2>(),
                           (int64_t)R * N);
                BEM_TRY(apply_fp64(xsol.as<double2>(), tmp.as<double2>(), R));
                BEM_LAUNCH(k_sub, blocks_for((int64_t)R * N, 256), 256, 0, s, sb.as<double2>(), tmp.as<double2>(),
                           (int64_t)R * N, rvec.as<double2>());
                BEM_TRY(norms(W, rvec.as<double2>(), R, rn.data(), s));
                ++outer;
                if (moved == 0) break;
            }
            outer_used = std::max(outer_used, outer);
        }
        for (int r = 0; r < R; ++r) {
            const double rel = beta[r] > 0.0 ? rn[r] / beta[r] : 0.0;
            const bool conv = beta[r] == 0.0 || rel <= o->gmres_tol;
            all_conv = all_conv && conv;
            worst_res = std::max(worst_res, rel);
            total_inner += total[r];
            if (!conv) result = BEM_E_NOT_CONVERGED;
        }
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        BEM_CUDA_TRY(cudaMemcpyAsync(phi + (int64_t)r0 * N, xsol.p, (size_t)R * colf, kind, s));
        BEM_CUDA_TRY(cudaStreamSynchronize(s));
    }
    cudaEventRecord(t_sol.b, s);
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    BEM_TRY(check_tile_flag(tperr));
    BEM_TRY(csync.check());
    if (result == BEM_E_NOT_CONVERGED)
        set_error("GMRES did not reach the tolerance within gmres_maxiter iterations; outputs hold the last iterate");
    if (rep) {
        rep->iterations = total_inner;
        rep->converged = all_conv ? 1 : 0;
        rep->residual = worst_res;
        rep->t_assembly_ms = t_asm.ms();
        rep->t_mortar_ms = t_mor.ms();
        rep->t_solve_ms = t_sol.ms();
        rep->mtf_variant = 0;
        rep->outer_iterations = outer_used;
    }
    return result;
}

}  // namespace bem
