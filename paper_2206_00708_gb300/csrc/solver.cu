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

#include <algorithm>
#include <cmath>
#include <functional>

namespace bem {

namespace {

constexpr int CHEB_STEPS = 34;        // error <= 2 * 3^-34 ~ 1e-16: FP64 applications
constexpr int CHEB_STEPS_INNER = 17;  // error <= 2 * 3^-17 ~ 1.6e-8: inner solves of the refinement
constexpr double CHEB_ALPHA = 0.5, CHEB_BETA = 2.0;
constexpr int RMAX = 8;               // right-hand sides per batch

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {  // a*b + c
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

__device__ __forceinline__ double2 warp_sum2(double2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------- right-hand sides
// f_j = <u_inc, theta_j>, g_j = <du_inc/dn, theta_j> on the exterior grid,
// u_inc = amp exp(i k x.d), du_inc/dn = i k (d.n) u_inc (paper eq. planewave);
// blockIdx.y = right-hand side.
struct Waves {
    double3 d[RMAX];
    double2 amp[RMAX];
};

__device__ __forceinline__ double3 sel_dir(const Waves& W, int r) {
    double3 d = W.d[0];
#pragma unroll
    for (int k = 1; k < RMAX; ++k)
        if (r == k) d = W.d[k];
    return d;
}
__device__ __forceinline__ double2 sel_amp(const Waves& W, int r) {
    double2 a = W.amp[0];
#pragma unroll
    for (int k = 1; k < RMAX; ++k)
        if (r == k) a = W.amp[k];
    return a;
}

__global__ void k_plane_wave(const TriRec* __restrict__ rec, const int32_t* __restrict__ tri, int64_t nt,
                             double kr, double ki, Waves W, int64_t Ne, double2* __restrict__ f,
                             double2* __restrict__ g) {
    const int r = blockIdx.y;
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const double3 d = sel_dir(W, r);
    const double2 amp = sel_amp(W, r);
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

// the block row of global row gw and its parameters
template <class MT>
struct RowBlock {
    const MT *a1, *a2;
    double c1, c2;
    int64_t N, i, x1, x2;
};

template <class MT>
__device__ __forceinline__ RowBlock<MT> row_block(const Blocks<MT>& B, int64_t gw) {
    int b = 0;
    while (b < 3 && gw >= B.base[b + 1]) ++b;
    RowBlock<MT> rb;
    rb.a1 = B.A1[b];
    rb.a2 = B.A2[b];
    rb.c1 = B.c1[b];
    rb.c2 = B.c2[b];
    rb.N = B.rows[b];
    rb.i = gw - B.base[b];
    rb.x1 = B.x1[b];
    rb.x2 = B.x2[b];
    return rb;
}

// complex128 blocks, FP64 arithmetic: one warp per row, R right-hand sides
template <int R>
__global__ void __launch_bounds__(256) k_gemm64(Blocks<double2> B, int64_t n, const double2* __restrict__ x,
                                                double2* __restrict__ z) {
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= n) return;
    const RowBlock<double2> rb = row_block(B, gw);
    const double2* __restrict__ a1 = rb.a1 + rb.i * rb.N;
    const double2* __restrict__ a2 = rb.a2 + rb.i * rb.N;
    double2 s1[R], s2[R];
#pragma unroll
    for (int r = 0; r < R; ++r) s1[r] = s2[r] = make_double2(0, 0);
    for (int64_t j = lane; j < rb.N; j += 32) {
        const double2 p = a1[j], q = a2[j];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            s1[r] = cfma(p, x[r * n + rb.x1 + j], s1[r]);
            s2[r] = cfma(q, x[r * n + rb.x2 + j], s2[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const double2 u = warp_sum2(s1[r]), v = warp_sum2(s2[r]);
        if (lane == 0) z[r * n + gw] = make_double2(rb.c1 * u.x + rb.c2 * v.x, rb.c1 * u.y + rb.c2 * v.y);
    }
}

// complex64 blocks, FP64 arithmetic (outer residual of the refinement)
template <int R>
__global__ void __launch_bounds__(256) k_gemm_c64_f64(Blocks<float2> B, int64_t n, const double2* __restrict__ x,
                                                      double2* __restrict__ z) {
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= n) return;
    const RowBlock<float2> rb = row_block(B, gw);
    const float2* __restrict__ a1 = rb.a1 + rb.i * rb.N;
    const float2* __restrict__ a2 = rb.a2 + rb.i * rb.N;
    double2 s1[R], s2[R];
#pragma unroll
    for (int r = 0; r < R; ++r) s1[r] = s2[r] = make_double2(0, 0);
    for (int64_t j = lane; j < rb.N; j += 32) {
        const float2 pf = a1[j], qf = a2[j];
        const double2 p = make_double2(pf.x, pf.y), q = make_double2(qf.x, qf.y);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            s1[r] = cfma(p, x[r * n + rb.x1 + j], s1[r]);
            s2[r] = cfma(q, x[r * n + rb.x2 + j], s2[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const double2 u = warp_sum2(s1[r]), v = warp_sum2(s2[r]);
        if (lane == 0) z[r * n + gw] = make_double2(rb.c1 * u.x + rb.c2 * v.x, rb.c1 * u.y + rb.c2 * v.y);
    }
}

// complex64 blocks, FP32 arithmetic: one warp per row, 16-byte loads (two complex
// entries per lane) shared by the R right-hand sides; products are summed plainly in
// groups of four and added to the lane's accumulator with a compensated (two-sum)
// update; warp totals are formed in FP64.
template <int R>
__global__ void __launch_bounds__(256) k_gemm32(Blocks<float2> B, int64_t n, const float2* __restrict__ x,
                                                double2* __restrict__ z) {
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= n) return;
    // block-row parameters are read where they are used (not held across the loop:
    // the single-column kernel is bandwidth-bound and wants few registers)
    int b = 0;
    while (b < 3 && gw >= B.base[b + 1]) ++b;
    const int64_t N = B.rows[b];
    const int64_t i = gw - B.base[b];
    double2 out[R];
#pragma unroll
    for (int r = 0; r < R; ++r) out[r] = make_double2(0, 0);
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const float2* __restrict__ a = (m == 0 ? B.A1[b] : B.A2[b]) + i * N;
        const int64_t xo = m == 0 ? B.x1[b] : B.x2[b];
        float sr[R], si[R], er[R], ei[R];
#pragma unroll
        for (int r = 0; r < R; ++r) sr[r] = si[r] = er[r] = ei[r] = 0.f;
        // row start may be only 8-byte aligned: peel to a 16-byte boundary
        const int64_t j0 = ((reinterpret_cast<uintptr_t>(a) & 15) != 0) ? 1 : 0;
        if (j0 && lane == 0 && N > 0) {
            const float2 av = a[0];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float2 xx = x[r * n + xo];
                sr[r] = fmaf(av.x, xx.x, -av.y * xx.y);
                si[r] = fmaf(av.x, xx.y, av.y * xx.x);
            }
        }
        const int64_t npair = (N - j0) / 2;
        const float4* __restrict__ a4 = reinterpret_cast<const float4*>(a + j0);
        for (int64_t p = lane; p < npair; p += 64) {
            // two 16-byte loads in flight per lane; four products summed plainly per
            // right-hand side before the compensated update
            float cr[R], ci[R];
#pragma unroll
            for (int r = 0; r < R; ++r) cr[r] = ci[r] = 0.f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t pp = p + 32 * h;
                if (pp < npair) {
                    const float4 av = a4[pp];
                    const int64_t j = j0 + 2 * pp;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const float2 x0 = x[r * n + xo + j], x1 = x[r * n + xo + j + 1];
                        cr[r] = fmaf(av.x, x0.x, cr[r]);
                        cr[r] = fmaf(-av.y, x0.y, cr[r]);
                        ci[r] = fmaf(av.x, x0.y, ci[r]);
                        ci[r] = fmaf(av.y, x0.x, ci[r]);
                        cr[r] = fmaf(av.z, x1.x, cr[r]);
                        cr[r] = fmaf(-av.w, x1.y, cr[r]);
                        ci[r] = fmaf(av.z, x1.y, ci[r]);
                        ci[r] = fmaf(av.w, x1.x, ci[r]);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float t, e;
                two_sum_f(sr[r], cr[r], t, e);
                sr[r] = t;
                er[r] += e;
                two_sum_f(si[r], ci[r], t, e);
                si[r] = t;
                ei[r] += e;
            }
        }
        if (((N - j0) & 1) && lane == 1) {  // odd tail
            const float2 av = a[N - 1];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float2 xx = x[r * n + xo + N - 1];
                float t, e;
                two_sum_f(sr[r], fmaf(av.x, xx.x, -av.y * xx.y), t, e);
                sr[r] = t;
                er[r] += e;
                two_sum_f(si[r], fmaf(av.x, xx.y, av.y * xx.x), t, e);
                si[r] = t;
                ei[r] += e;
            }
        }
        const double c = m == 0 ? B.c1[b] : B.c2[b];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const double2 v = warp_sum2(make_double2((double)sr[r] + (double)er[r], (double)si[r] + (double)ei[r]));
            out[r].x += c * v.x;
            out[r].y += c * v.y;
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int r = 0; r < R; ++r) z[r * n + gw] = out[r];
    }
}

__global__ void k_to_c64(const double2* __restrict__ x, int64_t n, float2* __restrict__ y) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) y[e] = make_float2((float)x[e].x, (float)x[e].y);
}

// mortar part: entries (r, c, p) of P_ie; z1[c] += a p v_i[r], z2[c] += b p w_i[r],
// z3[r] += c p v_e[c], z4[r] += d p w_e[c]; blockIdx.y = right-hand side
__global__ void k_transfer(const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                           const double* __restrict__ val, int64_t nnz, int64_t Ne, int64_t Ni, int64_t n,
                           double4 coef, const double2* __restrict__ xb, double2* __restrict__ zb) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const double p = val[e];
    if (p == 0.0) return;
    const double2* x = xb + blockIdx.y * n;
    double2* z = zb + blockIdx.y * n;
    const int64_t r = row[e], c = col[e];
    const double2 vi = x[2 * Ne + r], wi = x[2 * Ne + Ni + r], ve = x[c], we = x[Ne + c];
    atomicAdd(&z[c].x, coef.x * p * vi.x);
    atomicAdd(&z[c].y, coef.x * p * vi.y);
    atomicAdd(&z[Ne + c].x, coef.y * p * wi.x);
    atomicAdd(&z[Ne + c].y, coef.y * p * wi.y);
    atomicAdd(&z[2 * Ne + r].x, coef.z * p * ve.x);
    atomicAdd(&z[2 * Ne + r].y, coef.z * p * ve.y);
    atomicAdd(&z[2 * Ne + Ni + r].x, coef.w * p * we.x);
    atomicAdd(&z[2 * Ne + Ni + r].y, coef.w * p * we.y);
}

// ---------------------------------------------------------------- mass inverse
struct MassPair {
    const int32_t *rp[2], *ci[2];
    const double *v[2], *dinv[2];
    int64_t Ne, Ni, n;
};

struct MassRow {
    const int32_t *rp, *ci;
    const double *v, *dinv;
    int64_t i, base;
};

__device__ __forceinline__ MassRow mass_row(const MassPair& M, int64_t g) {
    MassRow m;
    const bool ext = g < 2 * M.Ne;
    m.rp = ext ? M.rp[0] : M.rp[1];
    m.ci = ext ? M.ci[0] : M.ci[1];
    m.v = ext ? M.v[0] : M.v[1];
    m.dinv = ext ? M.dinv[0] : M.dinv[1];
    if (g < M.Ne) { m.i = g; m.base = 0; }
    else if (g < 2 * M.Ne) { m.i = g - M.Ne; m.base = M.Ne; }
    else if (g < 2 * M.Ne + M.Ni) { m.i = g - 2 * M.Ne; m.base = 2 * M.Ne; }
    else { m.i = g - 2 * M.Ne - M.Ni; m.base = 2 * M.Ne + M.Ni; }
    return m;
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

// y += d_k; r -= M d_k; d_{k+1} = c1 d_k + c2 D^-1 r
__global__ void k_cheb_step(MassPair M, const double2* __restrict__ dk, double2* __restrict__ dn,
                            double2* __restrict__ y, double2* __restrict__ r, double c1, double c2) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= M.n) return;
    const int64_t off = blockIdx.y * M.n;
    const MassRow m = mass_row(M, g);
    double2 md = make_double2(0, 0);
    for (int32_t e = m.rp[m.i]; e < m.rp[m.i + 1]; ++e) {
        const double v = m.v[e];
        const double2 dd = dk[off + m.base + m.ci[e]];
        md.x += v * dd.x;
        md.y += v * dd.y;
    }
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

// ---------------------------------------------------------------- GMRES kernels
// Krylov basis: vector i of right-hand side r at V + (i * R + r) * n.
// Hessenberg of r: column-major, H + r * ldh * ldh, column j at + j * ldh.
constexpr int RED_BLOCKS = 64;

// partial[((r * m) + i) * RED_BLOCKS + bx] = chunk of conj(V_{i,r}) w_r
__global__ void k_dots_partial(const double2* __restrict__ Vb, int64_t n, int R, int m,
                               const double2* __restrict__ w, double2* __restrict__ partial) {
    const int i = blockIdx.y, r = blockIdx.z;
    const double2* __restrict__ v = Vb + ((int64_t)i * R + r) * n;
    const double2* __restrict__ wr = w + (int64_t)r * n;
    double2 s = make_double2(0, 0);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = v[e], b = wr[e];
        s.x += a.x * b.x + a.y * b.y;
        s.y += a.x * b.y - a.y * b.x;
    }
    __shared__ double2 sh[8];
    s = warp_sum2(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double2 t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : make_double2(0, 0);
        t = warp_sum2(t);
        if (threadIdx.x == 0) partial[((int64_t)r * m + i) * RED_BLOCKS + blockIdx.x] = t;
    }
}

// out[r * ostride + i] = sum_b partial[r][i][b]  (+= when accumulate)
__global__ void k_dots_final(const double2* __restrict__ partial, int m, double2* __restrict__ out,
                             int64_t ostride, int accumulate) {
    const int i = blockIdx.x, r = blockIdx.y;
    double2 s = make_double2(0, 0);
    for (int b = threadIdx.x; b < RED_BLOCKS; b += 32) {
        const double2 p = partial[((int64_t)r * m + i) * RED_BLOCKS + b];
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

// w_r -= sum_{i<m} h_r[i] V_{i,r}   or (overwrite) x_r = sum_{i<m_r} y_r[i] V_{i,r}
__global__ void k_combine(const double2* __restrict__ Vb, int64_t n, int R, int m, const int* __restrict__ mr,
                          const double2* __restrict__ h, int64_t hstride, double2* __restrict__ w, int overwrite) {
    const int r = blockIdx.y;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int mm = mr ? mr[r] : m;
    double2 s = make_double2(0, 0);
    for (int i = 0; i < mm; ++i) s = cfma(h[r * hstride + i], Vb[((int64_t)i * R + r) * n + e], s);
    double2* wr = w + (int64_t)r * n;
    if (overwrite) wr[e] = s;
    else {
        const double2 t = wr[e];
        wr[e] = make_double2(t.x - s.x, t.y - s.y);
    }
}

__global__ void k_add_cols(double2* __restrict__ a, int64_t astride, const double2* __restrict__ b,
                           int64_t bstride, int m) {
    const int r = blockIdx.y;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        a[r * astride + i].x += b[r * bstride + i].x;
        a[r * astride + i].y += b[r * bstride + i].y;
    }
}

// v_r = w_r / |w_r| (|w_r|^2 = real part of nrm2[r]); writes |w_r| to dst[r * dstride]
__global__ void k_normalize(const double2* __restrict__ w, int64_t n, const double2* __restrict__ nrm2,
                            double2* __restrict__ v, int64_t vstride, double2* __restrict__ dst, int64_t dstride) {
    const int r = blockIdx.y;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const double nr = sqrt(fmax(nrm2[r].x, 0.0));
    if (e == 0 && dst) dst[r * dstride] = make_double2(nr, 0.0);
    if (e >= n) return;
    const double inv = nr > 0.0 ? 1.0 / nr : 0.0;
    v[r * vstride + e] = make_double2(w[(int64_t)r * n + e].x * inv, w[(int64_t)r * n + e].y * inv);
}

// Givens update of column j of every Hessenberg (one thread per right-hand side)
__global__ void k_givens(double2* __restrict__ Hb, int64_t ldh, int j, double* __restrict__ csb,
                         double2* __restrict__ snb, double2* __restrict__ gb, int64_t gstride,
                         double* __restrict__ res, int R) {
    const int r = threadIdx.x;
    if (r >= R) return;
    double2* h = Hb + (int64_t)r * ldh * ldh + (int64_t)j * ldh;
    double* cs = csb + r * gstride;
    double2* sn = snb + r * gstride;
    double2* g = gb + r * gstride;
    for (int i = 0; i < j; ++i) {
        const double2 a = h[i], b = h[i + 1];
        const double2 t = make_double2(cs[i] * a.x + (sn[i].x * b.x - sn[i].y * b.y),
                                       cs[i] * a.y + (sn[i].x * b.y + sn[i].y * b.x));
        // h[i+1] = -conj(sn) a + cs b
        const double2 u = make_double2(-(sn[i].x * a.x + sn[i].y * a.y) + cs[i] * b.x,
                                       -(sn[i].x * a.y - sn[i].y * a.x) + cs[i] * b.y);
        h[i] = t;
        h[i + 1] = u;
    }
    const double2 a = h[j], b = h[j + 1];
    const double aa = hypot(a.x, a.y), bb = hypot(b.x, b.y);
    double c;
    double2 s, rr;
    if (aa == 0.0) {
        c = 0.0;
        s = make_double2(1.0, 0.0);
        rr = b;
    } else {
        const double t = hypot(aa, bb);
        c = aa / t;
        const double2 ph = make_double2(a.x / aa, a.y / aa);
        s = make_double2((ph.x * b.x + ph.y * b.y) / t, (ph.y * b.x - ph.x * b.y) / t);  // ph conj(b) / t
        rr = make_double2(ph.x * t, ph.y * t);
    }
    cs[j] = c;
    sn[j] = s;
    h[j] = rr;
    h[j + 1] = make_double2(0.0, 0.0);
    const double2 gj = g[j];
    g[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));  // -conj(s) g_j
    g[j] = make_double2(c * gj.x, c * gj.y);
    res[r] = hypot(g[j + 1].x, g[j + 1].y);
}

// y_r = H_r(0:m_r,0:m_r)^-1 g_r(0:m_r), column-oriented back substitution, one block per r
__global__ void k_backsolve(const double2* __restrict__ Hb, int64_t ldh, const int* __restrict__ mr,
                            const double2* __restrict__ gb, int64_t gstride, double2* __restrict__ yb,
                            double2* __restrict__ workb) {
    const int r = blockIdx.x;
    const int m = mr[r];
    const double2* H = Hb + (int64_t)r * ldh * ldh;
    const double2* g = gb + r * gstride;
    double2* y = yb + r * gstride;
    double2* work = workb + r * gstride;
    for (int i = threadIdx.x; i < m; i += blockDim.x) work[i] = g[i];
    __syncthreads();
    __shared__ double2 yc;
    for (int c = m - 1; c >= 0; --c) {
        if (threadIdx.x == 0) {
            const double2 d = H[(int64_t)c * ldh + c];
            const double den = d.x * d.x + d.y * d.y;
            const double2 wc = work[c];
            yc = den > 0.0 ? make_double2((wc.x * d.x + wc.y * d.y) / den, (wc.y * d.x - wc.x * d.y) / den)
                           : make_double2(0.0, 0.0);
            y[c] = yc;
        }
        __syncthreads();
        const double2 yy = yc;
        for (int i = threadIdx.x; i < c; i += blockDim.x) {
            const double2 hic = H[(int64_t)c * ldh + i];
            work[i].x -= hic.x * yy.x - hic.y * yy.y;
            work[i].y -= hic.x * yy.y + hic.y * yy.x;
        }
        __syncthreads();
    }
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
struct MassOp {
    MassPair M{};
    double2 *r = nullptr, *dA = nullptr, *dB = nullptr;  // workspaces [R * n]
};

struct TransferOp {
    const int32_t *prow = nullptr, *pcol = nullptr;
    const double* pval = nullptr;
    int64_t pnnz = 0;
    double4 coef{};
};

// M^-1 on the four blocks of R columns, Chebyshev on the Jacobi-scaled mass matrices
bem_status mass_solve(const MassOp& op, const double2* z, double2* y, int R, cudaStream_t s, int steps) {
    const int64_t n = op.M.n;
    const double theta = 0.5 * (CHEB_BETA + CHEB_ALPHA), delta = 0.5 * (CHEB_BETA - CHEB_ALPHA);
    const double sigma = theta / delta;
    const dim3 grid(blocks_for(n, 256), R);
    BEM_LAUNCH(k_cheb_init, grid, 256, 0, s, op.M, z, y, op.r, op.dA, 1.0 / theta);
    double rho = 1.0 / sigma;
    double2 *dk = op.dA, *dn = op.dB;
    for (int k = 0; k < steps; ++k) {
        const double rho_n = 1.0 / (2.0 * sigma - rho);
        BEM_LAUNCH(k_cheb_step, grid, 256, 0, s, op.M, dk, dn, y, op.r, rho_n * rho, 2.0 * rho_n / delta);
        rho = rho_n;
        std::swap(dk, dn);
    }
    return BEM_OK;
}

bem_status transfer_add(const TransferOp& t, int64_t Ne, int64_t Ni, int64_t n, int R, const double2* x,
                        double2* z, cudaStream_t s) {
    if (t.pnnz > 0)
        BEM_LAUNCH(k_transfer, dim3(blocks_for(t.pnnz, 256), R), 256, 0, s, t.prow, t.pcol, t.pval, t.pnnz, Ne, Ni,
                   n, t.coef, x, z);
    return BEM_OK;
}

// compiled widths of the multi-column kernels; a batch of R columns runs at the
// next width and the padding columns read and write spare, in-bounds slots
int gemm_width(int R) { return R <= 1 ? 1 : R <= 2 ? 2 : R <= 4 ? 4 : 8; }

using Apply = std::function<bem_status(const double2* in, double2* out, int R)>;
using StopCheck = std::function<bem_status()>;

struct GmresWork {
    int maxit = 0, R = 0, RW = 0;
    int64_t n = 0, ldh = 0, gstride = 0;
    DevBuf Vb, H, cs, sn, g, resd, partial, hbuf, y, work, w, nrm, mr;
    double* h_res = nullptr;  // pinned, [R]
    ~GmresWork() {
        if (h_res) cudaFreeHost(h_res);
    }
    bem_status init(int maxit_, int64_t n_, int R_, cudaStream_t s) {
        maxit = maxit_;
        n = n_;
        R = R_;
        RW = gemm_width(R_);
        ldh = maxit + 1;
        gstride = maxit + 2;
        // (maxit + 1) basis blocks of R columns, plus RW - R spare columns read by the
        // padded operator kernels past the last block
        const size_t vb = ((size_t)(maxit + 1) * R + (RW - R)) * n * 16;
        BEM_TRY(Vb.alloc(vb, s));
        BEM_CUDA_TRY(cudaMemsetAsync(Vb.p, 0, vb, s));
        BEM_TRY(H.alloc((size_t)R * ldh * ldh * 16, s));
        BEM_TRY(cs.alloc((size_t)R * gstride * 8, s));
        BEM_TRY(sn.alloc((size_t)R * gstride * 16, s));
        BEM_TRY(g.alloc((size_t)R * gstride * 16, s));
        BEM_TRY(resd.alloc(R * 8, s));
        BEM_TRY(partial.alloc((size_t)R * (maxit + 1) * RED_BLOCKS * 16, s));
        BEM_TRY(hbuf.alloc((size_t)R * gstride * 16, s));
        BEM_TRY(y.alloc((size_t)R * gstride * 16, s));
        BEM_TRY(work.alloc((size_t)R * gstride * 16, s));
        BEM_TRY(w.alloc((size_t)R * n * 16, s));
        BEM_TRY(nrm.alloc(R * 16, s));
        BEM_TRY(mr.alloc(R * 4, s));
        BEM_CUDA_TRY(cudaMallocHost(&h_res, R * 16 + 16));
        return BEM_OK;
    }
};

// 2-norms of R columns stored back to back -> host
bem_status norms(GmresWork& W, const double2* v, int R, double* out, cudaStream_t s) {
    // with "basis" width 1 and index 0, column r is v + r * n
    BEM_LAUNCH(k_dots_partial, dim3(RED_BLOCKS, 1, R), 256, 0, s, v, W.n, 1, 1, v, W.partial.as<double2>());
    BEM_LAUNCH(k_dots_final, dim3(1, R), 32, 0, s, W.partial.as<double2>(), 1, W.nrm.as<double2>(), 1, 0);
    BEM_CUDA_TRY(cudaMemcpyAsync(W.h_res, W.nrm.p, R * 16, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    const double2* h = reinterpret_cast<const double2*>(W.h_res);
    for (int r = 0; r < R; ++r) out[r] = std::sqrt(std::max(h[r].x, 0.0));
    return BEM_OK;
}

// Unrestarted GMRES from x0 = 0 on apply(x) = rhs for R columns in lockstep; column
// r stops counting once its residual estimate is <= tol_abs[r].  Writes x (R
// columns); returns per-column iterations and final estimates.
bem_status gmres_run(GmresWork& W, int R, const Apply& apply, const double2* rhs, const double* beta,
                     const double* tol_abs, double2* x, int* iters_out, double* res_out, cudaStream_t s,
                     const StopCheck& stop) {
    const int64_t n = W.n, ldh = W.ldh, gs = W.gstride;
    double2* Vp = W.Vb.as<double2>();
    const dim3 eb(blocks_for(n, 256), R);
    BEM_CUDA_TRY(cudaMemsetAsync(W.H.p, 0, (size_t)R * ldh * ldh * 16, s));
    BEM_CUDA_TRY(cudaMemsetAsync(W.g.p, 0, (size_t)R * gs * 16, s));
    std::vector<int> it(R, 0);
    std::vector<char> done(R, 0);
    int ndone = 0;
    for (int r = 0; r < R; ++r) {
        res_out[r] = beta[r];
        if (!(beta[r] > tol_abs[r])) {
            done[r] = 1;
            ++ndone;
        }
    }
    if (ndone < R) {
        // V_0 = rhs / beta, g_0 = beta (per column)
        BEM_LAUNCH(k_dots_partial, dim3(RED_BLOCKS, 1, R), 256, 0, s, rhs, n, 1, 1, rhs, W.partial.as<double2>());
        BEM_LAUNCH(k_dots_final, dim3(1, R), 32, 0, s, W.partial.as<double2>(), 1, W.nrm.as<double2>(), 1, 0);
        BEM_LAUNCH(k_normalize, eb, 256, 0, s, rhs, n, W.nrm.as<double2>(), Vp, n, W.g.as<double2>(), gs);
        for (int j = 0; j < W.maxit && ndone < R; ++j) {
            double2* vj = Vp + (int64_t)j * R * n;
            BEM_TRY(apply(vj, W.w.as<double2>(), R));
            double2* Hj = W.H.as<double2>() + (int64_t)j * ldh;  // + r * ldh * ldh per column
            for (int pass = 0; pass < 2; ++pass) {  // CGS2
                double2* h = pass == 0 ? Hj : W.hbuf.as<double2>();
                const int64_t hst = pass == 0 ? ldh * ldh : gs;
                BEM_LAUNCH(k_dots_partial, dim3(RED_BLOCKS, j + 1, R), 256, 0, s, Vp, n, R, j + 1,
                           W.w.as<double2>(), W.partial.as<double2>());
                BEM_LAUNCH(k_dots_final, dim3(j + 1, R), 32, 0, s, W.partial.as<double2>(), j + 1, h, hst, 0);
                BEM_LAUNCH(k_combine, eb, 256, 0, s, Vp, n, R, j + 1, nullptr, h, hst, W.w.as<double2>(), 0);
            }
            BEM_LAUNCH(k_add_cols, dim3(1, R), 256, 0, s, Hj, ldh * ldh, W.hbuf.as<double2>(), gs, j + 1);
            BEM_LAUNCH(k_dots_partial, dim3(RED_BLOCKS, 1, R), 256, 0, s, W.w.as<double2>(), n, 1, 1,
                       W.w.as<double2>(), W.partial.as<double2>());
            BEM_LAUNCH(k_dots_final, dim3(1, R), 32, 0, s, W.partial.as<double2>(), 1, W.nrm.as<double2>(), 1, 0);
            BEM_LAUNCH(k_normalize, eb, 256, 0, s, W.w.as<double2>(), n, W.nrm.as<double2>(),
                       Vp + (int64_t)(j + 1) * R * n, n, Hj + j + 1, ldh * ldh);
            BEM_LAUNCH(k_givens, 1, 32, 0, s, W.H.as<double2>(), ldh, j, W.cs.as<double>(), W.sn.as<double2>(),
                       W.g.as<double2>(), gs, W.resd.as<double>(), R);
            BEM_CUDA_TRY(cudaMemcpyAsync(W.h_res, W.resd.p, R * 8, cudaMemcpyDeviceToHost, s));
            BEM_CUDA_TRY(cudaStreamSynchronize(s));
            for (int r = 0; r < R; ++r) {
                if (done[r]) continue;
                it[r] = j + 1;
                res_out[r] = W.h_res[r];
                if (!(W.h_res[r] > tol_abs[r])) {
                    done[r] = 1;
                    ++ndone;
                }
            }
            if (stop) BEM_TRY(stop());
        }
    }
    BEM_CUDA_TRY(cudaMemcpyAsync(W.mr.p, it.data(), R * 4, cudaMemcpyHostToDevice, s));
    BEM_LAUNCH(k_backsolve, R, 256, 0, s, W.H.as<double2>(), ldh, W.mr.as<int>(), W.g.as<double2>(), gs,
               W.y.as<double2>(), W.work.as<double2>());
    BEM_LAUNCH(k_combine, eb, 256, 0, s, Vp, n, R, 0, W.mr.as<int>(), W.y.as<double2>(), gs, x, 1);
    BEM_CUDA_TRY(cudaStreamSynchronize(s));  // `it` must outlive the copy
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

}  // namespace

bem_status solve_transmission_impl(bem_context* ctx, const bem_grid* ge, const bem_grid* gi, bem_c128 k_int,
                                   bem_c128 k_ext, double rho_ratio, const bem_incident* inc,
                                   const bem_solve_opts* o, bem_c128* v_ext, bem_c128* w_ext, bem_c128* v_int,
                                   bem_c128* w_int, int on_device, bem_solve_report* rep) {
    cudaStream_t s = ctx->stream;
    const int64_t Ne = ge->nv, Ni = gi->nv, n = 2 * Ne + 2 * Ni;
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
    // ---- operators on both grids --------------------------------------------------
    const size_t esz = mixed ? 8 : 16;
    const size_t be = (size_t)Ne * Ne * esz, bi = (size_t)Ni * Ni * esz;
    DevBuf M[8];  // Ve, Ke, Te, De, Vi, Ki, Ti, Di
    for (int m = 0; m < 8; ++m) BEM_TRY(M[m].alloc(m < 4 ? be : bi, s));
    cudaEventRecord(t_asm.a, s);
    if (mixed) {
        for (int m = 0; m < 8; ++m) BEM_CUDA_TRY(cudaMemsetAsync(M[m].p, 0, m < 4 ? be : bi, s));
        for (int side = 0; side < 2; ++side) {
            const bem_grid* g = side == 0 ? ge : gi;
            const bem_c128 k = side == 0 ? k_ext : k_int;
            float2* P4[4];
            for (int m = 0; m < 4; ++m) P4[m] = M[4 * side + m].as<float2>();
            BEM_TRY(assemble_regular_fp32(g, k.re, k.im, P4[0], P4[1], P4[2], P4[3], s));
            BEM_TRY(assemble_singular_into_c64(g, k.re, k.im, o->n_singular, P4[0], P4[1], P4[2], P4[3], s));
        }
    } else {
        BEM_TRY(assemble_operators_fp64(ge, k_ext.re, k_ext.im, o->n_singular, M[0].as<double2>(), M[1].as<double2>(),
                                        M[2].as<double2>(), M[3].as<double2>(), s));
        BEM_TRY(assemble_operators_fp64(gi, k_int.re, k_int.im, o->n_singular, M[4].as<double2>(), M[5].as<double2>(),
                                        M[6].as<double2>(), M[7].as<double2>(), s));
    }
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
    cudaEventRecord(t_mor.b, s);
    // ---- workspaces for batches of RB right-hand sides ---------------------------------
    const int RB = std::min<int>(RMAX, inc->n_rhs);
    const int RW = gemm_width(RB);  // column count of everything the operator kernels touch
    const size_t colb = (size_t)n * 16;
    DevBuf wz, wr, wa, wb, x32;
    BEM_TRY(wz.alloc(RW * colb, s));
    BEM_TRY(wr.alloc(RB * colb, s));
    BEM_TRY(wa.alloc(RB * colb, s));
    BEM_TRY(wb.alloc(RB * colb, s));
    MassOp mop;
    mop.M.rp[0] = ge->m_rowptr.as<int32_t>(); mop.M.ci[0] = ge->m_col.as<int32_t>();
    mop.M.v[0] = mve.as<double>(); mop.M.dinv[0] = dve.as<double>();
    mop.M.rp[1] = gi->m_rowptr.as<int32_t>(); mop.M.ci[1] = gi->m_col.as<int32_t>();
    mop.M.v[1] = mvi.as<double>(); mop.M.dinv[1] = dvi.as<double>();
    mop.M.Ne = Ne; mop.M.Ni = Ni; mop.M.n = n;
    mop.r = wr.as<double2>(); mop.dA = wa.as<double2>(); mop.dB = wb.as<double2>();
    TransferOp top;
    const double sgn = o->mtf_variant == BEM_MTF_PRINTED ? -1.0 : 1.0;
    top.prow = prow.as<int32_t>(); top.pcol = pcol.as<int32_t>(); top.pval = pval.as<double>(); top.pnnz = pnnz;
    top.coef = make_double4(-0.5 * sgn, -0.5 * sgn / rho_ratio, 0.5 * sgn, 0.5 * sgn * rho_ratio);
    double2* z = wz.as<double2>();
    Blocks<double2> B64{};
    Blocks<float2> B32{};
    if (mixed) {
        BEM_TRY(x32.alloc((size_t)RW * n * 8, s));
        BEM_CUDA_TRY(cudaMemsetAsync(x32.p, 0, x32.bytes, s));
        const float2* m1[4] = {M[1].as<float2>(), M[3].as<float2>(), M[5].as<float2>(), M[7].as<float2>()};
        const float2* m2[4] = {M[0].as<float2>(), M[2].as<float2>(), M[4].as<float2>(), M[6].as<float2>()};
        fill_blocks(B32, m1, m2, Ne, Ni);
    } else {
        const double2* m1[4] = {M[1].as<double2>(), M[3].as<double2>(), M[5].as<double2>(), M[7].as<double2>()};
        const double2* m2[4] = {M[0].as<double2>(), M[2].as<double2>(), M[4].as<double2>(), M[6].as<double2>()};
        fill_blocks(B64, m1, m2, Ne, Ni);
    }
    const unsigned rows_blocks = blocks_for(n * 32, 256);
    // dense blocks for R columns in the working arithmetic (x must hold gemm_width(R) columns)
    auto gemm_work = [&](const double2* xin, int R) -> bem_status {
        const int Wd = gemm_width(R);
        if (mixed) {
            BEM_LAUNCH(k_to_c64, blocks_for((int64_t)R * n, 256), 256, 0, s, xin, (int64_t)R * n, x32.as<float2>());
            if (Wd == 1) BEM_LAUNCH(k_gemm32<1>, rows_blocks, 256, 0, s, B32, n, x32.as<float2>(), z);
            else if (Wd == 2) BEM_LAUNCH(k_gemm32<2>, rows_blocks, 256, 0, s, B32, n, x32.as<float2>(), z);
            else if (Wd == 4) BEM_LAUNCH(k_gemm32<4>, rows_blocks, 256, 0, s, B32, n, x32.as<float2>(), z);
            else BEM_LAUNCH(k_gemm32<8>, rows_blocks, 256, 0, s, B32, n, x32.as<float2>(), z);
        } else {
            if (Wd == 1) BEM_LAUNCH(k_gemm64<1>, rows_blocks, 256, 0, s, B64, n, xin, z);
            else if (Wd == 2) BEM_LAUNCH(k_gemm64<2>, rows_blocks, 256, 0, s, B64, n, xin, z);
            else if (Wd == 4) BEM_LAUNCH(k_gemm64<4>, rows_blocks, 256, 0, s, B64, n, xin, z);
            else BEM_LAUNCH(k_gemm64<8>, rows_blocks, 256, 0, s, B64, n, xin, z);
        }
        return BEM_OK;
    };
    auto gemm_fp64 = [&](const double2* xin, int R) -> bem_status {
        if (!mixed) return gemm_work(xin, R);
        const int Wd = gemm_width(R);
        if (Wd == 1) BEM_LAUNCH(k_gemm_c64_f64<1>, rows_blocks, 256, 0, s, B32, n, xin, z);
        else if (Wd == 2) BEM_LAUNCH(k_gemm_c64_f64<2>, rows_blocks, 256, 0, s, B32, n, xin, z);
        else if (Wd == 4) BEM_LAUNCH(k_gemm_c64_f64<4>, rows_blocks, 256, 0, s, B32, n, xin, z);
        else BEM_LAUNCH(k_gemm_c64_f64<8>, rows_blocks, 256, 0, s, B32, n, xin, z);
        return BEM_OK;
    };
    // S A x in the working precision, and with FP64 arithmetic on the stored matrices
    Apply apply_work = [&](const double2* xin, double2* yout, int R) -> bem_status {
        BEM_TRY(gemm_work(xin, R));
        BEM_TRY(transfer_add(top, Ne, Ni, n, R, xin, z, s));
        return mass_solve(mop, z, yout, R, s, mixed ? CHEB_STEPS_INNER : CHEB_STEPS);
    };
    Apply apply_fp64 = [&](const double2* xin, double2* yout, int R) -> bem_status {
        BEM_TRY(gemm_fp64(xin, R));
        BEM_TRY(transfer_add(top, Ne, Ni, n, R, xin, z, s));
        return mass_solve(mop, z, yout, R, s, CHEB_STEPS);
    };
    // ---- GMRES ------------------------------------------------------------------------
    const int maxit = (int)std::min<int64_t>(o->gmres_maxiter, n);
    GmresWork W;
    BEM_TRY(W.init(maxit, n, RB, s));
    DevBuf fvec, gvec, bvec, sb, xsol, dvec, rvec, tmp;
    BEM_TRY(fvec.alloc((size_t)RB * Ne * 16, s));
    BEM_TRY(gvec.alloc((size_t)RB * Ne * 16, s));
    BEM_TRY(bvec.alloc(RB * colb, s));
    BEM_TRY(sb.alloc(RB * colb, s));
    BEM_TRY(xsol.alloc(RW * colb, s));  // read with RW columns by the FP64 residual
    BEM_CUDA_TRY(cudaMemsetAsync(xsol.p, 0, RW * colb, s));
    BEM_TRY(dvec.alloc(RB * colb, s));
    BEM_TRY(rvec.alloc(RB * colb, s));
    BEM_TRY(tmp.alloc(RB * colb, s));
    bem_status result = BEM_OK;
    int total_inner = 0, outer_used = 0;
    double worst_res = 0.0;
    bool all_conv = true;
    cudaEventRecord(t_sol.a, s);
    for (int r0 = 0; r0 < inc->n_rhs; r0 += RB) {
        const int R = std::min(RB, inc->n_rhs - r0);
        Waves wv{};
        for (int r = 0; r < R; ++r) {
            const double* d = inc->dirs + 3 * (r0 + r);
            wv.d[r] = make_double3(d[0], d[1], d[2]);
            wv.amp[r] = inc->amps ? make_double2(inc->amps[r0 + r].re, inc->amps[r0 + r].im) : make_double2(1.0, 0.0);
        }
        BEM_CUDA_TRY(cudaMemsetAsync(fvec.p, 0, (size_t)R * Ne * 16, s));
        BEM_CUDA_TRY(cudaMemsetAsync(gvec.p, 0, (size_t)R * Ne * 16, s));
        BEM_LAUNCH(k_plane_wave, dim3(blocks_for(ge->nt, 128), R), 128, 0, s, ge->rec.as<TriRec>(),
                   ge->tri.as<int32_t>(), ge->nt, k_ext.re, k_ext.im, wv, Ne, fvec.as<double2>(), gvec.as<double2>());
        BEM_LAUNCH(k_rhs_pack, dim3(blocks_for(n, 256), R), 256, 0, s, fvec.as<double2>(), gvec.as<double2>(), Ne, n,
                   bvec.as<double2>());
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
            while (any_pending() && outer < max_outer) {
                // a column that is finished (or out of iterations) gets tolerance |r|,
                // so that its inner GMRES takes no step and its correction is zero
                for (int r = 0; r < R; ++r)
                    inner_tol[r] = pending(r) ? std::max(tol_abs[r], o->ir_inner_tol * rn[r]) : rn[r];
                BEM_TRY(gmres_run(W, R, apply_work, rvec.as<double2>(), rn.data(), inner_tol.data(),
                                  dvec.as<double2>(), its.data(), est.data(), s, stop));
                int moved = 0;
                for (int r = 0; r < R; ++r) {
                    total[r] += its[r];
                    moved += its[r];
                }
                BEM_LAUNCH(k_acc, blocks_for((int64_t)R * n, 256), 256, 0, s, xsol.as<double2>(), dvec.as<double2>(),
                           (int64_t)R * n);
                BEM_TRY(apply_fp64(xsol.as<double2>(), tmp.as<double2>(), R));
                BEM_LAUNCH(k_sub, blocks_for((int64_t)R * n, 256), 256, 0, s, sb.as<double2>(), tmp.as<double2>(),
                           (int64_t)R * n, rvec.as<double2>());
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
        for (int r = 0; r < R; ++r) {
            const double2* X = xsol.as<double2>() + (int64_t)r * n;
            const int64_t rr = r0 + r;
            BEM_CUDA_TRY(cudaMemcpyAsync(v_ext + rr * Ne, X, Ne * 16, kind, s));
            BEM_CUDA_TRY(cudaMemcpyAsync(w_ext + rr * Ne, X + Ne, Ne * 16, kind, s));
            BEM_CUDA_TRY(cudaMemcpyAsync(v_int + rr * Ni, X + 2 * Ne, Ni * 16, kind, s));
            BEM_CUDA_TRY(cudaMemcpyAsync(w_int + rr * Ni, X + 2 * Ne + Ni, Ni * 16, kind, s));
        }
        BEM_CUDA_TRY(cudaStreamSynchronize(s));
    }
    cudaEventRecord(t_sol.b, s);
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
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

}  // namespace bem
