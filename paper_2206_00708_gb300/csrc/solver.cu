// Transmission solve on the device (paper Sec. 2.2 unknowns and transmission
// conditions, eq. mtf:discrete, Sec. 3.3 mass-matrix preconditioning, Sec. 5.1
// unrestarted GMRES).
//
// Unknown vector x = [v_e (N_e), w_e (N_e), v_i (N_i), w_i (N_i)], complex128.
// Weak-form MTF (derived signs, s = +1; printed signs, s = -1):
//   z1 = -K_e v_e + V_e w_e - (s/2) P_ei v_i
//   z2 =  D_e v_e + T_e w_e - (s/2)(rho_e/rho_i) P_ei w_i
//   z3 = (s/2) P_ie v_e - K_i v_i + V_i w_i
//   z4 = (s/2)(rho_i/rho_e) P_ie w_e + D_i v_i + T_i w_i
// with P_ie = P_int,ext (mortar, COO) and P_ei = P_ie^T.  The strong form applies
// M_e^-1 to z1, z2 and M_i^-1 to z3, z4.
//
// Mass inverse: Chebyshev iteration on the Jacobi-scaled mass matrix.  For P1
// triangles every element matrix scaled by its diagonal has eigenvalues {2, 1/2, 1/2}
// (whatever the triangle's shape), so D^-1 M has its spectrum in [1/2, 2] and the
// Chebyshev error contracts by (sqrt(4) - 1)/(sqrt(4) + 1) = 1/3 per step with no
// inner products: 34 steps reach 2 * 3^-34 ~ 1e-16.
//
// GMRES: Arnoldi with classical Gram-Schmidt applied twice (CGS2), complex Givens
// rotations and the residual estimate kept on the device; the host reads one
// scalar per iteration to stop.  x0 = 0, stop when |g_{j+1}| <= tol * ||S b||.
#include "bem_internal.cuh"

#include <algorithm>
#include <cmath>
#include <functional>

namespace bem {

namespace {

constexpr int CHEB_STEPS = 34;        // error <= 2 * 3^-34 ~ 1e-16: FP64 applications
constexpr int CHEB_STEPS_INNER = 17;  // error <= 2 * 3^-17 ~ 1.6e-8: inner solves of the refinement
constexpr double CHEB_ALPHA = 0.5, CHEB_BETA = 2.0;

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

// ---------------------------------------------------------------- right-hand side
// f_j = <u_inc, theta_j>, g_j = <du_inc/dn, theta_j> on the exterior grid,
// u_inc = amp exp(i k x.d), du_inc/dn = i k (d.n) u_inc (paper eq. planewave).
__global__ void k_plane_wave(const TriRec* __restrict__ rec, const int32_t* __restrict__ tri, int64_t nt,
                             double kr, double ki, double3 d, double2 amp, double2* __restrict__ f,
                             double2* __restrict__ g) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const TriRec& R = rec[t];
    const double dn = d.x * R.n[0] + d.y * R.n[1] + d.z * R.n[2];
    double2 fa[3] = {}, ga[3] = {};
    for (int p = 0; p < 6; ++p) {
        double xd = d.x * R.q[p][0] + d.y * R.q[p][1] + d.z * R.q[p][2];
        double sn, cs;
        sincos(kr * xd, &sn, &cs);
        double mag = (ki != 0.0) ? exp(-ki * xd) : 1.0;
        double2 u = cmul(amp, make_double2(mag * cs, mag * sn));
        // i k (d.n) u
        double2 ik = make_double2(-ki * dn, kr * dn);
        double2 du = cmul(ik, u);
        for (int a = 0; a < 3; ++a) {
            fa[a].x += R.wl[p][a] * u.x;
            fa[a].y += R.wl[p][a] * u.y;
            ga[a].x += R.wl[p][a] * du.x;
            ga[a].y += R.wl[p][a] * du.y;
        }
    }
    for (int a = 0; a < 3; ++a) {
        int32_t v = tri[3 * t + a];
        atomicAdd(&f[v].x, fa[a].x);
        atomicAdd(&f[v].y, fa[a].y);
        atomicAdd(&g[v].x, ga[a].x);
        atomicAdd(&g[v].y, ga[a].y);
    }
}

// b = [-f, -g, 0, 0]
__global__ void k_rhs_pack(const double2* __restrict__ f, const double2* __restrict__ g, int64_t Ne, int64_t n,
                           double2* __restrict__ b) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    double2 v = make_double2(0.0, 0.0);
    if (e < Ne) v = make_double2(-f[e].x, -f[e].y);
    else if (e < 2 * Ne) v = make_double2(-g[e - Ne].x, -g[e - Ne].y);
    b[e] = v;
}

// ---------------------------------------------------------------- MTF operator
struct Blocks {
    const double2* A1[4];  // first matrix of each block row
    const double2* A2[4];  // second matrix
    double c1[4], c2[4];   // real coefficients
    int64_t rows[4];       // N of each block row
    int64_t base[4];       // offset of block row b in the vector
    int64_t x1[4], x2[4];  // offsets of the vectors multiplying A1, A2
};

// dense part: one warp per row of the 4 x 4 block system
__global__ void __launch_bounds__(256) k_gemv_mtf(Blocks B, int64_t n, const double2* __restrict__ x,
                                                  double2* __restrict__ z) {
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= n) return;
    int b = 0;
    while (b < 3 && gw >= B.base[b + 1]) ++b;
    const int64_t i = gw - B.base[b];
    const int64_t N = B.rows[b];
    const double2* __restrict__ a1 = B.A1[b] + i * N;
    const double2* __restrict__ a2 = B.A2[b] + i * N;
    const double2* __restrict__ x1 = x + B.x1[b];
    const double2* __restrict__ x2 = x + B.x2[b];
    double2 s1 = make_double2(0, 0), s2 = make_double2(0, 0);
    for (int64_t j = lane; j < N; j += 32) {
        s1 = cfma(a1[j], x1[j], s1);
        s2 = cfma(a2[j], x2[j], s2);
    }
    s1 = warp_sum2(s1);
    s2 = warp_sum2(s2);
    if (lane == 0) z[gw] = make_double2(B.c1[b] * s1.x + B.c2[b] * s2.x, B.c1[b] * s1.y + B.c2[b] * s2.y);
}

// mortar part: entries (r, c, p) of P_ie; z1[c] += a p v_i[r], z2[c] += b p w_i[r],
// z3[r] += c p v_e[c], z4[r] += d p w_e[c]
__global__ void k_transfer(const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                           const double* __restrict__ val, int64_t nnz, int64_t Ne, int64_t Ni, double4 coef,
                           const double2* __restrict__ x, double2* __restrict__ z) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const double p = val[e];
    if (p == 0.0) return;
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

struct MassPair {
    const int32_t *rp[2], *ci[2];
    const double *v[2], *dinv[2];
    int64_t Ne, Ni, n;
};

__device__ __forceinline__ void mass_row(const MassPair& M, int64_t g, int& m, int64_t& i, int64_t& base) {
    if (g < M.Ne) { m = 0; i = g; base = 0; }
    else if (g < 2 * M.Ne) { m = 0; i = g - M.Ne; base = M.Ne; }
    else if (g < 2 * M.Ne + M.Ni) { m = 1; i = g - 2 * M.Ne; base = 2 * M.Ne; }
    else { m = 1; i = g - 2 * M.Ne - M.Ni; base = 2 * M.Ne + M.Ni; }
}

// y = 0, r = z, d = D^-1 r / theta
__global__ void k_cheb_init(MassPair M, const double2* __restrict__ z, double2* __restrict__ y,
                            double2* __restrict__ r, double2* __restrict__ d, double inv_theta) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= M.n) return;
    int m;
    int64_t i, base;
    mass_row(M, g, m, i, base);
    const double2 zz = z[g];
    const double s = M.dinv[m][i] * inv_theta;
    y[g] = make_double2(0, 0);
    r[g] = zz;
    d[g] = make_double2(s * zz.x, s * zz.y);
}

// y += d_k; r -= M d_k; d_{k+1} = c1 d_k + c2 D^-1 r
__global__ void k_cheb_step(MassPair M, const double2* __restrict__ dk, double2* __restrict__ dn,
                            double2* __restrict__ y, double2* __restrict__ r, double c1, double c2) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= M.n) return;
    int m;
    int64_t i, base;
    mass_row(M, g, m, i, base);
    double2 md = make_double2(0, 0);
    for (int32_t e = M.rp[m][i]; e < M.rp[m][i + 1]; ++e) {
        const double v = M.v[m][e];
        const double2 dd = dk[base + M.ci[m][e]];
        md.x += v * dd.x;
        md.y += v * dd.y;
    }
    const double2 d0 = dk[g];
    double2 yy = y[g], rr = r[g];
    yy.x += d0.x;
    yy.y += d0.y;
    rr.x -= md.x;
    rr.y -= md.y;
    y[g] = yy;
    r[g] = rr;
    const double s = c2 * M.dinv[m][i];
    dn[g] = make_double2(c1 * d0.x + s * rr.x, c1 * d0.y + s * rr.y);
}

// ---------------------------------------------------------------- GMRES kernels
constexpr int RED_BLOCKS = 64;

// partial[i * RED_BLOCKS + bx] = sum over the block's chunk of conj(V_i) w
__global__ void k_dots_partial(const double2* __restrict__ Vb, int64_t n, int64_t ld, const double2* __restrict__ w,
                               double2* __restrict__ partial) {
    const int i = blockIdx.y;
    const double2* __restrict__ v = Vb + (int64_t)i * ld;
    double2 s = make_double2(0, 0);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = v[e], b = w[e];
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
        if (threadIdx.x == 0) partial[(int64_t)i * RED_BLOCKS + blockIdx.x] = t;
    }
}

// out[i] = sum_b partial[i][b]  (+= when accumulate)
__global__ void k_dots_final(const double2* __restrict__ partial, int m, double2* __restrict__ out, int accumulate) {
    const int i = blockIdx.x;
    if (i >= m) return;
    double2 s = make_double2(0, 0);
    for (int b = threadIdx.x; b < RED_BLOCKS; b += 32) {
        s.x += partial[(int64_t)i * RED_BLOCKS + b].x;
        s.y += partial[(int64_t)i * RED_BLOCKS + b].y;
    }
    s = warp_sum2(s);
    if (threadIdx.x == 0) {
        if (accumulate) { out[i].x += s.x; out[i].y += s.y; }
        else out[i] = s;
    }
}

// w -= sum_i h_i V_i   (sign = -1)   or   x = sum_i h_i V_i (sign = +1, overwrite)
__global__ void k_combine(const double2* __restrict__ Vb, int64_t n, int64_t ld, int m, const double2* __restrict__ h,
                          double2* __restrict__ w, int overwrite) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    double2 s = make_double2(0, 0);
    for (int i = 0; i < m; ++i) s = cfma(h[i], Vb[(int64_t)i * ld + e], s);
    if (overwrite) w[e] = s;
    else {
        double2 t = w[e];
        w[e] = make_double2(t.x - s.x, t.y - s.y);
    }
}

__global__ void k_add(double2* __restrict__ a, const double2* __restrict__ b, int m) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        a[i].x += b[i].x;
        a[i].y += b[i].y;
    }
}

// v = w / |w|, where |w|^2 = real part of nrm2[0]; also stores |w| to dst (complex)
__global__ void k_normalize(const double2* __restrict__ w, int64_t n, const double2* __restrict__ nrm2,
                            double2* __restrict__ v, double2* __restrict__ dst) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const double nr = sqrt(fmax(nrm2[0].x, 0.0));
    if (e == 0 && dst) *dst = make_double2(nr, 0.0);
    if (e >= n) return;
    const double inv = nr > 0.0 ? 1.0 / nr : 0.0;
    v[e] = make_double2(w[e].x * inv, w[e].y * inv);
}

// Givens update of Hessenberg column j (H column-major with leading dimension ldh)
__global__ void k_givens(double2* __restrict__ H, int64_t ldh, int j, double* __restrict__ cs,
                         double2* __restrict__ sn, double2* __restrict__ g, double* __restrict__ res) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double2* h = H + (int64_t)j * ldh;
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
    double2 s, r;
    if (aa == 0.0) {
        c = 0.0;
        s = make_double2(1.0, 0.0);
        r = b;
    } else {
        const double t = hypot(aa, bb);
        c = aa / t;
        const double2 ph = make_double2(a.x / aa, a.y / aa);
        // s = ph * conj(b) / t
        s = make_double2((ph.x * b.x + ph.y * b.y) / t, (ph.y * b.x - ph.x * b.y) / t);
        r = make_double2(ph.x * t, ph.y * t);
    }
    cs[j] = c;
    sn[j] = s;
    h[j] = r;
    h[j + 1] = make_double2(0.0, 0.0);
    const double2 gj = g[j];
    // g[j+1] = -conj(s) g[j]; g[j] = c g[j]
    g[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
    g[j] = make_double2(c * gj.x, c * gj.y);
    res[0] = hypot(g[j + 1].x, g[j + 1].y);
}

// y = H(0:m,0:m)^-1 g(0:m), column-oriented back substitution in one block
__global__ void k_backsolve(const double2* __restrict__ H, int64_t ldh, int m, const double2* __restrict__ g,
                            double2* __restrict__ y, double2* __restrict__ work) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) work[i] = g[i];
    __syncthreads();
    for (int c = m - 1; c >= 0; --c) {
        __shared__ double2 yc;
        if (threadIdx.x == 0) {
            const double2 d = H[(int64_t)c * ldh + c];
            const double den = d.x * d.x + d.y * d.y;
            const double2 wc = work[c];
            yc = make_double2((wc.x * d.x + wc.y * d.y) / den, (wc.y * d.x - wc.x * d.y) / den);
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

unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------- mixed precision
struct Blocks32 {
    const float2* A1[4];
    const float2* A2[4];
    double c1[4], c2[4];
    int64_t rows[4], base[4], x1[4], x2[4];
};

__global__ void k_to_c64(const double2* __restrict__ x, int64_t n, float2* __restrict__ y) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) y[e] = make_float2((float)x[e].x, (float)x[e].y);
}

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// complex64 matrices, FP32 arithmetic: one warp per row, 16-byte loads (two complex
// entries per lane), each 4-entry chunk summed plainly and added to the lane's
// accumulator with a compensated (two-sum) update; the warp total is formed in FP64.
__global__ void __launch_bounds__(256) k_gemv_mtf32(Blocks32 B, int64_t n, const float2* __restrict__ x,
                                                    double2* __restrict__ z) {
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= n) return;
    int b = 0;
    while (b < 3 && gw >= B.base[b + 1]) ++b;
    const int64_t i = gw - B.base[b];
    const int64_t N = B.rows[b];
    double2 out = make_double2(0, 0);
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const float2* __restrict__ a = (m == 0 ? B.A1[b] : B.A2[b]) + i * N;
        const float2* __restrict__ xv = x + (m == 0 ? B.x1[b] : B.x2[b]);
        float sr = 0.f, si = 0.f, er = 0.f, ei = 0.f;
        // row start may be only 8-byte aligned: peel to a 16-byte boundary
        int64_t j0 = ((reinterpret_cast<uintptr_t>(a) & 15) != 0) ? 1 : 0;
        if (j0 && lane == 0 && N > 0) {
            const float2 av = a[0], xx = xv[0];
            sr = fmaf(av.x, xx.x, -av.y * xx.y);
            si = fmaf(av.x, xx.y, av.y * xx.x);
        }
        const int64_t npair = (N - j0) / 2;
        const float4* __restrict__ a4 = reinterpret_cast<const float4*>(a + j0);
        for (int64_t p = lane; p < npair; p += 64) {
            float cr = 0.f, ci = 0.f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t pp = p + 32 * h;
                if (pp < npair) {
                    const float4 av = a4[pp];
                    const int64_t j = j0 + 2 * pp;
                    const float2 x0 = xv[j], x1 = xv[j + 1];
                    cr = fmaf(av.x, x0.x, cr); cr = fmaf(-av.y, x0.y, cr);
                    ci = fmaf(av.x, x0.y, ci); ci = fmaf(av.y, x0.x, ci);
                    cr = fmaf(av.z, x1.x, cr); cr = fmaf(-av.w, x1.y, cr);
                    ci = fmaf(av.z, x1.y, ci); ci = fmaf(av.w, x1.x, ci);
                }
            }
            float t, e;
            two_sum_f(sr, cr, t, e); sr = t; er += e;
            two_sum_f(si, ci, t, e); si = t; ei += e;
        }
        if (((N - j0) & 1) && lane == 1) {  // odd tail
            const int64_t j = N - 1;
            const float2 av = a[j], xx = xv[j];
            float t, e;
            two_sum_f(sr, fmaf(av.x, xx.x, -av.y * xx.y), t, e); sr = t; er += e;
            two_sum_f(si, fmaf(av.x, xx.y, av.y * xx.x), t, e); si = t; ei += e;
        }
        double2 v = make_double2((double)sr + (double)er, (double)si + (double)ei);
        v = warp_sum2(v);
        const double c = m == 0 ? B.c1[b] : B.c2[b];
        out.x += c * v.x;
        out.y += c * v.y;
    }
    if (lane == 0) z[gw] = out;
}

// complex64 matrices, FP64 arithmetic (outer residual of the refinement)
__global__ void __launch_bounds__(256) k_gemv_mtf_c64_f64(Blocks32 B, int64_t n, const double2* __restrict__ x,
                                                          double2* __restrict__ z) {
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= n) return;
    int b = 0;
    while (b < 3 && gw >= B.base[b + 1]) ++b;
    const int64_t i = gw - B.base[b];
    const int64_t N = B.rows[b];
    const float2* __restrict__ a1 = B.A1[b] + i * N;
    const float2* __restrict__ a2 = B.A2[b] + i * N;
    const double2* __restrict__ x1 = x + B.x1[b];
    const double2* __restrict__ x2 = x + B.x2[b];
    double2 s1 = make_double2(0, 0), s2 = make_double2(0, 0);
    for (int64_t j = lane; j < N; j += 32) {
        const float2 p = a1[j], q = a2[j];
        s1 = cfma(make_double2(p.x, p.y), x1[j], s1);
        s2 = cfma(make_double2(q.x, q.y), x2[j], s2);
    }
    s1 = warp_sum2(s1);
    s2 = warp_sum2(s2);
    if (lane == 0) z[gw] = make_double2(B.c1[b] * s1.x + B.c2[b] * s2.x, B.c1[b] * s1.y + B.c2[b] * s2.y);
}

// y = a - b
__global__ void k_sub(const double2* __restrict__ a, const double2* __restrict__ b, int64_t n,
                      double2* __restrict__ y) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) y[e] = make_double2(a[e].x - b[e].x, a[e].y - b[e].y);
}

// x += d
__global__ void k_acc(double2* __restrict__ x, const double2* __restrict__ d, int64_t n) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) {
        x[e].x += d[e].x;
        x[e].y += d[e].y;
    }
}

}  // namespace

// ------------------------------------------------------------------ host driver
namespace {

struct MassOp {
    MassPair M{};
    double2 *r = nullptr, *dA = nullptr, *dB = nullptr;  // workspaces [n]
};

struct TransferOp {
    const int32_t *prow = nullptr, *pcol = nullptr;
    const double* pval = nullptr;
    int64_t pnnz = 0;
    double4 coef{};
};

// M^-1 (z) -> y on the four blocks, Chebyshev on the Jacobi-scaled mass matrices
bem_status mass_solve(const MassOp& op, const double2* z, double2* y, cudaStream_t s, int steps = CHEB_STEPS) {
    const int64_t n = op.M.n;
    const double theta = 0.5 * (CHEB_BETA + CHEB_ALPHA), delta = 0.5 * (CHEB_BETA - CHEB_ALPHA);
    const double sigma = theta / delta;
    BEM_LAUNCH(k_cheb_init, blocks_for(n, 256), 256, 0, s, op.M, z, y, op.r, op.dA, 1.0 / theta);
    double rho = 1.0 / sigma;
    double2 *dk = op.dA, *dn = op.dB;
    for (int k = 0; k < steps; ++k) {
        const double rho_n = 1.0 / (2.0 * sigma - rho);
        BEM_LAUNCH(k_cheb_step, blocks_for(n, 256), 256, 0, s, op.M, dk, dn, y, op.r, rho_n * rho, 2.0 * rho_n / delta);
        rho = rho_n;
        std::swap(dk, dn);
    }
    return BEM_OK;
}

bem_status transfer_add(const TransferOp& t, int64_t Ne, int64_t Ni, const double2* x, double2* z, cudaStream_t s) {
    if (t.pnnz > 0)
        BEM_LAUNCH(k_transfer, blocks_for(t.pnnz, 256), 256, 0, s, t.prow, t.pcol, t.pval, t.pnnz, Ne, Ni, t.coef, x, z);
    return BEM_OK;
}

using Apply = std::function<bem_status(const double2* in, double2* out)>;

struct GmresWork {
    int maxit = 0;
    int64_t n = 0, ldh = 0;
    DevBuf Vb, H, cs, sn, g, resd, partial, hbuf, y, work, w, nrm;
    double* h_res = nullptr;
    ~GmresWork() {
        if (h_res) cudaFreeHost(h_res);
    }
    bem_status init(int maxit_, int64_t n_, cudaStream_t s) {
        maxit = maxit_;
        n = n_;
        ldh = maxit + 1;
        BEM_TRY(Vb.alloc((size_t)(maxit + 1) * n * 16, s));
        BEM_TRY(H.alloc((size_t)ldh * (maxit + 1) * 16, s));
        BEM_TRY(cs.alloc((maxit + 1) * 8, s));
        BEM_TRY(sn.alloc((maxit + 1) * 16, s));
        BEM_TRY(g.alloc((maxit + 2) * 16, s));
        BEM_TRY(resd.alloc(8, s));
        BEM_TRY(partial.alloc((size_t)(maxit + 1) * RED_BLOCKS * 16, s));
        BEM_TRY(hbuf.alloc((maxit + 1) * 16, s));
        BEM_TRY(y.alloc((maxit + 1) * 16, s));
        BEM_TRY(work.alloc((maxit + 1) * 16, s));
        BEM_TRY(w.alloc(n * 16, s));
        BEM_TRY(nrm.alloc(16, s));
        BEM_CUDA_TRY(cudaMallocHost(&h_res, 16));
        return BEM_OK;
    }
};

// ||v||_2 read back to the host
bem_status norm2(GmresWork& W, const double2* v, double* out, cudaStream_t s) {
    BEM_LAUNCH(k_dots_partial, dim3(RED_BLOCKS, 1), 256, 0, s, v, W.n, W.n, v, W.partial.as<double2>());
    BEM_LAUNCH(k_dots_final, 1, 32, 0, s, W.partial.as<double2>(), 1, W.nrm.as<double2>(), 0);
    BEM_CUDA_TRY(cudaMemcpyAsync(W.h_res, W.nrm.p, 8, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    *out = std::sqrt(std::max(W.h_res[0], 0.0));
    return BEM_OK;
}

// Unrestarted GMRES from x0 = 0 on apply(x) = rhs; stops when the residual estimate
// is <= tol_abs.  Writes x; returns iterations and the final estimate.
// stop check between iterations (serving: cancellation and deadlines)
using StopCheck = std::function<bem_status()>;

bem_status gmres_run(GmresWork& W, const Apply& apply, const double2* rhs, double beta, double tol_abs,
                     double2* x, int* iters_out, double* res_out, cudaStream_t s, const StopCheck& stop) {
    const int64_t n = W.n, ldv = n, ldh = W.ldh;
    double2* Vp = W.Vb.as<double2>();
    const unsigned eb = blocks_for(n, 256);
    BEM_CUDA_TRY(cudaMemsetAsync(W.H.p, 0, (size_t)ldh * (W.maxit + 1) * 16, s));
    BEM_CUDA_TRY(cudaMemsetAsync(W.g.p, 0, (W.maxit + 2) * 16, s));
    int iters = 0;
    double resid = beta;
    if (beta > 0.0) {
        // V_0 = rhs / beta, g_0 = beta
        BEM_LAUNCH(k_dots_partial, dim3(RED_BLOCKS, 1), 256, 0, s, rhs, n, ldv, rhs, W.partial.as<double2>());
        BEM_LAUNCH(k_dots_final, 1, 32, 0, s, W.partial.as<double2>(), 1, W.nrm.as<double2>(), 0);
        BEM_LAUNCH(k_normalize, eb, 256, 0, s, rhs, n, W.nrm.as<double2>(), Vp, W.g.as<double2>());
        for (int j = 0; j < W.maxit; ++j) {
            double2* vj = Vp + (int64_t)j * ldv;
            BEM_TRY(apply(vj, W.w.as<double2>()));
            double2* Hj = W.H.as<double2>() + (int64_t)j * ldh;
            for (int pass = 0; pass < 2; ++pass) {  // CGS2
                double2* h = pass == 0 ? Hj : W.hbuf.as<double2>();
                BEM_LAUNCH(k_dots_partial, dim3(RED_BLOCKS, j + 1), 256, 0, s, Vp, n, ldv, W.w.as<double2>(),
                           W.partial.as<double2>());
                BEM_LAUNCH(k_dots_final, j + 1, 32, 0, s, W.partial.as<double2>(), j + 1, h, 0);
                BEM_LAUNCH(k_combine, eb, 256, 0, s, Vp, n, ldv, j + 1, h, W.w.as<double2>(), 0);
            }
            BEM_LAUNCH(k_add, 1, 256, 0, s, Hj, W.hbuf.as<double2>(), j + 1);
            BEM_LAUNCH(k_dots_partial, dim3(RED_BLOCKS, 1), 256, 0, s, W.w.as<double2>(), n, ldv, W.w.as<double2>(),
                       W.partial.as<double2>());
            BEM_LAUNCH(k_dots_final, 1, 32, 0, s, W.partial.as<double2>(), 1, W.nrm.as<double2>(), 0);
            BEM_LAUNCH(k_normalize, eb, 256, 0, s, W.w.as<double2>(), n, W.nrm.as<double2>(),
                       Vp + (int64_t)(j + 1) * ldv, Hj + j + 1);
            BEM_LAUNCH(k_givens, 1, 32, 0, s, W.H.as<double2>(), ldh, j, W.cs.as<double>(), W.sn.as<double2>(),
                       W.g.as<double2>(), W.resd.as<double>());
            BEM_CUDA_TRY(cudaMemcpyAsync(W.h_res, W.resd.p, 8, cudaMemcpyDeviceToHost, s));
            BEM_CUDA_TRY(cudaStreamSynchronize(s));
            iters = j + 1;
            resid = W.h_res[0];
            if (!(resid > tol_abs)) break;
            if (stop) BEM_TRY(stop());
        }
    }
    if (iters > 0) {
        BEM_LAUNCH(k_backsolve, 1, 256, 0, s, W.H.as<double2>(), ldh, iters, W.g.as<double2>(), W.y.as<double2>(),
                   W.work.as<double2>());
        BEM_LAUNCH(k_combine, eb, 256, 0, s, Vp, n, ldv, iters, W.y.as<double2>(), x, 1);
    } else {
        BEM_CUDA_TRY(cudaMemsetAsync(x, 0, n * 16, s));
    }
    *iters_out = iters;
    *res_out = resid;
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
    // ---- operator application ------------------------------------------------------
    DevBuf wz, wr, wa, wb, x32;
    BEM_TRY(wz.alloc(n * 16, s)); BEM_TRY(wr.alloc(n * 16, s)); BEM_TRY(wa.alloc(n * 16, s)); BEM_TRY(wb.alloc(n * 16, s));
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
    Blocks B64{};
    Blocks32 B32{};
    if (mixed) {
        BEM_TRY(x32.alloc(n * 8, s));
        const float2* m1[4] = {M[1].as<float2>(), M[3].as<float2>(), M[5].as<float2>(), M[7].as<float2>()};
        const float2* m2[4] = {M[0].as<float2>(), M[2].as<float2>(), M[4].as<float2>(), M[6].as<float2>()};
        fill_blocks(B32, m1, m2, Ne, Ni);
    } else {
        const double2* m1[4] = {M[1].as<double2>(), M[3].as<double2>(), M[5].as<double2>(), M[7].as<double2>()};
        const double2* m2[4] = {M[0].as<double2>(), M[2].as<double2>(), M[4].as<double2>(), M[6].as<double2>()};
        fill_blocks(B64, m1, m2, Ne, Ni);
    }
    // S A x in the working precision (FP64, or FP32 arithmetic on complex64 storage)
    Apply apply_work = [&](const double2* xin, double2* yout) -> bem_status {
        if (mixed) {
            BEM_LAUNCH(k_to_c64, blocks_for(n, 256), 256, 0, s, xin, n, x32.as<float2>());
            BEM_LAUNCH(k_gemv_mtf32, blocks_for(n * 32, 256), 256, 0, s, B32, n, x32.as<float2>(), z);
        } else {
            BEM_LAUNCH(k_gemv_mtf, blocks_for(n * 32, 256), 256, 0, s, B64, n, xin, z);
        }
        BEM_TRY(transfer_add(top, Ne, Ni, xin, z, s));
        return mass_solve(mop, z, yout, s, mixed ? CHEB_STEPS_INNER : CHEB_STEPS);
    };
    // S A x with FP64 arithmetic on the stored matrices (outer residual of the refinement)
    Apply apply_fp64 = [&](const double2* xin, double2* yout) -> bem_status {
        if (mixed) BEM_LAUNCH(k_gemv_mtf_c64_f64, blocks_for(n * 32, 256), 256, 0, s, B32, n, xin, z);
        else BEM_LAUNCH(k_gemv_mtf, blocks_for(n * 32, 256), 256, 0, s, B64, n, xin, z);
        BEM_TRY(transfer_add(top, Ne, Ni, xin, z, s));
        return mass_solve(mop, z, yout, s);
    };
    // ---- GMRES ------------------------------------------------------------------------
    const int maxit = (int)std::min<int64_t>(o->gmres_maxiter, n);
    GmresWork W;
    BEM_TRY(W.init(maxit, n, s));
    DevBuf fvec, gvec, bvec, sb, xsol, dvec, rvec, tmp;
    BEM_TRY(fvec.alloc(Ne * 16, s)); BEM_TRY(gvec.alloc(Ne * 16, s)); BEM_TRY(bvec.alloc(n * 16, s));
    BEM_TRY(sb.alloc(n * 16, s)); BEM_TRY(xsol.alloc(n * 16, s)); BEM_TRY(dvec.alloc(n * 16, s));
    BEM_TRY(rvec.alloc(n * 16, s)); BEM_TRY(tmp.alloc(n * 16, s));
    bem_status result = BEM_OK;
    int total_inner = 0, outer_used = 0;
    double worst_res = 0.0;
    bool all_conv = true;
    const unsigned eb = blocks_for(n, 256);
    cudaEventRecord(t_sol.a, s);
    for (int rr = 0; rr < inc->n_rhs; ++rr) {
        double3 d = make_double3(inc->dirs[3 * rr], inc->dirs[3 * rr + 1], inc->dirs[3 * rr + 2]);
        double2 amp = inc->amps ? make_double2(inc->amps[rr].re, inc->amps[rr].im) : make_double2(1.0, 0.0);
        BEM_CUDA_TRY(cudaMemsetAsync(fvec.p, 0, Ne * 16, s));
        BEM_CUDA_TRY(cudaMemsetAsync(gvec.p, 0, Ne * 16, s));
        BEM_LAUNCH(k_plane_wave, blocks_for(ge->nt, 128), 128, 0, s, ge->rec.as<TriRec>(), ge->tri.as<int32_t>(),
                   ge->nt, k_ext.re, k_ext.im, d, amp, fvec.as<double2>(), gvec.as<double2>());
        BEM_LAUNCH(k_rhs_pack, eb, 256, 0, s, fvec.as<double2>(), gvec.as<double2>(), Ne, n, bvec.as<double2>());
        BEM_TRY(mass_solve(mop, bvec.as<double2>(), sb.as<double2>(), s));
        double beta = 0.0;
        BEM_TRY(norm2(W, sb.as<double2>(), &beta, s));
        const double tol_abs = o->gmres_tol * beta;
        int iters = 0;
        double rel = 0.0;
        if (!mixed) {
            double est = 0.0;
            BEM_TRY(gmres_run(W, apply_work, sb.as<double2>(), beta, tol_abs, xsol.as<double2>(), &iters, &est, s, stop));
            rel = beta > 0.0 ? est / beta : 0.0;
            total_inner += iters;
            outer_used = 1;
        } else {
            // iterative refinement: FP64 residual of the stored system, FP32-matvec GMRES corrections
            BEM_CUDA_TRY(cudaMemsetAsync(xsol.p, 0, n * 16, s));
            BEM_CUDA_TRY(cudaMemcpyAsync(rvec.p, sb.p, n * 16, cudaMemcpyDeviceToDevice, s));
            double rn = beta;
            int outer = 0;
            const int max_outer = 12;
            while (beta > 0.0 && rn > tol_abs && outer < max_outer && total_inner < o->gmres_maxiter) {
                const double inner_tol = std::max(tol_abs, o->ir_inner_tol * rn);
                int it = 0;
                double est = 0.0;
                BEM_TRY(gmres_run(W, apply_work, rvec.as<double2>(), rn, inner_tol, dvec.as<double2>(), &it, &est, s, stop));
                iters += it;
                total_inner += it;
                BEM_LAUNCH(k_acc, eb, 256, 0, s, xsol.as<double2>(), dvec.as<double2>(), n);
                BEM_TRY(apply_fp64(xsol.as<double2>(), tmp.as<double2>()));
                BEM_LAUNCH(k_sub, eb, 256, 0, s, sb.as<double2>(), tmp.as<double2>(), n, rvec.as<double2>());
                BEM_TRY(norm2(W, rvec.as<double2>(), &rn, s));
                ++outer;
                if (it == 0) break;
            }
            outer_used = std::max(outer_used, outer);
            rel = beta > 0.0 ? rn / beta : 0.0;
        }
        const bool conv = beta == 0.0 || rel <= o->gmres_tol;
        all_conv = all_conv && conv;
        worst_res = std::max(worst_res, rel);
        if (!conv) result = BEM_E_NOT_CONVERGED;
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        const double2* X = xsol.as<double2>();
        BEM_CUDA_TRY(cudaMemcpyAsync(v_ext + rr * Ne, X, Ne * 16, kind, s));
        BEM_CUDA_TRY(cudaMemcpyAsync(w_ext + rr * Ne, X + Ne, Ne * 16, kind, s));
        BEM_CUDA_TRY(cudaMemcpyAsync(v_int + rr * Ni, X + 2 * Ne, Ni * 16, kind, s));
        BEM_CUDA_TRY(cudaMemcpyAsync(w_int + rr * Ni, X + 2 * Ne + Ni, Ni * 16, kind, s));
        (void)iters;
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
