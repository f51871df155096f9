// Galerkin assembly of the Helmholtz boundary operators V, K, T, D on one P1 grid
// (paper Sec. 2.1 operator definitions, Sec. 2.4 P1 discretisation, Sec. 5.1
// quadrature: order-four rules with Sauter-Schwab transformations).
//
//   G(x,y)    = exp(i k r) / (4 pi r)
//   dG/dn(y)  = G (1 - i k r) ((x - y) . n(y)) / r^2
//   dG/dn(x)  = G (1 - i k r) ((y - x) . n(x)) / r^2
//   D_ij      = int int G [curl theta_i . curl phi_j - k^2 (n_x . n_y) theta_i phi_j]   (Maue)
//
// Regular pairs (no common vertex): tensor product of the 6-point degree-4 rule.
// Each unordered pair {tau, sigma} is integrated once: the same point pairs give
// V_{tau,sigma}, K_{tau,sigma} (normal of sigma) and T_{tau,sigma} (normal of tau);
// by the symmetry of G, V and D are symmetric and K_{sigma,tau} = T_{tau,sigma}^T,
// so the four matrices are written in both orientations.
// CTA tile: TB test triangles x TB trial triangles of the upper tile triangle;
// geometry is staged in shared memory (the trial side in field-major order so that
// the 32 lanes of a warp read consecutive words); each thread integrates whole
// triangle pairs and scatters its 3x3 blocks with FP64 atomics (the FP64 pipe, not
// the scatter, bounds this kernel).
//
// Singular pairs (coincident / edge / vertex): one warp per pair, lanes stride the
// Sauter-Schwab points, a butterfly reduction sums the 3x3 blocks.
#include "bem_internal.cuh"
#include "ddf.cuh"

namespace bem {

namespace {

constexpr int TB = 32;
constexpr int NTHREADS = 256;
constexpr double INV_4PI = 0.07957747154594767;  // 1 / (4 pi)

struct KParams {
    double kr, ki;        // wavenumber
    double k2r, k2i;      // k^2
    int64_t n;            // matrix order (vertices)
    int nt;               // 64 x 64 tiles per side (tiled layouts)
    int lay[4];           // storage layouts of V, K, T, D (OP_DENSE, OP_FULL, OP_SYM)
};

struct TrialTile {
    double q[6][3][TB];
    double wl[6][3][TB];
    float wlh[6][3][TB], wll[6][3][TB];  // the weights split into FP32 pairs (double-float sums)
    double n[3][TB];
    double curl[3][3][TB];
    int32_t v[3][TB];
};

// double-float accumulator: value h plus collected error c
struct DDAcc {
    float h, c;
};

__device__ __forceinline__ void kernel_values(bool complex_k, const KParams& P, double dx, double dy, double dz,
                                              double& Gr, double& Gi, double& Fr, double& Fi) {
    double r2 = dx * dx + dy * dy + dz * dz;
    double rinv = rsqrt(r2);
    double r = r2 * rinv;
    double ph = P.kr * r;
    double sn, cs;
    sincos(ph, &sn, &cs);
    double g = rinv * INV_4PI;
    if (complex_k) g *= exp(-P.ki * r);
    Gr = g * cs;
    Gi = g * sn;
    // F = G (1 - i k r) / r^2 with k = kr + i ki: (1 + ki r) - i kr r
    double ar = complex_k ? 1.0 + P.ki * r : 1.0;
    double ai = -ph;
    double ri2 = rinv * rinv;
    Fr = (Gr * ar - Gi * ai) * ri2;
    Fi = (Gr * ai + Gi * ar) * ri2;
}

__device__ __forceinline__ void add2(double2* M, int64_t idx, double re, double im) {
    if (idx < 0) return;  // a symmetric layout keeps the mirror entry, added by the caller too
    atomicAdd(&M[idx].x, re);
    atomicAdd(&M[idx].y, im);
}
__device__ __forceinline__ void add2(float2* M, int64_t idx, double re, double im) {
    if (idx < 0) return;
    atomicAdd(&M[idx], make_float2((float)re, (float)im));
}
// storage index of entry (i, j) of operator op (0 V, 1 K, 2 T, 3 D)
__device__ __forceinline__ int64_t at(const KParams& P, int op, int64_t i, int64_t j) {
    return op_index(P.lay[op], P.n, P.nt, i, j);
}

template <bool CK>
__global__ void __launch_bounds__(NTHREADS, 1)
k_regular(const TriRec* __restrict__ rec, const int32_t* __restrict__ tri, int64_t nt, KParams P,
          double2* __restrict__ V, double2* __restrict__ K, double2* __restrict__ T, double2* __restrict__ D) {
    const int it = blockIdx.y, is = blockIdx.x;
    if (it > is) return;
    __shared__ TriRec test[TB];
    __shared__ int32_t testv[TB][3];
    __shared__ TrialTile trial;
    const int64_t t0 = (int64_t)it * TB, s0 = (int64_t)is * TB;
    // stage geometry
    {
        const double* src = reinterpret_cast<const double*>(rec + t0);
        double* dst = reinterpret_cast<double*>(test);
        int64_t avail = nt - t0 < TB ? nt - t0 : TB;
        for (int e = threadIdx.x; e < TB * TRIREC_DOUBLES; e += NTHREADS)
            dst[e] = (e / TRIREC_DOUBLES < avail) ? src[e] : 0.0;
        for (int e = threadIdx.x; e < TB * 3; e += NTHREADS)
            testv[e / 3][e % 3] = (e / 3 < avail) ? tri[3 * t0 + e] : -1;
        int64_t savail = nt - s0 < TB ? nt - s0 : TB;
        for (int e = threadIdx.x; e < TB * 49; e += NTHREADS) {
            int s = e % TB, f = e / TB;  // field-major gather
            double val = (s < savail) ? reinterpret_cast<const double*>(rec + s0 + s)[f] : 0.0;
            if (f < 18) trial.q[f / 3][f % 3][s] = val;
            else if (f < 36) trial.wl[(f - 18) / 3][(f - 18) % 3][s] = val;
            else if (f < 39) trial.n[f - 36][s] = val;
            else if (f == 39) { /* J unused */ }
            else trial.curl[(f - 40) / 3][(f - 40) % 3][s] = val;
        }
        for (int e = threadIdx.x; e < TB * 3; e += NTHREADS) {
            int s = e % TB, a = e / TB;
            trial.v[a][s] = (s < savail) ? tri[3 * (s0 + s) + a] : -1;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < TB * 18; e += NTHREADS) {
        const int s = e % TB, f = e / TB;
        ddf::split(trial.wl[f / 3][f % 3][s], trial.wlh[f / 3][f % 3][s], trial.wll[f / 3][f % 3][s]);
    }
    __syncthreads();
    for (int pidx = threadIdx.x; pidx < TB * TB; pidx += NTHREADS) {
        const int tl = pidx / TB, sl = pidx % TB;
        if (t0 + tl >= nt || s0 + sl >= nt) continue;
        if (it == is && tl >= sl) continue;
        const int32_t ta = testv[tl][0], tb = testv[tl][1], tc = testv[tl][2];
        const int32_t sa = trial.v[0][sl], sb = trial.v[1][sl], sc = trial.v[2][sl];
        const bool touch = (ta == sa) | (ta == sb) | (ta == sc) | (tb == sa) | (tb == sb) | (tb == sc) |
                           (tc == sa) | (tc == sb) | (tc == sc);
        if (touch) continue;  // singular pair: Sauter-Schwab kernel
        const TriRec& tr = test[tl];
        const double nsx = trial.n[0][sl], nsy = trial.n[1][sl], nsz = trial.n[2][sl];
        const double ntx = tr.n[0], nty = tr.n[1], ntz = tr.n[2];
        // sums over the 36 point pairs in double-float on the FP32 pipe (the kernel values are
        // FP64): GB300's FP64 pipe, 1/64 of the FP32 rate, keeps only the geometry and the
        // kernel evaluation.  A[0..5][a][b] = V re, V im, K re, K im, T re, T im
        DDAcc A[6][3][3];
#pragma unroll
        for (int o = 0; o < 6; ++o)
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) A[o][a][b] = DDAcc{0.f, 0.f};
#pragma unroll 1
        for (int p = 0; p < 6; ++p) {
            const double xx = tr.q[p][0], xy = tr.q[p][1], xz = tr.q[p][2];
            DDAcc S[6][3];
#pragma unroll
            for (int o = 0; o < 6; ++o)
#pragma unroll
                for (int b = 0; b < 3; ++b) S[o][b] = DDAcc{0.f, 0.f};
#pragma unroll 2
            for (int q = 0; q < 6; ++q) {
                const double dx = xx - trial.q[q][0][sl], dy = xy - trial.q[q][1][sl], dz = xz - trial.q[q][2][sl];
                double Gr, Gi, Fr, Fi;
                kernel_values(CK, P, dx, dy, dz, Gr, Gi, Fr, Fi);
                const double dns = dx * nsx + dy * nsy + dz * nsz;
                const double dnt = -(dx * ntx + dy * nty + dz * ntz);
                float grh, grl, gih, gil, frh, frl, fih, fil, nsh, nsl, nth, ntl;
                ddf::split(Gr, grh, grl);
                ddf::split(Gi, gih, gil);
                ddf::split(Fr, frh, frl);
                ddf::split(Fi, fih, fil);
                ddf::split(dns, nsh, nsl);
                ddf::split(dnt, nth, ntl);
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const float wh = trial.wlh[q][b][sl], wlo = trial.wll[q][b][sl];
                    ddf::mac(S[0][b].h, S[0][b].c, wh, wlo, grh, grl);
                    ddf::mac(S[1][b].h, S[1][b].c, wh, wlo, gih, gil);
                    // w (x - y).n as a double-float pair, times F
                    const float csh = __fmul_rn(wh, nsh);
                    const float csl = fmaf(wlo, nsh, fmaf(wh, nsl, fmaf(wh, nsh, -csh)));
                    const float cth = __fmul_rn(wh, nth);
                    const float ctl = fmaf(wlo, nth, fmaf(wh, ntl, fmaf(wh, nth, -cth)));
                    ddf::mac(S[2][b].h, S[2][b].c, csh, csl, frh, frl);
                    ddf::mac(S[3][b].h, S[3][b].c, csh, csl, fih, fil);
                    ddf::mac(S[4][b].h, S[4][b].c, cth, ctl, frh, frl);
                    ddf::mac(S[5][b].h, S[5][b].c, cth, ctl, fih, fil);
                }
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float wh, wlo;
                ddf::split(tr.wl[p][a], wh, wlo);
#pragma unroll
                for (int o = 0; o < 6; ++o)
#pragma unroll
                    for (int b = 0; b < 3; ++b) ddf::mac(A[o][a][b].h, A[o][a][b].c, wh, wlo, S[o][b].h, S[o][b].c);
            }
        }
        double Vr[3][3], Vi[3][3], Kr[3][3], Ki[3][3], Tr[3][3], Ti[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                Vr[a][b] = ddf::widen(A[0][a][b].h) + ddf::widen(A[0][a][b].c);
                Vi[a][b] = ddf::widen(A[1][a][b].h) + ddf::widen(A[1][a][b].c);
                Kr[a][b] = ddf::widen(A[2][a][b].h) + ddf::widen(A[2][a][b].c);
                Ki[a][b] = ddf::widen(A[3][a][b].h) + ddf::widen(A[3][a][b].c);
                Tr[a][b] = ddf::widen(A[4][a][b].h) + ddf::widen(A[4][a][b].c);
                Ti[a][b] = ddf::widen(A[5][a][b].h) + ddf::widen(A[5][a][b].c);
            }
        double I0r = 0, I0i = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                I0r += Vr[a][b];
                I0i += Vi[a][b];
            }
        const double nn = ntx * nsx + nty * nsy + ntz * nsz;
        const int32_t tv[3] = {ta, tb, tc}, sv[3] = {sa, sb, sc};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const int64_t i = tv[a], j = sv[b];
                if (V) { add2(V, at(P, 0, i, j), Vr[a][b], Vi[a][b]); add2(V, at(P, 0, j, i), Vr[a][b], Vi[a][b]); }
                if (K) { add2(K, at(P, 1, i, j), Kr[a][b], Ki[a][b]); add2(K, at(P, 1, j, i), Tr[a][b], Ti[a][b]); }
                if (T) { add2(T, at(P, 2, i, j), Tr[a][b], Ti[a][b]); add2(T, at(P, 2, j, i), Kr[a][b], Ki[a][b]); }
                if (D) {
                    const double cc = tr.curl[a][0] * trial.curl[b][0][sl] + tr.curl[a][1] * trial.curl[b][1][sl] +
                                      tr.curl[a][2] * trial.curl[b][2][sl];
                    // D = cc I0 - k^2 nn V
                    const double dr = cc * I0r - nn * (P.k2r * Vr[a][b] - P.k2i * Vi[a][b]);
                    const double di = cc * I0i - nn * (P.k2r * Vi[a][b] + P.k2i * Vr[a][b]);
                    add2(D, at(P, 3, i, j), dr, di);
                    add2(D, at(P, 3, j, i), dr, di);
                }
            }
        }
    }
}

// One warp per singular pair.  Pairs [0, nt) are coincident (tau = sigma = w);
// then the edge- and vertex-adjacent list.
template <bool CK, typename Out>
__global__ void __launch_bounds__(128)
k_singular(const double* __restrict__ xyz, const int32_t* __restrict__ tri, const TriRec* __restrict__ rec,
           const SingPair* __restrict__ pairs, int64_t nt, int64_t npairs, const double* __restrict__ ss,
           int3 count, int3 offset, KParams P, Out* __restrict__ V, Out* __restrict__ K,
           Out* __restrict__ T, Out* __restrict__ D) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nt + npairs) return;
    int32_t t, s;
    int pt[3], ps[3], kind;
    if (w < nt) {
        t = s = (int32_t)w;
        pt[0] = ps[0] = 0; pt[1] = ps[1] = 1; pt[2] = ps[2] = 2;
        kind = 0;
    } else {
        const SingPair sp = pairs[w - nt];
        t = sp.t; s = sp.s;
        for (int m = 0; m < 3; ++m) { pt[m] = sp.pt[m]; ps[m] = sp.ps[m]; }
        kind = sp.kind;
    }
    // reordered vertex coordinates (Sauter-Schwab A, B, C)
    double X[3][3], Y[3][3];
    for (int m = 0; m < 3; ++m) {
        const int32_t iv = tri[3 * (int64_t)t + pt[m]], jv = tri[3 * (int64_t)s + ps[m]];
        for (int d = 0; d < 3; ++d) {
            X[m][d] = xyz[3 * (int64_t)iv + d];
            Y[m][d] = xyz[3 * (int64_t)jv + d];
        }
    }
    const TriRec& rt = rec[t];
    const TriRec& rs = rec[s];
    const double nt0 = rt.n[0], nt1 = rt.n[1], nt2 = rt.n[2];
    const double ns0 = rs.n[0], ns1 = rs.n[1], ns2 = rs.n[2];
    const double JJ = rt.J * rs.J;
    const int cnt = kind == 0 ? count.x : (kind == 1 ? count.y : count.z);
    const int off = kind == 0 ? offset.x : (kind == 1 ? offset.y : offset.z);
    // the 54 sums (3 x 3 blocks of V, K, T as re, im) in double-float on the FP32 pipe:
    // the kernel values are formed in FP64, each sum term (w_q L_a L_b times a kernel
    // value) is added as an exact FP32 product plus its rounded cross terms, every
    // rounding error collected in a second word (ddf.cuh); GB300's FP64 pipe (1/64 of
    // the FP32 rate) is left with the geometry and the kernel values
    float ah[54], ac[54];
#pragma unroll
    for (int e = 0; e < 54; ++e) ah[e] = ac[e] = 0.0f;
    for (int e = lane; e < cnt; e += 32) {
        const double* pnt = ss + 5 * (int64_t)(off + e);
        const double x1 = pnt[0], x2 = pnt[1], y1 = pnt[2], y2 = pnt[3], wq = pnt[4] * JJ;
        const double bx[3] = {1.0 - x1, x1 - x2, x2}, by[3] = {1.0 - y1, y1 - y2, y2};
        double x[3], y[3];
        for (int d = 0; d < 3; ++d) {
            x[d] = bx[0] * X[0][d] + bx[1] * X[1][d] + bx[2] * X[2][d];
            y[d] = by[0] * Y[0][d] + by[1] * Y[1][d] + by[2] * Y[2][d];
        }
        // shape values in the triangles' own vertex order: L[perm[m]] = b[m]
        double Lx[3], Ly[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Lx[a] = pt[0] == a ? bx[0] : (pt[1] == a ? bx[1] : bx[2]);
            Ly[a] = ps[0] == a ? by[0] : (ps[1] == a ? by[1] : by[2]);
        }
        const double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
        double Gr, Gi, Fr, Fi;
        kernel_values(CK, P, dx, dy, dz, Gr, Gi, Fr, Fi);
        const double dns = dx * ns0 + dy * ns1 + dz * ns2;
        const double dnt = -(dx * nt0 + dy * nt1 + dz * nt2);
        float ch[9], cl[9];
        {
            float xh[3], xl[3], yh[3], yl[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                ddf::split(wq * Lx[a], xh[a], xl[a]);
                ddf::split(Ly[a], yh[a], yl[a]);
            }
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {  // w_q L_a L_b as a double-float pair
                    ch[3 * a + b] = __fmul_rn(xh[a], yh[b]);
                    cl[3 * a + b] =
                        fmaf(xl[a], yh[b], fmaf(xh[a], yl[b], fmaf(xh[a], yh[b], -ch[3 * a + b])));
                }
        }
        const double kv[6] = {Gr, Gi, dns * Fr, dns * Fi, dnt * Fr, dnt * Fi};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float kh, kl;
            ddf::split(kv[k], kh, kl);
#pragma unroll
            for (int e9 = 0; e9 < 9; ++e9) ddf::mac(ah[9 * k + e9], ac[9 * k + e9], ch[e9], cl[e9], kh, kl);
        }
    }
#pragma unroll
    for (int e = 0; e < 54; ++e)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float qh = __shfl_xor_sync(0xffffffffu, ah[e], o), qc = __shfl_xor_sync(0xffffffffu, ac[e], o);
            float t;
            ddf::two_sum(ah[e], qh, ah[e], t);
            ac[e] = __fadd_rn(ac[e], __fadd_rn(qc, t));
        }
    // lanes 0..8 each write one (a, b) entry: stage the sums in shared memory so that
    // no register array is indexed by the lane number
    __shared__ double red[4][54];
    double* rw = red[(threadIdx.x >> 5) & 3];
    if (lane == 0) {
#pragma unroll
        for (int e = 0; e < 54; ++e) rw[e] = ddf::widen(ah[e]) + ddf::widen(ac[e]);
    }
    __syncwarp();
    if (lane >= 9) return;
    const int a = lane / 3, b = lane % 3;
    double I0r = 0, I0i = 0;
#pragma unroll
    for (int e = 0; e < 9; ++e) { I0r += rw[e]; I0i += rw[9 + e]; }
    const int e9 = lane;
    const double vr = rw[e9], vi = rw[9 + e9], kr = rw[18 + e9], ki = rw[27 + e9], tr = rw[36 + e9],
                 ti = rw[45 + e9];
    const double cc = rt.curl[a][0] * rs.curl[b][0] + rt.curl[a][1] * rs.curl[b][1] + rt.curl[a][2] * rs.curl[b][2];
    const double nn = nt0 * ns0 + nt1 * ns1 + nt2 * ns2;
    const double dr = cc * I0r - nn * (P.k2r * vr - P.k2i * vi);
    const double di = cc * I0i - nn * (P.k2r * vi + P.k2i * vr);
    const int64_t iv = tri[3 * (int64_t)t + a], jv = tri[3 * (int64_t)s + b];
    if (V) add2(V, at(P, 0, iv, jv), vr, vi);
    if (K) add2(K, at(P, 1, iv, jv), kr, ki);
    if (T) add2(T, at(P, 2, iv, jv), tr, ti);
    if (D) add2(D, at(P, 3, iv, jv), dr, di);
    if (kind != 0) {
        if (V) add2(V, at(P, 0, jv, iv), vr, vi);
        if (K) add2(K, at(P, 1, jv, iv), tr, ti);
        if (T) add2(T, at(P, 2, jv, iv), kr, ki);
        if (D) add2(D, at(P, 3, jv, iv), dr, di);
    }
}

}  // namespace

static KParams kparams(const bem_grid* g, double k_re, double k_im, const OpLayouts& L) {
    KParams P;
    P.kr = k_re;
    P.ki = k_im;
    P.k2r = k_re * k_re - k_im * k_im;
    P.k2i = 2.0 * k_re * k_im;
    P.n = g->nv;
    P.nt = op_tiles(g->nv);
    for (int i = 0; i < 4; ++i) P.lay[i] = L.lay[i];
    return P;
}

bem_status assemble_operators_fp64(const bem_grid* g, double k_re, double k_im, int n_singular, double2* V,
                                   double2* K, double2* T, double2* D, const OpLayouts& L, cudaStream_t s) {
    const int64_t N = g->nv, nt = g->nt;
    double2* const ops[4] = {V, K, T, D};
    for (int o = 0; o < 4; ++o)
        if (ops[o]) BEM_CUDA_TRY(cudaMemsetAsync(ops[o], 0, op_entries(L.lay[o], N) * sizeof(double2), s));
    const KParams P = kparams(g, k_re, k_im, L);
    const bool ck = k_im != 0.0;
    const int64_t ntile = (nt + TB - 1) / TB;
    if (ntile > 65535) {
        set_error("grid too large for the tile grid (more than 2M triangles)");
        return BEM_E_INVALID_ARG;
    }
    dim3 grid((unsigned)ntile, (unsigned)ntile);
    if (ck)
        BEM_LAUNCH(k_regular<true>, grid, NTHREADS, 0, s, g->rec.as<TriRec>(), g->tri.as<int32_t>(), nt, P, V, K, T, D);
    else
        BEM_LAUNCH(k_regular<false>, grid, NTHREADS, 0, s, g->rec.as<TriRec>(), g->tri.as<int32_t>(), nt, P, V, K, T, D);
    BEM_CHECK_LAUNCH();
    const double* ss;
    int cnt[3], off[3];
    BEM_TRY(ss_table_get(n_singular, s, &ss, cnt, off));
    const int64_t npairs = g->n_edge + g->n_vertex;
    const int64_t warps = nt + npairs;
    const unsigned blocks = (unsigned)((warps * 32 + 127) / 128);
    int3 c3 = make_int3(cnt[0], cnt[1], cnt[2]), o3 = make_int3(off[0], off[1], off[2]);
    if (ck)
        BEM_LAUNCH((k_singular<true, double2>), blocks, 128, 0, s, g->xyz.as<double>(), g->tri.as<int32_t>(), g->rec.as<TriRec>(),
                                                g->sing.as<SingPair>(), nt, npairs, ss, c3, o3, P, V, K, T, D);
    else
        BEM_LAUNCH((k_singular<false, double2>), blocks, 128, 0, s, g->xyz.as<double>(), g->tri.as<int32_t>(), g->rec.as<TriRec>(),
                                                 g->sing.as<SingPair>(), nt, npairs, ss, c3, o3, P, V, K, T, D);
    BEM_CHECK_LAUNCH();
    return BEM_OK;
}

bem_status assemble_singular_into_c64(const bem_grid* g, double k_re, double k_im, int n_singular, float2* V,
                                      float2* K, float2* T, float2* D, const OpLayouts& L, cudaStream_t s) {
    const KParams P = kparams(g, k_re, k_im, L);
    const double* ss;
    int cnt[3], off[3];
    BEM_TRY(ss_table_get(n_singular, s, &ss, cnt, off));
    const int64_t npairs = g->n_edge + g->n_vertex, nt = g->nt;
    const unsigned blocks = (unsigned)(((nt + npairs) * 32 + 127) / 128);
    int3 c3 = make_int3(cnt[0], cnt[1], cnt[2]), o3 = make_int3(off[0], off[1], off[2]);
    if (k_im != 0.0)
        BEM_LAUNCH((k_singular<true, float2>), blocks, 128, 0, s, g->xyz.as<double>(), g->tri.as<int32_t>(),
                   g->rec.as<TriRec>(), g->sing.as<SingPair>(), nt, npairs, ss, c3, o3, P, V, K, T, D);
    else
        BEM_LAUNCH((k_singular<false, float2>), blocks, 128, 0, s, g->xyz.as<double>(), g->tri.as<int32_t>(),
                   g->rec.as<TriRec>(), g->sing.as<SingPair>(), nt, npairs, ss, c3, o3, P, V, K, T, D);
    return BEM_OK;
}

}  // namespace bem
