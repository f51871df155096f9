// Regular-pair Galerkin assembly of V, K, T, D in FP32 on GB300's FP32 pipe (the
// mixed-precision mode; the operators and quadrature are those of assemble.cu:
// paper Sec. 2.1, Sec. 2.4, Sec. 5.1).  Results go to complex64 matrices.
//
// Accuracy design (target: relative entry errors ~1e-7, the FP32 storage rounding):
//  * geometry is stored relative to each triangle's centroid, so quadrature-point
//    offsets are small and exact to FP32 rounding;
//  * per triangle pair the centroid distance R = |c_tau - c_sigma| and the phase
//    reference k R mod 2 pi are formed in double-float arithmetic (two FP32 words,
//    error-free transformations), and exp(i k R) is evaluated once per pair;
//  * per point pair only the small offset delta = r - R enters the phase:
//    delta = (2 D.w + |w|^2) / (r + R) with D = c_tau - c_sigma and w the difference
//    of the centroid offsets, so exp(i k r) = exp(i k R) exp(i k delta) keeps an
//    absolute phase error ~1e-7 even where k r is large;
//  * the 3x3 blocks of a CTA's triangle pairs are summed in shared memory in fixed
//    point, with native integer atomics (FP32 atomic adds on shared memory are
//    compare-and-swap loops): each CTA first bounds every value it will produce
//    (smallest and largest point distance of its regular pairs, largest weight sums,
//    areas and curls, |k|), picks a power-of-two scale 2^e that maps the bound to
//    2^40, and adds round(v 2^e) split into a high word (units of 2^21) and a low
//    word, both int32.  A vertex lies in at most 32 triangles of a tile, so at most
//    1024 values meet in one entry and neither word can overflow; the in-tile sums
//    are exact (and independent of the order of the atomics) to 2^-40 of the bound.
// The tile buffers are flushed to the global matrices with vector float2 atomics.
#include "bem_internal.cuh"

#include <algorithm>
#include <vector>

namespace bem {

namespace {

constexpr int NT32 = 512;  // threads per CTA
constexpr float INV_4PI_F = 0.0795774715459476679f;

struct KP32 {
    float k_h, k_l;      // real wavenumber as a double-float pair
    float k_i;           // imaginary part
    float k2r, k2i;      // k^2
    int64_t n;           // matrix order
};

// ---- double-float helpers (error-free transformations) ----
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    e = b - (s - a);
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);  // never contracted into a following sum
    e = fmaf(a, b, -p);
}

// sin and cos of a moderate FP32 argument (|x| < 2^15): Cody-Waite reduction by
// pi/2 with a three-part constant (the first part has 8 significant bits, so n * P1 is
// exact), then the Taylor series of sin and cos on |r| <= pi/4 (truncation below
// 2e-9), evaluated by Horner's rule in r^2; the quadrant selects signs and swaps.
// Returned as a (cos, sin) pair; the two Horner recurrences run together as packed
// FP32x2 FMAs.
__device__ __forceinline__ float2 sincos_moderate2(float x) {
    const float n = rintf(x * 0.636619772367581343f);  // 2 / pi
    float r = fmaf(-n, 1.5703125f, x);                  // pi/2 = P1 + P2 + P3
    r = fmaf(-n, 4.838267923332751e-4f, r);
    r = fmaf(-n, 2.5632829192545614e-12f, r);
    const float r2 = r * r;
    const float2 R2 = make_float2(r2, r2);
    // (sin, cos) series in r^2: (1/9!, -1/10!) ... as in sincos_moderate
    float2 P = __ffma2_rn(R2, make_float2(2.75573192239858907e-6f, -2.75573192239858907e-7f),
                          make_float2(-1.98412698412698413e-4f, 2.48015873015873016e-5f));
    P = __ffma2_rn(R2, P, make_float2(8.33333333333333333e-3f, -1.38888888888888889e-3f));
    P = __ffma2_rn(R2, P, make_float2(-1.66666666666666667e-1f, 4.16666666666666667e-2f));
    const float sr = fmaf(r * r2, P.x, r);
    const float pc = fmaf(r2, P.y, -0.5f);
    const float cr = fmaf(r2, pc, 1.0f);
    const int q = ((int)n) & 3;
    const float ss = (q & 1) ? cr : sr, cc = (q & 1) ? sr : cr;
    return make_float2(((q + 1) & 2) ? -cc : cc, (q & 2) ? -ss : ss);
}

// sin and cos of a small FP32 argument (|x| <= pi/4, no reduction): the same Taylor
// series as sincos_moderate2 on r = x, returned as (cos, sin).
__device__ __forceinline__ float2 sincos_small2(float r) {
    const float r2 = r * r;
    const float2 R2 = make_float2(r2, r2);
    float2 P = __ffma2_rn(R2, make_float2(2.75573192239858907e-6f, -2.75573192239858907e-7f),
                          make_float2(-1.98412698412698413e-4f, 2.48015873015873016e-5f));
    P = __ffma2_rn(R2, P, make_float2(8.33333333333333333e-3f, -1.38888888888888889e-3f));
    P = __ffma2_rn(R2, P, make_float2(-1.66666666666666667e-1f, 4.16666666666666667e-2f));
    const float sr = fmaf(r * r2, P.x, r);
    const float pc = fmaf(r2, P.y, -0.5f);
    return make_float2(fmaf(r2, pc, 1.0f), sr);
}

struct TrialTile32 {
    float ch[3][TILE_TRI], cl[3][TILE_TRI];
    float u[6][3][TILE_TRI];
    float2 wl2[6][3][TILE_TRI];  // w_q J lambda_b(q), duplicated (an FP32x2 operand)
    float n[3][TILE_TRI];
    float curl[3][3][TILE_TRI];
    int32_t v[3][TILE_TRI];
    uint32_t slot[TILE_TRI];
};

// fixed-point shared-memory accumulation (see the header): value v at scale 2^e.
// c = v 2^e (|c| < 2^41) is split with FP32 operations only (a conversion to a
// 64-bit integer would run on the FP64 pipe, 1/64 of the FP32 rate on this part):
// h = rint(c 2^-21) and l = c - h 2^21 are exact, |h|, |l| <= 2^20, and adding
// 1.5 * 2^23 to a float of magnitude below 2^22 leaves rint(x) in its low mantissa
// bits.  Both words are signed; at most 1024 values meet in one entry, so neither
// 32-bit sum can overflow.
constexpr float FX_LIMIT = 2199023255552.0f;  // 2^41: twice the bound that sets the scale
constexpr float FX_MAGIC = 12582912.0f;       // 1.5 * 2^23
constexpr int FX_MAGIC_BITS = 0x4B400000;     // its bit pattern

__device__ __forceinline__ void fx_add(int32_t* H, int32_t* L, int idx, float v, float scale, int* overflow) {
    const float c = v * scale;
    if (!(fabsf(c) < FX_LIMIT)) {  // the bound was violated (or v is not finite)
        *overflow = 1;
        return;
    }
    const float th = fmaf(c, 4.76837158203125e-7f, FX_MAGIC);  // c 2^-21 + magic
    const float h = th - FX_MAGIC;                              // rint(c 2^-21)
    const float l = fmaf(-h, 2097152.0f, c);                    // c - h 2^21, exact
    const int32_t hi = __float_as_int(th) - FX_MAGIC_BITS;
    const int32_t lo = __float_as_int(l + FX_MAGIC) - FX_MAGIC_BITS;
    // unconditional: skipping zero words costs more (tests, divergence) than it saves
    atomicAdd(&L[idx], lo);
    atomicAdd(&H[idx], hi);
}

// largest |v| of a positive float kept as its bit pattern (monotone for x >= 0)
__device__ __forceinline__ void smax(float* a, float v) { atomicMax(reinterpret_cast<int*>(a), __float_as_int(v)); }
__device__ __forceinline__ void smin(float* a, float v) { atomicMin(reinterpret_cast<int*>(a), __float_as_int(v)); }

// true for a regular (non-touching) pair of the tile pair (it, is)
__device__ __forceinline__ bool regular_pair(int it, int is, int tl, int sl, const int32_t (*testv)[3],
                                             const TrialTile32* trial) {
    if (it == is && tl >= sl) return false;
    const int32_t ta = testv[tl][0], tb = testv[tl][1], tc = testv[tl][2];
    const int32_t sa = trial->v[0][sl], sb = trial->v[1][sl], sc = trial->v[2][sl];
    return !((ta == sa) | (ta == sb) | (ta == sc) | (tb == sa) | (tb == sb) | (tb == sc) | (tc == sa) |
             (tc == sb) | (tc == sc));
}

// everything one regular-pair tile pair needs from its grid
struct Grid32 {
    const TriRec32* rec;
    const int32_t* tverts;
    const uint32_t* tslots;
    const int32_t* tstart;
    const int32_t* vstart;
    const int32_t* tvert;
    KP32 P;
    float2 *Vm, *Km, *Tm, *Dm;
    int* err;
    int ck;      // complex wavenumber
    int nt;      // 64 x 64 tiles per side (tiled layouts)
    int lay[4];  // storage layouts of V, K, T, D
};

// The regular pairs of test tile it and trial tile is: kernel values at the 6 x 6 point
// pairs of each triangle pair, their 3x3 blocks summed in fixed point into acc.  SMALL:
// every phase offset k delta of the tile pair is below pi/4 (no argument reduction).
template <bool CK, bool SMALL>
__device__ __forceinline__ void regular32_pairs(const Grid32& G, const int it, const int is, const int nI,
                                                const int nJ, const TriRec32* test, const TrialTile32* trial,
                                                const int32_t (*testv)[3], const uint32_t* testslot, int32_t* acc,
                                                const float scale, int* overflow) {
    const KP32 P = G.P;
    constexpr int SLAB = TILE_NV * TILE_NV;
    const float tp_h = 6.28318548202514648f, tp_l = -1.7484555314695172e-7f;  // 2 pi as hi + lo
    const float inv_tp = 0.159154943091895336f;
    for (int pidx = threadIdx.x; pidx < TILE_TRI * TILE_TRI; pidx += NT32) {
        const int tl = pidx / TILE_TRI, sl = pidx % TILE_TRI;
        if (tl >= nI || sl >= nJ || !regular_pair(it, is, tl, sl, testv, trial)) continue;
        const TriRec32& tr = test[tl];
        // ---- per-pair reference in double-float: D = c_tau - c_sigma, R, exp(i k R)
        float Dh[3], R2h = 0.f, R2l = 0.f;
        for (int d = 0; d < 3; ++d) {
            float s, e;
            two_sum(tr.ch[d], -trial->ch[d][sl], s, e);
            e += tr.cl[d] - trial->cl[d][sl];
            float dh, dl;
            fast_two_sum(s, e, dh, dl);
            Dh[d] = dh;
            float p, pe;
            two_prod(dh, dh, p, pe);
            pe += 2.0f * dh * dl;
            float ns, ne;
            two_sum(R2h, p, ns, ne);
            ne += R2l + pe;
            fast_two_sum(ns, ne, R2h, R2l);
        }
        // R = sqrt(R^2) as a double-float: one Newton correction of the FP32 root
        const float r0 = sqrtf(R2h);
        float Rh, Rlo;
        fast_two_sum(r0, (fmaf(-r0, r0, R2h) + R2l) / (2.0f * r0), Rh, Rlo);
        // k R as a double-float, reduced modulo 2 pi (the multiple of 2 pi is subtracted
        // exactly: two_prod for n * (2 pi)_hi, Sterbenz for the leading difference)
        float ph, pe;
        two_prod(P.k_h, Rh, ph, pe);
        pe += P.k_h * Rlo + P.k_l * Rh;
        float Ph, Pl;
        fast_two_sum(ph, pe, Ph, Pl);
        const float nn = rintf(Ph * inv_tp);
        float mh, ml;
        two_prod(nn, tp_h, mh, ml);
        float th, tl2;
        fast_two_sum(Ph - mh, Pl - ml - nn * tp_l, th, tl2);
        float sn0, cs0;
        sincosf(th, &sn0, &cs0);
        {  // exp(i (th + tl2)) = exp(i th) (1 + i tl2) to FP32 rounding
            const float c1 = cs0 - sn0 * tl2, s1 = sn0 + cs0 * tl2;
            cs0 = c1;
            sn0 = s1;
        }
        // exp(i k R), times exp(-k_i R) for a complex wavenumber
        const float amp0 = CK ? expf(-P.k_i * Rh) : 1.0f;
        {
            // complex values as (re, im) pairs, products with real scalars as packed
            // FP32x2 FMAs: E0 = exp(i k R) as (E0r, E0r) and (-E0i, E0i) for E0 (c, s)
            const float E0r = amp0 * cs0, E0i = amp0 * sn0;
            const float2 E0rr = make_float2(E0r, E0r), E0im = make_float2(-E0i, E0i);
            const float R2f = R2h + R2l;
            const float Dns = Dh[0] * trial->n[0][sl] + Dh[1] * trial->n[1][sl] + Dh[2] * trial->n[2][sl];
            const float Dnt = Dh[0] * tr.n[0] + Dh[1] * tr.n[1] + Dh[2] * tr.n[2];
            const float nsx = trial->n[0][sl], nsy = trial->n[1][sl], nsz = trial->n[2][sl];
            float2 V[3][3], K[3][3], T[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) V[a][b] = K[a][b] = T[a][b] = make_float2(0.f, 0.f);
#pragma unroll 1
            for (int p = 0; p < 6; ++p) {
                const float ux = tr.u[p][0], uy = tr.u[p][1], uz = tr.u[p][2];
                float2 SV[3], SK[3], ST[3];
#pragma unroll
                for (int b = 0; b < 3; ++b) SV[b] = SK[b] = ST[b] = make_float2(0.f, 0.f);
#pragma unroll 3
                for (int q = 0; q < 6; ++q) {
                    const float wx = ux - trial->u[q][0][sl], wy = uy - trial->u[q][1][sl],
                                wz = uz - trial->u[q][2][sl];
                    const float Dw = Dh[0] * wx + Dh[1] * wy + Dh[2] * wz;
                    const float ww = wx * wx + wy * wy + wz * wz;
                    const float num = fmaf(2.0f, Dw, ww);
                    const float r2 = R2f + num;
                    const float rinv = rsqrtf(r2);
                    const float r = r2 * rinv;
                    const float delta = __fdividef(num, r + Rh);
                    const float2 cs = SMALL ? sincos_small2(P.k_h * delta) : sincos_moderate2(P.k_h * delta);  // (cos, sin)
                    float g = rinv * INV_4PI_F;
                    if (CK) g *= __expf(-P.k_i * delta);
                    // G = g exp(i k R) exp(i k delta)
                    const float2 E = __ffma2_rn(E0rr, cs, __fmul2_rn(E0im, make_float2(cs.y, cs.x)));
                    const float2 G = __fmul2_rn(make_float2(g, g), E);
                    // F = G (1 - i k r) / r^2, k = k_h + i k_i: (1 + k_i r) - i k_h r
                    const float ar = CK ? 1.0f + P.k_i * r : 1.0f;
                    const float ai = -P.k_h * r;
                    const float ri2 = rinv * rinv;
                    const float Fr = (G.x * ar - G.y * ai) * ri2, Fi = (G.x * ai + G.y * ar) * ri2;
                    // (x - y).n = (D + w).n
                    const float dns = Dns + wx * nsx + wy * nsy + wz * nsz;
                    const float dnt = -(Dnt + wx * tr.n[0] + wy * tr.n[1] + wz * tr.n[2]);
                    const float2 KF = make_float2(dns * Fr, dns * Fi), TF = make_float2(dnt * Fr, dnt * Fi);
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        const float2 wl = trial->wl2[q][b][sl];
                        SV[b] = __ffma2_rn(wl, G, SV[b]);
                        SK[b] = __ffma2_rn(wl, KF, SK[b]);
                        ST[b] = __ffma2_rn(wl, TF, ST[b]);
                    }
                }
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float2 wl = make_float2(tr.wl[p][a], tr.wl[p][a]);
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        V[a][b] = __ffma2_rn(wl, SV[b], V[a][b]);
                        K[a][b] = __ffma2_rn(wl, SK[b], K[a][b]);
                        T[a][b] = __ffma2_rn(wl, ST[b], T[a][b]);
                    }
                }
            }
            float I0r = 0.f, I0i = 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    I0r += V[a][b].x;
                    I0i += V[a][b].y;
                }
            const float nn2 = tr.n[0] * trial->n[0][sl] + tr.n[1] * trial->n[1][sl] + tr.n[2] * trial->n[2][sl];
            const uint32_t ts = testslot[tl], ss = trial->slot[sl];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int li = (ts >> (8 * a)) & 0xff;
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const int lj = (ss >> (8 * b)) & 0xff;
                    const int idx = li * TILE_NV + lj;
                    const float cc = tr.curl[a][0] * trial->curl[b][0][sl] + tr.curl[a][1] * trial->curl[b][1][sl] +
                                     tr.curl[a][2] * trial->curl[b][2][sl];
                    const float dr = cc * I0r - nn2 * (P.k2r * V[a][b].x - P.k2i * V[a][b].y);
                    const float di = cc * I0i - nn2 * (P.k2r * V[a][b].y + P.k2i * V[a][b].x);
                    // slab of value o: high words at acc + 2 o SLAB, low words SLAB further
                    auto put = [&](int o, float v) {
                        int32_t* H = acc + (2 * o) * SLAB;
                        fx_add(H, H + SLAB, idx, v, scale, overflow);
                    };
                    put(0, V[a][b].x);
                    put(1, V[a][b].y);
                    put(2, K[a][b].x);
                    put(3, K[a][b].y);
                    put(4, T[a][b].x);
                    put(5, T[a][b].y);
                    put(6, dr);
                    put(7, di);
                }
            }
        }
    }
}

// Adds the tile sums (high * 2^21 + low, unscaled) of every touched (i, j) to the global
// matrices, both orientations.
__device__ __forceinline__ void regular32_flush(const Grid32& G, const int32_t* acc, const int32_t* vI,
                                                const int32_t* vJ, const int nvI, const int nvJ,
                                                const float inv_scale) {
    const int64_t N = G.P.n;
    float2* __restrict__ Vm = G.Vm;
    float2* __restrict__ Km = G.Km;
    float2* __restrict__ Tm = G.Tm;
    float2* __restrict__ Dm = G.Dm;
    constexpr int SLAB = TILE_NV * TILE_NV;
    for (int e = threadIdx.x; e < nvI * nvJ; e += NT32) {
        const int li = e / nvJ, lj = e % nvJ;
        const int idx = li * TILE_NV + lj;
        float v[8];
        bool any = false;
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            // high * 2^21 + low, rounded to FP32 (one extra rounding at most) and unscaled
            const int32_t hs = acc[(2 * o) * SLAB + idx], ls = acc[(2 * o + 1) * SLAB + idx];
            any = any || (hs | ls) != 0;
            v[o] = fmaf((float)hs, 2097152.0f, (float)ls) * inv_scale;
        }
        if (!any) continue;
        const int64_t i = vI[li], j = vJ[lj];
        // storage index per layout (-1: a symmetric layout keeps the mirror, added here too)
        auto put = [&](float2* M, int op, int64_t a, int64_t b, float re, float im) {
            const int64_t x = op_index(G.lay[op], N, G.nt, a, b);
            if (x >= 0) atomicAdd(&M[x], make_float2(re, im));
        };
        if (Vm) { put(Vm, 0, i, j, v[0], v[1]); put(Vm, 0, j, i, v[0], v[1]); }
        if (Km) { put(Km, 1, i, j, v[2], v[3]); put(Km, 1, j, i, v[4], v[5]); }
        if (Tm) { put(Tm, 2, i, j, v[4], v[5]); put(Tm, 2, j, i, v[2], v[3]); }
        if (Dm) { put(Dm, 3, i, j, v[6], v[7]); put(Dm, 3, j, i, v[6], v[7]); }
    }
}


// One CTA's work: the regular pairs of test tile it and trial tile is (it <= is).
template <bool CK>
__device__ __forceinline__ void regular32_tile(const Grid32& G, const int it, const int is) {
    const TriRec32* __restrict__ rec = G.rec;
    const int32_t* __restrict__ tverts = G.tverts;
    const uint32_t* __restrict__ tslots = G.tslots;
    const int32_t* __restrict__ tstart = G.tstart;
    const int32_t* __restrict__ vstart = G.vstart;
    const int32_t* __restrict__ tvert = G.tvert;
    const KP32 P = G.P;
    extern __shared__ float smem[];
    // accumulation slabs: [op V,K,T,D][re,im][high | low int32][TILE_NV * TILE_NV]
    constexpr int SLAB = TILE_NV * TILE_NV;
    int32_t* acc = reinterpret_cast<int32_t*>(smem);
    TriRec32* test = reinterpret_cast<TriRec32*>(smem + 16 * SLAB);
    TrialTile32* trial = reinterpret_cast<TrialTile32*>(test + TILE_TRI);
    __shared__ int32_t testv[TILE_TRI][3];
    __shared__ uint32_t testslot[TILE_TRI];
    __shared__ int32_t vI[TILE_NV], vJ[TILE_NV];
    __shared__ float rho_t[TILE_TRI], rho_s[TILE_TRI];
    // bound factors: [0] min r, [1] max r, [2..3] max weight sum, [4..5] max area, [6..7] max |curl|,
    // [8..9] largest quadrature-point radius of a test / trial triangle
    __shared__ float bnd[10];
    __shared__ float s_scale, s_inv_scale;
    __shared__ int s_overflow, s_small;

    const int t0 = tstart[it], nI = tstart[it + 1] - t0;
    const int s0 = tstart[is], nJ = tstart[is + 1] - s0;
    const int nvI = vstart[it + 1] - vstart[it], nvJ = vstart[is + 1] - vstart[is];
    for (int e = threadIdx.x; e < 16 * SLAB; e += NT32) acc[e] = 0;
    if (threadIdx.x < 10) bnd[threadIdx.x] = threadIdx.x == 0 ? 3.0e38f : 0.0f;
    if (threadIdx.x == 0) s_overflow = 0;
    {
        const float* src = reinterpret_cast<const float*>(rec + t0);
        float* dst = reinterpret_cast<float*>(test);
        for (int e = threadIdx.x; e < nI * TRIREC32_FLOATS; e += NT32) dst[e] = src[e];
        for (int e = threadIdx.x; e < nI * 3; e += NT32) testv[e / 3][e % 3] = tverts[3 * t0 + e];
        for (int e = threadIdx.x; e < nI; e += NT32) testslot[e] = tslots[t0 + e];
        for (int e = threadIdx.x; e < 54 * TILE_TRI; e += NT32) {
            const int s = e % TILE_TRI, f = e / TILE_TRI;
            const float val = s < nJ ? reinterpret_cast<const float*>(rec + s0 + s)[f] : 0.0f;
            if (f < 3) trial->ch[f][s] = val;
            else if (f < 6) trial->cl[f - 3][s] = val;
            else if (f < 24) trial->u[(f - 6) / 3][(f - 6) % 3][s] = val;
            else if (f < 42) trial->wl2[(f - 24) / 3][(f - 24) % 3][s] = make_float2(val, val);
            else if (f < 45) trial->n[f - 42][s] = val;
            else trial->curl[(f - 45) / 3][(f - 45) % 3][s] = val;
        }
        for (int e = threadIdx.x; e < 3 * TILE_TRI; e += NT32) {
            const int s = e % TILE_TRI, a = e / TILE_TRI;
            trial->v[a][s] = s < nJ ? tverts[3 * (s0 + s) + a] : -1;
        }
        for (int e = threadIdx.x; e < TILE_TRI; e += NT32) trial->slot[e] = e < nJ ? tslots[s0 + e] : 0u;
        for (int e = threadIdx.x; e < nvI; e += NT32) vI[e] = tvert[vstart[it] + e];
        for (int e = threadIdx.x; e < nvJ; e += NT32) vJ[e] = tvert[vstart[is] + e];
    }
    __syncthreads();

    // ---- bound of every value this CTA produces, and the fixed-point scale
    if (threadIdx.x < 2 * TILE_TRI) {  // per-triangle radius, weight sums, area, curls
        const bool tside = threadIdx.x < TILE_TRI;
        const int t = tside ? threadIdx.x : threadIdx.x - TILE_TRI;
        if (t < (tside ? nI : nJ)) {
            float rho = 0.f, area = 0.f, wmax = 0.f, cmax = 0.f;
            for (int p = 0; p < 6; ++p) {
                float u2 = 0.f;
                for (int d = 0; d < 3; ++d) {
                    const float u = tside ? test[t].u[p][d] : trial->u[p][d][t];
                    u2 = fmaf(u, u, u2);
                }
                rho = fmaxf(rho, sqrtf(u2));
            }
            for (int a = 0; a < 3; ++a) {
                float w = 0.f, c2 = 0.f;
                for (int p = 0; p < 6; ++p) w += fabsf(tside ? test[t].wl[p][a] : trial->wl2[p][a][t].x);
                for (int d = 0; d < 3; ++d) {
                    const float c = tside ? test[t].curl[a][d] : trial->curl[a][d][t];
                    c2 = fmaf(c, c, c2);
                }
                area += w;
                wmax = fmaxf(wmax, w);
                cmax = fmaxf(cmax, sqrtf(c2));
            }
            rho *= 1.0001f;
            (tside ? rho_t : rho_s)[t] = rho;
            smax(&bnd[tside ? 8 : 9], rho);
            smax(&bnd[tside ? 2 : 3], wmax);
            smax(&bnd[tside ? 4 : 5], area);
            smax(&bnd[tside ? 6 : 7], cmax);
        }
    }
    __syncthreads();
    for (int pidx = threadIdx.x; pidx < TILE_TRI * TILE_TRI; pidx += NT32) {  // point distances
        const int tl = pidx / TILE_TRI, sl = pidx % TILE_TRI;
        if (tl >= nI || sl >= nJ || !regular_pair(it, is, tl, sl, testv, trial)) continue;
        const TriRec32& tr = test[tl];
        float D[3], R2 = 0.f;
        for (int d = 0; d < 3; ++d) {
            D[d] = (tr.ch[d] - trial->ch[d][sl]) + (tr.cl[d] - trial->cl[d][sl]);
            R2 = fmaf(D[d], D[d], R2);
        }
        const float R = sqrtf(R2), ro = rho_t[tl] + rho_s[sl];
        float rmin = R - ro;
        if (rmin < 0.5f * R) {  // near pair: the smallest of its 36 point distances
            float m2 = 3.0e38f;
            for (int p = 0; p < 6; ++p)
                for (int q = 0; q < 6; ++q) {
                    float r2 = 0.f;
                    for (int d = 0; d < 3; ++d) {
                        const float x = D[d] + tr.u[p][d] - trial->u[q][d][sl];
                        r2 = fmaf(x, x, r2);
                    }
                    m2 = fminf(m2, r2);
                }
            rmin = 0.999f * sqrtf(m2);
        }
        smin(&bnd[0], fmaxf(rmin, 1e-30f));
        smax(&bnd[1], R + ro);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const float rmin = bnd[0], rmax = bnd[1];
        const float kabs = sqrtf(P.k_h * P.k_h + P.k_i * P.k_i);
        const float amp = CK ? expf(fmaxf(0.0f, -P.k_i) * rmax) : 1.0f;
        const float g = INV_4PI_F / rmin;
        const float ww = bnd[2] * bnd[3];
        const float bV = ww * g;
        const float bK = ww * g * (1.0f + kabs * rmin) / rmin;
        const float bD = (bnd[6] * bnd[7] * bnd[4] * bnd[5] + kabs * kabs * ww) * g;
        float B = 2.0f * amp * fmaxf(bV, fmaxf(bK, bD));  // factor 2: FP32 rounding of the values
        B = fminf(fmaxf(B, 1e-30f), 1e30f);                // also maps NaN (no regular pair) to 1e-30
        int e = 40 - ilogbf(B) - 1;                        // B < 2^(ilogb B + 1), so |v| 2^e < 2^40
        e = max(-120, min(120, e));
        s_scale = ldexpf(1.0f, e);
        s_inv_scale = ldexpf(1.0f, -e);
        // |k delta| <= |k| (rho_t + rho_s) for every point pair (delta = r - R, |delta| <= |w|):
        // below pi/4 the phase offsets need no reduction
        s_small = fabsf(P.k_h) * (bnd[8] + bnd[9]) <= 0.78f;
    }
    __syncthreads();
    const float scale = s_scale;
    if (s_small) regular32_pairs<CK, true>(G, it, is, nI, nJ, test, trial, testv, testslot, acc, scale, &s_overflow);
    else regular32_pairs<CK, false>(G, it, is, nI, nJ, test, trial, testv, testslot, acc, scale, &s_overflow);
    __syncthreads();
    if (s_overflow) {  // cannot happen for finite inputs if the bound holds; reported, tile not written
        if (threadIdx.x == 0) atomicOr(G.err, 1);
        return;
    }
    regular32_flush(G, acc, vI, vJ, nvI, nvJ, s_inv_scale);
}

template <bool CK>
__global__ void __launch_bounds__(NT32, 1) k_regular32(Grid32 G) {
    const int it = blockIdx.y, is = blockIdx.x;
    if (it > is) return;
    regular32_tile<CK>(G, it, is);
}

// Persistent form for many grids of uneven sizes in one launch: one CTA per SM
// takes (grid, it, is) items from a shared counter until the list is exhausted.
__global__ void __launch_bounds__(NT32, 1) k_regular32_many(const Grid32* __restrict__ grids,
                                                            const int4* __restrict__ items, int nitems,
                                                            int* __restrict__ counter) {
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int w = s_item;
        __syncthreads();  // every thread has read s_item before it is overwritten
        if (w >= nitems) break;
        const int4 item = items[w];
        if (grids[item.x].ck) regular32_tile<true>(grids[item.x], item.y, item.z);
        else regular32_tile<false>(grids[item.x], item.y, item.z);
        __syncthreads();  // the tile's shared memory is reused by the next item
    }
}

__global__ void k_sincos_check(int n, float xmax, float* __restrict__ err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = -xmax + 2.0f * xmax * ((float)i + 0.5f) / (float)n;
    float s0, c0;
    sincosf(x, &s0, &c0);
    const float2 cs = sincos_moderate2(x);
    err[i] = fmaxf(fabsf(cs.y - s0), fabsf(cs.x - c0));
}

}  // namespace

// Largest absolute difference between sincos_moderate and CUDA's sincosf on n
// evenly spaced arguments in [-xmax, xmax].
bem_status selftest_sincos(int n, float xmax, double* max_err, cudaStream_t s) {
    DevBuf e;
    BEM_TRY(e.alloc((size_t)n * 4, s));
    BEM_LAUNCH(k_sincos_check, (unsigned)((n + 255) / 256), 256, 0, s, n, xmax, e.as<float>());
    std::vector<float> h(n);
    BEM_CUDA_TRY(cudaMemcpyAsync(h.data(), e.p, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    double m = 0.0;
    for (float v : h) m = std::max(m, (double)v);
    *max_err = m;
    return BEM_OK;
}

namespace {

size_t regular32_smem() {
    return 16 * TILE_NV * TILE_NV * sizeof(float) + TILE_TRI * sizeof(TriRec32) + sizeof(TrialTile32);
}

Grid32 grid32_args(const bem_grid* g, double k_re, double k_im, float2* V, float2* K, float2* T, float2* D,
                   const OpLayouts& L, int* flag) {
    Grid32 G{};
    G.rec = g->rec32.as<TriRec32>();
    G.tverts = g->t_verts.as<int32_t>();
    G.tslots = g->t_slots.as<uint32_t>();
    G.tstart = g->tile_tstart.as<int32_t>();
    G.vstart = g->tile_vstart.as<int32_t>();
    G.tvert = g->tile_vert.as<int32_t>();
    G.P.k_h = (float)k_re;
    G.P.k_l = (float)(k_re - (double)G.P.k_h);
    G.P.k_i = (float)k_im;
    G.P.k2r = (float)(k_re * k_re - k_im * k_im);
    G.P.k2i = (float)(2.0 * k_re * k_im);
    G.P.n = g->nv;
    G.Vm = V;
    G.Km = K;
    G.Tm = T;
    G.Dm = D;
    G.err = flag;
    G.ck = k_im != 0.0;
    G.nt = op_tiles(g->nv);
    for (int i = 0; i < 4; ++i) G.lay[i] = L.lay[i];
    return G;
}

bem_status check_flag(const DevBuf& flag, cudaStream_t s) {
    int h_flag = 0;
    BEM_CUDA_TRY(cudaMemcpyAsync(&h_flag, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_flag) {
        set_error("FP32 assembly: a value exceeded the fixed-point range of its tile (non-finite input or "
                  "a degenerate grid)");
        return BEM_E_NONFINITE;
    }
    return BEM_OK;
}

}  // namespace

bem_status assemble_regular_fp32(const bem_grid* g, double k_re, double k_im, float2* V, float2* K, float2* T,
                                 float2* D, const OpLayouts& L, cudaStream_t s) {
    if (g->ntile > 65535) {
        set_error("grid too large for the tile grid of the mixed-precision assembly");
        return BEM_E_INVALID_ARG;
    }
    const size_t smem = regular32_smem();
    // the attribute is per device and per function; setting it on every call is cheap and thread-safe
    BEM_CUDA_TRY(cudaFuncSetAttribute(k_regular32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    BEM_CUDA_TRY(cudaFuncSetAttribute(k_regular32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((unsigned)g->ntile, (unsigned)g->ntile);
    DevBuf flag;
    BEM_TRY(flag.alloc(sizeof(int), s));
    BEM_CUDA_TRY(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
    const Grid32 G = grid32_args(g, k_re, k_im, V, K, T, D, L, flag.as<int>());
    if (G.ck) BEM_LAUNCH(k_regular32<true>, grid, NT32, smem, s, G);
    else BEM_LAUNCH(k_regular32<false>, grid, NT32, smem, s, G);
    return check_flag(flag, s);
}

bem_status assemble_regular_fp32_many(int count, const bem_grid* const* g, const double* k_re, const double* k_im,
                                      float2* const* V, float2* const* K, float2* const* T, float2* const* D,
                                      const OpLayouts& L, cudaStream_t s) {
    if (count <= 0) return BEM_OK;
    DevBuf flag, dgrids, ditems, counter;
    BEM_TRY(flag.alloc(sizeof(int), s));
    BEM_CUDA_TRY(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
    std::vector<Grid32> grids(count);
    std::vector<int4> items;
    for (int i = 0; i < count; ++i) {
        grids[i] = grid32_args(g[i], k_re[i], k_im[i], V[i], K[i], T[i], D[i], L, flag.as<int>());
        for (int it = 0; it < (int)g[i]->ntile; ++it)
            for (int is = it; is < (int)g[i]->ntile; ++is) items.push_back(make_int4(i, it, is, 0));
    }
    BEM_TRY(dgrids.alloc(grids.size() * sizeof(Grid32), s));
    BEM_TRY(ditems.alloc(items.size() * sizeof(int4), s));
    BEM_TRY(counter.alloc(sizeof(int), s));
    BEM_CUDA_TRY(cudaMemcpyAsync(dgrids.p, grids.data(), grids.size() * sizeof(Grid32), cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(ditems.p, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(cudaMemsetAsync(counter.p, 0, sizeof(int), s));
    const size_t smem = regular32_smem();
    BEM_CUDA_TRY(cudaFuncSetAttribute(k_regular32_many, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0;
    BEM_CUDA_TRY(cudaGetDevice(&dev));
    BEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int ctas = std::max(1, std::min<int>(sms, (int)items.size()));
    BEM_LAUNCH(k_regular32_many, ctas, NT32, smem, s, dgrids.as<Grid32>(), ditems.as<int4>(), (int)items.size(),
               counter.as<int>());
    return check_flag(flag, s);  // also keeps the host vectors alive until the copies are done
}

}  // namespace bem
