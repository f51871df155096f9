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
//  * the 3x3 blocks of a CTA's triangle pairs are summed in shared memory with
//    compensated atomics: each thread recovers the exact rounding error of its own
//    atomic add (the returned old value makes a two-sum possible) and adds it to a
//    second buffer, so the in-tile sums are double-float accurate.
// The tile buffers are flushed to the global matrices with vector float2 atomics.
#include "bem_internal.cuh"

#include <algorithm>

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
    p = a * b;
    e = fmaf(a, b, -p);
}

// sin and cos of a moderate FP32 argument (|x| < 2^15): Cody-Waite reduction by
// pi/2 with a three-part constant (the first part has 8 significant bits, so n * P1 is
// exact), then the Taylor series of sin and cos on |r| <= pi/4 (truncation below
// 2e-9), evaluated by Horner's rule in r^2; the quadrant selects signs and swaps.
__device__ __forceinline__ void sincos_moderate(float x, float* s, float* c) {
    const float n = rintf(x * 0.636619772367581343f);  // 2 / pi
    float r = fmaf(-n, 1.5703125f, x);                  // pi/2 = P1 + P2 + P3
    r = fmaf(-n, 4.838267923332751e-4f, r);
    r = fmaf(-n, 2.5632829192545614e-12f, r);
    const float r2 = r * r;
    // sin r = r (1 - r^2/3! + r^4/5! - r^6/7! + r^8/9!)
    float ps = fmaf(r2, 2.75573192239858907e-6f, -1.98412698412698413e-4f);
    ps = fmaf(r2, ps, 8.33333333333333333e-3f);
    ps = fmaf(r2, ps, -1.66666666666666667e-1f);
    const float sr = fmaf(r * r2, ps, r);
    // cos r = 1 - r^2/2! + r^4/4! - r^6/6! + r^8/8! - r^10/10!
    float pc = fmaf(r2, -2.75573192239858907e-7f, 2.48015873015873016e-5f);
    pc = fmaf(r2, pc, -1.38888888888888889e-3f);
    pc = fmaf(r2, pc, 4.16666666666666667e-2f);
    pc = fmaf(r2, pc, -0.5f);
    const float cr = fmaf(r2, pc, 1.0f);
    const int q = ((int)n) & 3;
    const float ss = (q & 1) ? cr : sr, cc = (q & 1) ? sr : cr;
    *s = (q & 2) ? -ss : ss;
    *c = ((q + 1) & 2) ? -cc : cc;
}

struct TrialTile32 {
    float ch[3][TILE_TRI], cl[3][TILE_TRI];
    float u[6][3][TILE_TRI];
    float wl[6][3][TILE_TRI];
    float n[3][TILE_TRI];
    float curl[3][3][TILE_TRI];
    int32_t v[3][TILE_TRI];
    uint32_t slot[TILE_TRI];
};

// compensated shared-memory accumulation: S += c exactly up to the rounding of E
__device__ __forceinline__ void comp_add(float* S, float* E, int idx, float c) {
    const float old = atomicAdd(&S[idx], c);
    float s, e;
    two_sum(old, c, s, e);  // s is the value the atomic stored; e its exact rounding error
    if (e != 0.0f) atomicAdd(&E[idx], e);
}

template <bool CK>
__global__ void __launch_bounds__(NT32, 1)
k_regular32(const TriRec32* __restrict__ rec, const int32_t* __restrict__ tverts, const uint32_t* __restrict__ tslots,
            const int32_t* __restrict__ tstart, const int32_t* __restrict__ vstart,
            const int32_t* __restrict__ tvert, KP32 P, float2* __restrict__ Vm, float2* __restrict__ Km,
            float2* __restrict__ Tm, float2* __restrict__ Dm) {
    const int it = blockIdx.y, is = blockIdx.x;
    if (it > is) return;
    extern __shared__ float smem[];
    // accumulation slabs: [op V,K,T,D][re,im][S,E][TILE_NV * TILE_NV]
    constexpr int SLAB = TILE_NV * TILE_NV;
    float* acc = smem;
    TriRec32* test = reinterpret_cast<TriRec32*>(smem + 16 * SLAB);
    TrialTile32* trial = reinterpret_cast<TrialTile32*>(test + TILE_TRI);
    __shared__ int32_t testv[TILE_TRI][3];
    __shared__ uint32_t testslot[TILE_TRI];
    __shared__ int32_t vI[TILE_NV], vJ[TILE_NV];

    const int t0 = tstart[it], nI = tstart[it + 1] - t0;
    const int s0 = tstart[is], nJ = tstart[is + 1] - s0;
    const int nvI = vstart[it + 1] - vstart[it], nvJ = vstart[is + 1] - vstart[is];
    for (int e = threadIdx.x; e < 16 * SLAB; e += NT32) acc[e] = 0.0f;
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
            else if (f < 42) trial->wl[(f - 24) / 3][(f - 24) % 3][s] = val;
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

    const float tp_h = 6.28318548202514648f, tp_l = -1.7484555314695172e-7f;  // 2 pi as hi + lo
    const float inv_tp = 0.159154943091895336f;
    for (int pidx = threadIdx.x; pidx < TILE_TRI * TILE_TRI; pidx += NT32) {
        const int tl = pidx / TILE_TRI, sl = pidx % TILE_TRI;
        if (tl >= nI || sl >= nJ) continue;
        if (it == is && tl >= sl) continue;
        const int32_t ta = testv[tl][0], tb = testv[tl][1], tc = testv[tl][2];
        const int32_t sa = trial->v[0][sl], sb = trial->v[1][sl], sc = trial->v[2][sl];
        if ((ta == sa) | (ta == sb) | (ta == sc) | (tb == sa) | (tb == sb) | (tb == sc) | (tc == sa) |
            (tc == sb) | (tc == sc))
            continue;  // singular pair
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
            const float E0r = amp0 * cs0, E0i = amp0 * sn0;
            const float R2f = R2h + R2l;
            const float Dns = Dh[0] * trial->n[0][sl] + Dh[1] * trial->n[1][sl] + Dh[2] * trial->n[2][sl];
            const float Dnt = Dh[0] * tr.n[0] + Dh[1] * tr.n[1] + Dh[2] * tr.n[2];
            float Vr[3][3] = {}, Vi[3][3] = {}, Kr[3][3] = {}, Ki[3][3] = {}, Tr[3][3] = {}, Ti[3][3] = {};
#pragma unroll 1
            for (int p = 0; p < 6; ++p) {
                const float ux = tr.u[p][0], uy = tr.u[p][1], uz = tr.u[p][2];
                float SVr[3] = {}, SVi[3] = {}, SKr[3] = {}, SKi[3] = {}, STr[3] = {}, STi[3] = {};
#pragma unroll 2
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
                    float sd, cd;
                    sincos_moderate(P.k_h * delta, &sd, &cd);
                    float g = rinv * INV_4PI_F;
                    if (CK) g *= __expf(-P.k_i * delta);
                    // G = g exp(i k R) exp(i k delta)
                    const float Er = E0r * cd - E0i * sd, Ei = E0r * sd + E0i * cd;
                    const float Gr = g * Er, Gi = g * Ei;
                    // F = G (1 - i k r) / r^2, k = k_h + i k_i: (1 + k_i r) - i k_h r
                    const float ar = CK ? 1.0f + P.k_i * r : 1.0f;
                    const float ai = -P.k_h * r;
                    const float ri2 = rinv * rinv;
                    const float Fr = (Gr * ar - Gi * ai) * ri2, Fi = (Gr * ai + Gi * ar) * ri2;
                    // (x - y).n = (D + w).n
                    const float dns = Dns + wx * trial->n[0][sl] + wy * trial->n[1][sl] + wz * trial->n[2][sl];
                    const float dnt = -(Dnt + wx * tr.n[0] + wy * tr.n[1] + wz * tr.n[2]);
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        const float wl = trial->wl[q][b][sl];
                        SVr[b] = fmaf(wl, Gr, SVr[b]);
                        SVi[b] = fmaf(wl, Gi, SVi[b]);
                        const float cs = wl * dns, ct = wl * dnt;
                        SKr[b] = fmaf(cs, Fr, SKr[b]);
                        SKi[b] = fmaf(cs, Fi, SKi[b]);
                        STr[b] = fmaf(ct, Fr, STr[b]);
                        STi[b] = fmaf(ct, Fi, STi[b]);
                    }
                }
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float wl = tr.wl[p][a];
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        Vr[a][b] = fmaf(wl, SVr[b], Vr[a][b]);
                        Vi[a][b] = fmaf(wl, SVi[b], Vi[a][b]);
                        Kr[a][b] = fmaf(wl, SKr[b], Kr[a][b]);
                        Ki[a][b] = fmaf(wl, SKi[b], Ki[a][b]);
                        Tr[a][b] = fmaf(wl, STr[b], Tr[a][b]);
                        Ti[a][b] = fmaf(wl, STi[b], Ti[a][b]);
                    }
                }
            }
            float I0r = 0.f, I0i = 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    I0r += Vr[a][b];
                    I0i += Vi[a][b];
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
                    const float dr = cc * I0r - nn2 * (P.k2r * Vr[a][b] - P.k2i * Vi[a][b]);
                    const float di = cc * I0i - nn2 * (P.k2r * Vi[a][b] + P.k2i * Vr[a][b]);
                    const float vals[8] = {Vr[a][b], Vi[a][b], Kr[a][b], Ki[a][b], Tr[a][b], Ti[a][b], dr, di};
#pragma unroll
                    for (int o = 0; o < 8; ++o) {
                        float* S = acc + (2 * o) * SLAB;
                        comp_add(S, S + SLAB, idx, vals[o]);
                    }
                }
            }
        }
    }
    __syncthreads();
    // flush: S + E of every touched (i, j) to the global matrices, both orientations
    const int64_t N = P.n;
    for (int e = threadIdx.x; e < nvI * nvJ; e += NT32) {
        const int li = e / nvJ, lj = e % nvJ;
        const int idx = li * TILE_NV + lj;
        float v[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) v[o] = acc[(2 * o) * SLAB + idx] + acc[(2 * o + 1) * SLAB + idx];
        if (v[0] == 0.f && v[1] == 0.f && v[2] == 0.f && v[3] == 0.f && v[4] == 0.f && v[5] == 0.f) continue;
        const int64_t i = vI[li], j = vJ[lj];
        const int64_t ij = i * N + j, ji = j * N + i;
        if (Vm) { atomicAdd(&Vm[ij], make_float2(v[0], v[1])); atomicAdd(&Vm[ji], make_float2(v[0], v[1])); }
        if (Km) { atomicAdd(&Km[ij], make_float2(v[2], v[3])); atomicAdd(&Km[ji], make_float2(v[4], v[5])); }
        if (Tm) { atomicAdd(&Tm[ij], make_float2(v[4], v[5])); atomicAdd(&Tm[ji], make_float2(v[2], v[3])); }
        if (Dm) { atomicAdd(&Dm[ij], make_float2(v[6], v[7])); atomicAdd(&Dm[ji], make_float2(v[6], v[7])); }
    }
}

__global__ void k_sincos_check(int n, float xmax, float* __restrict__ err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = -xmax + 2.0f * xmax * ((float)i + 0.5f) / (float)n;
    float s0, c0, s1, c1;
    sincosf(x, &s0, &c0);
    sincos_moderate(x, &s1, &c1);
    err[i] = fmaxf(fabsf(s1 - s0), fabsf(c1 - c0));
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

bem_status assemble_regular_fp32(const bem_grid* g, double k_re, double k_im, float2* V, float2* K, float2* T,
                                 float2* D, cudaStream_t s) {
    KP32 P;
    P.k_h = (float)k_re;
    P.k_l = (float)(k_re - (double)P.k_h);
    P.k_i = (float)k_im;
    P.k2r = (float)(k_re * k_re - k_im * k_im);
    P.k2i = (float)(2.0 * k_re * k_im);
    P.n = g->nv;
    if (g->ntile > 65535) {
        set_error("grid too large for the tile grid of the mixed-precision assembly");
        return BEM_E_INVALID_ARG;
    }
    const size_t smem = 16 * TILE_NV * TILE_NV * sizeof(float) + TILE_TRI * sizeof(TriRec32) + sizeof(TrialTile32);
    // the attribute is per device and per function; setting it on every call is cheap and thread-safe
    BEM_CUDA_TRY(cudaFuncSetAttribute(k_regular32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    BEM_CUDA_TRY(cudaFuncSetAttribute(k_regular32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((unsigned)g->ntile, (unsigned)g->ntile);
    const bool ck = k_im != 0.0;
    if (ck)
        BEM_LAUNCH(k_regular32<true>, grid, NT32, smem, s, g->rec32.as<TriRec32>(), g->t_verts.as<int32_t>(),
                   g->t_slots.as<uint32_t>(), g->tile_tstart.as<int32_t>(), g->tile_vstart.as<int32_t>(),
                   g->tile_vert.as<int32_t>(), P, V, K, T, D);
    else
        BEM_LAUNCH(k_regular32<false>, grid, NT32, smem, s, g->rec32.as<TriRec32>(), g->t_verts.as<int32_t>(),
                   g->t_slots.as<uint32_t>(), g->tile_tstart.as<int32_t>(), g->tile_vstart.as<int32_t>(),
                   g->tile_vert.as<int32_t>(), P, V, K, T, D);
    return BEM_OK;
}

}  // namespace bem
