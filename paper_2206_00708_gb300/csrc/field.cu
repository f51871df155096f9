// Field evaluation with the potential operators (paper Sec. 2.1 and eq.
// representation): u(x) = [V psi](x) - [K phi](x) for P1 densities on one grid, at
// points off the surface, with the 6-point degree-4 rule per triangle.
//
// A preparation kernel turns every (triangle, quadrature point) into a record: the
// point y, the triangle's normal, and the weighted densities sum_a w_p J lambda_a(p)
// psi_a and the same for phi.  The field kernel gives each thread one point; a block
// stages a tile of records in shared memory and its threads sweep it.  To fill the
// GPU for a few thousand points the record range is cut into S slices (blockIdx.y),
// whose partial sums are added in a fixed order by a second kernel, so the result
// does not depend on scheduling.  FP64 throughout.
#include "bem_internal.cuh"

#include <algorithm>

namespace bem {

namespace {

constexpr double INV_4PI_D = 0.07957747154594767;  // 1 / (4 pi)
constexpr int FIELD_THREADS = 64;
constexpr int FIELD_TILE = 256;  // records staged per block and sweep

struct FieldRec {
    double y[3], n[3];
    double2 wpsi, wphi;
};

__global__ void k_field_prep(const TriRec* __restrict__ rec, const int32_t* __restrict__ tri, int64_t nt,
                             const double2* __restrict__ phi, const double2* __restrict__ psi,
                             FieldRec* __restrict__ out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= 6 * nt) return;
    const int64_t t = e / 6;
    const int p = (int)(e % 6);
    const TriRec& R = rec[t];
    FieldRec f;
    for (int d = 0; d < 3; ++d) {
        f.y[d] = R.q[p][d];
        f.n[d] = R.n[d];
    }
    double2 a = make_double2(0, 0), b = make_double2(0, 0);
    for (int k = 0; k < 3; ++k) {
        const int32_t v = tri[3 * t + k];
        const double w = R.wl[p][k];
        if (psi) {
            a.x += w * psi[v].x;
            a.y += w * psi[v].y;
        }
        if (phi) {
            b.x += w * phi[v].x;
            b.y += w * phi[v].y;
        }
    }
    f.wpsi = a;
    f.wphi = b;
    out[e] = f;
}

// partial[slice][point] = sum over the slice's records of G wpsi - dG/dn(y) wphi
template <bool CK>
__global__ void __launch_bounds__(FIELD_THREADS) k_field(const FieldRec* __restrict__ recs, int64_t nrec,
                                                         double kr, double ki, const double* __restrict__ pts,
                                                         int64_t npts, double2* __restrict__ partial) {
    __shared__ FieldRec tile[FIELD_TILE];
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t per = (nrec + gridDim.y - 1) / gridDim.y;
    const int64_t r0 = blockIdx.y * per, r1 = (r0 + per < nrec) ? r0 + per : nrec;
    double x0 = 0, x1 = 0, x2 = 0;
    if (m < npts) {
        x0 = pts[3 * m];
        x1 = pts[3 * m + 1];
        x2 = pts[3 * m + 2];
    }
    double ur = 0.0, ui = 0.0;
    for (int64_t base = r0; base < r1; base += FIELD_TILE) {
        const int cnt = (int)((r1 - base) < FIELD_TILE ? (r1 - base) : FIELD_TILE);
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) tile[i] = recs[base + i];
        __syncthreads();
        if (m < npts) {
            for (int i = 0; i < cnt; ++i) {
                const FieldRec& f = tile[i];
                const double d0 = x0 - f.y[0], d1 = x1 - f.y[1], d2 = x2 - f.y[2];
                const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
                const double rinv = rsqrt(r2);
                const double r = r2 * rinv;
                double sn, cs;
                sincos(kr * r, &sn, &cs);
                double g = rinv * INV_4PI_D;
                if (CK) g *= exp(-ki * r);
                const double Gr = g * cs, Gi = g * sn;
                // dG/dn(y) = G (1 - i k r) ((x - y) . n) / r^2, k = kr + i ki
                const double dn = (d0 * f.n[0] + d1 * f.n[1] + d2 * f.n[2]) * rinv * rinv;
                const double ar = CK ? 1.0 + ki * r : 1.0, ai = -kr * r;
                const double Fr = (Gr * ar - Gi * ai) * dn, Fi = (Gr * ai + Gi * ar) * dn;
                ur += Gr * f.wpsi.x - Gi * f.wpsi.y - (Fr * f.wphi.x - Fi * f.wphi.y);
                ui += Gr * f.wpsi.y + Gi * f.wpsi.x - (Fr * f.wphi.y + Fi * f.wphi.x);
            }
        }
    }
    if (m < npts) partial[blockIdx.y * npts + m] = make_double2(ur, ui);
}

__global__ void k_field_sum(const double2* __restrict__ partial, int S, int64_t npts, double2* __restrict__ u) {
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= npts) return;
    double2 s = make_double2(0, 0);
    for (int k = 0; k < S; ++k) {
        s.x += partial[k * npts + m].x;
        s.y += partial[k * npts + m].y;
    }
    u[m] = s;
}

}  // namespace

bem_status field_impl(bem_context* ctx, const bem_grid* g, bem_c128 k, const bem_c128* phi, const bem_c128* psi,
                      const double* points, int64_t npts, bem_c128* u, int on_device) {
    cudaStream_t s = ctx->stream;
    const int64_t nt = g->nt, nv = g->nv, nrec = 6 * nt;
    DevBuf dphi, dpsi, dpts, du, recs, part;
    const double2 *phi_d = nullptr, *psi_d = nullptr;
    const double* pts_d = nullptr;
    double2* u_d = nullptr;
    if (on_device) {
        phi_d = reinterpret_cast<const double2*>(phi);
        psi_d = reinterpret_cast<const double2*>(psi);
        pts_d = points;
        u_d = reinterpret_cast<double2*>(u);
    } else {
        if (phi) {
            BEM_TRY(dphi.alloc(nv * 16, s));
            BEM_CUDA_TRY(cudaMemcpyAsync(dphi.p, phi, nv * 16, cudaMemcpyHostToDevice, s));
            phi_d = dphi.as<double2>();
        }
        if (psi) {
            BEM_TRY(dpsi.alloc(nv * 16, s));
            BEM_CUDA_TRY(cudaMemcpyAsync(dpsi.p, psi, nv * 16, cudaMemcpyHostToDevice, s));
            psi_d = dpsi.as<double2>();
        }
        BEM_TRY(dpts.alloc(npts * 24, s));
        BEM_CUDA_TRY(cudaMemcpyAsync(dpts.p, points, npts * 24, cudaMemcpyHostToDevice, s));
        pts_d = dpts.as<double>();
        BEM_TRY(du.alloc(npts * 16, s));
        u_d = du.as<double2>();
    }
    BEM_TRY(recs.alloc(nrec * sizeof(FieldRec), s));
    BEM_LAUNCH(k_field_prep, (unsigned)((nrec + 255) / 256), 256, 0, s, g->rec.as<TriRec>(), g->tri.as<int32_t>(), nt,
               phi_d, psi_d, recs.as<FieldRec>());
    int dev = 0, sms = 0;
    BEM_CUDA_TRY(cudaGetDevice(&dev));
    BEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t bx = (npts + FIELD_THREADS - 1) / FIELD_THREADS;
    // slices of the record range: about 8 blocks per SM in total, each slice at least one tile
    int S = (int)std::max<int64_t>(1, std::min<int64_t>((8LL * sms + bx - 1) / bx, (nrec + FIELD_TILE - 1) / FIELD_TILE));
    S = std::min(S, 65535);
    BEM_TRY(part.alloc((size_t)S * npts * 16, s));
    const dim3 grid((unsigned)bx, (unsigned)S);
    if (k.im != 0.0)
        BEM_LAUNCH(k_field<true>, grid, FIELD_THREADS, 0, s, recs.as<FieldRec>(), nrec, k.re, k.im, pts_d, npts,
                   part.as<double2>());
    else
        BEM_LAUNCH(k_field<false>, grid, FIELD_THREADS, 0, s, recs.as<FieldRec>(), nrec, k.re, k.im, pts_d, npts,
                   part.as<double2>());
    BEM_LAUNCH(k_field_sum, (unsigned)((npts + 255) / 256), 256, 0, s, part.as<double2>(), S, npts, u_d);
    if (!on_device) BEM_CUDA_TRY(cudaMemcpyAsync(u, u_d, npts * 16, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    return BEM_OK;
}

}  // namespace bem
