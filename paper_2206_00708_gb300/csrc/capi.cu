// C ABI entry points (include/bem.h): argument checks, handle management, error
// strings.  Every entry point makes the handle's device current and runs its work
// on the context's stream.
#include "bem_internal.cuh"

#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>

namespace bem {

namespace {
thread_local std::string g_last_error = "no error";
std::atomic<uint64_t> g_launches{0};
}

void set_error(const std::string& msg) { g_last_error = msg; }

void count_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
thread_local int g_capturing = 0;

bem_status DevBuf::alloc(size_t nbytes, cudaStream_t s) {
    release();
    if (nbytes == 0) nbytes = 16;
    cudaError_t e = cudaMallocAsync(&p, nbytes, s);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        set_error(std::string("device allocation of ") + std::to_string(nbytes) + " bytes failed: " +
                  cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? BEM_E_OOM : BEM_E_CUDA;
    }
    bytes = nbytes;
    stream = s;
    return BEM_OK;
}

void DevBuf::release() {
    if (p) {
        if (stream) cudaFreeAsync(p, stream);
        else cudaFree(p);
    }
    p = nullptr;
    bytes = 0;
}

bem_status solve_transmission_impl(bem_context* ctx, const bem_grid* ge, const bem_grid* gi, bem_c128 k_int,
                                   bem_c128 k_ext, double rho_ratio, const bem_incident* inc,
                                   const bem_solve_opts* o, bem_c128* v_ext, bem_c128* w_ext, bem_c128* v_int,
                                   bem_c128* w_int, int on_device, bem_solve_report* rep);
bem_status solve_screen_impl(bem_context* ctx, const bem_grid* gf, const bem_grid* gc, bem_c128 k,
                             const bem_incident* inc, const bem_solve_opts* o, int precond, bem_c128* phi,
                             int on_device, bem_solve_report* rep);
bem_status autotune_impl(bem_context* ctx, const bem_grid* ge, const bem_grid* gi, int n_rhs, int reps);
bem_status field_impl(bem_context* ctx, const bem_grid* g, bem_c128 k, const bem_c128* phi, const bem_c128* psi,
                      const double* points, int64_t npts, bem_c128* u, int on_device);

}  // namespace bem

using namespace bem;

#define CTX_GUARD(ctx)                                         \
    do {                                                       \
        BEM_REQUIRE((ctx) != nullptr, "null context");         \
        BEM_CUDA_TRY(cudaSetDevice((ctx)->device));            \
    } while (0)

namespace {

// Validation of an incident field (bem_incident) on the host: kind, sizes and finite,
// unit or present inputs.
bem_status check_incident(const bem_incident* inc) {
    BEM_REQUIRE(inc != nullptr && inc->n_rhs >= 1, "incident field needs n_rhs >= 1");
    BEM_REQUIRE(inc->kind == BEM_INC_PLANE_WAVE || inc->kind == BEM_INC_POINT_SOURCE ||
                    inc->kind == BEM_INC_USER_TRACES, "unknown incident-field kind");
    if (inc->kind == BEM_INC_USER_TRACES) {
        BEM_REQUIRE(inc->g != nullptr, "BEM_INC_USER_TRACES needs g (and f, except for a screen)");
        return BEM_OK;
    }
    const double* p = inc->kind == BEM_INC_PLANE_WAVE ? inc->dirs : inc->sources;
    BEM_REQUIRE(p != nullptr, inc->kind == BEM_INC_PLANE_WAVE ? "plane waves need dirs" : "point sources need sources");
    for (int r = 0; r < inc->n_rhs; ++r) {
        const double* d = p + 3 * r;
        BEM_REQUIRE(std::isfinite(d[0]) && std::isfinite(d[1]) && std::isfinite(d[2]),
                    "incident directions or source positions are not finite");
        if (inc->kind == BEM_INC_PLANE_WAVE) {
            const double nd = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            BEM_REQUIRE(std::fabs(nd - 1.0) < 1e-6, "incident directions must be unit vectors");
        }
        if (inc->amps)
            BEM_REQUIRE(std::isfinite(inc->amps[r].re) && std::isfinite(inc->amps[r].im), "amplitude not finite");
    }
    return BEM_OK;
}

}  // namespace

extern "C" {

const char* bem_last_error(void) { return g_last_error.c_str(); }

const char* bem_version(void) { return "bem-gb300 0.1 (sm_103a)"; }

uint64_t bem_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

bem_status bem_selftest(bem_context* ctx, int which, double* result) {
    CTX_GUARD(ctx);
    BEM_REQUIRE(result != nullptr, "null result");
    BEM_REQUIRE(which >= 0 && which <= 12, "unknown self-test");
    if (which == 0) return selftest_sincos(1 << 20, 64.0f, result, ctx->stream);
    if (which == 3) return selftest_barrier(result, ctx->stream);
    if (which == 12) return selftest_tc(24, result, ctx->stream, 3);
    if (which >= 10) return selftest_tc(which == 10 ? 24 : 128, result, ctx->stream, 2);
    if (which >= 4) {
        // tile products: (arithmetic, storage bytes, columns)
        const int cfg[6][3] = {{TP_F32, 8, 1}, {TP_F32, 8, 5}, {TP_DD, 8, 1}, {TP_DD, 8, 3}, {TP_DD, 16, 1},
                               {TP_DD, 16, 8}};
        const int* c = cfg[which - 4];
        return selftest_tile(c[0], c[1], c[2], result, ctx->stream);
    }
    return selftest_tc(which == 1 ? 24 : 8, result, ctx->stream, 1);
}

bem_status bem_context_create(int device, void* stream, bem_context** out) {
    BEM_REQUIRE(out != nullptr, "out is null");
    *out = nullptr;
    int ndev = 0;
    BEM_CUDA_TRY(cudaGetDeviceCount(&ndev));
    BEM_REQUIRE(device >= 0 && device < ndev, "device index out of range");
    BEM_CUDA_TRY(cudaSetDevice(device));
    auto* c = new (std::nothrow) bem_context();
    if (!c) {
        set_error("host allocation failed");
        return BEM_E_OOM;
    }
    c->device = device;
    if (stream) {
        c->stream = static_cast<cudaStream_t>(stream);
        c->own_stream = false;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            set_error(std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
            return BEM_E_CUDA;
        }
        c->own_stream = true;
    }
    *out = c;
    return BEM_OK;
}

bem_status bem_context_destroy(bem_context* ctx) {
    if (!ctx) return BEM_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return BEM_OK;
}

bem_status bem_context_synchronize(bem_context* ctx) {
    CTX_GUARD(ctx);
    BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return BEM_OK;
}

bem_status bem_grid_create(bem_context* ctx, const double* xyz, int64_t nv, const int32_t* tri, int64_t nt,
                           int on_device, bem_grid** out) {
    CTX_GUARD(ctx);
    BEM_REQUIRE(out != nullptr, "out is null");
    *out = nullptr;
    BEM_REQUIRE(xyz != nullptr && tri != nullptr, "null vertex or triangle array");
    BEM_REQUIRE(nv >= 3 && nt >= 1, "a grid needs at least 3 vertices and 1 triangle");
    BEM_REQUIRE(nv < (int64_t)1 << 31 && nt < (int64_t)1 << 30, "grid too large for int32 indices");
    std::unique_ptr<bem_grid> g(new (std::nothrow) bem_grid());
    if (!g) {
        set_error("host allocation failed");
        return BEM_E_OOM;
    }
    g->ctx = ctx;
    g->nv = nv;
    g->nt = nt;
    g->h_xyz.resize(3 * nv);
    g->h_tri.resize(3 * nt);
    cudaStream_t s = ctx->stream;
    if (on_device) {
        BEM_CUDA_TRY(cudaMemcpyAsync(g->h_xyz.data(), xyz, 24 * nv, cudaMemcpyDeviceToHost, s));
        BEM_CUDA_TRY(cudaMemcpyAsync(g->h_tri.data(), tri, 12 * nt, cudaMemcpyDeviceToHost, s));
        BEM_CUDA_TRY(cudaStreamSynchronize(s));
    } else {
        std::memcpy(g->h_xyz.data(), xyz, 24 * nv);
        std::memcpy(g->h_tri.data(), tri, 12 * nt);
    }
    // validation
    for (int64_t i = 0; i < 3 * nv; ++i)
        if (!std::isfinite(g->h_xyz[i])) {
            set_error("vertex coordinate is not finite");
            return BEM_E_NONFINITE;
        }
    double vol6 = 0.0;
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t a = g->h_tri[3 * t], b = g->h_tri[3 * t + 1], c = g->h_tri[3 * t + 2];
        BEM_REQUIRE(a >= 0 && a < nv && b >= 0 && b < nv && c >= 0 && c < nv,
                    "triangle " + std::to_string(t) + " has a vertex index outside [0, nv)");
        BEM_REQUIRE(a != b && b != c && a != c, "triangle " + std::to_string(t) + " repeats a vertex");
        const double* A = &g->h_xyz[3 * (int64_t)a];
        const double* B = &g->h_xyz[3 * (int64_t)b];
        const double* C = &g->h_xyz[3 * (int64_t)c];
        const double e1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        const double e2[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
        const double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                              e1[0] * e2[1] - e1[1] * e2[0]};
        const double J = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        BEM_REQUIRE(J > 0.0, "triangle " + std::to_string(t) + " has zero area");
        g->surface_area += 0.5 * J;
        vol6 += A[0] * cr[0] + A[1] * cr[1] + A[2] * cr[2];
    }
    (void)vol6;
    BEM_TRY(g->xyz.alloc(24 * nv, s));
    BEM_TRY(g->tri.alloc(12 * nt, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(g->xyz.p, g->h_xyz.data(), 24 * nv, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(g->tri.p, g->h_tri.data(), 12 * nt, cudaMemcpyHostToDevice, s));
    BEM_TRY(grid_build_geometry(g.get()));
    *out = g.release();
    return BEM_OK;
}

bem_status bem_grid_destroy(bem_grid* g) {
    if (!g) return BEM_OK;
    cudaSetDevice(g->ctx->device);
    delete g;
    return BEM_OK;
}

int64_t bem_grid_num_vertices(const bem_grid* g) { return g ? g->nv : -1; }
int64_t bem_grid_num_triangles(const bem_grid* g) { return g ? g->nt : -1; }

bem_status bem_assemble(bem_context* ctx, int op, bem_c128 k, const bem_grid* test, const bem_grid* trial,
                        int precision, int n_singular, bem_matrix** out) {
    CTX_GUARD(ctx);
    BEM_REQUIRE(out != nullptr, "out is null");
    *out = nullptr;
    BEM_REQUIRE(test != nullptr && trial != nullptr, "null grid");
    BEM_REQUIRE(test == trial, "test and trial grids must be the same grid for V, K, T, D");
    BEM_REQUIRE(op >= BEM_OP_V && op <= BEM_OP_D, "unknown operator");
    BEM_REQUIRE(precision == BEM_PREC_FP64 || precision == BEM_PREC_MIXED, "unsupported precision");
    BEM_REQUIRE(n_singular >= 1 && n_singular <= 16, "n_singular must be in [1, 16]");
    BEM_REQUIRE(std::isfinite(k.re) && std::isfinite(k.im), "wavenumber is not finite");
    std::unique_ptr<bem_matrix> m(new (std::nothrow) bem_matrix());
    if (!m) {
        set_error("host allocation failed");
        return BEM_E_OOM;
    }
    const int64_t N = test->nv;
    m->rows = m->cols = N;
    cudaStream_t s = ctx->stream;
    if (precision == BEM_PREC_FP64) {
        m->entry_bytes = 16;
        BEM_TRY(m->data.alloc((size_t)N * N * 16, s));
        double2* p = m->data.as<double2>();
        BEM_TRY(assemble_operators_fp64(test, k.re, k.im, n_singular, op == BEM_OP_V ? p : nullptr,
                                        op == BEM_OP_K ? p : nullptr, op == BEM_OP_T ? p : nullptr,
                                        op == BEM_OP_D ? p : nullptr, op_layouts_dense(), s));
    } else {
        m->entry_bytes = 8;
        BEM_TRY(m->data.alloc((size_t)N * N * 8, s));
        BEM_CUDA_TRY(cudaMemsetAsync(m->data.p, 0, (size_t)N * N * 8, s));
        float2* p = m->data.as<float2>();
        float2* V = op == BEM_OP_V ? p : nullptr;
        float2* K = op == BEM_OP_K ? p : nullptr;
        float2* T = op == BEM_OP_T ? p : nullptr;
        float2* D = op == BEM_OP_D ? p : nullptr;
        BEM_TRY(assemble_regular_fp32(test, k.re, k.im, V, K, T, D, op_layouts_dense(), s));
        BEM_TRY(assemble_singular_into_c64(test, k.re, k.im, n_singular, V, K, T, D, op_layouts_dense(), s));
    }
    *out = m.release();
    return BEM_OK;
}

int bem_matrix_entry_bytes(const bem_matrix* m) { return m ? m->entry_bytes : 0; }

bem_status bem_matrix_destroy(bem_matrix* m) {
    delete m;
    return BEM_OK;
}

bem_status bem_matrix_shape(const bem_matrix* m, int64_t* rows, int64_t* cols) {
    BEM_REQUIRE(m != nullptr, "null matrix");
    if (rows) *rows = m->rows;
    if (cols) *cols = m->cols;
    return BEM_OK;
}

bem_status bem_matrix_copy_out(bem_context* ctx, const bem_matrix* m, void* dst, int64_t dst_bytes, int on_device) {
    CTX_GUARD(ctx);
    BEM_REQUIRE(m != nullptr && dst != nullptr, "null matrix or destination");
    const int64_t need = m->rows * m->cols * m->entry_bytes;
    BEM_REQUIRE(dst_bytes >= need, "destination smaller than rows*cols*entry_bytes");
    BEM_CUDA_TRY(cudaMemcpyAsync(dst, m->data.p, need, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 ctx->stream));
    if (!on_device) BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return BEM_OK;
}

bem_status bem_mass(bem_context* ctx, const bem_grid* g, bem_sparse** out) {
    CTX_GUARD(ctx);
    BEM_REQUIRE(out != nullptr && g != nullptr, "null argument");
    *out = nullptr;
    std::unique_ptr<bem_sparse> sp(new (std::nothrow) bem_sparse());
    if (!sp) {
        set_error("host allocation failed");
        return BEM_E_OOM;
    }
    cudaStream_t s = ctx->stream;
    sp->rows = sp->cols = g->nv;
    sp->nnz = g->m_nnz;
    BEM_TRY(sp->val.alloc(g->m_nnz * 8, s));
    BEM_TRY(mass_values(g, sp->val.as<double>(), s));
    // expand the CSR row pointer to COO rows on the host (pattern only)
    std::vector<int32_t> rowptr(g->nv + 1), rows(g->m_nnz);
    BEM_CUDA_TRY(cudaMemcpyAsync(rowptr.data(), g->m_rowptr.p, (g->nv + 1) * 4, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    for (int64_t i = 0; i < g->nv; ++i)
        for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) rows[e] = (int32_t)i;
    BEM_TRY(sp->row.alloc(g->m_nnz * 4, s));
    BEM_TRY(sp->col.alloc(g->m_nnz * 4, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(sp->row.p, rows.data(), g->m_nnz * 4, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(sp->col.p, g->m_col.p, g->m_nnz * 4, cudaMemcpyDeviceToDevice, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    *out = sp.release();
    return BEM_OK;
}

bem_status bem_projection(bem_context* ctx, const bem_grid* a, const bem_grid* b, const double* center,
                          bem_sparse** out) {
    CTX_GUARD(ctx);
    BEM_REQUIRE(out != nullptr && a != nullptr && b != nullptr, "null argument");
    *out = nullptr;
    double c0[3] = {0.0, 0.0, 0.0};
    if (center) {
        for (int d = 0; d < 3; ++d) c0[d] = center[d];
        BEM_REQUIRE(std::isfinite(c0[0]) && std::isfinite(c0[1]) && std::isfinite(c0[2]), "centre not finite");
    }
    std::unique_ptr<bem_sparse> sp(new (std::nothrow) bem_sparse());
    if (!sp) {
        set_error("host allocation failed");
        return BEM_E_OOM;
    }
    sp->rows = a->nv;
    sp->cols = b->nv;
    BEM_TRY(mortar_coo(a, b, c0, sp->row, sp->col, sp->val, &sp->nnz, ctx->stream));
    BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    *out = sp.release();
    return BEM_OK;
}

bem_status bem_sparse_destroy(bem_sparse* s) {
    delete s;
    return BEM_OK;
}

bem_status bem_sparse_info(const bem_sparse* s, int64_t* rows, int64_t* cols, int64_t* nnz) {
    BEM_REQUIRE(s != nullptr, "null sparse matrix");
    if (rows) *rows = s->rows;
    if (cols) *cols = s->cols;
    if (nnz) *nnz = s->nnz;
    return BEM_OK;
}

bem_status bem_sparse_copy_out(bem_context* ctx, const bem_sparse* sp, int32_t* row, int32_t* col, double* val,
                               int64_t capacity) {
    CTX_GUARD(ctx);
    BEM_REQUIRE(sp != nullptr && row != nullptr && col != nullptr && val != nullptr, "null argument");
    BEM_REQUIRE(capacity >= sp->nnz, "capacity smaller than nnz");
    if (sp->nnz == 0) return BEM_OK;
    cudaStream_t s = ctx->stream;
    BEM_CUDA_TRY(cudaMemcpyAsync(row, sp->row.p, sp->nnz * 4, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(col, sp->col.p, sp->nnz * 4, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(val, sp->val.p, sp->nnz * 8, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    return BEM_OK;
}

void bem_solve_opts_default(bem_solve_opts* o) {
    if (!o) return;
    o->gmres_tol = 1e-8;
    o->gmres_maxiter = 2000;
    o->precision = BEM_PREC_FP64;
    o->n_singular = 4;
    o->mtf_variant = BEM_MTF_DERIVED;
    o->center[0] = o->center[1] = o->center[2] = 0.0;
    o->ir_inner_tol = 0.0;  // chosen per solve (one right-hand side or a batch)
    o->batch_columns = 0;
    o->tensor_cores = 2;
    o->formulation = BEM_FORM_MTF;
    o->dd_switch = 1.0;
    o->cuda_graphs = 1;
}

bem_status bem_solve_transmission(bem_context* ctx, const bem_grid* ext, const bem_grid* intr, bem_c128 k_int,
                                  bem_c128 k_ext, double rho_int_over_rho_ext, const bem_incident* inc,
                                  const bem_solve_opts* opts, bem_c128* v_ext, bem_c128* w_ext, bem_c128* v_int,
                                  bem_c128* w_int, int on_device, bem_solve_report* rep) {
    CTX_GUARD(ctx);
    BEM_REQUIRE(ext != nullptr && intr != nullptr, "null grid");
    BEM_TRY(check_incident(inc));
    BEM_REQUIRE(inc->kind != BEM_INC_USER_TRACES || inc->f != nullptr, "BEM_INC_USER_TRACES needs f and g");
    BEM_REQUIRE(v_ext && w_ext && v_int && w_int, "null output array");
    BEM_REQUIRE(std::isfinite(rho_int_over_rho_ext) && rho_int_over_rho_ext > 0.0, "density ratio must be > 0");
    BEM_REQUIRE(std::isfinite(k_int.re) && std::isfinite(k_int.im) && std::isfinite(k_ext.re) &&
                    std::isfinite(k_ext.im), "wavenumber is not finite");
    bem_solve_opts o;
    if (opts) o = *opts;
    else bem_solve_opts_default(&o);
    BEM_REQUIRE(o.gmres_tol >= 0.0 && o.gmres_maxiter >= 1, "bad GMRES options");
    BEM_REQUIRE(o.n_singular >= 1 && o.n_singular <= 16, "n_singular must be in [1, 16]");
    BEM_REQUIRE(o.mtf_variant == BEM_MTF_DERIVED || o.mtf_variant == BEM_MTF_PRINTED, "unknown MTF variant");
    BEM_REQUIRE(o.precision == BEM_PREC_FP64 || o.precision == BEM_PREC_MIXED, "unsupported precision");
    BEM_REQUIRE(o.ir_inner_tol >= 0.0 && o.ir_inner_tol < 1.0, "ir_inner_tol must be 0 or in (0, 1)");
    BEM_REQUIRE(o.batch_columns >= 0 && o.batch_columns <= 128, "batch_columns must be in [0, 128]");
    BEM_REQUIRE(o.tensor_cores >= 0 && o.tensor_cores <= 3, "tensor_cores must be 0, 1, 2 or 3");
    BEM_REQUIRE(o.formulation >= BEM_FORM_MTF && o.formulation <= BEM_FORM_HC_INT_DIR, "unknown formulation");
    BEM_REQUIRE(o.cuda_graphs == 0 || o.cuda_graphs == 1, "cuda_graphs must be 0 or 1");
    BEM_REQUIRE(o.dd_switch >= 0.0 && o.dd_switch <= 1.0, "dd_switch must be in [0, 1]");
    return solve_transmission_impl(ctx, ext, intr, k_int, k_ext, rho_int_over_rho_ext, inc, &o, v_ext, w_ext, v_int,
                                   w_int, on_device, rep);
}

bem_status bem_context_set_exclusive(bem_context* ctx, int exclusive) {
    CTX_GUARD(ctx);
    BEM_REQUIRE(exclusive == 0 || exclusive == 1, "exclusive must be 0 or 1");
    ctx->exclusive = exclusive != 0;
    return BEM_OK;
}

bem_status bem_solve_screen(bem_context* ctx, const bem_grid* screen, const bem_grid* coarse, bem_c128 k,
                            const bem_incident* inc, const bem_solve_opts* opts, int32_t precond, bem_c128* phi,
                            int on_device, bem_solve_report* rep) {
    CTX_GUARD(ctx);
    BEM_REQUIRE(screen != nullptr, "null screen grid");
    BEM_REQUIRE(precond == BEM_SCREEN_MASS || precond == BEM_SCREEN_OO, "unknown screen preconditioner");
    BEM_REQUIRE(precond == BEM_SCREEN_MASS || coarse != nullptr, "the opposite-order preconditioner needs a grid");
    BEM_TRY(check_incident(inc));
    BEM_REQUIRE(phi != nullptr, "null output array");
    BEM_REQUIRE(std::isfinite(k.re) && std::isfinite(k.im), "wavenumber is not finite");
    bem_solve_opts o;
    if (opts) o = *opts;
    else bem_solve_opts_default(&o);
    BEM_REQUIRE(o.gmres_tol >= 0.0 && o.gmres_maxiter >= 1, "bad GMRES options");
    BEM_REQUIRE(o.n_singular >= 1 && o.n_singular <= 16, "n_singular must be in [1, 16]");
    BEM_REQUIRE(o.precision == BEM_PREC_FP64 || o.precision == BEM_PREC_MIXED, "unsupported precision");
    BEM_REQUIRE(o.ir_inner_tol >= 0.0 && o.ir_inner_tol < 1.0, "ir_inner_tol must be 0 or in (0, 1)");
    BEM_REQUIRE(o.batch_columns >= 0 && o.batch_columns <= 128, "batch_columns must be in [0, 128]");
    BEM_REQUIRE(o.cuda_graphs == 0 || o.cuda_graphs == 1, "cuda_graphs must be 0 or 1");
    BEM_REQUIRE(o.dd_switch >= 0.0 && o.dd_switch <= 1.0, "dd_switch must be in [0, 1]");
    return solve_screen_impl(ctx, screen, coarse, k, inc, &o, precond, phi, on_device, rep);
}

bem_status bem_autotune(bem_context* ctx, const bem_grid* ext, const bem_grid* intr, int32_t n_rhs) {
    CTX_GUARD(ctx);
    BEM_REQUIRE(ext != nullptr && intr != nullptr, "null grid");
    BEM_REQUIRE(n_rhs >= 1 && n_rhs <= 4096, "n_rhs must be in [1, 4096]");
    return autotune_impl(ctx, ext, intr, n_rhs, 5);
}

bem_status bem_field(bem_context* ctx, const bem_grid* g, bem_c128 k, const bem_c128* phi, const bem_c128* psi,
                     const double* points, int64_t npts, bem_c128* u, int on_device) {
    CTX_GUARD(ctx);
    BEM_REQUIRE(g != nullptr, "null grid");
    BEM_REQUIRE(phi != nullptr || psi != nullptr, "need phi or psi");
    BEM_REQUIRE(npts >= 0 && (npts == 0 || (points != nullptr && u != nullptr)), "bad points or output");
    BEM_REQUIRE(std::isfinite(k.re) && std::isfinite(k.im), "wavenumber is not finite");
    if (npts == 0) return BEM_OK;
    if (!on_device)
        for (int64_t i = 0; i < 3 * npts; ++i) BEM_REQUIRE(std::isfinite(points[i]), "point is not finite");
    return field_impl(ctx, g, k, phi, psi, points, npts, u, on_device);
}

bem_status bem_solve_many(bem_context* ctx, int32_t count, const bem_instance* instances, const bem_solve_opts* opts,
                          int on_device, bem_solve_report* reports) {
    CTX_GUARD(ctx);
    BEM_REQUIRE(count >= 1 && instances != nullptr, "need count >= 1 instances");
    bem_solve_opts o;
    if (opts) o = *opts;
    else {
        bem_solve_opts_default(&o);
        o.precision = BEM_PREC_MIXED;
    }
    BEM_REQUIRE(o.precision == BEM_PREC_MIXED, "bem_solve_many runs the mixed-precision mode");
    BEM_REQUIRE(o.formulation == BEM_FORM_MTF, "bem_solve_many solves the multiple-traces system only");
    BEM_REQUIRE(o.cuda_graphs == 0 || o.cuda_graphs == 1, "cuda_graphs must be 0 or 1");
    BEM_REQUIRE(o.dd_switch >= 0.0 && o.dd_switch <= 1.0, "dd_switch must be in [0, 1]");
    BEM_REQUIRE(o.gmres_tol >= 0.0 && o.gmres_maxiter >= 1, "bad GMRES options");
    BEM_REQUIRE(o.n_singular >= 1 && o.n_singular <= 16, "n_singular must be in [1, 16]");
    BEM_REQUIRE(o.mtf_variant == BEM_MTF_DERIVED || o.mtf_variant == BEM_MTF_PRINTED, "unknown MTF variant");
    BEM_REQUIRE(o.ir_inner_tol >= 0.0 && o.ir_inner_tol < 1.0, "ir_inner_tol must be 0 or in (0, 1)");
    for (int i = 0; i < count; ++i) {
        const bem_instance& q = instances[i];
        BEM_REQUIRE(q.ext != nullptr && q.intr != nullptr, "null grid");
        BEM_REQUIRE(q.v_ext && q.w_ext && q.v_int && q.w_int, "null output array");
        BEM_REQUIRE(std::isfinite(q.rho_int_over_rho_ext) && q.rho_int_over_rho_ext > 0.0, "density ratio must be > 0");
        BEM_REQUIRE(std::isfinite(q.k_int.re) && std::isfinite(q.k_int.im) && std::isfinite(q.k_ext.re) &&
                        std::isfinite(q.k_ext.im) && std::isfinite(q.amp.re) && std::isfinite(q.amp.im),
                    "wavenumber or amplitude is not finite");
        const double nd = std::sqrt(q.dir[0] * q.dir[0] + q.dir[1] * q.dir[1] + q.dir[2] * q.dir[2]);
        BEM_REQUIRE(std::isfinite(nd) && std::fabs(nd - 1.0) < 1e-6, "incident directions must be unit vectors");
    }
    return solve_many_impl(ctx, count, instances, &o, on_device, reports);
}

}  // extern "C"
