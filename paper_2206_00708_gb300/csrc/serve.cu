// Request server for streams of transmission solves (continuous batching with
// admission by HBM budget).  Host-side C++: worker threads, each with its own context
// and CUDA stream, take requests from a FIFO queue when a slot is free and the
// request's device working set fits in what is left of the budget; the GPU work of
// different requests overlaps on the streams.  Small mixed-precision requests that
// wait together at the head of the queue are taken as one lockstep group and solved
// through the many-instance path (one launch per GMRES step for all their waves).
#include "bem_internal.cuh"

#include <condition_variable>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>

namespace bem {

// lockstep groups: at most this many bytes of complex64 operator tiles in one group
// (the operators of a group are read once per wave and product, so they should stay
// in L2), at most this many plane waves, and only requests of at most GROUP_RHS waves
// (a request with more waves runs faster alone, its waves as columns of one product)
constexpr int64_t GROUP_OP_BYTES = 64ll << 20;
constexpr int GROUP_MAX_WAVES = 64;
constexpr int GROUP_RHS = 2;
constexpr int GROUP_MAX_DEFAULT = 8;
constexpr int GROUP_SCAN = 4;  // a group looks at the first GROUP_SCAN * group_max queued requests

bem_status solve_transmission_impl(bem_context* ctx, const bem_grid* ge, const bem_grid* gi, bem_c128 k_int,
                                   bem_c128 k_ext, double rho_ratio, const bem_incident* inc,
                                   const bem_solve_opts* o, bem_c128* v_ext, bem_c128* w_ext, bem_c128* v_int,
                                   bem_c128* w_int, int on_device, bem_solve_report* rep);

namespace {

enum class RState { Queued, Running, Done };

struct Request {
    uint64_t ticket = 0;
    std::vector<double> xe, xi, dirs;
    std::vector<int32_t> te, ti;
    std::vector<bem_c128> amps;
    bem_c128 k_ext{}, k_int{};
    double rho = 1.0;
    int32_t n_rhs = 1, precision = BEM_PREC_MIXED;
    double tol = 1e-8;
    int32_t maxiter = 2000;
    double t_submit = 0, t_start = 0, t_end = 0, deadline = 0;
    int64_t bytes = 0, op_bytes = 0;
    std::atomic<int> cancel{0};
    RState state = RState::Queued;
    bem_result result{};
    std::vector<bem_c128> v_ext, w_ext, v_int, w_int;
};

}  // namespace
}  // namespace bem

struct bem_server {
    bem_server_opts opts{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<bem::Request>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<bem::Request>> all;
    std::vector<std::thread> workers;
    std::vector<bem_context*> contexts;
    bool stopping = false;
    uint64_t next_ticket = 1;
    int64_t reserved = 0, high_water = 0;
    int group_max = 1;
    bem_serve_stats stats{};
};

namespace bem {
namespace {

// Upper estimate of a request's device working set.  A served request always solves
// the multiple-traces system (bem_request carries no formulation): its operators are the
// four blocks of each grid, its Krylov vectors have 2 N_e + 2 N_i entries.
int64_t working_set_bytes(int64_t ne, int64_t ni, int precision, int maxiter, int n_rhs) {
    const int64_t n = 2 * ne + 2 * ni;
    const int64_t esz = precision == BEM_PREC_MIXED ? 8 : 16;
    // tiled operators: V, D as upper tile triangles, K in full (64 x 64 tiles)
    const int64_t te = op_tiles(ne), ti = op_tiles(ni);
    const int64_t ops = (te * (te + 1) + te * te + ti * (ti + 1) + ti * ti) * OPT * OPT * esz;
    const int64_t m = std::min<int64_t>(maxiter, n) + 1;
    // the solver advances up to 64 (mixed precision, tensor-core products) or 8
    // right-hand sides together, each with its own Krylov basis and Hessenberg matrix
    const int64_t R = std::max(1, std::min(n_rhs, precision == BEM_PREC_MIXED ? 64 : 8));
    // basis (counted at 16 bytes per entry: complex128, or complex64 plus slack), Hessenberg,
    // and the inner-product partials of the row chunks (256 rows, or 128 for the fused pass)
    const int64_t chunks = std::max<int64_t>(std::min<int64_t>(1216, (n + 255) / 256), (n + 127) / 128);
    const int64_t krylov = R * (m * n * 16 + m * m * 16 + m * chunks * 16) + (R + 8) * n * 16;
    const int64_t vectors = 16 * (R + 8) * n * 16;
    // partial sums of the tile products (8 columns, double-float) and the input splits
    const int64_t partial = 2 * (te * te + ti * ti) * OPT * 8 * 16 + 8 * n * 16;
    // tensor-core batches (mixed, more than 8 waves) also keep a copy of the blocks (dense
    // complex64, from which the FP16 split copy is made: both exist for a moment)
    const int64_t dense = precision == BEM_PREC_MIXED && R > 8 ? 2 * 4 * (ne * ne + ni * ni) * 8 : 0;
    const int64_t tc = precision == BEM_PREC_MIXED ? 128 * ((R + 7) / 8 * 8) * (ne + ni + 16) + dense : 0;
    const int64_t grids = 600 * (ne + ni) * 2;
    const int64_t mortar = 2 * 9 * 40 * (ne + ni) * 16;
    return ops + krylov + vectors + partial + tc + grids + mortar + (int64_t)(16 << 20);
}

// complex64 tile bytes of a request's operators (V, D upper tile triangles, K)
int64_t operator_bytes_c64(int64_t ne, int64_t ni) {
    const int64_t te = op_tiles(ne), ti = op_tiles(ni);
    return (te * (te + 1) + te * te + ti * (ti + 1) + ti * ti) * OPT * OPT * 8;
}

bool groupable(const Request& r) {
    return r.precision == BEM_PREC_MIXED && r.op_bytes <= GROUP_OP_BYTES && r.n_rhs <= GROUP_RHS;
}

void finish_locked(bem_server* srv, const std::shared_ptr<Request>& r, int32_t status) {
    r->t_end = now_seconds();
    r->state = RState::Done;
    r->result.status = status;
    r->result.queue_ms = 1e3 * ((r->t_start > 0 ? r->t_start : r->t_end) - r->t_submit);
    r->result.run_ms = r->t_start > 0 ? 1e3 * (r->t_end - r->t_start) : 0.0;
    r->result.total_ms = 1e3 * (r->t_end - r->t_submit);
    switch (status) {
        case BEM_OK: srv->stats.completed++; break;
        case BEM_E_CANCELLED: srv->stats.cancelled++; break;
        case BEM_E_TIMEOUT: srv->stats.timed_out++; break;
        default: srv->stats.failed++; break;
    }
}

// a member's stop condition (cancellation, its deadline)
bem_status member_halt(const Request& r) {
    if (r.cancel.load()) return BEM_E_CANCELLED;
    if (r.deadline > 0 && now_seconds() > r.deadline) return BEM_E_TIMEOUT;
    return BEM_OK;
}

// one request alone, through the single-problem solver (its waves batched as columns)
int32_t run_alone(bem_context* ctx, Request& r) {
    const int64_t ne = (int64_t)r.xe.size() / 3, ni = (int64_t)r.xi.size() / 3;
    ctx->cancel = &r.cancel;
    ctx->deadline = r.deadline;
    bem_grid *ge = nullptr, *gi = nullptr;
    bem_status st = bem_grid_create(ctx, r.xe.data(), ne, r.te.data(), (int64_t)r.te.size() / 3, 0, &ge);
    if (st == BEM_OK) st = bem_grid_create(ctx, r.xi.data(), ni, r.ti.data(), (int64_t)r.ti.size() / 3, 0, &gi);
    if (st == BEM_OK) {
        bem_incident inc{};
        inc.n_rhs = r.n_rhs;
        inc.dirs = r.dirs.data();
        inc.amps = r.amps.empty() ? nullptr : r.amps.data();
        bem_solve_opts o;
        bem_solve_opts_default(&o);
        o.precision = r.precision;
        o.gmres_tol = r.tol;
        o.gmres_maxiter = r.maxiter;
        bem_solve_report rep{};
        st = solve_transmission_impl(ctx, ge, gi, r.k_int, r.k_ext, r.rho, &inc, &o, r.v_ext.data(), r.w_ext.data(),
                                     r.v_int.data(), r.w_int.data(), 0, &rep);
        r.result.iterations = rep.iterations;
        r.result.residual = rep.residual;
    }
    if (ge) bem_grid_destroy(ge);
    if (gi) bem_grid_destroy(gi);
    cudaStreamSynchronize(ctx->stream);
    ctx->cancel = nullptr;
    ctx->deadline = 0.0;
    return st;
}

// the waves of all members as instances of one lockstep solve; statuses per member
void run_lockstep(bem_context* ctx, std::vector<std::shared_ptr<Request>>& g, std::vector<int32_t>& status) {
    const int m = (int)g.size();
    std::vector<bem_grid*> grids(2 * m, nullptr);
    bem_status st = BEM_OK;
    for (int i = 0; i < m && st == BEM_OK; ++i) {
        Request& r = *g[i];
        st = bem_grid_create(ctx, r.xe.data(), (int64_t)r.xe.size() / 3, r.te.data(), (int64_t)r.te.size() / 3, 0,
                             &grids[2 * i]);
        if (st == BEM_OK)
            st = bem_grid_create(ctx, r.xi.data(), (int64_t)r.xi.size() / 3, r.ti.data(), (int64_t)r.ti.size() / 3,
                                 0, &grids[2 * i + 1]);
    }
    std::vector<bem_instance> inst;
    std::vector<int> owner;
    if (st == BEM_OK) {
        for (int i = 0; i < m; ++i) {
            Request& r = *g[i];
            const int64_t ne = (int64_t)r.xe.size() / 3, ni = (int64_t)r.xi.size() / 3;
            for (int w = 0; w < r.n_rhs; ++w) {
                bem_instance q{};
                q.ext = grids[2 * i];
                q.intr = grids[2 * i + 1];
                q.k_ext = r.k_ext;
                q.k_int = r.k_int;
                q.rho_int_over_rho_ext = r.rho;
                for (int d = 0; d < 3; ++d) q.dir[d] = r.dirs[3 * w + d];
                q.amp = r.amps.empty() ? bem_c128{1.0, 0.0} : r.amps[w];
                q.v_ext = r.v_ext.data() + w * ne;
                q.w_ext = r.w_ext.data() + w * ne;
                q.v_int = r.v_int.data() + w * ni;
                q.w_int = r.w_int.data() + w * ni;
                inst.push_back(q);
                owner.push_back(i);
            }
        }
        bem_solve_opts o;
        bem_solve_opts_default(&o);
        o.precision = BEM_PREC_MIXED;
        o.gmres_tol = g[0]->tol;
        o.gmres_maxiter = g[0]->maxiter;
        const HaltCheck halt = [&](int k) { return member_halt(*g[owner[k]]); };
        const int n = (int)inst.size();
        std::vector<int32_t> ist(n, BEM_OK);
        std::vector<bem_solve_report> reps(n);
        st = solve_many_impl(ctx, n, inst.data(), &o, 0, reps.data(), &halt, ist.data());
        for (int i = 0; i < m; ++i) {
            g[i]->result.iterations = 0;
            g[i]->result.residual = 0.0;
        }
        for (int k = 0; k < n; ++k) {
            Request& r = *g[owner[k]];
            r.result.iterations = std::max(r.result.iterations, reps[k].iterations);
            r.result.residual = std::max(r.result.residual, reps[k].residual);
            if (status[owner[k]] == BEM_OK) status[owner[k]] = ist[k];
        }
    }
    if (st != BEM_OK && st != BEM_E_NOT_CONVERGED)
        for (int i = 0; i < m; ++i) status[i] = st;
    for (bem_grid* gr : grids)
        if (gr) bem_grid_destroy(gr);
    cudaStreamSynchronize(ctx->stream);
}

// runs a group (one request or a lockstep group) and sets each member's status
void run_group(bem_server* srv, bem_context* ctx, std::vector<std::shared_ptr<Request>>& g,
               std::vector<int32_t>& status) {
    const int m = (int)g.size();
    status.assign(m, BEM_OK);
    for (auto& r : g) {
        const int64_t ne = (int64_t)r->xe.size() / 3, ni = (int64_t)r->xi.size() / 3;
        r->v_ext.assign((size_t)r->n_rhs * ne, bem_c128{0, 0});
        r->w_ext.assign((size_t)r->n_rhs * ne, bem_c128{0, 0});
        r->v_int.assign((size_t)r->n_rhs * ni, bem_c128{0, 0});
        r->w_int.assign((size_t)r->n_rhs * ni, bem_c128{0, 0});
    }
    if (srv->opts.dry_run) {
        // simulated service time (the longest member's), with the members' stop checks
        double us = 0.0;
        for (auto& r : g)
            us = std::max(us, srv->opts.dry_run_us_per_unknown * (double)(r->xe.size() / 3 * 2 + r->xi.size() / 3 * 2) *
                                  r->n_rhs);
        const double t_end = now_seconds() + us * 1e-6;
        for (;;) {
            bool live = false;
            for (int i = 0; i < m; ++i) {
                if (status[i] == BEM_OK) status[i] = member_halt(*g[i]);
                live = live || status[i] == BEM_OK;
            }
            if (!live || now_seconds() >= t_end) break;
            std::this_thread::sleep_for(std::chrono::microseconds(200));
        }
        for (auto& r : g) {
            r->result.iterations = 0;
            r->result.residual = 0.0;
        }
        return;
    }
    if (m == 1) status[0] = run_alone(ctx, *g[0]);
    else run_lockstep(ctx, g, status);
}

void worker_main(bem_server* srv, int idx) {
    bem_context* ctx = srv->opts.dry_run ? nullptr : srv->contexts[idx];
    if (ctx) cudaSetDevice(ctx->device);
    for (;;) {
        std::vector<std::shared_ptr<Request>> g;
        int64_t gbytes = 0;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv_work.wait(lk, [&] {
                if (srv->stopping) return true;
                if (srv->queue.empty()) return false;
                const auto& h = srv->queue.front();
                return h->cancel.load() || srv->reserved + h->bytes <= srv->opts.hbm_budget_bytes;
            });
            if (srv->stopping) return;
            std::shared_ptr<Request> r = srv->queue.front();
            srv->queue.pop_front();
            if (r->cancel.load()) {
                srv->stats.queued = (int64_t)srv->queue.size();
                finish_locked(srv, r, BEM_E_CANCELLED);
                srv->cv_done.notify_all();
                srv->cv_work.notify_all();
                continue;
            }
            g.push_back(r);
            gbytes = r->bytes;
            // requests of the same kind from the first places of the queue join its
            // lockstep group while they fit; those passed over keep their order and
            // their room in the budget (they are next for the following free slot)
            if (srv->group_max > 1 && groupable(*r)) {
                int64_t ops = r->op_bytes, passed = 0;
                int waves = r->n_rhs;
                size_t pos = 0;
                const size_t window = (size_t)GROUP_SCAN * (size_t)srv->group_max;
                while (pos < srv->queue.size() && pos < window && (int)g.size() < srv->group_max) {
                    std::shared_ptr<Request> q = srv->queue[pos];
                    if (q->cancel.load()) {
                        srv->queue.erase(srv->queue.begin() + (std::ptrdiff_t)pos);
                        finish_locked(srv, q, BEM_E_CANCELLED);
                        continue;
                    }
                    if (groupable(*q) && q->tol == r->tol && q->maxiter == r->maxiter &&
                        waves + q->n_rhs <= GROUP_MAX_WAVES && ops + q->op_bytes <= GROUP_OP_BYTES &&
                        srv->reserved + gbytes + passed + q->bytes <= srv->opts.hbm_budget_bytes) {
                        srv->queue.erase(srv->queue.begin() + (std::ptrdiff_t)pos);
                        g.push_back(q);
                        gbytes += q->bytes;
                        ops += q->op_bytes;
                        waves += q->n_rhs;
                    } else {
                        passed += q->bytes;
                        ++pos;
                    }
                }
            }
            srv->stats.queued = (int64_t)srv->queue.size();
            const double t0 = now_seconds();
            int waves = 0;
            for (auto& q : g) waves += q->n_rhs;
            for (auto& q : g) {
                q->state = RState::Running;
                q->t_start = t0;
                q->result.group_size = (int32_t)g.size();
                q->result.group_waves = waves;
            }
            if (g.size() > 1) {
                srv->stats.groups++;
                srv->stats.grouped += (int64_t)g.size();
            }
            srv->reserved += gbytes;
            srv->high_water = std::max(srv->high_water, srv->reserved);
            srv->stats.running += (int64_t)g.size();
        }
        std::vector<int32_t> status;
        run_group(srv, ctx, g, status);
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->reserved -= gbytes;
            srv->stats.running -= (int64_t)g.size();
            for (size_t i = 0; i < g.size(); ++i) finish_locked(srv, g[i], status[i]);
        }
        srv->cv_done.notify_all();
        srv->cv_work.notify_all();
    }
}

}  // namespace
}  // namespace bem

using namespace bem;

extern "C" {

void bem_serve_opts_default(bem_server_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->device = 0;
    o->max_inflight = 4;
    o->hbm_budget_bytes = 0;
    o->precision = BEM_PREC_MIXED;
    o->gmres_maxiter = 2000;
    o->gmres_tol = 1e-8;
    o->dry_run = 0;
    o->group_max = 0;
    o->dry_run_us_per_unknown = 1.0;
}

bem_status bem_serve_create(const bem_server_opts* opts, bem_server** out) {
    BEM_REQUIRE(out != nullptr, "out is null");
    *out = nullptr;
    bem_server_opts o;
    if (opts) o = *opts;
    else bem_serve_opts_default(&o);
    BEM_REQUIRE(o.max_inflight >= 1 && o.max_inflight <= 64, "max_inflight must be in [1, 64]");
    BEM_REQUIRE(o.precision == BEM_PREC_FP64 || o.precision == BEM_PREC_MIXED, "unknown precision");
    BEM_REQUIRE(o.gmres_maxiter >= 1 && o.gmres_tol >= 0.0, "bad GMRES options");
    BEM_REQUIRE(o.group_max >= 0 && o.group_max <= 64, "group_max must be in [0, 64]");
    std::unique_ptr<bem_server> srv(new (std::nothrow) bem_server());
    if (!srv) {
        set_error("host allocation failed");
        return BEM_E_OOM;
    }
    if (!o.dry_run) {
        BEM_CUDA_TRY(cudaSetDevice(o.device));
        size_t free_b = 0, total_b = 0;
        BEM_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
        if (o.hbm_budget_bytes <= 0) o.hbm_budget_bytes = (int64_t)(0.8 * (double)free_b);
        // keep freed stream-ordered allocations in the pool between requests
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, o.device) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        for (int i = 0; i < o.max_inflight; ++i) {
            bem_context* c = nullptr;
            bem_status st = bem_context_create(o.device, nullptr, &c);
            if (st != BEM_OK) {
                for (bem_context* x : srv->contexts) bem_context_destroy(x);
                return st;
            }
            c->exclusive = false;  // the workers' solves overlap on the device (never fused)
            srv->contexts.push_back(c);
        }
    } else {
        BEM_REQUIRE(o.hbm_budget_bytes > 0, "dry-run servers need an explicit hbm_budget_bytes");
        BEM_REQUIRE(o.dry_run_us_per_unknown >= 0.0, "dry_run_us_per_unknown must be >= 0");
    }
    srv->opts = o;
    srv->group_max = o.group_max == 0 ? GROUP_MAX_DEFAULT : o.group_max;
    srv->stats.hbm_budget_bytes = o.hbm_budget_bytes;
    bem_server* p = srv.release();
    for (int i = 0; i < o.max_inflight; ++i) p->workers.emplace_back(worker_main, p, i);
    *out = p;
    return BEM_OK;
}

bem_status bem_serve_destroy(bem_server* srv) {
    if (!srv) return BEM_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stopping = true;
        for (auto& kv : srv->all) kv.second->cancel.store(1);
    }
    srv->cv_work.notify_all();
    for (auto& t : srv->workers) t.join();
    for (bem_context* c : srv->contexts) bem_context_destroy(c);
    delete srv;
    return BEM_OK;
}

bem_status bem_serve_submit(bem_server* srv, const bem_request* q, uint64_t* ticket) {
    BEM_REQUIRE(srv != nullptr && q != nullptr && ticket != nullptr, "null argument");
    BEM_REQUIRE(q->xyz_ext && q->tri_ext && q->xyz_int && q->tri_int && q->dirs, "null request array");
    BEM_REQUIRE(q->nv_ext >= 3 && q->nt_ext >= 1 && q->nv_int >= 3 && q->nt_int >= 1, "empty grid");
    BEM_REQUIRE(q->n_rhs >= 1, "n_rhs must be >= 1");
    BEM_REQUIRE(std::isfinite(q->rho_int_over_rho_ext) && q->rho_int_over_rho_ext > 0.0, "density ratio must be > 0");
    BEM_REQUIRE(q->precision == -1 || q->precision == BEM_PREC_FP64 || q->precision == BEM_PREC_MIXED,
                "unknown precision");
    BEM_REQUIRE(q->timeout_ms >= 0.0, "timeout must be >= 0");
    auto r = std::make_shared<Request>();
    r->xe.assign(q->xyz_ext, q->xyz_ext + 3 * q->nv_ext);
    r->te.assign(q->tri_ext, q->tri_ext + 3 * q->nt_ext);
    r->xi.assign(q->xyz_int, q->xyz_int + 3 * q->nv_int);
    r->ti.assign(q->tri_int, q->tri_int + 3 * q->nt_int);
    r->dirs.assign(q->dirs, q->dirs + 3 * q->n_rhs);
    if (q->amps) r->amps.assign(q->amps, q->amps + q->n_rhs);
    r->k_ext = q->k_ext;
    r->k_int = q->k_int;
    r->rho = q->rho_int_over_rho_ext;
    r->n_rhs = q->n_rhs;
    r->precision = q->precision < 0 ? srv->opts.precision : q->precision;
    r->tol = srv->opts.gmres_tol;
    r->maxiter = srv->opts.gmres_maxiter;
    r->bytes = working_set_bytes(q->nv_ext, q->nv_int, r->precision, srv->opts.gmres_maxiter, q->n_rhs);
    r->op_bytes = operator_bytes_c64(q->nv_ext, q->nv_int);
    r->result.group_size = 1;
    r->result.group_waves = q->n_rhs;
    r->result.nv_ext = q->nv_ext;
    r->result.nv_int = q->nv_int;
    r->result.n_rhs = q->n_rhs;
    r->result.precision = r->precision;
    r->result.bytes_reserved = r->bytes;
    std::lock_guard<std::mutex> lk(srv->mu);
    BEM_REQUIRE(!srv->stopping, "server is shutting down");
    if (r->bytes > srv->opts.hbm_budget_bytes) {
        srv->stats.refused++;
        set_error("request needs about " + std::to_string(r->bytes) + " device bytes, more than the budget of " +
                  std::to_string(srv->opts.hbm_budget_bytes));
        return BEM_E_ADMISSION_REFUSED;
    }
    r->t_submit = now_seconds();
    r->deadline = q->timeout_ms > 0 ? r->t_submit + 1e-3 * q->timeout_ms : 0.0;
    r->ticket = srv->next_ticket++;
    srv->all[r->ticket] = r;
    srv->queue.push_back(r);
    srv->stats.submitted++;
    srv->stats.queued = (int64_t)srv->queue.size();
    *ticket = r->ticket;
    srv->cv_work.notify_one();
    return BEM_OK;
}

bem_status bem_serve_poll(bem_server* srv, uint64_t ticket, bem_result* info, bem_c128* v_ext, bem_c128* w_ext,
                          bem_c128* v_int, bem_c128* w_int) {
    BEM_REQUIRE(srv != nullptr, "null server");
    std::shared_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = srv->all.find(ticket);
        BEM_REQUIRE(it != srv->all.end(), "unknown or released ticket");
        r = it->second;
        if (r->state != RState::Done) return BEM_E_BUSY;
        srv->all.erase(it);
    }
    if (info) *info = r->result;
    auto copy = [](bem_c128* dst, const std::vector<bem_c128>& src) {
        if (dst && !src.empty()) std::memcpy(dst, src.data(), src.size() * sizeof(bem_c128));
    };
    copy(v_ext, r->v_ext);
    copy(w_ext, r->w_ext);
    copy(v_int, r->v_int);
    copy(w_int, r->w_int);
    return BEM_OK;
}

bem_status bem_serve_wait(bem_server* srv, uint64_t ticket, double timeout_ms) {
    BEM_REQUIRE(srv != nullptr, "null server");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->all.find(ticket);
    BEM_REQUIRE(it != srv->all.end(), "unknown or released ticket");
    std::shared_ptr<Request> r = it->second;
    const auto pred = [&] { return r->state == RState::Done; };
    if (timeout_ms <= 0) srv->cv_done.wait(lk, pred);
    else if (!srv->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), pred))
        return BEM_E_BUSY;
    return BEM_OK;
}

bem_status bem_serve_cancel(bem_server* srv, uint64_t ticket) {
    BEM_REQUIRE(srv != nullptr, "null server");
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = srv->all.find(ticket);
        BEM_REQUIRE(it != srv->all.end(), "unknown or released ticket");
        std::shared_ptr<Request> r = it->second;
        if (r->state == RState::Done) return BEM_OK;
        r->cancel.store(1);
        if (r->state == RState::Queued) {
            for (auto q = srv->queue.begin(); q != srv->queue.end(); ++q)
                if (*q == r) {
                    srv->queue.erase(q);
                    break;
                }
            srv->stats.queued = (int64_t)srv->queue.size();
            finish_locked(srv, r, BEM_E_CANCELLED);
        }
    }
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
    return BEM_OK;
}

bem_status bem_serve_get_stats(bem_server* srv, bem_serve_stats* st) {
    BEM_REQUIRE(srv != nullptr && st != nullptr, "null argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    *st = srv->stats;
    st->hbm_reserved_bytes = srv->reserved;
    st->hbm_high_water_bytes = srv->high_water;
    st->queued = (int64_t)srv->queue.size();
    return BEM_OK;
}

}  // extern "C"
