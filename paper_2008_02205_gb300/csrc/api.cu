// C ABI of the library (include/mlpg.h): argument checks, the call-order state
// machine, host<->device copies, stage outputs and statistics.  Every entry
// point returns a status; nothing throws across the ABI.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <thread>

#include "internal.h"

namespace mlpg {

mlpg_status set_err(mlpg_ctx *ctx, mlpg_status s, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return s;
}

mlpg_status cuda_fail(mlpg_ctx *ctx, cudaError_t e, const char *what, const char *file, int line) {
    std::string m = std::string("CUDA error '") + cudaGetErrorString(e) + "' in " + what + " (" + file + ":" +
                    std::to_string(line) + ")";
    cudaGetLastError();
    return set_err(ctx, MLPG_ERR_CUDA, m);
}

mlpg_status shard_sum_host(mlpg_ctx *ctx, double *host, int64_t count) {
    if (!ctx->reduce_fn) return MLPG_OK;
    if (ctx->reduce_fn(host, count, ctx->reduce_user) != 0)
        return set_err(ctx, MLPG_ERR_ARG, "cross-shard sum failed");
    return MLPG_OK;
}

mlpg_status shard_sum_dev(mlpg_ctx *ctx, double *dev, int64_t count) {
    if (!ctx->reduce_fn) return MLPG_OK;
    if (count > ctx->n + 8) return set_err(ctx, MLPG_ERR_ARG, "cross-shard sum too long");
    if (!ctx->reduce_host) {
        void *hp = nullptr;
        CU(ctx, cudaHostAlloc(&hp, sizeof(double) * (ctx->n + 8), cudaHostAllocDefault));
        ctx->host_allocs.push_back(hp);
        ctx->reduce_host = static_cast<double *>(hp);
    }
    CU(ctx, cudaMemcpyAsync(ctx->reduce_host, dev, sizeof(double) * count, cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    MLPG_TRY(shard_sum_host(ctx, ctx->reduce_host, count));
    CU(ctx, cudaMemcpyAsync(dev, ctx->reduce_host, sizeof(double) * count, cudaMemcpyHostToDevice, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));   // the host buffer is reused by the next sum
    return MLPG_OK;
}

void harvest_timing(mlpg_ctx *ctx) {
    for (int k = 0; k < ctx->ev_used; ++k) {
        float ms = 0.f;
        cudaEventSynchronize(ctx->ev_pool[k].second);
        if (cudaEventElapsedTime(&ms, ctx->ev_pool[k].first, ctx->ev_pool[k].second) == cudaSuccess)
            ctx->st.spmm_ms += ms;
    }
    ctx->ev_used = 0;
}

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool finite_all(const double *a, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

__global__ void k_tau(int64_t n, double f, const double *__restrict__ R, double *__restrict__ tau) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) tau[i] = f * 0.5 * R[i];
}

mlpg_status create_common(const mlpg_options *opt, int64_t n, const double *points, const double *extent,
                          int32_t m, const double *omega, const double *w, const double *st, const double *ss,
                          const double *q, bool on_device, mlpg_ctx **out) {
    if (!out) return MLPG_ERR_ARG;
    *out = nullptr;
    if (!opt || !points || !extent || !omega || !w || !st || !ss || !q) return MLPG_ERR_ARG;
    if ((opt->dim != 2 && opt->dim != 3) || n < 4 || m < 1 || m > MLPG_MAX_DIR) return MLPG_ERR_ARG;
    if (n >= (int64_t(1) << 31)) return MLPG_ERR_ARG;
    if (opt->inner_restart < 1 || opt->inner_restart > MLPG_MAX_RESTART || opt->outer_restart < 1 ||
        opt->outer_restart > MLPG_MAX_RESTART || opt->mixed_restart < 1 || opt->mixed_restart > MLPG_MAX_RESTART ||
        (opt->mixed_reorth != 0 && opt->mixed_reorth != 1) ||
        (opt->mixed_half_prec != 0 && opt->mixed_half_prec != 1) || opt->rk_order < 0 || opt->rk_order > 2 ||
        (opt->outer_method != 0 && opt->outer_method != 1) || opt->apply_kernel < 0 || opt->apply_kernel > 4 ||
        ((opt->apply_kernel == 2 || opt->apply_kernel == 4) && (m & 3) != 0) ||
        (opt->apply_kernel == 3 && (m & 7) != 0) ||
        (opt->tile_rows != 0 && opt->tile_rows != 4 && opt->tile_rows != 8 && opt->tile_rows != 16 &&
         opt->tile_rows != 32 && opt->tile_rows != 64) ||
        (opt->tile_rows > 0 && opt->tile_rows < 32 && opt->apply_kernel != 4) ||
        (opt->tile_rows == 64 && opt->apply_kernel == 4) ||
        (opt->tile_dpt != 0 && opt->tile_dpt != 4 && opt->tile_dpt != 8) ||
        (opt->outer_precond != 0 && opt->outer_precond != 1) || (opt->outer_precond == 1 && opt->outer_method != 0) ||
        (opt->outer_precond == 1 && (!(opt->dsa_tol > 0.0) || opt->dsa_max < 1)) ||
        (opt->cells_3d != 0 && opt->cells_3d != 1) ||
        (opt->dim == 3 && opt->rk_order > 1) || opt->check_every < 1 || !(opt->c > 0) ||
        !(opt->tau_factor >= 0) || (opt->precision != MLPG_FP64 && opt->precision != MLPG_MIXED))
        return MLPG_ERR_ARG;
    for (int a = 0; a < opt->dim; ++a)
        if (!(opt->hi[a] > opt->lo[a])) return MLPG_ERR_ARG;
    mlpg_ctx *ctx = new (std::nothrow) mlpg_ctx();
    if (!ctx) return MLPG_ERR_OOM;
    ctx->opt = *opt;
    ctx->n = n;
    ctx->m = m;
    ctx->dim = opt->dim;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return MLPG_ERR_CUDA;
    }
    if (opt->stream) {
        ctx->stream = (cudaStream_t)opt->stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete ctx;
            return MLPG_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    *out = ctx;
    const int d = ctx->dim;
    ctx->h_x.resize(n * d);
    ctx->h_R.resize(n);
    ctx->h_omega.resize(3 * (size_t)m);
    ctx->h_w.resize(m);
    cudaStream_t s = ctx->stream;
    auto fetch = [&](double *dst, const double *src, size_t cnt) -> mlpg_status {
        if (on_device) CU(ctx, cudaMemcpyAsync(dst, src, cnt * sizeof(double), cudaMemcpyDeviceToHost, s));
        else std::memcpy(dst, src, cnt * sizeof(double));
        return MLPG_OK;
    };
    MLPG_TRY(fetch(ctx->h_x.data(), points, n * d));
    MLPG_TRY(fetch(ctx->h_R.data(), extent, n));
    MLPG_TRY(fetch(ctx->h_omega.data(), omega, 3 * (size_t)m));
    MLPG_TRY(fetch(ctx->h_w.data(), w, m));
    std::vector<double> hst(n), hss(n), hq(n);
    MLPG_TRY(fetch(hst.data(), st, n));
    MLPG_TRY(fetch(hss.data(), ss, n));
    MLPG_TRY(fetch(hq.data(), q, n));
    CU(ctx, cudaStreamSynchronize(s));
    if (!finite_all(ctx->h_x.data(), n * d) || !finite_all(ctx->h_R.data(), n) ||
        !finite_all(ctx->h_omega.data(), 3 * m) || !finite_all(ctx->h_w.data(), m) || !finite_all(hst.data(), n) ||
        !finite_all(hss.data(), n) || !finite_all(hq.data(), n))
        return set_err(ctx, MLPG_ERR_ARG, "non-finite input");
    for (int64_t i = 0; i < n; ++i) {
        if (!(ctx->h_R[i] > 0.0)) return set_err(ctx, MLPG_ERR_ARG, "kernel extents must be positive");
        for (int a = 0; a < d; ++a) {
            double v = ctx->h_x[i * d + a];
            if (!(v >= opt->lo[a] && v <= opt->hi[a])) return set_err(ctx, MLPG_ERR_GEOMETRY, "point outside the box");
        }
    }
    for (int k = 0; k < m; ++k) {
        const double *o = &ctx->h_omega[3 * k];
        if (std::fabs(o[0] * o[0] + o[1] * o[1] + o[2] * o[2] - 1.0) > 1e-10)
            return set_err(ctx, MLPG_ERR_ARG, "ordinates must be unit vectors");
    }
    MLPG_TRY(dalloc(ctx, &ctx->x, n * d));
    MLPG_TRY(dalloc(ctx, &ctx->R, n));
    MLPG_TRY(dalloc(ctx, &ctx->V, n));
    MLPG_TRY(dalloc(ctx, &ctx->tau, n));
    MLPG_TRY(dalloc(ctx, &ctx->sig_t, n));
    MLPG_TRY(dalloc(ctx, &ctx->sig_s, n));
    MLPG_TRY(dalloc(ctx, &ctx->q, n));
    MLPG_TRY(dalloc(ctx, &ctx->omega, 3 * m));
    MLPG_TRY(dalloc(ctx, &ctx->w, m));
    MLPG_TRY(dalloc(ctx, &ctx->Psi, (size_t)n * m));
    MLPG_TRY(dalloc(ctx, &ctx->Phi, n));
    auto put = [&](double *dst, const double *src, size_t cnt) -> mlpg_status {
        CU(ctx, cudaMemcpyAsync(dst, src, cnt * sizeof(double),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        return MLPG_OK;
    };
    MLPG_TRY(put(ctx->x, points, n * d));
    MLPG_TRY(put(ctx->R, extent, n));
    MLPG_TRY(put(ctx->sig_t, st, n));
    MLPG_TRY(put(ctx->sig_s, ss, n));
    MLPG_TRY(put(ctx->q, q, n));
    MLPG_TRY(put(ctx->omega, omega, 3 * (size_t)m));
    MLPG_TRY(put(ctx->w, w, m));
    k_tau<<<(n + 255) / 256, 256, 0, s>>>(n, opt->tau_factor, ctx->R, ctx->tau);
    CU_LAUNCH(ctx);
    CU(ctx, cudaMemsetAsync(ctx->Psi, 0, sizeof(double) * n * m, s));
    CU(ctx, cudaMemsetAsync(ctx->Phi, 0, sizeof(double) * n, s));
    CU(ctx, cudaStreamSynchronize(s));
    ctx->st.n = n;
    ctx->st.m = m;
    return MLPG_OK;
}

__global__ void k_phi_from_psi(int64_t n, int m, const double *__restrict__ w, const double *__restrict__ psi,
                               double *__restrict__ phi) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int k = 0; k < m; ++k) s += w[k] * psi[i * m + k];
    phi[i] = s;
}

}  // namespace
}  // namespace mlpg

using namespace mlpg;

#define GUARD(ctx) DeviceGuard _dg((ctx)->device)
#define CATCH_ALL(ctx)                                                   \
    catch (const std::bad_alloc &) {                                     \
        return set_err(ctx, MLPG_ERR_OOM, "host allocation failed");    \
    }                                                                    \
    catch (...) {                                                        \
        return set_err(ctx, MLPG_ERR_ARG, "unexpected host exception");  \
    }

extern "C" {

void mlpg_default_options(mlpg_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->dim = 2;
    o->lo[0] = o->lo[1] = o->lo[2] = 0.0;
    o->hi[0] = o->hi[1] = o->hi[2] = 1.0;
    o->tau_factor = 1.0;
    o->c = 1.0;
    o->precision = MLPG_FP64;
    o->inner_tol = 1e-12;
    o->outer_tol = 1e-12;
    o->inner_restart = 20;
    o->outer_restart = 30;
    o->max_inner = 2000;
    o->max_outer = 500;
    o->refine_tol = 1e-11;
    o->max_refine = 12;
    o->mixed_inner_tol = 1e-2;
    o->check_every = 3;
    o->mixed_restart = 20;
    o->mixed_reorth = 0;
    o->mixed_half_prec = 1;
    o->outer_method = 0;
    o->rk_order = 1;
    o->stream = nullptr;
    o->apply_kernel = 0;
    o->tile_rows = 0;
    o->tile_dpt = 0;
    o->outer_precond = 0;
    o->dsa_tol = 1e-10;
    o->dsa_max = 500;
    o->cells_3d = 0;
}

mlpg_status mlpg_create(const mlpg_options *opt, int64_t n, const double *points, const double *kernel_extent,
                        int32_t m, const double *omega, const double *w, const double *sigma_t,
                        const double *sigma_s, const double *q, mlpg_ctx **out) {
    try {
        return create_common(opt, n, points, kernel_extent, m, omega, w, sigma_t, sigma_s, q, false, out);
    } catch (...) {
        return MLPG_ERR_OOM;
    }
}

mlpg_status mlpg_create_dev(const mlpg_options *opt, int64_t n, const double *points, const double *kernel_extent,
                            int32_t m, const double *omega, const double *w, const double *sigma_t,
                            const double *sigma_s, const double *q, mlpg_ctx **out) {
    try {
        return create_common(opt, n, points, kernel_extent, m, omega, w, sigma_t, sigma_s, q, true, out);
    } catch (...) {
        return MLPG_ERR_OOM;
    }
}

mlpg_status mlpg_set_inflow(mlpg_ctx *ctx, int face, double psi_b) {
    if (!ctx) return MLPG_ERR_ARG;
    if (face < 0 || face >= 2 * ctx->dim || !std::isfinite(psi_b)) return set_err(ctx, MLPG_ERR_ARG, "bad inflow");
    ctx->psi_b[face] = psi_b;
    return MLPG_OK;
}

mlpg_status mlpg_set_initial(mlpg_ctx *ctx, const double *psi0) {
    if (!ctx) return MLPG_ERR_ARG;
    GUARD(ctx);
    const int64_t N = ctx->n * ctx->m;
    if (psi0) CU(ctx, cudaMemcpyAsync(ctx->Psi, psi0, N * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    else CU(ctx, cudaMemsetAsync(ctx->Psi, 0, N * sizeof(double), ctx->stream));
    k_phi_from_psi<<<(ctx->n + 255) / 256, 256, 0, ctx->stream>>>(ctx->n, ctx->m, ctx->w, ctx->Psi, ctx->Phi);
    CU_LAUNCH(ctx);
    MLPG_TRY(shard_sum_dev(ctx, ctx->Phi, ctx->n));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->nhist = 0;   // a new state: no history for the initial guess
    return MLPG_OK;
}

mlpg_status mlpg_integrate(mlpg_ctx *ctx) {
    if (!ctx) return MLPG_ERR_ARG;
    if (ctx->state != 0) return set_err(ctx, MLPG_ERR_STATE, "integrate must follow create");
    GUARD(ctx);
    try {
        MLPG_TRY(run_neighbors(ctx));
        if (ctx->dim == 3 && ctx->opt.cells_3d == 0) {   // cells on the device
            MLPG_TRY(run_cells_3d(ctx));
            MLPG_TRY(run_interp_3d(ctx));
            MLPG_TRY(build_blocks(ctx));
            ctx->st.nnz = ctx->nnz;
            ctx->st.n_volume_qp = ctx->nvq;
            ctx->st.n_boundary_qp = ctx->nbq;
            ctx->state = 1;
            return MLPG_OK;
        }
        if (ctx->dim == 3) {   // cells on the host cores
            HostCells3 c3;
            int64_t bad = build_cells_3d(ctx->n, ctx->h_x.data(), ctx->h_R.data(), ctx->opt.lo, ctx->opt.hi,
                                         ctx->h_rowptr.data(), ctx->h_col.data(), c3);
            if (bad >= 0) return set_err(ctx, MLPG_ERR_GEOMETRY, "empty cell at point " + std::to_string(bad));
            ctx->ntet = (int64_t)c3.tet_owner.size();
            ctx->nbtri = (int64_t)c3.tri_owner.size();
            ctx->nvq = 8 * ctx->ntet;
            ctx->nbq = 4 * ctx->nbtri;
            cudaStream_t s = ctx->stream;
            MLPG_TRY(dalloc(ctx, &ctx->tet_owner, ctx->ntet));
            MLPG_TRY(dalloc(ctx, &ctx->tet_v, 9 * ctx->ntet));
            MLPG_TRY(dalloc(ctx, &ctx->tri_owner, ctx->nbtri + 1));
            MLPG_TRY(dalloc(ctx, &ctx->tri_face, ctx->nbtri + 1));
            MLPG_TRY(dalloc(ctx, &ctx->tri_v, 9 * ctx->nbtri + 9));
            CU(ctx, cudaMemcpyAsync(ctx->tet_owner, c3.tet_owner.data(), ctx->ntet * sizeof(int32_t), cudaMemcpyHostToDevice, s));
            CU(ctx, cudaMemcpyAsync(ctx->tet_v, c3.tet_v.data(), 9 * ctx->ntet * sizeof(double), cudaMemcpyHostToDevice, s));
            if (ctx->nbtri > 0) {
                CU(ctx, cudaMemcpyAsync(ctx->tri_owner, c3.tri_owner.data(), ctx->nbtri * sizeof(int32_t), cudaMemcpyHostToDevice, s));
                CU(ctx, cudaMemcpyAsync(ctx->tri_face, c3.tri_face.data(), ctx->nbtri * sizeof(int32_t), cudaMemcpyHostToDevice, s));
                CU(ctx, cudaMemcpyAsync(ctx->tri_v, c3.tri_v.data(), 9 * ctx->nbtri * sizeof(double), cudaMemcpyHostToDevice, s));
            }
            CU(ctx, cudaMemcpyAsync(ctx->V, c3.volume.data(), ctx->n * sizeof(double), cudaMemcpyHostToDevice, s));
            MLPG_TRY(run_interp_3d(ctx));  // synchronises: the host vectors may go
            MLPG_TRY(build_blocks(ctx));
            ctx->st.nnz = ctx->nnz;
            ctx->st.n_volume_qp = ctx->nvq;
            ctx->st.n_boundary_qp = ctx->nbq;
            ctx->state = 1;
            return MLPG_OK;
        }
        // 2D cells on the device: 25-point triangle rule, 5-point edge rule
        MLPG_TRY(run_cells_2d(ctx, 25, 5));
        MLPG_TRY(run_interp(ctx));  // synchronises
        MLPG_TRY(build_blocks(ctx));
        ctx->st.nnz = ctx->nnz;
        ctx->st.n_volume_qp = ctx->nvq;
        ctx->st.n_boundary_qp = ctx->nbq;
        ctx->state = 1;
        return MLPG_OK;
    }
    CATCH_ALL(ctx)
}

mlpg_status mlpg_assemble(mlpg_ctx *ctx) {
    if (!ctx) return MLPG_ERR_ARG;
    if (ctx->state != 1) return set_err(ctx, MLPG_ERR_STATE, "assemble must follow integrate");
    GUARD(ctx);
    try {
        MLPG_TRY(ctx->dim == 3 ? run_assemble_3d(ctx) : run_assemble(ctx));
        ctx->kappa = -1.0;
        ctx->state = 2;
        return MLPG_OK;
    }
    CATCH_ALL(ctx)
}

mlpg_status mlpg_step(mlpg_ctx *ctx, double dt) {
    if (!ctx) return MLPG_ERR_ARG;
    if (ctx->state != 2) return set_err(ctx, MLPG_ERR_STATE, "step needs an assembled problem");
    if (!(dt > 0.0)) return set_err(ctx, MLPG_ERR_ARG, "dt must be positive (INFINITY: steady)");
    GUARD(ctx);
    try {
        return ctx->opt.precision == MLPG_MIXED ? step_mixed(ctx, dt) : step_fp64(ctx, dt);
    }
    CATCH_ALL(ctx)
}

mlpg_status mlpg_step_batch(mlpg_ctx *const *ctxs, const double *dt, int count, mlpg_status *status) {
    if (!ctxs || !dt || count < 0) return MLPG_ERR_ARG;
    for (int i = 0; i < count; ++i) {
        if (!ctxs[i]) return MLPG_ERR_ARG;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i] || ctxs[j]->stream == ctxs[i]->stream)
                return set_err(ctxs[i], MLPG_ERR_ARG, "batched contexts must be distinct and on distinct streams");
    }
    if (count == 0) return MLPG_OK;
    std::vector<mlpg_status> st(count, MLPG_OK);
    std::vector<std::thread> th;
    int next = 1;   // contexts [next, count) still to run on the caller's thread
    try {
        th.reserve(count - 1);
        for (; next < count; ++next) th.emplace_back([&st, ctxs, dt, i = next] { st[i] = mlpg_step(ctxs[i], dt[i]); });
    } catch (...) {   // no thread: run the rest here
    }
    st[0] = mlpg_step(ctxs[0], dt[0]);
    for (int i = next; i < count; ++i) st[i] = mlpg_step(ctxs[i], dt[i]);
    for (auto &t : th) t.join();
    if (status) std::copy(st.begin(), st.end(), status);
    for (int i = 0; i < count; ++i)
        if (st[i] != MLPG_OK) return st[i];
    return MLPG_OK;
}

mlpg_status mlpg_scalar_flux_dev(mlpg_ctx *ctx, double *out, int kind) {
    if (!ctx || !out || (kind != 0 && kind != 1)) return ctx ? set_err(ctx, MLPG_ERR_ARG, "bad flux request") : MLPG_ERR_ARG;
    if (ctx->state < 1) return set_err(ctx, MLPG_ERR_STATE, "scalar flux needs integrate");
    GUARD(ctx);
    return interp_flux(ctx, out, kind);
}

mlpg_status mlpg_scalar_flux(mlpg_ctx *ctx, double *out, int kind) {
    if (!ctx || !out || (kind != 0 && kind != 1)) return ctx ? set_err(ctx, MLPG_ERR_ARG, "bad flux request") : MLPG_ERR_ARG;
    if (ctx->state < 1) return set_err(ctx, MLPG_ERR_STATE, "scalar flux needs integrate");
    GUARD(ctx);
    if (!ctx->nvec) {
        // before the first step: a private buffer
        MLPG_TRY(dalloc(ctx, &ctx->nvec, 8 * ctx->n));
    }
    double *tmp = ctx->nvec + 7 * ctx->n;
    MLPG_TRY(interp_flux(ctx, tmp, kind));
    CU(ctx, cudaMemcpyAsync(out, tmp, ctx->n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    return MLPG_OK;
}

mlpg_status mlpg_get_state(const mlpg_ctx *cctx, double *psi) {
    mlpg_ctx *ctx = const_cast<mlpg_ctx *>(cctx);
    if (!ctx || !psi) return MLPG_ERR_ARG;
    GUARD(ctx);
    CU(ctx, cudaMemcpyAsync(psi, ctx->Psi, ctx->n * ctx->m * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    return MLPG_OK;
}

mlpg_status mlpg_set_state(mlpg_ctx *ctx, const double *psi) {
    if (!ctx || !psi) return MLPG_ERR_ARG;
    return mlpg_set_initial(ctx, psi);
}

mlpg_status mlpg_get_stats(const mlpg_ctx *cctx, mlpg_stats *st) {
    mlpg_ctx *ctx = const_cast<mlpg_ctx *>(cctx);
    if (!ctx || !st) return MLPG_ERR_ARG;
    GUARD(ctx);
    if (ctx->timing) harvest_timing(ctx);
    // algorithmic bytes of one batched L-apply
    const int64_t nnz = ctx->nnz, n = ctx->n, m = ctx->m, d = ctx->dim;
    const int64_t na = 1 + d + d * (d + 1) / 2, nf = 2 * d;   // base arrays, faces
    if (ctx->opt.precision == MLPG_MIXED)
        ctx->st.spmm_bytes = nnz * (4 + na * 4) + ctx->nb * (4 + nf * 4) + 2 * 4 * (n + 1) + 2 * n * m * 4;
    else
        ctx->st.spmm_bytes = nnz * (4 + 8 * m) + 4 * (n + 1) + 2 * n * m * 8;
    ctx->st.apply_kernel = ctx->A32 ? (ctx->t_rec ? (ctx->tile_mma ? 3 : (ctx->tile_gather ? 4 : 2)) : 1) : 0;
    ctx->st.tile_chunk = ctx->t_rec ? ctx->tile_chunk : 0;
    ctx->st.tile_max_halo = ctx->t_rec ? ctx->tile_max_halo : 0;
    *st = ctx->st;
    return MLPG_OK;
}

mlpg_status mlpg_enable_timing(mlpg_ctx *ctx, int on) {
    if (!ctx) return MLPG_ERR_ARG;
    GUARD(ctx);
    if (on && ctx->ev_pool.empty()) {
        ctx->ev_pool.resize(512);
        for (auto &p : ctx->ev_pool) {
            CU(ctx, cudaEventCreate(&p.first));
            CU(ctx, cudaEventCreate(&p.second));
        }
    }
    if (!on && ctx->timing) harvest_timing(ctx);
    ctx->timing = on != 0;
    ctx->st.spmm_ms = 0.0;
    ctx->st.spmm_launches = 0;
    return MLPG_OK;
}

mlpg_status mlpg_get_neighbors(const mlpg_ctx *ctx, int64_t *rowptr, int32_t *col) {
    if (!ctx || !rowptr || !col) return MLPG_ERR_ARG;
    if (ctx->state < 1) return MLPG_ERR_STATE;
    for (int64_t i = 0; i <= ctx->n; ++i) rowptr[i] = ctx->h_rowptr[i];
    std::memcpy(col, ctx->h_col.data(), ctx->nnz * sizeof(int32_t));
    return MLPG_OK;
}

mlpg_status mlpg_get_volumes(const mlpg_ctx *cctx, double *out) {
    mlpg_ctx *ctx = const_cast<mlpg_ctx *>(cctx);
    if (!ctx || !out) return MLPG_ERR_ARG;
    if (ctx->state < 1) return set_err(ctx, MLPG_ERR_STATE, "volumes need integrate");
    GUARD(ctx);
    CU(ctx, cudaStreamSynchronize(ctx->stream));   // the library stream does not block with the legacy one
    CU(ctx, cudaMemcpy(out, ctx->V, ctx->n * sizeof(double), cudaMemcpyDeviceToHost));
    return MLPG_OK;
}

int mlpg_n_matrices(int dim) { return 3 + 3 * dim + dim * dim + 2 * dim; }
int mlpg_n_vectors(int dim) { return 1 + dim + 2 * dim; }

mlpg_status mlpg_get_forms(const mlpg_ctx *cctx, double *mats, double *vecs) {
    mlpg_ctx *ctx = const_cast<mlpg_ctx *>(cctx);
    if (!ctx || !mats || !vecs) return MLPG_ERR_ARG;
    if (ctx->state < 2) return set_err(ctx, MLPG_ERR_STATE, "forms need assemble");
    GUARD(ctx);
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    CU(ctx, cudaMemcpy(mats, ctx->mats, sizeof(double) * ctx->nmats * ctx->nnz, cudaMemcpyDeviceToHost));
    CU(ctx, cudaMemcpy(vecs, ctx->vecs, sizeof(double) * ctx->nvecs * ctx->n, cudaMemcpyDeviceToHost));
    return MLPG_OK;
}

mlpg_status mlpg_apply_L_dev(mlpg_ctx *ctx, double dt, int precision, const void *X, void *Y) {
    if (!ctx || !X || !Y || !(dt > 0.0)) return ctx ? set_err(ctx, MLPG_ERR_ARG, "bad apply arguments") : MLPG_ERR_ARG;
    if (ctx->state != 2) return set_err(ctx, MLPG_ERR_STATE, "apply needs an assembled problem");
    {
        const uintptr_t x = (uintptr_t)X, y = (uintptr_t)Y;
        const uintptr_t bytes = (uintptr_t)ctx->n * ctx->m * (precision == MLPG_FP64 ? 8 : 4);
        if ((x & 15) || (y & 15)) return set_err(ctx, MLPG_ERR_ARG, "X and Y must be 16-byte aligned");
        if (x < y + bytes && y < x + bytes) return set_err(ctx, MLPG_ERR_ARG, "X and Y overlap");
    }
    GUARD(ctx);
    try {
        double kappa = std::isfinite(dt) ? 1.0 / (ctx->opt.c * dt) : 0.0;
        if (kappa != ctx->kappa) MLPG_TRY(form_operators(ctx, kappa));
        if (precision == MLPG_FP64) return apply_L64(ctx, (const double *)X, (double *)Y);
        if (precision == MLPG_MIXED) return apply_L32(ctx, (const float *)X, (float *)Y);
        return set_err(ctx, MLPG_ERR_ARG, "bad precision");
    }
    CATCH_ALL(ctx)
}

mlpg_status mlpg_set_reduce(mlpg_ctx *ctx, mlpg_reduce_fn fn, void *user) {
    if (!ctx) return MLPG_ERR_ARG;
    ctx->reduce_fn = fn;
    ctx->reduce_user = fn ? user : nullptr;
    return MLPG_OK;
}

const char *mlpg_last_error(const mlpg_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void mlpg_destroy(mlpg_ctx *ctx) {
    if (!ctx) return;
    {
        DeviceGuard g(ctx->device);
        if (ctx->stream) cudaStreamSynchronize(ctx->stream);
        for (auto &p : ctx->ev_pool) {
            cudaEventDestroy(p.first);
            cudaEventDestroy(p.second);
        }
        for (void *p : ctx->allocs)
            if (p) cudaFree(p);
        for (void *p : ctx->host_allocs)
            if (p) cudaFreeHost(p);
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        cudaGetLastError();
    }
    delete ctx;
}

}  // extern "C"
