// C ABI of the self-consistency accelerators (App. E): step-size logic on the
// host from device reductions (accel.cu).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>

#include "accel.cuh"
#include "context.hpp"

namespace {

using sc_internal::set_err;

#define ACK(expr)                                                                       \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return set_err(ctx, e_ == cudaErrorMemoryAllocation ? SC_ENOMEM : SC_ECUDA, \
                           std::string(#expr) + ": " + cudaGetErrorString(e_));          \
    } while (0)

#define ACKS(expr)                  \
    do {                            \
        sc_status s_ = (expr);      \
        if (s_ != SC_OK) return s_; \
    } while (0)

template <typename P>
cudaError_t alloc_once(sc_ctx *ctx, P **p, size_t bytes) {
    if (*p) return cudaSuccess;
    void *v = nullptr;
    cudaError_t e = sc_internal::dalloc_bytes(ctx, &v, bytes);
    if (e == cudaSuccess) *p = (P *)v;
    return e;
}

double clamp(double a, const sc_accel_params *p) {
    return std::fmin(std::fmax(a, p->step_size_min), p->step_size_max);
}

double cos_from_sums(double w, double md, double mm, double dd) {
    const double num = w * md + (1.0 - w) * dd;
    const double nv2 = w * w * mm + 2.0 * w * (1.0 - w) * md + (1.0 - w) * (1.0 - w) * dd;
    return num / (std::sqrt(nv2) * std::sqrt(dd));
}

// w in [0, 1] with cos(w m + (1 - w) d, d) = s_min (cos is 1 at w = 0 and below
// s_min at w = 1), 60 bisection steps
double similarity_weight(double md, double mm, double dd, double s_min) {
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (cos_from_sums(mid, md, mm, dd) >= s_min)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

}  // namespace

extern "C" {

sc_status sc_accel_params_default(int32_t kind, sc_accel_params *p) {
    if (!p || kind < SC_ACC_PICARD || kind > SC_ACC_CONGACC) return SC_EINVAL;
    std::memset(p, 0, sizeof *p);
    p->kind = kind;
    p->step_size = kind == SC_ACC_POLYAK ? 2.0 : (kind == SC_ACC_CONGACC ? 0.5 : 1.0);
    p->drag = 0.5;
    p->step_size_factor = 1.234;
    p->cos_similarity_min = 0.7;
    p->step_size_max = 100.0;
    p->step_size_min = 0.001;
    return SC_OK;
}

sc_status sc_accel_reset(sc_ctx *ctx) {
    if (!ctx) return SC_EINVAL;
    ctx->acc_kind = -1;
    ctx->acc_iter = 0;
    return SC_OK;
}

sc_status sc_accel_get_state(const sc_ctx *ctx, int32_t *iterations, double *alpha, double *w) {
    if (!ctx) return SC_EINVAL;
    if (iterations) *iterations = ctx->acc_kind < 0 ? 0 : (int32_t)ctx->acc_iter;
    const int ncomp = 2 * ctx->geo.n_comp + 2;
    for (int c = 0; c < ncomp; ++c) {
        if (alpha) alpha[c] = ctx->acc_kind == SC_ACC_CONGACC ? ctx->acc_alpha_c[c] : (c == 0 ? ctx->acc_alpha : 0.0);
        if (w) w[c] = ctx->acc_kind == SC_ACC_CONGACC ? ctx->acc_w_c[c] : 0.0;
    }
    return SC_OK;
}

sc_status sc_accelerate(sc_ctx *ctx, const sc_accel_params *p, void *stream) {
    ACKS(sc_internal::check_ctx(ctx));
    if (!p) return set_err(ctx, SC_EINVAL, "accelerator parameters are required");
    if (p->kind < SC_ACC_PICARD || p->kind > SC_ACC_CONGACC) return set_err(ctx, SC_EINVAL, "unknown accelerator");
    if (!(p->step_size > 0.0) || !(p->drag > 0.0 && p->drag <= 1.0) || !(p->step_size_factor > 0.0) ||
        !(p->cos_similarity_min >= -1.0 && p->cos_similarity_min <= 1.0) || !(p->step_size_min > 0.0) ||
        !(p->step_size_max >= p->step_size_min))
        return set_err(ctx, SC_EINVAL, "accelerator parameters out of range");
    if (!ctx->have_sweep) return set_err(ctx, SC_ESTATE, "the accelerator needs a sweep of the current fields");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = (int64_t)ctx->geo.nx * ctx->geo.ny;
    ACKS(sc_internal::ensure_outputs(ctx, st));
    const bool magn = ctx->d_G != nullptr;
    const double kappa = ctx->geo.prm.kappa;
    if (magn) {
        ACK(alloc_once(ctx, &ctx->d_anew, 2 * n * sizeof(double)));
        ACK(scd::launch_mean_current(ctx->grid, ctx->d_mask, ctx->d_j, ctx->d_jsum, ctx->d_part, st));
        ACK(sc_internal::induced_field(ctx, ctx->d_anew, st));
    }
    const int blocks = scd::accel_reduce_blocks(n, ctx->sm_count);
    ACK(alloc_once(ctx, &ctx->d_acc_v, scd::kAccelComps * n * sizeof(double)));
    ACK(alloc_once(ctx, &ctx->d_acc_prev, scd::kAccelComps * n * sizeof(double)));
    ACK(alloc_once(ctx, &ctx->d_acc_m, scd::kAccelComps * n * sizeof(double)));
    ACK(alloc_once(ctx, &ctx->d_acc_part, (size_t)blocks * scd::kAccelSums * sizeof(double)));
    ACK(alloc_once(ctx, &ctx->d_acc_sums, scd::kAccelSums * sizeof(double)));
    if (ctx->acc_kind != p->kind) {  // a new history
        ACK(cudaMemsetAsync(ctx->d_acc_v, 0, scd::kAccelComps * n * sizeof(double), st));
        ACK(cudaMemsetAsync(ctx->d_acc_prev, 0, scd::kAccelComps * n * sizeof(double), st));
        ACK(cudaMemsetAsync(ctx->d_acc_m, 0, scd::kAccelComps * n * sizeof(double), st));
        ctx->acc_kind = p->kind;
        ctx->acc_iter = 0;
        ctx->acc_alpha = p->step_size;
        for (int c = 0; c < scd::kAccelComps; ++c) {
            ctx->acc_alpha_c[c] = p->step_size;
            ctx->acc_w_c[c] = 0.0;
        }
    }
    scd::AccelArgs a{};
    a.npts = n;
    a.nc = ctx->geo.n_comp;
    a.mask = ctx->d_mask;
    a.delta = ctx->d_delta;
    a.aind = magn ? ctx->d_aind : nullptr;
    a.dnew = ctx->d_dnew;
    a.anew = magn ? ctx->d_anew : nullptr;
    a.k2 = magn ? kappa * kappa : 1.0;
    a.v = ctx->d_acc_v;
    a.dprev = ctx->d_acc_prev;
    a.m = ctx->d_acc_m;
    const bool reduce = ctx->acc_iter >= 1 && (p->kind == SC_ACC_BARZILAI_BORWEIN || p->kind == SC_ACC_CONGACC);
    if (reduce) {
        double s[scd::kAccelSums];
        ACK(scd::launch_accel_reduce(a, ctx->d_acc_part, blocks, ctx->d_acc_sums, st));
        ACK(cudaMemcpyAsync(s, ctx->d_acc_sums, sizeof s, cudaMemcpyDeviceToHost, st));
        ACK(cudaStreamSynchronize(st));
        if (p->kind == SC_ACC_BARZILAI_BORWEIN) {
            // s0 = |d_{i-1}|^2, s1 = d_{i-1}.(d_i - d_{i-1}), s2 = |d_i - d_{i-1}|^2
            const double q = std::fabs(s[1]);
            const bool bb1 = ctx->acc_iter % 2 == 1;
            const double num = bb1 ? s[0] : q, den = bb1 ? q : s[2];
            if (den > 0.0) ctx->acc_alpha = clamp(ctx->acc_alpha * num / den, p);
        } else {
            for (int c = 0; c < scd::kAccelComps; ++c) {
                const double md = s[3 + 3 * c], mm = s[4 + 3 * c], dd = s[5 + 3 * c];
                if (!(mm > 0.0) || !(dd > 0.0)) continue;  // component absent or at rest
                const double sim = md / std::sqrt(mm * dd);
                ctx->acc_alpha_c[c] = clamp(ctx->acc_alpha_c[c] * std::pow(p->step_size_factor, sim), p);
                if (sim < p->cos_similarity_min)
                    ctx->acc_w_c[c] = similarity_weight(md, mm, dd, p->cos_similarity_min);
            }
        }
    }
    const double alpha = p->kind == SC_ACC_BARZILAI_BORWEIN ? ctx->acc_alpha : p->step_size;
    ACK(scd::launch_accel_update(a, p->kind, alpha, p->drag, ctx->acc_alpha_c, ctx->acc_w_c, st));
    ++ctx->acc_iter;
    ctx->have_sweep = false;
    ctx->have_outputs = false;
    if (magn) ctx->have_aind = true;
    return SC_OK;
}

}  // extern "C"

extern "C" sc_status sc_self_consistency(sc_ctx *ctx, const sc_accel_params *p, int32_t max_iter, double tol,
                                         int32_t check_every, int32_t *iterations, double *eps_G, void *stream) {
    ACKS(sc_internal::check_ctx(ctx));
    if (!p || max_iter < 1 || !(tol >= 0.0) || check_every < 1)
        return set_err(ctx, SC_EINVAL, "self-consistency needs parameters, max_iter >= 1, tol >= 0, check_every >= 1");
    double eps = -1.0;
    int it = 0;
    bool converged = false;
    for (it = 1; it <= max_iter; ++it) {
        ACKS(sc_riccati_sweep(ctx, stream));
        if (it % check_every == 0 || it == max_iter) {
            ACKS(sc_gap_update(ctx, nullptr, &eps, 1, stream));
            if (eps < tol) {
                converged = true;
                break;
            }
        }
        if (it == max_iter) break;
        ACKS(sc_accelerate(ctx, p, stream));
    }
    if (iterations) *iterations = it > max_iter ? max_iter : it;
    if (eps_G) *eps_G = eps;
    return converged ? SC_OK : SC_ENOTCONV;
}
