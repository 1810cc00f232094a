// C ABI of the Riccati sweep: context, device memory, launch plans.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "adjoint.cuh"
#include "context.hpp"

namespace {
thread_local std::string g_create_error;
}  // namespace

namespace sc_internal {
void set_thread_error(const char *msg) { g_create_error = msg ? msg : ""; }
}  // namespace sc_internal

namespace sc_internal {

sc_status set_err(sc_ctx *c, sc_status st, const std::string &msg) {
    c->err = msg;
    if (st == SC_ECUDA || st == SC_ENOMEM) c->failed = true;
    return st;
}

cudaError_t dalloc_bytes(sc_ctx *ctx, void **p, size_t bytes) {
    void *v = nullptr;
    if (ctx->fail_alloc_at >= 0 && ctx->alloc_count++ == ctx->fail_alloc_at) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(&v, bytes > 0 ? bytes : 16);
    if (e == cudaSuccess) {
        ctx->allocs.push_back(v);
        *p = v;
    }
    return e;
}

void dfree(sc_ctx *ctx, void *p) {
    if (!p) return;
    auto f = std::find(ctx->allocs.begin(), ctx->allocs.end(), p);
    if (f != ctx->allocs.end()) ctx->allocs.erase(f);
    cudaFree(p);
}

}  // namespace sc_internal

namespace {

int64_t count_bad_indices(const scg::Geometry &G);  // defined with sc_debug_validate_tables

using sc_internal::dfree;
using sc_internal::set_err;

#define CK(expr)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return set_err(ctx, e_ == cudaErrorMemoryAllocation ? SC_ENOMEM : SC_ECUDA, \
                           std::string(#expr) + ": " + cudaGetErrorString(e_));          \
    } while (0)

#define CKS(expr)                   \
    do {                            \
        sc_status s_ = (expr);      \
        if (s_ != SC_OK) return s_; \
    } while (0)

template <typename P>
cudaError_t dalloc(sc_ctx *ctx, P **p, size_t bytes) {
    void *v = nullptr;
    cudaError_t e = sc_internal::dalloc_bytes(ctx, &v, bytes);
    if (e == cudaSuccess) *p = (P *)v;
    return e;
}

// energy lanes per line and energies per lane: least padding, then EPT near 4.
// wide (the FP32 sweep on packed energy pairs, at most 256 energies): 16 or 32
// lanes per line may carry up to 10 energies each, so may 2 lanes per line (16
// lines per warp, at most 20 energies), and among layouts with equal
// padding the one with fewer issue units per line (lanes x energy pairs, an odd
// energy counting as a pair) wins (c5, 160 energies: 16 x 10 against 32 x 5,
// sweep 119.9 -> 110.4 ms; 8 lanes x 10 on c2 is slower than 16 x 5, its four
// lines per warp differing in length)
void choose_lanes(int n_e, int forced_lanes, int forced_ept, int &lanes, int &ept, bool wide) {
    if (forced_ept) {
        ept = forced_ept;
        lanes = 32;
        for (int l : {4, 8, 16, 32})
            if (l * ept >= n_e) {
                lanes = l;
                break;
            }
        return;
    }
    if (forced_lanes) {
        lanes = forced_lanes;
        ept = (n_e + lanes - 1) / lanes;
        return;
    }
    int best_pad = 1 << 30, best_l = 32, best_e = 8;
    if (n_e > 32 * 8) {
        // several energy blocks per line: the fewest padded lane slots, each block
        // counted with 32 slots of per-block overhead (samples, coefficients)
        for (int l : {32, 16, 8, 4})
            for (int e = 8; e >= 1; --e) {
                const int nb = (n_e + l * e - 1) / (l * e);
                const int cost = nb * (l * e + 32);
                if (cost < best_pad) {
                    best_pad = cost;
                    best_l = l;
                    best_e = e;
                }
            }
        lanes = best_l;
        ept = best_e;
        return;
    }
    for (int l : {32, 16, 8, 4, 2}) {
        if (l == 2 && !wide) continue;
        const int e = (n_e + l - 1) / l;
        if (e > (wide && (l >= 16 || l == 2) ? 10 : 8)) continue;
        const int pad = l * e;
        bool better = pad < best_pad;
        if (pad == best_pad) {
            const int units = l * ((e + 1) / 2), best_units = best_l * ((best_e + 1) / 2);
            better = wide && units != best_units ? units < best_units
                                                 : std::abs(e - 4) < std::abs(best_e - 4);
        }
        if (better) {
            best_pad = pad;
            best_l = l;
            best_e = e;
        }
    }
    lanes = best_l;
    ept = best_e;
}

sc_status ensure_scratch(sc_ctx *ctx, size_t need) {
    if (need <= ctx->scratch_bytes) return SC_OK;
    dfree(ctx, ctx->d_scratch);
    ctx->d_scratch = nullptr;
    ctx->scratch_bytes = 0;
    CK(dalloc(ctx, &ctx->d_scratch, need));
    ctx->scratch_bytes = need;
    return SC_OK;
}

size_t npts(const sc_ctx *ctx) { return (size_t)ctx->geo.nx * ctx->geo.ny; }

}  // namespace

namespace sc_internal {

sc_status check_ctx(sc_ctx *ctx) {
    if (!ctx) return SC_EINVAL;
    if (ctx->host_only) return set_err(ctx, SC_ESTATE, "context was created with host_only = 1");
    if (ctx->failed) return SC_ESTATE;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return set_err(ctx, SC_ECUDA, cudaGetErrorString(e));
    return SC_OK;
}

sc_status make_plan(sc_ctx *ctx, int n_e, int forced_ept, Plan **out, bool wide) {
    int lanes, ept;
    choose_lanes(n_e, ctx->forced_lanes, forced_ept, lanes, ept, wide && !ctx->fp64 && n_e <= 32 * 8);
    return make_plan_layout(ctx, n_e, lanes, ept, out);
}

sc_status make_plan_layout(sc_ctx *ctx, int n_e, int lanes, int ept, Plan **out) {
    if (lanes != 2 && lanes != 4 && lanes != 8 && lanes != 16 && lanes != 32)
        return set_err(ctx, SC_EINVAL, "energy lanes per line must be 2, 4, 8, 16 or 32");
    if (ept < 1 || ept > (ctx->fp64 ? 8 : 10))
        return set_err(ctx, SC_EINVAL, ctx->fp64 ? "energies per lane must be 1 to 8" : "energies per lane must be 1 to 10");
    const int n_blocks = (n_e + lanes * ept - 1) / (lanes * ept);
    const int key = n_blocks * 1024 + lanes * 16 + ept;
    auto it = ctx->plans.find(key);
    if (it != ctx->plans.end()) {
        *out = &it->second;
        return SC_OK;
    }
    Plan pl;
    pl.lanes = lanes;
    pl.ept = ept;
    pl.lines_per_warp = 32 / lanes;
    const int G = pl.lines_per_warp;
    // groups of G lines of one pair, the pair's lines taken longest first: a warp
    // steps its lines as long as the longest, so lines of equal length share a warp
    std::vector<int32_t> flat;
    std::vector<int32_t> by_len;
    for (const auto &pp : ctx->geo.pairs) {
        const int n = pp.n_lines;
        by_len.resize(n);
        for (int i = 0; i < n; ++i) by_len[i] = pp.line0 + i;
        std::stable_sort(by_len.begin(), by_len.end(),
                         [&](int32_t a, int32_t b) { return ctx->geo.lines[a].ns > ctx->geo.lines[b].ns; });
        for (int i = 0; i < n; i += G) {
            int c = 0;
            for (int k = 0; k < G; ++k) {
                if (i + k < n) {
                    flat.push_back(by_len[i + k]);
                    c = std::max(c, ctx->geo.lines[by_len[i + k]].ns + 1);
                } else {
                    flat.push_back(-1);
                }
            }
            pl.group_cost.push_back(c);
        }
    }
    pl.n_groups = (int32_t)pl.group_cost.size();
    pl.n_blocks = n_blocks;
    pl.n_items = pl.n_groups * pl.n_blocks;
    std::vector<int> order(pl.n_groups);
    for (int i = 0; i < pl.n_groups; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return pl.group_cost[a] > pl.group_cost[b]; });
    // every energy block of a group is one item of the group's cost
    std::vector<int2> items(pl.n_items);
    for (int i = 0; i < pl.n_groups; ++i)
        for (int k = 0; k < pl.n_blocks; ++k) items[(size_t)i * pl.n_blocks + k] = make_int2(0, order[i] * pl.n_blocks + k);
    CK(dalloc(ctx, &pl.d_groups, flat.size() * sizeof(int32_t)));
    CK(cudaMemcpy(pl.d_groups, flat.data(), flat.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(dalloc(ctx, &pl.d_items, items.size() * sizeof(int2)));
    CK(cudaMemcpy(pl.d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice));
    const int bs = 128;
    int occ = scd::sweep_occupancy(ctx->fp64, ept, bs, ctx->stepper, ctx->d_ewt != nullptr);
    if (occ < 1) occ = 1;
    pl.grid_blocks = std::max(1, std::min(ctx->sm_count * occ, (pl.n_items + 3) / 4));
    pl.stride = (int64_t)G * std::max(ctx->geo.max_ns, 1) * lanes * ept;
    // descriptor of the context's own Matsubara sweep
    scd::GrainSweep gs{};
    gs.lines = ctx->d_lines;
    gs.groups = pl.d_groups;
    gs.image_in = ctx->d_img_in;
    gs.image_out = ctx->d_img_out;
    if (pl.n_blocks > 1) {  // each energy block writes its own image; launch_block_sum adds them
        CK(dalloc(ctx, &pl.d_img_blocks, (size_t)pl.n_blocks * ctx->geo.n_slots * (ctx->fp64 ? 32 : 16)));
        gs.image_out = pl.d_img_blocks;
    }
    gs.n_slots = ctx->geo.n_slots;
    gs.n_lines = (int32_t)ctx->geo.lines.size();
    gs.n_groups = pl.n_groups;
    gs.exits[0] = ctx->d_exit[0];
    gs.exits[1] = ctx->d_exit[1];
    gs.energies = nullptr;
    gs.mats_eps = ctx->d_eps;  // nullptr for plain Matsubara energies
    gs.mats_w = ctx->d_ewt;
    gs.t = ctx->geo.prm.t;
    gs.h = ctx->geo.prm.h;
    gs.broadening = 0.0;
    gs.n_e = n_e;
    gs.lanes = lanes;
    gs.lines_per_warp = G;
    gs.ne_pad = lanes * ept;
    gs.n_blocks = pl.n_blocks;
    gs.max_ns = std::max(ctx->geo.max_ns, 1);
    gs.ept = ept;
    CK(dalloc(ctx, &pl.d_grain, sizeof(gs)));
    CK(cudaMemcpy(pl.d_grain, &gs, sizeof(gs), cudaMemcpyHostToDevice));
    auto res = ctx->plans.emplace(key, std::move(pl));
    *out = &res.first->second;
    return SC_OK;
}

// A = -(1/kappa^2) G * (j - <j>) from d_j and d_jsum (App. D): FFT convolution
// where the padded grid fits, else the direct sum
cudaError_t induced_field(sc_ctx *ctx, double *aind, cudaStream_t st) {
    const double k = ctx->geo.prm.kappa;
    if (ctx->vp_fft)
        return scd::vecpot_fft_apply(ctx->vp, ctx->grid, ctx->d_mask, ctx->d_j, ctx->d_jsum, (double)ctx->geo.n_in,
                                     1.0 / (k * k), aind, st);
    return scd::launch_vector_potential(ctx->grid, ctx->d_mask, ctx->d_j, ctx->d_jsum, (double)ctx->geo.n_in, ctx->d_G,
                                        ctx->G_width, 1.0 / (k * k), aind, st);
}

sc_status rotate_fields(sc_ctx *ctx, cudaStream_t st) {
    if (ctx->fp64) {
        CK(scd::launch_rotate(true, ctx->d_geo, ctx->d_slot_line, ctx->geo.n_slots, ctx->d_pairs, ctx->grid,
                              ctx->d_ghost, ctx->d_delta, ctx->have_aind ? ctx->d_aind : nullptr, ctx->d_img_in,
                              st));
    } else {
        CK(scd::launch_fields_f32(ctx->grid, ctx->d_ghost, ctx->d_delta, ctx->have_aind ? ctx->d_aind : nullptr,
                                  ctx->d_pad0, ctx->d_padc, st));
        CK(scd::launch_rotate_f32(ctx->d_line_f32, ctx->d_slot_line, ctx->geo.n_slots, ctx->d_pair_f32, ctx->grid,
                                  ctx->d_ghost, ctx->d_pad0, ctx->d_padc, (float4 *)ctx->d_img_in, st));
    }
    return SC_OK;
}

sc_status rotate_back(sc_ctx *ctx, cudaStream_t st) {
    if (ctx->fp64)
        CK(scd::launch_rotate_back(true, ctx->d_pairs, ctx->geo.n_pairs, ctx->d_back, ctx->grid, ctx->d_mask,
                                   ctx->d_img_out, ctx->d_acc, st));
    else
        CK(scd::launch_rotate_back_f32(ctx->d_pair_f32, ctx->geo.n_pairs, ctx->d_back, ctx->grid, ctx->d_mask,
                                       (const float4 *)ctx->d_img_out, ctx->d_acc, st));
    return SC_OK;
}

}  // namespace sc_internal

namespace {

using sc_internal::check_ctx;
using sc_internal::make_plan;
using sc_internal::make_plan_layout;

// one persistent sweep launch over the plan's items for one grain descriptor
sc_status launch_plan_sweep(sc_ctx *ctx, const Plan &pl, const scd::GrainSweep *d_grain, bool retarded,
                            bool first, int parity, cudaStream_t st) {
    CKS(ensure_scratch(ctx, (size_t)pl.grid_blocks * 4 * (size_t)pl.stride * 2 * ctx->real_bytes));
    CK(cudaMemsetAsync(ctx->d_counter, 0, sizeof(int32_t), st));
    scd::SweepLaunch a{};
    a.grains = d_grain;
    a.items = pl.d_items;
    a.n_items = pl.n_items;
    a.counter = ctx->d_counter;
    a.scratch = ctx->d_scratch;
    a.scratch_stride = pl.stride;
    a.scratch_elems = (int64_t)(ctx->scratch_bytes / (2 * ctx->real_bytes));
    a.n_grains = 1;
    a.energies_per_lane = pl.ept;
    a.first_sweep = first ? 1 : 0;
    a.parity = parity;
    a.retarded = retarded ? 1 : 0;
    a.grid_blocks = pl.grid_blocks;
    a.block_threads = 128;
    a.stepper = ctx->stepper;
    a.weighted = ctx->d_ewt != nullptr ? 1 : 0;
    a.blocked = !retarded && pl.n_blocks > 1 ? 1 : 0;
    CK(scd::launch_sweep(ctx->fp64, a, st));
    if (a.blocked)  // the energy blocks' images, added in block order
        CK(scd::launch_block_sum(ctx->fp64, pl.d_img_blocks, pl.n_blocks, ctx->geo.n_slots, ctx->d_img_out, st));
    return SC_OK;
}

sc_status ensure_outputs_impl(sc_ctx *ctx, cudaStream_t st) {
    if (!ctx->have_sweep) return set_err(ctx, SC_ESTATE, "no sweep since the fields were last set");
    if (ctx->have_outputs) return SC_OK;
    const double kappa = ctx->geo.prm.kappa;
    const bool magn = kappa > 0.0 && std::isfinite(kappa) && ctx->have_aind;
    CK(scd::launch_outputs(ctx->grid, ctx->d_mask, ctx->d_acc, ctx->d_delta, magn ? ctx->d_aind : nullptr,
                           ctx->geo.prm.t, ctx->norms, magn ? kappa : 0.0, ctx->d_dnew, ctx->d_j, ctx->d_F,
                           ctx->d_sums, ctx->d_part, st));
    ctx->have_outputs = true;
    return SC_OK;
}

sc_status copy_out(sc_ctx *ctx, void *dst, const void *src, size_t bytes, int on_device, cudaStream_t st) {
    if (!dst) return SC_OK;
    CK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    if (!on_device) CK(cudaStreamSynchronize(st));
    return SC_OK;
}

}  // namespace

namespace sc_internal {
sc_status ensure_outputs(sc_ctx *ctx, cudaStream_t st) { return ensure_outputs_impl(ctx, st); }
}  // namespace sc_internal

extern "C" {

const char *sc_version(void) { return "sc-riccati 0.1 (sm_103a)"; }

const char *sc_last_error(const sc_ctx *ctx) {
    if (!ctx) return g_create_error.c_str();
    return ctx->err.c_str();
}

sc_status sc_params_default(sc_params *p) {
    if (!p) return SC_EINVAL;
    std::memset(p, 0, sizeof *p);
    p->nx = p->ny = 64;
    p->h = 1.0;
    p->x0 = p->y0 = -32.0;
    p->shape_kind = 0;
    p->disc_r = 30.0;
    p->pairing = SC_PAIR_S;
    p->t = 0.5;
    p->kappa = 0.0;
    p->charge_sign = -1;
    p->n_angles = 32;
    p->n_energies = 16;
    p->lattice_ox = 0.1;
    p->lattice_oy = 0.2;
    p->precision = SC_PREC_FP32;
    return SC_OK;
}

sc_status sc_destroy(sc_ctx *ctx) {
    if (!ctx) return SC_EINVAL;
    if (!ctx->allocs.empty()) cudaSetDevice(ctx->device);
    for (void *p : ctx->allocs) cudaFree(p);
    for (cudaEvent_t e : ctx->ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->ev_adj)
        if (e) cudaEventDestroy(e);
    if (!ctx->allocs.empty()) (void)cudaGetLastError();  // teardown errors are not the caller's
    delete ctx;
    return SC_OK;
}

sc_status sc_create(const sc_params *p, sc_ctx **out) {
    g_create_error.clear();
    if (!p || !out) {
        g_create_error = "null argument";
        return SC_EINVAL;
    }
    *out = nullptr;
    if (p->precision != SC_PREC_FP32 && p->precision != SC_PREC_FP64) {
        g_create_error = "unknown precision";
        return SC_EINVAL;
    }
    if (p->lanes_per_line != 0 && p->lanes_per_line != 2 && p->lanes_per_line != 4 && p->lanes_per_line != 8 &&
        p->lanes_per_line != 16 && p->lanes_per_line != 32) {
        g_create_error = "lanes_per_line must be 0, 2, 4, 8, 16 or 32";
        return SC_EINVAL;
    }
    if (p->stepper != SC_STEP_CLOSED && p->stepper != SC_STEP_MIDPOINT) {
        g_create_error = "stepper must be SC_STEP_CLOSED or SC_STEP_MIDPOINT";
        return SC_EINVAL;
    }
    if (p->energy_sum != SC_SUM_MATSUBARA && p->energy_sum != SC_SUM_OZAKI) {
        g_create_error = "energy_sum must be SC_SUM_MATSUBARA or SC_SUM_OZAKI";
        return SC_EINVAL;
    }
    if (p->adjoint_checkpoint != 0 &&
        (p->adjoint_checkpoint < 2 || p->precision != SC_PREC_FP32 || p->stepper != SC_STEP_CLOSED)) {
        g_create_error = "adjoint_checkpoint must be 0, or >= 2 with precision FP32 and the closed-form stepper";
        return SC_EINVAL;
    }
    // n_energies = 0: the count follows from the energy cutoff
    sc_params resolved = *p;
    if (resolved.n_energies == 0) {
        if (!(p->eps_cut > 0.0) || !(p->t > 0.0)) {
            g_create_error = "n_energies = 0 needs eps_cut > 0 and t > 0";
            return SC_EINVAL;
        }
        resolved.n_energies = p->energy_sum == SC_SUM_OZAKI ? sc_ozaki_poles_for_cutoff(p->t, p->eps_cut)
                                                            : (int32_t)std::ceil(p->eps_cut / p->t - 0.5);
        if (resolved.n_energies < 1) {
            g_create_error = "eps_cut gives no energy";
            return SC_EINVAL;
        }
    }
    p = &resolved;
    if (p->energy_sum == SC_SUM_OZAKI && (p->n_energies < 1 || p->n_energies > 1024)) {
        g_create_error = "Ozaki sums take 1 to 1024 poles (n_energies)";
        return SC_EINVAL;
    }
    sc_ctx *ctx = new (std::nothrow) sc_ctx();
    if (!ctx) {
        g_create_error = "host allocation failed";
        return SC_ENOMEM;
    }
    std::string why = ctx->geo.build(*p);
    if (why.empty() && p->mask &&
        std::memcmp(p->mask, ctx->geo.mask.data(), ctx->geo.mask.size()) != 0)
        why = "the given mask does not match the mask of the shape";
    if (!why.empty()) {
        g_create_error = why;
        delete ctx;
        return SC_EINVAL;
    }
    const scg::Geometry &G = ctx->geo;
    ctx->fp64 = p->precision == SC_PREC_FP64;
    ctx->real_bytes = ctx->fp64 ? 8 : 4;
    ctx->n_e = p->n_energies;
    ctx->forced_lanes = p->lanes_per_line;
    ctx->stepper = p->stepper;
    ctx->adj_ckpt = p->adjoint_checkpoint;
    // energies and weights of the energy sums; D = ln t + t sum_n w_n / eps_n
    // (Matsubara: eps_n = t (n + 1/2), w_n = 1, i.e. 2 sum 1/(2n + 1))
    ctx->energy_sum = p->energy_sum;
    ctx->eps.resize(ctx->n_e);
    ctx->ewt.assign(ctx->n_e, 1.0);
    if (p->energy_sum == SC_SUM_OZAKI) {
        std::vector<double> z(ctx->n_e);
        sc_ozaki_poles(ctx->n_e, z.data(), ctx->ewt.data());
        for (int n = 0; n < ctx->n_e; ++n) ctx->eps[n] = p->t * z[n] / (2.0 * M_PI);
    } else {
        for (int n = 0; n < ctx->n_e; ++n) ctx->eps[n] = p->t * (n + 0.5);
    }
    {
        double s = 0.0;
        for (int n = 0; n < ctx->n_e; ++n) s += ctx->ewt[n] / ctx->eps[n];
        ctx->normD = std::log(p->t) + p->t * s;
    }
    if (p->host_only) {
        ctx->host_only = true;
        *out = ctx;
        return SC_OK;
    }
    if (const char *fa = std::getenv("SC_TEST_FAIL_ALLOC_AT")) ctx->fail_alloc_at = std::atol(fa);
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) {
        g_create_error = std::string("no CUDA device: ") + cudaGetErrorString(e);
        delete ctx;
        return SC_ECUDA;
    }
    // grid description for the kernels
    scd::GridDev &gd = ctx->grid;
    gd.nx = G.nx;
    gd.ny = G.ny;
    gd.h = p->h;
    gd.x0 = p->x0;
    gd.y0 = p->y0;
    gd.ox = G.ox;
    gd.oy = G.oy;
    gd.bfield = M_PI * p->flux_quanta / G.area;  // B = pi alpha / area in units of B0
    gd.n_comp = G.n_comp;
    for (int c = 0; c < 4; ++c) {
        ctx->norms.D[c] = ctx->normD - std::log(G.tc_ratio[c]);
        ctx->norms.kD[c] = p->t / (2.0 * 3.141592653589793) / ctx->norms.D[c];
    }
    gd.gx = p->gauge_cx;
    gd.gy = p->gauge_cy;
    gd.gauge = p->gauge;
    gd.flux = p->flux_quanta;
    gd.charge_sign = p->charge_sign;
    gd.n_slots = G.n_slots;
    gd.n_lines = (int32_t)G.lines.size();
    gd.n_pairs = G.n_pairs;

    // host tables
    const int P = G.n_pairs;
    const size_t nL = G.lines.size();
    std::vector<scd::LineGeo> lgeo(nL);
    std::vector<scd::LineDev> ldev(nL);
    std::vector<int32_t> slot_line(G.n_slots);
    for (size_t L = 0; L < nL; ++L) {
        const scg::LineInfo &li = G.lines[L];
        scd::LineGeo &lg = lgeo[L];
        lg.pair = li.pair;
        lg.l = li.l;
        lg.m0 = li.m0;
        lg.ns = li.ns;
        lg.slot0 = li.slot0;
        lg.pad = 0;
        lg.smid = 0.5 * (li.smin + li.smax);
        for (int q = 0; q < std::max(li.ns, 1); ++q) slot_line[li.slot0 + q] = (int32_t)L;
        scd::LineDev &ld = ldev[L];
        ld.ns = li.ns;
        ld.slot0 = li.slot0;
        ld.exit_f = (int32_t)L;
        ld.exit_b = (int32_t)(nL + L);
        if (li.ns > 0) {
            ld.lead = std::max(0.0, li.m0 * p->h - li.smin);
            ld.tail = std::max(0.0, li.smax - li.m1 * p->h);
        } else {
            ld.lead = ld.tail = li.smax - li.smin;
        }
        for (int q = 0; q < 4; ++q) {
            ld.tap_f[q] = li.fwd[q].slot;
            ld.w_f[q] = li.fwd[q].w;
            ld.tap_b[q] = li.bwd[q].slot;
            ld.w_b[q] = li.bwd[q].w;
        }
    }
    // rotate-back table: per lattice line, the sampled chords of the nearest
    // lattice line that has some; one chord inline, several in a list after
    // the per-line records
    std::vector<scd::BackLine> lback(G.lats.size());
    for (int q = 0; q < G.n_pairs; ++q) {
        const scg::PairInfo &pp = G.pairs[q];
        for (int l = pp.l_lo; l <= pp.l_hi; ++l) {
            const scg::LatticeLine &src = G.lat(q, G.lat(q, l).sampled);
            std::vector<int> cand;
            for (int c = src.c0; c < src.c0 + src.nc; ++c)
                if (G.lines[c].ns > 0) cand.push_back(c);
            const scg::LineInfo &c0 = G.lines[cand[0]];
            scd::BackLine &b = lback[pp.lat0 + (l - pp.l_lo)];
            b = scd::BackLine{-1, c0.m0, c0.ns, c0.slot0};
            if (cand.size() > 1) {
                b.more = (int32_t)lback.size();
                for (int c : cand) {
                    const scg::LineInfo &lc = G.lines[c];
                    lback.push_back(scd::BackLine{(int32_t)cand.size(), lc.m0, lc.ns, lc.slot0});
                }
            }
        }
    }
    const size_t nBack = lback.size();
    gd.n_back = (int32_t)nBack;
    std::vector<scd::PairDev> pdev(P);
    const double cx = 0.5 + (p->x0 - G.ox) / p->h, cy = 0.5 + (p->y0 - G.oy) / p->h;
    for (int q = 0; q < P; ++q) {
        const scg::PairInfo &pp = G.pairs[q];
        scd::PairDev &d = pdev[q];
        d.ex = pp.ex;
        d.ey = pp.ey;
        d.u0 = cx * (-pp.ey) + cy * pp.ex;  // (R - O).e_perp / h at grid point (0, 0)
        d.v0 = cx * pp.ex + cy * pp.ey;
        d.eta = pp.eta;
        for (int c = 0; c < 4; ++c) d.eta_c[c] = pp.eta_c[c];
        d.wa = G.weight[q];
        d.wb = G.weight[q + P];
        d.l_lo = pp.l_lo;
        d.l_hi = pp.l_hi;
        d.lat0 = pp.lat0;
        d.pad = 0;
    }

    // FP32 production path: fixed-point lattice coordinates (2^-40 grid units)
    const double fix = std::ldexp(1.0, scd::kFixBits);
    auto to_fix = [&](double v) { return (int64_t)std::llround(v * fix); };
    std::vector<scd::LineF32> lf(nL);
    std::vector<scd::PairF32> pf(P);
    {
        const double cxo = (G.ox - p->x0) / p->h - 0.5, cyo = (G.oy - p->y0) / p->h - 0.5;
        const double half_b = 0.5 * gd.bfield;
        for (size_t L = 0; L < nL; ++L) {
            const scg::LineInfo &li = G.lines[L];
            const scg::PairInfo &pp = G.pairs[li.pair];
            const double sh = li.ns > 0 ? (double)li.m0 : 0.5 * (li.smin + li.smax) / p->h;  // along, units of h
            lf[L].gx0 = to_fix(cxo + li.l * (-pp.ey) + sh * pp.ex);
            lf[L].gy0 = to_fix(cyo + li.l * pp.ex + sh * pp.ey);
            // symmetric gauge: v.A_ext is constant on a line, B/2 (e_y (Ox - gx) - e_x (Oy - gy) - l h);
            // the other gauges are evaluated at every sample
            lf[L].aext = p->gauge != SC_GAUGE_SYMMETRIC
                             ? 0.0f
                             : (float)(p->charge_sign * half_b *
                                       (pp.ey * (G.ox - p->gauge_cx) - pp.ex * (G.oy - p->gauge_cy) - li.l * p->h));
            lf[L].pair = li.pair;
            lf[L].ns = li.ns;
            lf[L].slot0 = li.slot0;
            lf[L].m0 = li.ns > 0 ? li.m0 : (int32_t)std::floor(sh);
        }
        const double cx = 0.5 + (p->x0 - G.ox) / p->h, cy = 0.5 + (p->y0 - G.oy) / p->h;
        for (int q = 0; q < P; ++q) {
            const scg::PairInfo &pp = G.pairs[q];
            scd::PairF32 &d = pf[q];
            d.dx = to_fix(pp.ex);
            d.dy = to_fix(pp.ey);
            d.ui = to_fix(-pp.ey);
            d.uj = to_fix(pp.ex);
            d.u0 = to_fix(cx * (-pp.ey) + cy * pp.ex);
            d.vi = to_fix(pp.ex);
            d.vj = to_fix(pp.ey);
            d.v0 = to_fix(cx * pp.ex + cy * pp.ey);
            const double ws = G.weight[q] + G.weight[q + P];
            d.eta = (float)pp.eta;
            d.w_eta = (float)(ws * pp.eta);
            for (int c = 0; c < 4; ++c) {
                d.eta_c[c] = (float)pp.eta_c[c];
                d.w_eta_c[c] = (float)(ws * pp.eta_c[c]);
            }
            d.w_ex = (float)(ws * pp.ex);
            d.w_ey = (float)(ws * pp.ey);
            d.w_sum = (float)ws;
            d.wa = (float)G.weight[q];
            d.wb = (float)G.weight[q + P];
            d.ex_f = (float)pp.ex;
            d.ey_f = (float)pp.ey;
            d.l_lo = pp.l_lo;
            d.l_hi = pp.l_hi;
            d.lat0 = pp.lat0;
            d.pad = 0;
        }
        // gauge origin in the same fixed-point grid coordinates
        gd.gfx = to_fix((p->gauge_cx - p->x0) / p->h - 0.5);
        gd.gfy = to_fix((p->gauge_cy - p->y0) / p->h - 0.5);
    }

    // device memory
    const size_t np = npts(ctx);
    const size_t t4 = ctx->fp64 ? 32 : 16;
    const size_t cplx = 2 * ctx->real_bytes;
    auto fail_cuda = [&](cudaError_t err, const char *what) {
        g_create_error = std::string(what) + ": " + cudaGetErrorString(err);
        sc_status st = err == cudaErrorMemoryAllocation ? SC_ENOMEM : SC_ECUDA;
        sc_destroy(ctx);
        return st;
    };
#define CA(ptr, bytes)                                      \
    do {                                                    \
        cudaError_t err_ = dalloc(ctx, &(ptr), (bytes));    \
        if (err_ != cudaSuccess) return fail_cuda(err_, #ptr); \
    } while (0)
#define CP(dst, src, bytes)                                                      \
    do {                                                                         \
        cudaError_t err_ = cudaMemcpy((dst), (src), (bytes), cudaMemcpyHostToDevice); \
        if (err_ != cudaSuccess) return fail_cuda(err_, "upload " #dst);        \
    } while (0)
    if (count_bad_indices(G) != 0) {
        g_create_error = "internal error: an index of the sweep tables is out of range";
        sc_destroy(ctx);
        return SC_ESTATE;
    }
    CA(ctx->d_mask, np);
    CP(ctx->d_mask, G.mask.data(), np);
    CA(ctx->d_ghost, G.ghost.size() * sizeof(int32_t));
    CP(ctx->d_ghost, G.ghost.data(), G.ghost.size() * sizeof(int32_t));
    CA(ctx->d_geo, nL * sizeof(scd::LineGeo));
    CP(ctx->d_geo, lgeo.data(), nL * sizeof(scd::LineGeo));
    CA(ctx->d_lines, nL * sizeof(scd::LineDev));
    CP(ctx->d_lines, ldev.data(), nL * sizeof(scd::LineDev));
    CA(ctx->d_back, nBack * sizeof(scd::BackLine));
    CP(ctx->d_back, lback.data(), nBack * sizeof(scd::BackLine));
    CA(ctx->d_slot_line, slot_line.size() * sizeof(int32_t));
    CP(ctx->d_slot_line, slot_line.data(), slot_line.size() * sizeof(int32_t));
    CA(ctx->d_pairs, P * sizeof(scd::PairDev));
    CP(ctx->d_pairs, pdev.data(), P * sizeof(scd::PairDev));
    const size_t nc = (size_t)G.n_comp;
    CA(ctx->d_delta, 2 * np * nc * sizeof(double));
    CA(ctx->d_aind, 2 * np * sizeof(double));
    CA(ctx->d_acc, (3 + 2 * nc) * np * sizeof(double));
    CA(ctx->d_dnew, 2 * np * nc * sizeof(double));
    CA(ctx->d_j, 2 * np * sizeof(double));
    CA(ctx->d_F, np * sizeof(double));
    CA(ctx->d_sums, 8 * sizeof(double));
    CA(ctx->d_part, (size_t)scd::reduce_blocks((int64_t)np) * 4 * sizeof(double));
    CA(ctx->d_jsum, 2 * sizeof(double));
    CA(ctx->d_diff, sizeof(double));
    CA(ctx->d_counter, sizeof(int32_t));
    CA(ctx->d_img_in, G.n_slots * t4);
    CA(ctx->d_img_out, G.n_slots * t4);
    for (int b = 0; b < 2; ++b) CA(ctx->d_exit[b], 2 * nL * (size_t)ctx->n_e * cplx);
    if (ctx->energy_sum == SC_SUM_OZAKI) {
        CA(ctx->d_eps, ctx->n_e * sizeof(double));
        CP(ctx->d_eps, ctx->eps.data(), ctx->n_e * sizeof(double));
        CA(ctx->d_ewt, ctx->n_e * sizeof(double));
        CP(ctx->d_ewt, ctx->ewt.data(), ctx->n_e * sizeof(double));
    }
    if (!ctx->fp64) {
        CA(ctx->d_line_f32, nL * sizeof(scd::LineF32));
        CP(ctx->d_line_f32, lf.data(), nL * sizeof(scd::LineF32));
        CA(ctx->d_pair_f32, P * sizeof(scd::PairF32));
        CP(ctx->d_pair_f32, pf.data(), P * sizeof(scd::PairF32));
        const size_t npad = (size_t)(ctx->geo.nx + 2) * (ctx->geo.ny + 2);
        CA(ctx->d_pad0, npad * sizeof(float4));
        CA(ctx->d_padc, npad * (nc > 1 ? nc - 1 : 1) * sizeof(float2));
    }
    if (p->record_timings) {
        ctx->timing = true;
        for (auto &e : ctx->ev) {
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) return fail_cuda(err, "cudaEventCreate");
        }
        for (auto &e : ctx->ev_adj) {
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) return fail_cuda(err, "cudaEventCreate");
        }
    }
    {
        cudaError_t err = cudaMemset(ctx->d_delta, 0, 2 * np * nc * sizeof(double));
        if (err == cudaSuccess) err = cudaMemset(ctx->d_aind, 0, 2 * np * sizeof(double));
        if (err == cudaSuccess) err = cudaMemset(ctx->d_img_out, 0, G.n_slots * t4);
        if (err != cudaSuccess) return fail_cuda(err, "memset");
    }
    const double kappa = p->kappa;
    if (kappa > 0.0 && std::isfinite(kappa)) {
        // cell-integrated Green's function of the 2D Laplacian (App. D)
        const int W = std::max(G.nx, G.ny);
        ctx->G_width = W;
        std::vector<double> Gt((size_t)W * W);
        const double h = p->h;
        auto alpha = [](double m, double n) {
            return (1 + 2 * m) * (1 + 2 * n) * std::log(0.5 * (1 + 2 * m) * (1 + 2 * m) + 0.5 * (1 + 2 * n) * (1 + 2 * n));
        };
        auto beta = [](double m, double n) { return (-2 * m * m + 2 * n * n + 4 * n + 1) * std::atan((1 + 2 * m) / (1 + 2 * n)); };
        for (int a = 0; a < W; ++a)
            for (int b = 0; b < W; ++b) {
                double s = 0.0;
                for (int sa = -1; sa <= 1; sa += 2)
                    for (int sb = -1; sb <= 1; sb += 2) {
                        const double m = sa * (double)a, n = sb * (double)b;
                        s += alpha(m, n) + beta(m, n) + beta(n, m);
                    }
                Gt[(size_t)a * W + b] = h * h / (4 * M_PI) * (2 * std::log(h) - std::log(2.0) - 3 + 0.25 * s);
            }
        CA(ctx->d_G, Gt.size() * sizeof(double));
        CP(ctx->d_G, Gt.data(), Gt.size() * sizeof(double));
        // zero-padded FFT convolution (App. D) where the padded grid fits one
        // shared-memory transform per row; larger grids keep the direct sum
        scd::VecpotFft &f = ctx->vp;
        f.lx = scd::vecpot_fft_log2(G.nx);
        f.ly = scd::vecpot_fft_log2(G.ny);
        f.px = 1 << f.lx;
        f.py = 1 << f.ly;
        if (f.px <= scd::kVecpotMaxFft && f.py <= scd::kVecpotMaxFft) {
            auto twiddles = [](int n) {
                std::vector<double2> t(n / 2);
                for (int k = 0; k < n / 2; ++k)
                    t[k] = make_double2(std::cos(2.0 * M_PI * k / n), -std::sin(2.0 * M_PI * k / n));
                return t;
            };
            const std::vector<double2> tx = twiddles(f.px), ty = twiddles(f.py);
            const size_t nb = (size_t)f.px * f.py * sizeof(double2);
            CA(f.tw_x, tx.size() * sizeof(double2));
            CP(f.tw_x, tx.data(), tx.size() * sizeof(double2));
            CA(f.tw_y, ty.size() * sizeof(double2));
            CP(f.tw_y, ty.data(), ty.size() * sizeof(double2));
            CA(f.buf, nb);
            CA(f.tbuf, nb);
            CA(f.ghat, nb);
            cudaError_t err = scd::vecpot_fft_attributes();
            if (err == cudaSuccess) err = scd::vecpot_fft_prepare(f, ctx->d_G, W, G.nx, G.ny, 0);
            if (err == cudaSuccess) err = cudaStreamSynchronize(0);
            if (err != cudaSuccess) return fail_cuda(err, "vector-potential transform");
            ctx->vp_fft = true;
        }
    }
#undef CA
#undef CP
    sc_status st = make_plan(ctx, ctx->n_e, 0, &ctx->main_plan, true);
    if (st == SC_OK && !ctx->forced_lanes) {
        // A small grain (few lines, few energies) leaves resident warps without
        // work: one doubling of the lanes per line doubles the work items, kept
        // while the items stay fewer than the resident warps and >= 3/4 of the
        // lane slots carry an energy (measured: 14 Ozaki poles on 256^2, 0.56 ->
        // 0.44 ms; a grain that fills the GPU is left alone).
        Plan *pl = ctx->main_plan;
        const int occ = std::max(1, scd::sweep_occupancy(ctx->fp64, pl->ept, 128, ctx->stepper, ctx->d_ewt != nullptr));
        const int64_t resident = (int64_t)ctx->sm_count * occ * 4;
        const int l2 = 2 * pl->lanes, e2 = (ctx->n_e + l2 - 1) / l2;
        if (pl->lanes < 32 && pl->n_blocks == 1 && pl->n_groups < resident && 4 * ctx->n_e >= 3 * l2 * e2)
            st = make_plan_layout(ctx, ctx->n_e, l2, e2, &ctx->main_plan);
    }
    if (st != SC_OK) {
        g_create_error = ctx->err;
        sc_destroy(ctx);
        return st;
    }
    *out = ctx;
    return SC_OK;
}

sc_status sc_get_info(const sc_ctx *ctx, sc_info *info) {
    if (!ctx || !info) return SC_EINVAL;
    const scg::Geometry &G = ctx->geo;
    std::memset(info, 0, sizeof *info);
    info->n_pairs = G.n_pairs;
    info->n_lines = (int32_t)G.lines.size();
    info->n_samples = G.n_samples;
    info->n_in = G.n_in;
    int64_t steps = 0;
    for (const auto &li : G.lines) steps += 2 * (int64_t)(li.ns + 1);
    info->steps_per_sweep = steps * ctx->n_e;
    info->points_per_sweep = 2 * G.n_samples * ctx->n_e;
    info->area = G.area;
    info->norm_D = ctx->normD;
    if (ctx->main_plan) {
        info->lanes_per_line = ctx->main_plan->lanes;
        info->energies_per_lane = ctx->main_plan->ept;
        info->lines_per_warp = ctx->main_plan->lines_per_warp;
    }
    info->scratch_bytes = (int64_t)ctx->scratch_bytes;
    if (ctx->timing && ctx->timed) {
        float a = 0.f, b = 0.f, c = 0.f;
        if (cudaEventSynchronize(ctx->ev[3]) == cudaSuccess && cudaEventElapsedTime(&a, ctx->ev[0], ctx->ev[1]) == cudaSuccess &&
            cudaEventElapsedTime(&b, ctx->ev[1], ctx->ev[2]) == cudaSuccess &&
            cudaEventElapsedTime(&c, ctx->ev[2], ctx->ev[3]) == cudaSuccess) {
            info->ms_rotate = a;
            info->ms_sweep = b;
            info->ms_rotate_back = c;
        } else {
            (void)cudaGetLastError();  // a failed query must not linger as the thread's last error
        }
    }
    if (ctx->timing && ctx->adj_timed) {
        float a = 0.f;
        if (cudaEventSynchronize(ctx->ev_adj[1]) == cudaSuccess &&
            cudaEventElapsedTime(&a, ctx->ev_adj[0], ctx->ev_adj[1]) == cudaSuccess)
            info->ms_adjoint = a;
        else
            (void)cudaGetLastError();
    }
    return SC_OK;
}

sc_status sc_energy_grid(const sc_ctx *ctx, double *eps, double *weights) {
    if (!ctx) return SC_EINVAL;
    for (int n = 0; n < ctx->n_e; ++n) {
        if (eps) eps[n] = ctx->eps[n];
        if (weights) weights[n] = ctx->ewt[n];
    }
    return SC_OK;
}

sc_status sc_get_mask(const sc_ctx *ctx, uint8_t *mask) {
    if (!ctx || !mask) return SC_EINVAL;
    std::memcpy(mask, ctx->geo.mask.data(), ctx->geo.mask.size());
    return SC_OK;
}

sc_status sc_set_fields(sc_ctx *ctx, const double *delta, const double *a_ind, int on_device, void *stream) {
    CKS(check_ctx(ctx));
    if (!delta) return set_err(ctx, SC_EINVAL, "delta is required");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = 2 * npts(ctx) * sizeof(double);
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(ctx->d_delta, delta, bytes * ctx->geo.n_comp, k, st));
    if (a_ind) {
        CK(cudaMemcpyAsync(ctx->d_aind, a_ind, bytes, k, st));
        ctx->have_aind = true;
    } else {
        CK(cudaMemsetAsync(ctx->d_aind, 0, bytes, st));
        ctx->have_aind = false;
    }
    if (!on_device) CK(cudaStreamSynchronize(st));
    ctx->have_sweep = false;
    ctx->have_outputs = false;
    ctx->acc_kind = -1;  // new fields start a new accelerator history
    return SC_OK;
}

sc_status sc_get_fields(sc_ctx *ctx, double *delta, double *a_ind, int on_device, void *stream) {
    CKS(check_ctx(ctx));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = 2 * npts(ctx) * sizeof(double);
    if (delta) CKS(copy_out(ctx, delta, ctx->d_delta, bytes * ctx->geo.n_comp, on_device, st));
    if (a_ind) CKS(copy_out(ctx, a_ind, ctx->d_aind, bytes, on_device, st));
    return SC_OK;
}

sc_status sc_reset_boundary(sc_ctx *ctx) {
    CKS(check_ctx(ctx));
    ctx->have_boundary = false;
    return SC_OK;
}

sc_status sc_riccati_sweep(sc_ctx *ctx, void *stream) {
    CKS(check_ctx(ctx));
    if (ctx->batch_member) return set_err(ctx, SC_ESTATE, "this context belongs to a batch: use sc_batch_sweep");
    cudaStream_t st = (cudaStream_t)stream;
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[0], st));
    CKS(sc_internal::rotate_fields(ctx, st));
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[1], st));
    const Plan &pl = *ctx->main_plan;
    ctx->last_first = !ctx->have_boundary;
    CKS(launch_plan_sweep(ctx, pl, pl.d_grain, false, ctx->last_first, ctx->cur, st));
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[2], st));
    CKS(sc_internal::rotate_back(ctx, st));
    if (ctx->timing) {
        CK(cudaEventRecord(ctx->ev[3], st));
        ctx->timed = true;
    }
    ctx->cur ^= 1;
    ctx->have_boundary = true;
    ctx->have_sweep = true;
    ctx->have_outputs = false;
    ++ctx->sweeps;
    return SC_OK;
}

sc_status sc_burnin(sc_ctx *ctx, int32_t max_sweeps, double tol, void *stream) {
    CKS(check_ctx(ctx));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = 2 * (int64_t)ctx->geo.lines.size() * ctx->n_e;
    for (int it = 0; it < max_sweeps; ++it) {
        const bool had = ctx->have_boundary;
        CKS(sc_riccati_sweep(ctx, stream));
        if (!had) continue;
        CK(scd::launch_max_diff(n, ctx->d_exit[ctx->cur], ctx->d_exit[1 - ctx->cur], ctx->fp64, ctx->d_diff, st));
        double diff = 0.0;
        CK(cudaMemcpyAsync(&diff, ctx->d_diff, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (diff <= tol) return SC_OK;
    }
    return max_sweeps > 0 ? SC_ENOTCONV : SC_OK;
}

sc_status sc_gap_update(sc_ctx *ctx, double *delta_out, double *eps_G, int on_device, void *stream) {
    CKS(check_ctx(ctx));
    cudaStream_t st = (cudaStream_t)stream;
    CKS(ensure_outputs_impl(ctx, st));
    CKS(copy_out(ctx, delta_out, ctx->d_dnew, 2 * npts(ctx) * ctx->geo.n_comp * sizeof(double), on_device, st));
    if (eps_G) {
        double s[4];
        CK(cudaMemcpyAsync(s, ctx->d_sums, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (s[3] != 0.0) return set_err(ctx, SC_ENUMERIC, "non-finite values in the sweep outputs");
        *eps_G = s[1] > 0.0 ? std::sqrt(s[0] / s[1]) : 0.0;
        if (ctx->history.size() == sc_ctx::kHistory) ctx->history.pop_front();
        ctx->history.emplace_back(ctx->sweeps, *eps_G);
    }
    return SC_OK;
}

sc_status sc_get_history(const sc_ctx *ctx, int32_t *n, int64_t *sweeps, double *eps_G) {
    if (!ctx || !n || *n < 0 || (*n > 0 && (!sweeps || !eps_G))) {
        sc_internal::set_thread_error("sc_get_history needs a context, n >= 0 and, for n > 0, both arrays");
        return SC_EINVAL;
    }
    const size_t cap = (size_t)*n;
    size_t k = 0;
    for (const auto &r : ctx->history) {
        if (k == cap) break;
        sweeps[k] = r.first;
        eps_G[k] = r.second;
        ++k;
    }
    *n = (int32_t)ctx->history.size();
    return SC_OK;
}

sc_status sc_clear_history(sc_ctx *ctx) {
    if (!ctx) return SC_EINVAL;
    ctx->history.clear();
    return SC_OK;
}

sc_status sc_current(sc_ctx *ctx, double *j_out, int on_device, void *stream) {
    CKS(check_ctx(ctx));
    cudaStream_t st = (cudaStream_t)stream;
    CKS(ensure_outputs_impl(ctx, st));
    return copy_out(ctx, j_out, ctx->d_j, 2 * npts(ctx) * sizeof(double), on_device, st);
}

sc_status sc_free_energy(sc_ctx *ctx, double *F_total, double *density_out, int on_device, void *stream) {
    CKS(check_ctx(ctx));
    cudaStream_t st = (cudaStream_t)stream;
    CKS(ensure_outputs_impl(ctx, st));
    CKS(copy_out(ctx, density_out, ctx->d_F, npts(ctx) * sizeof(double), on_device, st));
    if (F_total) {
        double s[4];
        CK(cudaMemcpyAsync(s, ctx->d_sums, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (s[3] != 0.0) return set_err(ctx, SC_ENUMERIC, "non-finite values in the sweep outputs");
        *F_total = s[2] / (double)ctx->geo.n_in;
    }
    return SC_OK;
}

sc_status sc_update_vector_potential(sc_ctx *ctx, void *stream) {
    CKS(check_ctx(ctx));
    if (!ctx->d_G) return SC_OK;  // kappa <= 0: no induced field
    cudaStream_t st = (cudaStream_t)stream;
    CKS(ensure_outputs_impl(ctx, st));
    CK(scd::launch_mean_current(ctx->grid, ctx->d_mask, ctx->d_j, ctx->d_jsum, ctx->d_part, st));
    CK(sc_internal::induced_field(ctx, ctx->d_aind, st));
    ctx->have_aind = true;
    return SC_OK;
}

sc_status sc_picard_step(sc_ctx *ctx, void *stream) {
    CKS(check_ctx(ctx));
    cudaStream_t st = (cudaStream_t)stream;
    CKS(ensure_outputs_impl(ctx, st));
    if (ctx->d_G) CKS(sc_update_vector_potential(ctx, stream));
    CK(scd::launch_copy_delta(2 * (int64_t)npts(ctx) * ctx->geo.n_comp, ctx->d_dnew, ctx->d_delta, st));
    ctx->have_sweep = false;
    ctx->have_outputs = false;
    return SC_OK;
}

}  // extern "C"

namespace {

// Buffers of one LDOS evaluation (retarded sweeps with their own boundary values).
struct LdosRun {
    Plan *pl = nullptr;
    double *d_en = nullptr;
    void *d_ex[2] = {nullptr, nullptr};
    void *d_img = nullptr;
    scd::GrainSweep *d_gs = nullptr;
    int last_parity = 0;
    bool last_first = true;
};

void ldos_release(sc_ctx *ctx, LdosRun &R, cudaStream_t st) {
    cudaStreamSynchronize(st);
    dfree(ctx, R.d_en);
    dfree(ctx, R.d_ex[0]);
    dfree(ctx, R.d_ex[1]);
    dfree(ctx, R.d_img);
    dfree(ctx, R.d_gs);
    R = LdosRun();
}

sc_status ldos_check(sc_ctx *ctx, const double *energies, int32_t n_e, double broadening) {
    if (!energies || n_e < 1) return set_err(ctx, SC_EINVAL, "energies are required");
    if (!(broadening > 0.0)) return set_err(ctx, SC_EINVAL, "broadening must be > 0");
    // gamma~ at eps comes from gamma at -eps parked by the same warp: one energy block
    if (n_e > 32 * 8) return set_err(ctx, SC_EINVAL, "the LDOS takes at most 256 energies per call");
    for (int k = 0; k < n_e; ++k)
        if (std::fabs(energies[k] + energies[n_e - 1 - k]) > 1e-12 * (1.0 + std::fabs(energies[k])))
            return set_err(ctx, SC_EINVAL, "energies must be symmetric about zero");
    return SC_OK;
}

// Allocate, rotate the fields and run n_burnin retarded sweeps (Delta, A frozen).
sc_status ldos_burnin(sc_ctx *ctx, const double *energies, int32_t n_e, double broadening, int32_t n_burnin,
                      LdosRun &R, cudaStream_t st) {
    CKS(make_plan(ctx, n_e, 0, &R.pl));
    const Plan *pl = R.pl;
    const size_t nL = ctx->geo.lines.size();
    const size_t cplx = 2 * ctx->real_bytes;
    CK(dalloc(ctx, &R.d_en, n_e * sizeof(double)));
    CK(dalloc(ctx, &R.d_ex[0], 2 * nL * n_e * cplx));
    CK(dalloc(ctx, &R.d_ex[1], 2 * nL * n_e * cplx));
    CK(dalloc(ctx, &R.d_gs, sizeof(scd::GrainSweep)));
    CK(dalloc(ctx, &R.d_img, (size_t)ctx->geo.n_slots * n_e * ctx->real_bytes));
    scd::GrainSweep gs{};
    gs.lines = ctx->d_lines;
    gs.groups = pl->d_groups;
    gs.image_in = ctx->d_img_in;
    gs.image_out = R.d_img;
    gs.exits[0] = R.d_ex[0];
    gs.exits[1] = R.d_ex[1];
    gs.energies = R.d_en;
    gs.t = ctx->geo.prm.t;
    gs.h = ctx->geo.prm.h;
    gs.broadening = broadening;
    gs.n_e = n_e;
    gs.lanes = pl->lanes;
    gs.lines_per_warp = pl->lines_per_warp;
    gs.ne_pad = pl->lanes * pl->ept;
    gs.max_ns = std::max(ctx->geo.max_ns, 1);
    gs.ept = pl->ept;
    gs.n_blocks = 1;
    gs.n_slots = ctx->geo.n_slots;
    gs.n_lines = (int32_t)nL;
    gs.n_groups = pl->n_groups;
    CK(cudaMemcpyAsync(R.d_en, energies, n_e * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(R.d_gs, &gs, sizeof(gs), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(R.d_img, 0, (size_t)ctx->geo.n_slots * n_e * ctx->real_bytes, st));
    CK(cudaStreamSynchronize(st));  // gs lives on this stack frame
    CKS(sc_internal::rotate_fields(ctx, st));
    const int nb = std::max(1, n_burnin);
    for (int it = 0; it < nb; ++it) {
        CKS(launch_plan_sweep(ctx, *pl, R.d_gs, true, it == 0, it & 1, st));
        R.last_parity = it & 1;
        R.last_first = it == 0;
    }
    return SC_OK;
}

}  // namespace

extern "C" {

sc_status sc_ldos(sc_ctx *ctx, const double *energies, int32_t n_e, double broadening, int32_t n_burnin,
                  double *ldos_out, int on_device, void *stream) {
    CKS(check_ctx(ctx));
    if (!ldos_out) return set_err(ctx, SC_EINVAL, "ldos_out is required");
    CKS(ldos_check(ctx, energies, n_e, broadening));
    cudaStream_t st = (cudaStream_t)stream;
    LdosRun R;
    double *d_out = nullptr;
    sc_status rc = ldos_burnin(ctx, energies, n_e, broadening, n_burnin, R, st);
    if (rc == SC_OK) {
        cudaError_t e = cudaSuccess;
        if (on_device) d_out = ldos_out;
        else e = dalloc(ctx, &d_out, (size_t)n_e * npts(ctx) * sizeof(double));
        if (e == cudaSuccess)
            e = scd::launch_ldos_back(ctx->fp64, ctx->d_pairs, ctx->geo.n_pairs, ctx->d_back, ctx->grid, ctx->d_mask,
                                      R.d_img, n_e, d_out, st);
        if (e == cudaSuccess && !on_device)
            e = cudaMemcpyAsync(ldos_out, d_out, (size_t)n_e * npts(ctx) * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = set_err(ctx, SC_ECUDA, std::string("ldos: ") + cudaGetErrorString(e));
    }
    ldos_release(ctx, R, st);
    if (d_out && d_out != ldos_out) dfree(ctx, d_out);
    return rc;
}

sc_status sc_ldos_adjoint(sc_ctx *ctx, const double *energies, int32_t n_e, double broadening, int32_t n_burnin,
                          const double *g_ldos, double *dL_ddelta, double *dL_daind, int on_device, void *stream) {
    CKS(check_ctx(ctx));
    if (!g_ldos || !dL_ddelta) return set_err(ctx, SC_EINVAL, "g_ldos and dL_ddelta are required");
    CKS(ldos_check(ctx, energies, n_e, broadening));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t np = npts(ctx);
    LdosRun R;
    double *d_gN = nullptr, *d_gd = nullptr, *d_ga = nullptr;
    void *d_w = nullptr, *d_g = nullptr, *d_scr = nullptr;
    sc_status rc = ldos_burnin(ctx, energies, n_e, broadening, n_burnin, R, st);
    do {
        if (rc != SC_OK) break;
        const Plan &pl = *R.pl;
        const size_t t4 = ctx->fp64 ? 32 : 16;
        const int occ = std::max(1, scd::adjoint_occupancy(ctx->fp64, pl.ept, 128, ctx->stepper));
        const int blocks = std::max(1, std::min(ctx->sm_count * occ, (pl.n_items + 3) / 4));
        const int64_t stride = 3 * pl.stride;
        cudaError_t e = cudaSuccess;
        const size_t nc = (size_t)ctx->geo.n_comp;
        if ((e = dalloc(ctx, &d_gd, 2 * np * nc * sizeof(double))) != cudaSuccess ||
            (e = dalloc(ctx, &d_ga, 2 * np * sizeof(double))) != cudaSuccess ||
            (e = dalloc(ctx, &d_w, (size_t)ctx->geo.n_slots * n_e * ctx->real_bytes)) != cudaSuccess ||
            (e = dalloc(ctx, &d_g, (size_t)ctx->geo.n_slots * t4)) != cudaSuccess ||
            (e = dalloc(ctx, &d_scr, (size_t)blocks * 4 * stride * 2 * ctx->real_bytes)) != cudaSuccess) {
            rc = set_err(ctx, SC_ENOMEM, std::string("ldos adjoint buffers: ") + cudaGetErrorString(e));
            break;
        }
        const double *gN = g_ldos;
        if (!on_device) {
            if ((e = dalloc(ctx, &d_gN, (size_t)n_e * np * sizeof(double))) != cudaSuccess ||
                (e = cudaMemcpyAsync(d_gN, g_ldos, (size_t)n_e * np * sizeof(double), cudaMemcpyHostToDevice, st)) !=
                    cudaSuccess) {
                rc = set_err(ctx, SC_ECUDA, cudaGetErrorString(e));
                break;
            }
            gN = d_gN;
        }
        if ((e = cudaMemsetAsync(d_gd, 0, 2 * np * nc * sizeof(double), st)) != cudaSuccess ||
            (e = cudaMemsetAsync(d_ga, 0, 2 * np * sizeof(double), st)) != cudaSuccess ||
            (e = cudaMemsetAsync(d_w, 0, (size_t)ctx->geo.n_slots * n_e * ctx->real_bytes, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(d_g, 0, (size_t)ctx->geo.n_slots * t4, st)) != cudaSuccess ||
            (e = scd::launch_adjoint_ldos_back(ctx->fp64, ctx->d_pairs, ctx->geo.n_pairs, ctx->d_back, ctx->grid,
                                               ctx->d_mask, gN, n_e, d_w, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(ctx->d_counter, 0, sizeof(int32_t), st)) != cudaSuccess) {
            rc = set_err(ctx, SC_ECUDA, cudaGetErrorString(e));
            break;
        }
        scd::AdjointLaunch a{};
        a.grain = R.d_gs;
        a.items = pl.d_items;
        a.n_items = pl.n_items;
        a.counter = ctx->d_counter;
        a.scratch = d_scr;
        a.scratch_stride = stride;
        a.scratch_elems = (int64_t)blocks * 4 * stride;
        a.wimg = d_w;
        a.gimg = d_g;
        a.first_sweep = R.last_first ? 1 : 0;
        a.parity = R.last_parity;
        a.energies_per_lane = pl.ept;
        a.retarded = 1;
        a.stepper = ctx->stepper;
        a.grid_blocks = blocks;
        a.block_threads = 128;
        if ((e = scd::launch_adjoint_sweep(ctx->fp64, a, st)) != cudaSuccess ||
            (e = scd::launch_adjoint_rotate(ctx->fp64, ctx->d_geo, ctx->d_slot_line, ctx->geo.n_slots, ctx->d_pairs,
                                            ctx->grid, ctx->d_ghost, d_g, d_gd, d_ga, st)) != cudaSuccess) {
            rc = set_err(ctx, SC_ECUDA, cudaGetErrorString(e));
            break;
        }
        rc = copy_out(ctx, dL_ddelta, d_gd, 2 * np * nc * sizeof(double), on_device, st);
        if (rc == SC_OK) rc = copy_out(ctx, dL_daind, d_ga, 2 * np * sizeof(double), on_device, st);
    } while (0);
    ldos_release(ctx, R, st);
    dfree(ctx, d_gN);
    dfree(ctx, d_gd);
    dfree(ctx, d_ga);
    dfree(ctx, d_w);
    dfree(ctx, d_g);
    dfree(ctx, d_scr);
    return rc;
}

// Layout of the adjoint sweep: the forward sweep's, unless its work items fill
// less than half of the warps the adjoint kernel keeps resident (a small grain);
// then twice the lanes per line (twice the items, fewer energies per lane) as
// long as at least 3/4 of the lane slots carry an energy.
static sc_status adjoint_plan(sc_ctx *ctx, Plan **out) {
    Plan *pl = ctx->main_plan;
    *out = pl;
    if (pl->ept > 8) {
        // the adjoint kernel keeps at most 8 energies per lane
        if (ctx->forced_lanes)
            return set_err(ctx, SC_EINVAL, "the adjoint takes at most 8 energies per lane: more lanes per line");
        CKS(make_plan(ctx, ctx->n_e, 0, &pl));
        *out = pl;
    }
    if (ctx->forced_lanes) return SC_OK;
    const int occ = std::max(1, scd::adjoint_occupancy(ctx->fp64, pl->ept, 128, ctx->stepper));
    const int64_t resident = (int64_t)ctx->sm_count * occ * 4;
    int lanes = pl->lanes, ept = pl->ept;
    int64_t items = pl->n_items;
    while (lanes < 32 && pl->n_blocks == 1 && 2 * items <= resident) {
        const int l2 = 2 * lanes, e2 = (ctx->n_e + l2 - 1) / l2;
        if (4 * ctx->n_e < 3 * l2 * e2) break;
        lanes = l2;
        ept = e2;
        items *= 2;
    }
    if (lanes == pl->lanes) return SC_OK;
    return make_plan_layout(ctx, ctx->n_e, lanes, ept, out);
}

sc_status sc_sweep_adjoint(sc_ctx *ctx, const double *g_delta_new, const double *g_j, const double *g_F,
                           double g_Ftotal, double *dL_ddelta, double *dL_daind, int on_device, void *stream) {
    CKS(check_ctx(ctx));
    if (!ctx->have_sweep) return set_err(ctx, SC_ESTATE, "the adjoint needs a sweep of the current fields");
    if (!dL_ddelta) return set_err(ctx, SC_EINVAL, "dL_ddelta is required");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t np = npts(ctx);
    const size_t nc = (size_t)ctx->geo.n_comp;
    const size_t t4 = ctx->fp64 ? 32 : 16;
    Plan *apl = nullptr;
    CKS(adjoint_plan(ctx, &apl));
    const Plan &pl = *apl;
    if (!ctx->d_gacc) {
        CK(dalloc(ctx, &ctx->d_gacc, (3 + 2 * nc) * np * sizeof(double)));
        CK(dalloc(ctx, &ctx->d_gdelta, 2 * np * nc * sizeof(double)));
        CK(dalloc(ctx, &ctx->d_gaind, 2 * np * sizeof(double)));
        CK(dalloc(ctx, &ctx->d_gin, (2 * nc + 3) * np * sizeof(double)));
        CK(dalloc(ctx, &ctx->d_wimg, ctx->geo.n_slots * t4));
        CK(dalloc(ctx, &ctx->d_gimg, ctx->geo.n_slots * t4));
    }
    const int occ = std::max(1, scd::adjoint_occupancy(ctx->fp64, pl.ept, 128, ctx->stepper));
    const int blocks = std::max(1, std::min(ctx->sm_count * occ, (pl.n_items + 3) / 4));
    // per line: two rows per sample (gamma then beta; beta cotangent), with
    // checkpoints one row per kept gamma, and the entry values of gamma and beta
    const int64_t max_ns = std::max(ctx->geo.max_ns, 1);
    const int64_t lrows = 2 * max_ns + (ctx->adj_ckpt > 0 ? (max_ns + ctx->adj_ckpt - 1) / ctx->adj_ckpt : 0) + 2;
    const int64_t stride = (int64_t)pl.lines_per_warp * lrows * pl.lanes * pl.ept;
    const size_t need = (size_t)blocks * 4 * (size_t)stride * 2 * ctx->real_bytes;
    if (need > ctx->adj_scratch_bytes) {
        dfree(ctx, ctx->d_adj_scratch);
        ctx->d_adj_scratch = nullptr;
        ctx->adj_scratch_bytes = 0;
        CK(dalloc(ctx, &ctx->d_adj_scratch, need));
        ctx->adj_scratch_bytes = need;
    }
    // output cotangents on the device
    const double *gdn = g_delta_new, *gj = g_j, *gF = g_F;
    if (!on_device) {
        if (g_delta_new) {
            CK(cudaMemcpyAsync(ctx->d_gin, g_delta_new, 2 * np * nc * sizeof(double), cudaMemcpyHostToDevice, st));
            gdn = ctx->d_gin;
        }
        if (g_j) {
            CK(cudaMemcpyAsync(ctx->d_gin + 2 * np * nc, g_j, 2 * np * sizeof(double), cudaMemcpyHostToDevice, st));
            gj = ctx->d_gin + 2 * np * nc;
        }
        if (g_F) {
            CK(cudaMemcpyAsync(ctx->d_gin + (2 * nc + 2) * np, g_F, np * sizeof(double), cudaMemcpyHostToDevice, st));
            gF = ctx->d_gin + (2 * nc + 2) * np;
        }
    }
    CK(cudaMemsetAsync(ctx->d_gdelta, 0, 2 * np * nc * sizeof(double), st));
    CK(cudaMemsetAsync(ctx->d_gaind, 0, 2 * np * sizeof(double), st));
    CK(cudaMemsetAsync(ctx->d_wimg, 0, ctx->geo.n_slots * t4, st));
    CK(cudaMemsetAsync(ctx->d_gimg, 0, ctx->geo.n_slots * t4, st));
    const double kappa = ctx->geo.prm.kappa;
    const bool magn = kappa > 0.0 && std::isfinite(kappa) && ctx->have_aind;
    CK(scd::launch_adjoint_outputs(ctx->grid, ctx->d_mask, ctx->d_delta, magn ? ctx->d_aind : nullptr,
                                   ctx->geo.prm.t, ctx->norms, magn ? kappa : 0.0, (double)ctx->geo.n_in, gdn, gj, gF,
                                   g_Ftotal, ctx->d_gacc, ctx->d_gdelta, ctx->d_gaind, st));
    CK(scd::launch_adjoint_rotate_back(ctx->fp64, ctx->d_pairs, ctx->geo.n_pairs, ctx->d_back, ctx->grid, ctx->d_mask,
                                       ctx->d_gacc, ctx->d_wimg, st));
    CK(cudaMemsetAsync(ctx->d_counter, 0, sizeof(int32_t), st));
    scd::AdjointLaunch a{};
    a.grain = pl.d_grain;
    a.items = pl.d_items;
    a.n_items = pl.n_items;
    a.counter = ctx->d_counter;
    a.scratch = ctx->d_adj_scratch;
    a.scratch_stride = stride;
    a.ckpt = ctx->adj_ckpt;
    a.scratch_elems = (int64_t)(ctx->adj_scratch_bytes / (2 * ctx->real_bytes));
    a.wimg = ctx->d_wimg;
    a.gimg = ctx->d_gimg;
    a.first_sweep = ctx->last_first ? 1 : 0;
    a.parity = ctx->cur ^ 1;  // the buffer the last sweep read its entry values from
    a.energies_per_lane = pl.ept;
    a.retarded = 0;
    a.stepper = ctx->stepper;
    a.blocked = pl.n_blocks > 1 ? 1 : 0;
    a.grid_blocks = blocks;
    a.block_threads = 128;
    if (ctx->timing) CK(cudaEventRecord(ctx->ev_adj[0], st));
    CK(scd::launch_adjoint_sweep(ctx->fp64, a, st));
    if (ctx->timing) {
        CK(cudaEventRecord(ctx->ev_adj[1], st));
        ctx->adj_timed = true;
    }
    CK(scd::launch_adjoint_rotate(ctx->fp64, ctx->d_geo, ctx->d_slot_line, ctx->geo.n_slots, ctx->d_pairs, ctx->grid,
                                  ctx->d_ghost, ctx->d_gimg, ctx->d_gdelta, ctx->d_gaind, st));
    CKS(copy_out(ctx, dL_ddelta, ctx->d_gdelta, 2 * np * nc * sizeof(double), on_device, st));
    CKS(copy_out(ctx, dL_daind, ctx->d_gaind, 2 * np * sizeof(double), on_device, st));
    return SC_OK;
}

// ---- inspection ----------------------------------------------------------
sc_status sc_debug_lines(const sc_ctx *ctx, int32_t *l_lo, int32_t *l_hi, double *smin, double *smax, int32_t *m0,
                         int32_t *m1) {
    if (!ctx) return SC_EINVAL;
    const scg::Geometry &G = ctx->geo;
    for (int q = 0; q < G.n_pairs; ++q) {
        if (l_lo) l_lo[q] = G.pairs[q].l_lo;
        if (l_hi) l_hi[q] = G.pairs[q].l_hi;
    }
    for (size_t L = 0; L < G.lines.size(); ++L) {
        if (smin) smin[L] = G.lines[L].smin;
        if (smax) smax[L] = G.lines[L].smax;
        if (m0) m0[L] = G.lines[L].m0;
        if (m1) m1[L] = G.lines[L].m1;
    }
    return SC_OK;
}

sc_status sc_debug_ghost(const sc_ctx *ctx, int32_t *ghost) {
    if (!ctx || !ghost) return SC_EINVAL;
    std::memcpy(ghost, ctx->geo.ghost.data(), ctx->geo.ghost.size() * sizeof(int32_t));
    return SC_OK;
}

sc_status sc_debug_links(const sc_ctx *ctx, int32_t *ta, int32_t *tl, int32_t *tc, double *tw) {
    if (!ctx) return SC_EINVAL;
    const scg::Geometry &G = ctx->geo;
    size_t o = 0;
    for (int k = 0; k < G.n_angles; ++k) {
        const scg::PairInfo &pp = G.pairs[k % G.n_pairs];
        for (int L = pp.line0; L < pp.line0 + pp.n_lines; ++L) {
            const scg::LineInfo &li = G.lines[L];
            for (int q = 0; q < 4; ++q, ++o) {
                const bool f = k < G.n_pairs;
                if (ta) ta[o] = f ? li.dbg_fwd_angle[q] : li.dbg_bwd_angle[q];
                if (tl) tl[o] = f ? li.dbg_fwd_line[q] : li.dbg_bwd_line[q];
                if (tc) tc[o] = f ? li.dbg_fwd_chord[q] : li.dbg_bwd_chord[q];
                if (tw) tw[o] = f ? li.fwd[q].w : li.bwd[q].w;
            }
        }
    }
    return SC_OK;
}

sc_status sc_debug_fp64_math(const double *x, int64_t n, double *rcp, double *rsqrt, void *stream) {
    g_create_error.clear();
    if (n < 0 || (n > 0 && (!x || !rcp || !rsqrt))) {
        g_create_error = "sc_debug_fp64_math: n < 0 or a null pointer";
        return SC_EINVAL;
    }
    cudaError_t e = scd::launch_fp64_math(x, n, rcp, rsqrt, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) {
        g_create_error = cudaGetErrorString(e);
        return SC_ECUDA;
    }
    return SC_OK;
}

sc_status sc_debug_fma_rate(int32_t packed, double *lane_ops_per_s, void *stream) {
    g_create_error.clear();
    if (!lane_ops_per_s) return SC_EINVAL;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = scd::measure_fma_rate(packed != 0, sms, lane_ops_per_s, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        g_create_error = cudaGetErrorString(e);
        return SC_ECUDA;
    }
    return SC_OK;
}

sc_status sc_debug_chords(const sc_ctx *ctx, int32_t *pair, int32_t *l) {
    if (!ctx) return SC_EINVAL;
    const scg::Geometry &G = ctx->geo;
    for (size_t L = 0; L < G.lines.size(); ++L) {
        if (pair) pair[L] = G.lines[L].pair;
        if (l) l[L] = G.lines[L].l;
    }
    return SC_OK;
}

sc_status sc_debug_exits(sc_ctx *ctx, double *exits) {
    CKS(check_ctx(ctx));
    if (!exits) return SC_EINVAL;
    const size_t nL = ctx->geo.lines.size();
    const size_t n = 2 * nL * ctx->n_e;  // complex values, [angle half][line][energy]
    std::vector<char> buf(n * 2 * ctx->real_bytes);
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(buf.data(), ctx->d_exit[ctx->cur], buf.size(), cudaMemcpyDeviceToHost));
    // slots: [0, nL) = angle p (pair-major lines) ; [nL, 2nL) = angle p + P
    const scg::Geometry &G = ctx->geo;
    size_t o = 0;
    for (int k = 0; k < G.n_angles; ++k) {
        const scg::PairInfo &pp = G.pairs[k % G.n_pairs];
        for (size_t L = pp.line0; L < (size_t)(pp.line0 + pp.n_lines); ++L) {
            const size_t slot = k < G.n_pairs ? L : nL + L;
            for (int n2 = 0; n2 < ctx->n_e; ++n2, ++o) {
                const size_t i = slot * ctx->n_e + n2;
                if (ctx->fp64) {
                    exits[2 * o] = ((double *)buf.data())[2 * i];
                    exits[2 * o + 1] = ((double *)buf.data())[2 * i + 1];
                } else {
                    exits[2 * o] = ((float *)buf.data())[2 * i];
                    exits[2 * o + 1] = ((float *)buf.data())[2 * i + 1];
                }
            }
        }
    }
    return SC_OK;
}

sc_status sc_debug_images(sc_ctx *ctx, double *images) {
    CKS(check_ctx(ctx));
    if (!images) return SC_EINVAL;
    const scg::Geometry &G = ctx->geo;
    std::vector<char> buf(G.n_slots * (ctx->fp64 ? 32 : 16));
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(buf.data(), ctx->d_img_out, buf.size(), cudaMemcpyDeviceToHost));
    size_t o = 0;
    for (const auto &li : G.lines) {
        for (int q = 0; q < li.ns; ++q, ++o)
            for (int c = 0; c < 4; ++c) {
                const size_t i = 4 * (size_t)(li.slot0 + q) + c;
                images[4 * o + c] = ctx->fp64 ? ((double *)buf.data())[i] : ((float *)buf.data())[i];
            }
    }
    return SC_OK;
}

}  // extern "C"

namespace {

// every index of the host tables against the size of its table (see
// sc_debug_validate_tables)
int64_t count_bad_indices(const scg::Geometry &G) {
    int64_t bad = 0;
    const int64_t nL = (int64_t)G.lines.size(), rows = 2 * nL;
    auto in = [](int64_t i, int64_t n) { return i >= 0 && i < n; };
    for (const scg::LineInfo &li : G.lines) {
        const int64_t nsl = li.ns > 0 ? li.ns : 1;
        if (!in(li.slot0, G.n_slots) || !in(li.slot0 + nsl - 1, G.n_slots)) ++bad;
        if (!in(li.pair, G.n_pairs)) ++bad;
        for (int q = 0; q < 4; ++q) {
            if (!in(li.fwd[q].slot, rows)) ++bad;
            if (!in(li.bwd[q].slot, rows)) ++bad;
        }
    }
    for (const scg::PairInfo &pp : G.pairs) {
        if (pp.n_lines < 0 || !in(pp.line0, nL + 1) || pp.line0 + pp.n_lines > nL) ++bad;
        const int64_t nlat = (int64_t)pp.l_hi - pp.l_lo + 1;
        if (nlat < 1 || !in(pp.lat0, (int64_t)G.lats.size()) || pp.lat0 + nlat > (int64_t)G.lats.size()) ++bad;
    }
    for (const scg::LatticeLine &lt : G.lats)
        if (lt.nc < 0 || (lt.nc > 0 && (!in(lt.c0, nL) || lt.c0 + lt.nc > nL))) ++bad;
    return bad;
}

}  // namespace

extern "C" {

sc_status sc_debug_validate_tables(const sc_ctx *ctx, int64_t *n_bad) {
    if (!ctx || !n_bad) return SC_EINVAL;
    *n_bad = count_bad_indices(ctx->geo);
    return SC_OK;
}

sc_status sc_debug_corrupt_table(sc_ctx *ctx, int32_t which) {
    if (!ctx) return SC_EINVAL;
    if (!ctx->host_only) return set_err(ctx, SC_ESTATE, "only host_only contexts can be corrupted");
    scg::Geometry &G = ctx->geo;
    if (G.lines.empty() || G.pairs.empty()) return set_err(ctx, SC_ESTATE, "no tables");
    switch (which) {
        case 0: G.lines.back().slot0 = (int32_t)G.n_slots; break;
        case 1: G.lines[0].fwd[2].slot = (int32_t)(2 * G.lines.size()); break;
        case 2: G.pairs.back().lat0 = (int32_t)G.lats.size(); break;
        default: return set_err(ctx, SC_EINVAL, "which must be 0, 1 or 2");
    }
    return SC_OK;
}

sc_status sc_debug_bounds(uint64_t *violations, int32_t *checked_build, int32_t reset) {
    g_create_error.clear();
    if (!violations || !checked_build) return SC_EINVAL;
#ifdef SC_DEBUG_BOUNDS
    *checked_build = 1;
#else
    *checked_build = 0;
#endif
    cudaError_t (*const units[])(unsigned long long *, bool) = {
        scd::bounds_sweep_f32, scd::bounds_sweep_side_f32, scd::bounds_sweep_f64, scd::bounds_adjoint_f32, scd::bounds_adjoint_f64,
        scd::bounds_adjoint_transposes, scd::bounds_lattice_f32, scd::bounds_kernels};
    unsigned long long total = 0;
    cudaError_t e = cudaDeviceSynchronize();
    for (auto f : units) {
        unsigned long long v = 0;
        if (e == cudaSuccess) e = f(&v, reset != 0);
        total += v;
    }
    if (e != cudaSuccess) {
        g_create_error = std::string("reading the index-check counters: ") + cudaGetErrorString(e);
        return SC_ECUDA;
    }
    *violations = total;
    return SC_OK;
}

}  // extern "C"
