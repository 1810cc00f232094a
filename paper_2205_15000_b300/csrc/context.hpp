// Private definitions shared by the C-ABI implementation files (api.cpp, batch.cpp).
#pragma once
#include <cuda_runtime.h>

#include <deque>
#include <map>
#include <string>
#include <vector>

#include "geometry.hpp"
#include "kernels.cuh"
#include "vecpot.cuh"
#include "sc.h"

// How the sweep kernel maps (line, energy) work to lanes for one energy count.
struct Plan {
    int lanes = 0, ept = 0, lines_per_warp = 0;
    int32_t *d_groups = nullptr;         // [n_groups][lines_per_warp] line indices, -1 padded
    int32_t n_groups = 0;
    std::vector<int> group_cost;         // steps of the longest line of each group
    int n_blocks = 1;                    // energy blocks of lanes x ept energies
    int32_t n_items = 0;                 // n_groups x n_blocks work items
    int2 *d_items = nullptr;             // (0, group x n_blocks + block), longest first: single-context launches
    scd::GrainSweep *d_grain = nullptr;  // descriptor of the context's Matsubara sweep
    void *d_img_blocks = nullptr;        // n_blocks > 1: one image per energy block (n_blocks x n_slots)
    int grid_blocks = 0;
    int64_t stride = 0;                  // scratch elements (complex) per warp
};

struct sc_ctx {
    scg::Geometry geo;
    int device = 0;
    bool fp64 = false;
    int n_e = 0;
    int forced_lanes = 0;
    int stepper = 0;  // sc_stepper
    int adj_ckpt = 0;  // adjoint: forward gamma kept every adj_ckpt samples (0: every sample)
    int energy_sum = 0;  // sc_energy_sum
    std::vector<double> eps, ewt;  // energies and weights of the energy sums (host)
    double *d_eps = nullptr, *d_ewt = nullptr;  // on the device for Ozaki sums, else nullptr
    double normD = 0.0;
    scd::CompNorm norms{};  // per order-parameter component: normD - ln(T_c^c / T_c)
    size_t real_bytes = 4;
    scd::GridDev grid{};
    // geometry on the device
    uint8_t *d_mask = nullptr;
    int32_t *d_ghost = nullptr;
    scd::LineGeo *d_geo = nullptr;
    int32_t *d_slot_line = nullptr;
    scd::PairDev *d_pairs = nullptr;
    scd::BackLine *d_back = nullptr;
    scd::LineDev *d_lines = nullptr;
    std::map<int, Plan> plans;  // key: lanes * 16 + ept
    Plan *main_plan = nullptr;
    // fields and results
    double *d_delta = nullptr, *d_aind = nullptr, *d_acc = nullptr, *d_dnew = nullptr, *d_j = nullptr,
           *d_F = nullptr, *d_sums = nullptr, *d_jsum = nullptr, *d_G = nullptr, *d_diff = nullptr;
    double *d_part = nullptr;  // per-block partial sums of the grid reductions
    int G_width = 0;
    scd::VecpotFft vp{};        // FFT convolution buffers (grids up to 2048 points a side)
    bool vp_fft = false;
    bool have_aind = false;
    void *d_img_in = nullptr, *d_img_out = nullptr;
    void *d_exit[2] = {nullptr, nullptr};
    int cur = 0;  // d_exit[cur] holds the latest exit values
    bool have_boundary = false;
    bool have_sweep = false;
    bool have_outputs = false;
    void *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    int32_t *d_counter = nullptr;
    int sm_count = 0;
    // FP32 production path tables and buffers
    scd::LineF32 *d_line_f32 = nullptr;
    scd::PairF32 *d_pair_f32 = nullptr;
    // FP32 fields on the ghost-padded grid ((nx+2) x (ny+2)): (Re, Im Delta_0, A_ind)
    // and Delta of components c >= 1
    float4 *d_pad0 = nullptr;
    float2 *d_padc = nullptr;
    // kernel timings
    bool timing = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_adj[2] = {nullptr, nullptr};
    bool timed = false;
    bool adj_timed = false;
    bool failed = false;
    bool host_only = false;
    bool batch_member = false;  // swept only through its batch
    // residual history (sc_get_history): sweeps run so far, and per residual that
    // sc_gap_update computed, the sweep count then and eps_G (the newest kHistory)
    int64_t sweeps = 0;
    static constexpr size_t kHistory = 65536;
    std::deque<std::pair<int64_t, double>> history;
    // failure injection for tests: the fail_alloc_at-th device allocation of this
    // context reports cudaErrorMemoryAllocation without touching the device (-1 = off)
    long fail_alloc_at = -1;
    long alloc_count = 0;
    bool last_first = false;    // the last sweep started from homogeneous values
    // adjoint buffers (allocated on first use)
    double *d_gacc = nullptr, *d_gdelta = nullptr, *d_gaind = nullptr, *d_gin = nullptr;
    void *d_wimg = nullptr, *d_gimg = nullptr, *d_adj_scratch = nullptr;
    size_t adj_scratch_bytes = 0;
    // self-consistency accelerator (App. E), buffers allocated on first use
    double *d_anew = nullptr, *d_acc_v = nullptr, *d_acc_prev = nullptr, *d_acc_m = nullptr;
    double *d_acc_part = nullptr, *d_acc_sums = nullptr;
    int acc_kind = -1;  // kind of the running history; -1: none (next call starts one)
    long acc_iter = 0;
    double acc_alpha = 0.0, acc_alpha_c[10] = {}, acc_w_c[10] = {};  // per x component (Re, Im of each Delta_c, A)
    std::string err;
    std::vector<void *> allocs;
};

namespace sc_internal {
cudaError_t induced_field(sc_ctx *ctx, double *aind, cudaStream_t st);
sc_status set_err(sc_ctx *c, sc_status st, const std::string &msg);
cudaError_t dalloc_bytes(sc_ctx *ctx, void **p, size_t bytes);
void dfree(sc_ctx *ctx, void *p);
// lanes/EPT plan for n_e energies (forced_ept = 0: choose); builds the line groups
sc_status make_plan(sc_ctx *ctx, int n_e, int forced_ept, Plan **out, bool wide = false);
// plan for an explicit layout: lanes in {4, 8, 16, 32}, lanes * ept >= n_e
sc_status make_plan_layout(sc_ctx *ctx, int n_e, int lanes, int ept, Plan **out);
// fields of the context onto its lattices (rotate kernels)
sc_status rotate_fields(sc_ctx *ctx, cudaStream_t st);
// FS average of the context's image into its accumulators (rotate-back kernels)
sc_status rotate_back(sc_ctx *ctx, cudaStream_t st);
sc_status check_ctx(sc_ctx *ctx);
// Delta_new, j, F of the last sweep on the device (outputs kernel, once per sweep)
sc_status ensure_outputs(sc_ctx *ctx, cudaStream_t st);
void set_thread_error(const char *msg);
}  // namespace sc_internal
