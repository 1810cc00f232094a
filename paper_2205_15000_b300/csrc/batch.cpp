// Batched sweep: many grains of uneven size, shape, pairing, temperature,
// field and angle count swept by persistent launches over one work list of
// (grain, line group) items, longest first.  Each grain has its own energy
// layout (lanes per line, energies per lane); the energies per lane are the
// kernel's template parameter, so the items form one class per distinct
// count, and the classes run as back-to-back uniform launches on one stream.
// The bound on energies per lane is chosen by timing (sc_batch_autotune).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "context.hpp"

struct sc_batch {
    std::vector<sc_ctx *> members;
    std::vector<int> member_blocks;  // energy blocks of each member's layout
    std::vector<Plan *> member_plan; // each member's layout (owned by the member context)
    std::vector<int> member_parts;   // 2: the member's energies in two parts of their own layouts
    std::vector<void *> part_img;    // per member: the two parts' images (2 n_slots float4), lazily
    bool split = false;              // FP32: members may take two energy parts (autotuned)
    float split_ms[2] = {0.f, 0.f};  // the autotune's sweep times with and without parts
    int blocked = 0;                 // some member splits its energies into blocks
    int device = 0;
    bool fp64 = false;
    int ept = 0;  // bound on energies per lane
    int min_lanes = 2;  // fewest energy lanes per line a member may take (at most 32 / min_lanes lines per warp)
    int stepper = 0;  // sc_stepper, shared by all members
    bool weighted = false;  // Ozaki energy sums, shared by all members
    int sm_count = 0;
    scd::GrainSweep *d_grains = nullptr;
    int32_t n_gs = 0;  // sweep descriptors: one per member, two for a member in two energy parts
    int2 *d_items = nullptr;
    int32_t n_items = 0;
    int64_t stride = 0;
    // one uniform launch per energies-per-lane class: items [first, first + n)
    struct Class {
        int ept, first, n, grid_blocks;
        int occ, bps;  // occupancy (blocks per SM) and the blocks per SM the grid is sized for
        int64_t side_first, side_n;  // its lattice-transfer items: d_side[side_first, + side_n)
        int blocked;                 // it holds a member whose energies are split into blocks
    };
    std::vector<Class> classes;
    void *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    static constexpr int kMaxClasses = 16;  // energies-per-lane classes (1..10 energies per lane)
    int32_t *d_counter = nullptr;  // one work counter per class
    // every member's small kernels in single launches: member tables and offsets
    // (prefix sums over the members, n + 1 each) of their thread blocks: 256
    // padded points, 16 lines, tiles of 8 x 4 grid points per component count 1..4, and
    // reduction blocks of 256 grid points
    scd::MemberDev *d_members = nullptr;
    int64_t *d_off = nullptr;  // [7][n + 1]: pad, slots, back (nc = 1..4), outputs
    int64_t tot_pad = 0, tot_slots = 0, tot_back[4] = {0, 0, 0, 0}, tot_out = 0;
    // arrays of all members' fields and outputs (sc_batch_set_fields / _get_outputs):
    // [0] prefix of n_comp nx ny (complex Delta values), [1] prefix of nx ny
    int64_t *d_pt = nullptr;
    int64_t tot_cplx = 0, tot_pts = 0;
    double *d_stage_in = nullptr, *d_stage_out = nullptr;  // host-pointer transfers (lazy)
    int parity = 0;
    bool have_boundary = false;
    int64_t steps_per_sweep = 0;
    int64_t lane_steps_per_sweep = 0;  // with padded energy slots, for the current layout
    // FP32: the members' rotations and rotate-backs as work items of the class
    // launches (sc_batch_set_fused_transfers; chosen by sc_batch_autotune)
    bool fuse = false;   // wanted
    bool fused = false;  // the current layout carries transfer items
    float fuse_ms[2] = {0.f, 0.f};  // the autotune's iteration times with and without
    int2 *d_side = nullptr;
    int64_t n_side = 0;
    // [2][n + 1] prefixes: blocks of 16 lines rotated before the first class launch,
    // tiles (one-component members) rotated back after the last
    int64_t *d_solo = nullptr;
    int64_t tot_solo_rot = 0, tot_solo_back = 0;
    cudaEvent_t iev[2] = {nullptr, nullptr};  // around a whole batch sweep (rotation to rotate-back)
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaEvent_t cev[kMaxClasses + 1] = {};  // around each class launch of the last sweep
    std::vector<int> bps_choice;  // autotuned blocks per SM of the class of each energies-per-lane
                                  // count (index; empty or 0: occupancy)
    bool timed = false;
    // captured iterations: graph[p] = one sweep starting from parity p (+ outputs)
    cudaStream_t gstream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_outputs = -1;
    int graph_ept = 0;
    cudaEvent_t sync_ev[2] = {nullptr, nullptr};
    // per-member kernels (rotate, rotate-back, outputs) are small: spread them over
    // auxiliary streams forked from and joined back to the sweep's stream
    static constexpr int kAux = 8;
    cudaStream_t aux[kAux] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kAux] = {};
    bool failed = false;
    std::string err;
};

namespace {

sc_status berr(sc_batch *b, sc_status st, const std::string &msg) {
    b->err = msg;
    if (st == SC_ECUDA || st == SC_ENOMEM) b->failed = true;
    sc_internal::set_thread_error(msg.c_str());
    return st;
}

#define BCK(expr)                                                                    \
    do {                                                                             \
        cudaError_t e_ = (expr);                                                     \
        if (e_ != cudaSuccess)                                                       \
            return berr(b, e_ == cudaErrorMemoryAllocation ? SC_ENOMEM : SC_ECUDA,   \
                        std::string(#expr) + ": " + cudaGetErrorString(e_));         \
    } while (0)

void free_graphs(sc_batch *b) {
    for (auto &g : b->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    b->graph_outputs = -1;
}

void free_plan_buffers(sc_batch *b) {
    cudaFree(b->d_grains);
    cudaFree(b->d_items);
    cudaFree(b->d_side);
    cudaFree(b->d_solo);
    b->d_grains = nullptr;
    b->d_items = nullptr;
    b->d_side = nullptr;
    b->d_solo = nullptr;
    b->n_side = 0;
}

// Energy layout of one member with at most `ept_max` energies per lane: the
// fewest padded lane slots (lanes x energies per lane >= n_e), then the most
// energies per lane (fewer lanes: fewer shuffle rounds, more lines per warp).
void member_layout(int n_e, int ept_max, int min_lanes, int &lanes, int &ept) {
    int best = 1 << 30;
    // among equal padding the fewer lanes (fewer issue units per line, fewer
    // shuffle rounds) come first
    for (int l : {2, 4, 8, 16, 32}) {
        if (l < min_lanes) continue;
        const int e = (n_e + l - 1) / l;
        if (e < 1 || e > ept_max) continue;
        if (l * e < best) {
            best = l * e;
            lanes = l;
            ept = e;
        }
    }
    if (best < (1 << 30)) return;
    // more energies than one layout holds: energy blocks, each counted with 32
    // slots of per-block overhead
    for (int l : {32, 16, 8, 4})
        for (int e = std::min(ept_max, 8); e >= 1 && l >= min_lanes; --e) {
            const int nb = (n_e + l * e - 1) / (l * e);
            const int cost = nb * (l * e + 32);
            if (cost < best) {
                best = cost;
                lanes = l;
                ept = e;
            }
        }
}

// Relative cost of a lane layout per line and sample: its lane slots over the
// fraction of the FP32 peak a lane-step reaches with that many energies per lane
// (measured per class on the 64-grain batch: 0.58-0.61 from 5 energies per lane
// up, 0.53 at 4, 0.45 at 3; 1 and 2 estimated).
double layout_cost(int lanes, int ept) {
    static const double rate[5] = {1.0, 0.25, 0.35, 0.45, 0.53};
    return (double)lanes * ept / (ept < 5 ? rate[ept] : 0.6);
}

struct Part {
    int first, n, lanes, ept;
};

// The member's energies as one layout, or (FP32) as two parts [0, n1) and
// [n1, n_e), each in its own layout with at least 5 energies per lane, where
// that costs at least 5 % less than the padded single layout (e.g. 132
// energies: 2 x 10 and 16 x 7 lanes x energies instead of 16 x 9).
std::vector<Part> member_parts(int n_e, int ept_max, int min_lanes, bool split) {
    int lanes = 32, ept = ept_max;
    member_layout(n_e, ept_max, min_lanes, lanes, ept);
    std::vector<Part> one{{0, n_e, lanes, ept}};
    if (!split || lanes * ept <= n_e || n_e > 32 * ept_max) return one;  // no padding, or blocks
    double best = 0.95 * layout_cost(lanes, ept);
    std::vector<Part> res = one;
    for (int n1 = 1; n1 < n_e; ++n1) {
        int l1 = 32, e1 = ept_max, l2 = 32, e2 = ept_max;
        member_layout(n1, ept_max, min_lanes, l1, e1);
        member_layout(n_e - n1, ept_max, min_lanes, l2, e2);
        if (e1 < 5 || e2 < 5) continue;  // a part repeats the per-sample work of every line
        const double c = layout_cost(l1, e1) + layout_cost(l2, e2);
        if (c < best) {
            best = c;
            res = {{0, n1, l1, e1}, {n1, n_e - n1, l2, e2}};
        }
    }
    return res;
}

// Cost of the lattice transfers in sweep lane-steps (one energy slot of one lane
// over one segment), from the B300 rates of the transfer kernels and of the
// FP32 sweep on the 256^2 grain with 128 angles: about 3.4e11 lane-steps, 6.6e10
// rotated slots and 1.1e11 rotated-back (grid point, pair) terms per second.
constexpr double kRotLaneSteps = 5.3;   // per image slot
constexpr double kBackLaneSteps = 3.3;  // per grid point and angle pair

// Where the members' lattice transfers run when the class launches carry them.
// A one-part member of class k is rotated during one of the launches before k
// and rotated back during one after k; each transfer goes, largest first, to
// the eligible launch whose transfer load relative to its own sweep work stays
// lowest, and runs in the separate launches (solo) when none is eligible or it
// would exceed that launch's sweep work.  The launch order puts the class with
// the least rotation work first and, of the others, the one with the least
// rotate-back work last.  Members in two energy parts, and the rotate-back of
// members with several order-parameter components, stay solo.
void plan_transfers(sc_batch *b, const std::vector<scd::GrainSweep> &gs, const std::vector<int> &member_gi,
                    std::vector<sc_batch::Class> &classes, std::vector<double> &class_cost, std::vector<int2> &side,
                    std::vector<int64_t> &solo) {
    const size_t n = b->members.size(), K = classes.size();
    std::vector<int> kc(n, -1);
    std::vector<double> rot(n, 0.0), back(n, 0.0), crot(K, 0.0), cback(K, 0.0);
    for (size_t g = 0; g < n; ++g) {
        const sc_ctx *c = b->members[g];
        rot[g] = kRotLaneSteps * (double)c->geo.n_slots;
        if (c->geo.n_comp == 1) back[g] = kBackLaneSteps * (double)c->geo.nx * c->geo.ny * c->geo.n_pairs;
        if (member_gi[g] < 0) continue;
        for (size_t k = 0; k < K; ++k)
            if (classes[k].ept == gs[member_gi[g]].ept) kc[g] = (int)k;
        if (kc[g] >= 0) {
            crot[kc[g]] += rot[g];
            cback[kc[g]] += back[g];
        }
    }
    // launch order: position -> class
    size_t f = 0;
    for (size_t k = 1; k < K; ++k)
        if (crot[k] < crot[f]) f = k;
    size_t l = f == 0 ? 1 : 0;
    for (size_t k = 0; k < K; ++k)
        if (k != f && cback[k] < cback[l]) l = k;
    std::vector<size_t> order{f};
    for (size_t k = 0; k < K; ++k)
        if (k != f && k != l) order.push_back(k);
    order.push_back(l);
    std::vector<int> pos_of(K);
    std::vector<sc_batch::Class> cl(K);
    std::vector<double> cc(K);
    for (size_t q = 0; q < K; ++q) {
        cl[q] = classes[order[q]];
        cc[q] = class_cost[order[q]];
        pos_of[order[q]] = (int)q;
    }
    classes = cl;
    class_cost = cc;
    for (size_t g = 0; g < n; ++g)
        if (kc[g] >= 0) kc[g] = pos_of[kc[g]];
    // transfers (member, kind 0 rotation / 1 rotate-back), largest first
    struct Job {
        double cost;
        int g, kind;
    };
    std::vector<Job> jobs;
    for (size_t g = 0; g < n; ++g) {
        if (kc[g] < 0) continue;
        if (kc[g] > 0) jobs.push_back({rot[g], (int)g, 0});
        if (kc[g] < (int)K - 1 && back[g] > 0.0) jobs.push_back({back[g], (int)g, 1});
    }
    std::stable_sort(jobs.begin(), jobs.end(), [](const Job &x, const Job &y) { return x.cost > y.cost; });
    std::vector<double> load(K, 0.0);
    std::vector<std::vector<Job>> at(K);
    std::vector<char> rot_fused(n, 0), back_fused(n, 0);
    for (const Job &j : jobs) {
        const int lo = j.kind == 0 ? 0 : kc[j.g] + 1, hi = j.kind == 0 ? kc[j.g] : (int)K;
        int best = -1;
        double best_r = 1.0;  // at most the launch's own sweep work
        for (int q = lo; q < hi; ++q) {
            const double r = (load[q] + j.cost) / std::max(class_cost[q], 1.0);
            if (r <= best_r) {
                best_r = r;
                best = q;
            }
        }
        if (best < 0) continue;
        load[best] += j.cost;
        at[best].push_back(j);
        (j.kind == 0 ? rot_fused : back_fused)[j.g] = 1;
    }
    side.clear();
    for (size_t q = 0; q < K; ++q) {
        classes[q].side_first = (int64_t)side.size();
        for (const Job &j : at[q]) {
            const sc_ctx *c = b->members[j.g];
            const int64_t cnt = j.kind == 0 ? ((int64_t)c->geo.lines.size() + 3) / 4 : scd::back_tiles(c->geo.nx, c->geo.ny);
            for (int64_t i = 0; i < cnt; ++i) side.push_back(make_int2(2 * j.g + j.kind, (int)i));
        }
        classes[q].side_n = (int64_t)side.size() - classes[q].side_first;
    }
    solo.assign(2 * (n + 1), 0);
    for (size_t g = 0; g < n; ++g) {
        const sc_ctx *c = b->members[g];
        solo[g + 1] = solo[g] + (rot_fused[g] ? 0 : ((int64_t)c->geo.lines.size() + 15) / 16);
        solo[n + 1 + g + 1] = solo[n + 1 + g] + (back_fused[g] || c->geo.n_comp != 1 ? 0 : scd::back_tiles(c->geo.nx, c->geo.ny));
    }
}

// Lay out the work list for at most `ept` energies per lane.
sc_status build(sc_batch *b, int ept) {
    free_graphs(b);  // captured graphs refer to the buffers rebuilt here
    std::vector<scd::GrainSweep> gs;
    b->member_blocks.assign(b->members.size(), 1);
    b->member_plan.assign(b->members.size(), nullptr);
    b->member_parts.assign(b->members.size(), 1);
    b->part_img.resize(b->members.size(), nullptr);
    struct It {
        int cost, grain, group;
    };
    std::vector<It> items;
    int64_t stride = 0;
    int64_t lane_steps = 0;
    std::vector<int> member_gi(b->members.size(), -1);  // sweep descriptor of a one-part member
    for (size_t g = 0; g < b->members.size(); ++g) {
        sc_ctx *c = b->members[g];
        const std::vector<Part> parts = member_parts(c->n_e, ept, b->min_lanes, b->split && !b->fp64);
        const bool two = parts.size() > 1;
        if (!two) member_gi[g] = (int)gs.size();
        b->member_parts[g] = (int)parts.size();
        if (two && !b->part_img[g]) {  // zeroed once: slots no sample writes stay zero
            BCK(cudaMalloc(&b->part_img[g], 2 * (size_t)c->geo.n_slots * sizeof(float4)));
            BCK(cudaMemset(b->part_img[g], 0, 2 * (size_t)c->geo.n_slots * sizeof(float4)));
        }
        for (size_t k = 0; k < parts.size(); ++k) {
            const int lanes = parts[k].lanes, eg = parts[k].ept;
            Plan *pl = nullptr;
            sc_status st = sc_internal::make_plan_layout(c, two ? parts[k].n : c->n_e, lanes, eg, &pl);
            if (st != SC_OK) return berr(b, st, c->err);
            gs.emplace_back();
            scd::GrainSweep &d = gs.back();
            const int gi = (int)gs.size() - 1;
            d.lines = c->d_lines;
            d.groups = pl->d_groups;
            d.image_in = c->d_img_in;
            // a blocked member writes one image per energy block (added after the sweep)
            d.image_out = pl->n_blocks > 1 ? pl->d_img_blocks : c->d_img_out;
            d.n_slots = c->geo.n_slots;
            d.n_lines = (int32_t)c->geo.lines.size();
            d.n_groups = pl->n_groups;
            d.exits[0] = c->d_exit[0];
            d.exits[1] = c->d_exit[1];
            d.energies = nullptr;
            d.mats_eps = c->d_eps;
            d.mats_w = c->d_ewt;
            d.t = c->geo.prm.t;
            d.h = c->geo.prm.h;
            d.broadening = 0.0;
            d.n_e = c->n_e;
            d.lanes = pl->lanes;
            d.lines_per_warp = pl->lines_per_warp;
            d.ne_pad = pl->lanes * pl->ept;
            d.max_ns = std::max(c->geo.max_ns, 1);
            d.ept = pl->ept;
            d.n_blocks = pl->n_blocks;
            d.e_first = parts[k].first;
            d.e_count = two ? parts[k].n : 0;
            if (two)  // each part sums into its own image; the two are added after the sweep
                d.image_out = (char *)b->part_img[g] + k * (size_t)c->geo.n_slots * sizeof(float4);
            b->member_blocks[g] = pl->n_blocks;
            b->member_plan[g] = pl;
            stride = std::max(stride, pl->stride);
            int64_t steps = 0;
            for (const auto &li : c->geo.lines) steps += 2 * (int64_t)(li.ns + 1);
            lane_steps += steps * pl->lanes * pl->ept * pl->n_blocks;
            // cost of a group ~ steps x energies handled per lane; one item per energy block
            for (int q = 0; q < pl->n_groups; ++q)
                for (int kb = 0; kb < pl->n_blocks; ++kb)
                    items.push_back({pl->group_cost[q] * pl->ept, gi, q * pl->n_blocks + kb});
        }
    }
    // classes by energies per lane (largest first), longest items first within each
    std::stable_sort(items.begin(), items.end(), [&](const It &x, const It &y) {
        const int ex = gs[x.grain].ept, ey = gs[y.grain].ept;
        return ex != ey ? ex > ey : x.cost > y.cost;
    });
    std::vector<int2> flat(items.size());
    for (size_t i = 0; i < items.size(); ++i) flat[i] = make_int2(items[i].grain, items[i].group);
    std::vector<sc_batch::Class> classes;
    std::vector<double> class_cost;  // lane-steps of each class's items
    for (size_t i = 0; i < items.size(); ++i) {
        const int e = gs[items[i].grain].ept;
        if (classes.empty() || classes.back().ept != e) {
            classes.push_back({e, (int)i, 0, 0, 0, 0, 0, 0, 0});
            class_cost.push_back(0.0);
        }
        ++classes.back().n;
        // the block-aware kernels (at most 8 energies per lane, as every blocked
        // member's layout) only where a member of the class is blocked
        if (gs[items[i].grain].n_blocks > 1) classes.back().blocked = 1;
        class_cost.back() += 64.0 * items[i].cost;  // both directions, 32 lanes
    }
    bool any_blocks = false;
    for (int nbk : b->member_blocks) any_blocks = any_blocks || nbk > 1;
    std::vector<int2> side;
    std::vector<int64_t> solo;
    if (b->fuse && !b->fp64 && !any_blocks && classes.size() >= 2)
        plan_transfers(b, gs, member_gi, classes, class_cost, side, solo);
    const bool fused = !side.empty();
    int max_blocks = 1;
    for (size_t k = 0; k < classes.size(); ++k) {
        auto &c = classes[k];
        if (!fused) c.side_first = c.side_n = 0;
        int occ = c.side_n > 0 ? scd::sweep_side_occupancy_f32(c.ept, 128, b->stepper, b->weighted)
                               : scd::sweep_occupancy(b->fp64, c.ept, 128, b->stepper, b->weighted);
        if (occ < 1) occ = 1;
        c.occ = occ;
        const size_t e = (size_t)c.ept;
        c.bps = e < b->bps_choice.size() && b->bps_choice[e] > 0 ? std::min(b->bps_choice[e], occ) : occ;
        c.grid_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)b->sm_count * c.bps, (c.n + c.side_n + 3) / 4));
        max_blocks = std::max(max_blocks, c.grid_blocks);
    }
    free_plan_buffers(b);
    b->fused = fused;
    if (fused) {
        BCK(cudaMalloc(&b->d_side, side.size() * sizeof(int2)));
        BCK(cudaMemcpy(b->d_side, side.data(), side.size() * sizeof(int2), cudaMemcpyHostToDevice));
        BCK(cudaMalloc(&b->d_solo, solo.size() * sizeof(int64_t)));
        BCK(cudaMemcpy(b->d_solo, solo.data(), solo.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
        b->n_side = (int64_t)side.size();
        const size_t n = b->members.size();
        b->tot_solo_rot = solo[n];
        b->tot_solo_back = solo[2 * n + 1];
    }
    BCK(cudaMalloc(&b->d_grains, gs.size() * sizeof(scd::GrainSweep)));
    BCK(cudaMemcpy(b->d_grains, gs.data(), gs.size() * sizeof(scd::GrainSweep), cudaMemcpyHostToDevice));
    BCK(cudaMalloc(&b->d_items, flat.size() * sizeof(int2)));
    BCK(cudaMemcpy(b->d_items, flat.data(), flat.size() * sizeof(int2), cudaMemcpyHostToDevice));
    b->n_items = (int32_t)flat.size();
    b->n_gs = (int32_t)gs.size();
    b->stride = stride;
    b->classes = classes;
    const size_t need = (size_t)max_blocks * 4 * (size_t)stride * 2 * (b->fp64 ? 8 : 4);
    if (need > b->scratch_bytes) {
        cudaFree(b->d_scratch);
        b->d_scratch = nullptr;
        b->scratch_bytes = 0;
        BCK(cudaMalloc(&b->d_scratch, need));
        b->scratch_bytes = need;
    }
    b->ept = ept;
    b->lane_steps_per_sweep = lane_steps;
    b->blocked = 0;
    for (int nbk : b->member_blocks) b->blocked |= nbk > 1 ? 1 : 0;
    return SC_OK;
}

sc_status fork(sc_batch *b, cudaStream_t st) {
    BCK(cudaEventRecord(b->fork_ev, st));
    for (int k = 0; k < sc_batch::kAux; ++k) BCK(cudaStreamWaitEvent(b->aux[k], b->fork_ev, 0));
    return SC_OK;
}

sc_status join(sc_batch *b, cudaStream_t st) {
    for (int k = 0; k < sc_batch::kAux; ++k) {
        BCK(cudaEventRecord(b->join_ev[k], b->aux[k]));
        BCK(cudaStreamWaitEvent(st, b->join_ev[k], 0));
    }
    return SC_OK;
}

// Member tables of the single-launch per-member kernels (static for the life
// of the batch: every pointer belongs to a member context).
sc_status build_member_tables(sc_batch *b) {
    const size_t n = b->members.size();
    std::vector<scd::MemberDev> md(n);
    std::vector<int64_t> off(7 * (n + 1), 0);
    for (size_t g = 0; g < n; ++g) {
        sc_ctx *c = b->members[g];
        scd::MemberDev &m = md[g];
        std::memset(&m, 0, sizeof m);
        m.grid = c->grid;
        m.ghost = c->d_ghost;
        m.mask = c->d_mask;
        m.delta = c->d_delta;
        m.aind = c->d_aind;  // zero while no induced potential is set
        m.pad0 = c->d_pad0;
        m.padc = c->d_padc;
        m.lines = c->d_line_f32;
        m.slot_line = c->d_slot_line;
        m.pairs = c->d_pair_f32;
        m.n_pairs = c->geo.n_pairs;
        m.back = c->d_back;
        m.image_in = (float4 *)c->d_img_in;
        m.image_out = (const float4 *)c->d_img_out;
        m.acc = c->d_acc;
        m.t = c->geo.prm.t;
        const double kappa = c->geo.prm.kappa;
        m.kappa = kappa > 0.0 && std::isfinite(kappa) ? kappa : 0.0;
        m.norms = c->norms;
        m.dnew = c->d_dnew;
        m.j = c->d_j;
        m.F = c->d_F;
        m.sums = c->d_sums;
        m.partials = c->d_part;
        const int64_t nx = c->geo.nx, ny = c->geo.ny;
        const int nc = c->geo.n_comp;
        m.n_slots = c->geo.n_slots;
        m.n_pad = (nx + 2) * (ny + 2);
        off[0 * (n + 1) + g + 1] = (m.n_pad + 255) / 256;     // blocks of 256 padded points
        off[1 * (n + 1) + g + 1] = ((int64_t)c->geo.lines.size() + 15) / 16;  // blocks of 16 lines
        for (int k = 1; k <= 4; ++k) off[(1 + k) * (n + 1) + g + 1] = nc == k ? scd::back_tiles(nx, ny) : 0;
        off[6 * (n + 1) + g + 1] = scd::reduce_blocks(nx * ny);
    }
    for (int a = 0; a < 7; ++a)
        for (size_t g = 0; g < n; ++g) off[a * (n + 1) + g + 1] += off[a * (n + 1) + g];
    b->tot_pad = off[0 * (n + 1) + n];
    b->tot_slots = off[1 * (n + 1) + n];
    for (int k = 0; k < 4; ++k) b->tot_back[k] = off[(2 + k) * (n + 1) + n];
    b->tot_out = off[6 * (n + 1) + n];
    BCK(cudaMalloc(&b->d_members, n * sizeof(scd::MemberDev)));
    BCK(cudaMemcpy(b->d_members, md.data(), n * sizeof(scd::MemberDev), cudaMemcpyHostToDevice));
    BCK(cudaMalloc(&b->d_off, off.size() * sizeof(int64_t)));
    BCK(cudaMemcpy(b->d_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    std::vector<int64_t> pt(2 * (n + 1), 0);
    for (size_t g = 0; g < n; ++g) {
        const int64_t np = (int64_t)b->members[g]->geo.nx * b->members[g]->geo.ny;
        pt[g + 1] = pt[g] + np * b->members[g]->geo.n_comp;
        pt[(n + 1) + g + 1] = pt[(n + 1) + g] + np;
    }
    b->tot_cplx = pt[n];
    b->tot_pts = pt[2 * n + 1];
    BCK(cudaMalloc(&b->d_pt, pt.size() * sizeof(int64_t)));
    BCK(cudaMemcpy(b->d_pt, pt.data(), pt.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    return SC_OK;
}

const int64_t *member_off(const sc_batch *b, int a) { return b->d_off + (size_t)a * (b->members.size() + 1); }

}  // namespace

extern "C" {

sc_status sc_batch_destroy(sc_batch *b) {
    if (!b) return SC_EINVAL;
    cudaSetDevice(b->device);
    for (sc_ctx *c : b->members) sc_destroy(c);
    free_plan_buffers(b);
    cudaFree(b->d_scratch);
    cudaFree(b->d_counter);
    cudaFree(b->d_members);
    cudaFree(b->d_off);
    cudaFree(b->d_pt);
    cudaFree(b->d_stage_in);
    cudaFree(b->d_stage_out);
    for (void *q : b->part_img) cudaFree(q);
    for (cudaEvent_t e : b->ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : b->iev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : b->cev)
        if (e) cudaEventDestroy(e);
    free_graphs(b);
    for (cudaEvent_t e : b->sync_ev)
        if (e) cudaEventDestroy(e);
    if (b->gstream) cudaStreamDestroy(b->gstream);
    for (int k = 0; k < sc_batch::kAux; ++k) {
        if (b->aux[k]) cudaStreamDestroy(b->aux[k]);
        if (b->join_ev[k]) cudaEventDestroy(b->join_ev[k]);
    }
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    (void)cudaGetLastError();  // teardown errors are not the caller's
    delete b;
    return SC_OK;
}

sc_status sc_batch_create(const sc_params *params, int32_t n, int32_t energies_per_lane, sc_batch **out) {
    sc_internal::set_thread_error("");
    if (!params || !out || n < 1) {
        sc_internal::set_thread_error("need params, out and n >= 1");
        return SC_EINVAL;
    }
    const int ept_cap = params[0].precision == SC_PREC_FP64 ? 8 : 10;
    if (energies_per_lane < 0 || energies_per_lane > ept_cap) {
        sc_internal::set_thread_error(ept_cap == 8 ? "energies_per_lane must be 0 (automatic) or 1..8"
                                                   : "energies_per_lane must be 0 (automatic) or 1..10");
        return SC_EINVAL;
    }
    *out = nullptr;
    sc_batch *b = new (std::nothrow) sc_batch();
    if (!b) return SC_ENOMEM;
    int max_ne = 0;
    for (int g = 0; g < n; ++g) {
        if (params[g].precision != params[0].precision || params[g].stepper != params[0].stepper ||
            params[g].energy_sum != params[0].energy_sum) {
            sc_batch_destroy(b);
            sc_internal::set_thread_error("all members of a batch need the same precision, stepper and energy sum");
            return SC_EINVAL;
        }
        if (params[g].host_only) {
            sc_batch_destroy(b);
            sc_internal::set_thread_error("batch members cannot be host_only");
            return SC_EINVAL;
        }
        sc_ctx *c = nullptr;
        sc_status st = sc_create(&params[g], &c);
        if (st != SC_OK) {
            std::string why = std::string("member ") + std::to_string(g) + ": " + sc_last_error(nullptr);
            sc_batch_destroy(b);
            sc_internal::set_thread_error(why.c_str());
            return st;
        }
        c->batch_member = true;
        b->members.push_back(c);
        max_ne = std::max(max_ne, c->n_e);
        int64_t steps = 0;
        for (const auto &li : c->geo.lines) steps += 2 * (int64_t)(li.ns + 1);
        b->steps_per_sweep += steps * c->n_e;
    }
    b->fp64 = params[0].precision == SC_PREC_FP64;
    b->stepper = params[0].stepper;
    b->weighted = params[0].energy_sum == SC_SUM_OZAKI;
    b->device = b->members[0]->device;
    b->sm_count = b->members[0]->sm_count;
    sc_status st = SC_OK;
    cudaError_t e = cudaMalloc(&b->d_counter, sc_batch::kMaxClasses * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev[1]);
    if (e == cudaSuccess) e = cudaEventCreate(&b->iev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&b->iev[1]);
    for (int k = 0; k <= sc_batch::kMaxClasses && e == cudaSuccess; ++k) e = cudaEventCreate(&b->cev[k]);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
    for (int k = 0; k < sc_batch::kAux && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&b->aux[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join_ev[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) st = SC_ECUDA;
    int ept = energies_per_lane;
    if (!ept) ept = std::min(8, std::max(4, (max_ne + 31) / 32));
    if (st == SC_OK) st = build(b, ept);
    if (st == SC_OK) st = build_member_tables(b);
    if (st != SC_OK) {
        std::string why = b->err.empty() ? "device setup failed" : b->err;
        sc_batch_destroy(b);
        sc_internal::set_thread_error(why.c_str());
        return st;
    }
    *out = b;
    return SC_OK;
}

sc_status sc_batch_member(sc_batch *b, int32_t i, sc_ctx **out) {
    if (!b || !out || i < 0 || i >= (int32_t)b->members.size()) return SC_EINVAL;
    *out = b->members[i];
    return SC_OK;
}

sc_status sc_batch_sweep(sc_batch *b, void *stream) {
    if (!b) return SC_EINVAL;
    if (b->failed) return SC_ESTATE;
    BCK(cudaSetDevice(b->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int n = (int)b->members.size();
    for (sc_ctx *c : b->members)
        if (c->failed) return berr(b, SC_ESTATE, "a member context failed");
    sc_status fs = SC_OK;
    // while a graph is being captured the timing events become external event
    // nodes, so that every replay records them
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    BCK(cudaStreamIsCapturing(st, &cap));
    const unsigned ev_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
    BCK(cudaEventRecordWithFlags(b->iev[0], st, ev_flags));
    if (!b->fp64) {
        // every member's fields onto its lattices: two launches over all members (with
        // transfer items, the rotation only of the members no class launch rotates)
        BCK(scd::launch_batch_fields_rotate_f32(b->d_members, member_off(b, 0), b->tot_pad,
                                                b->fused ? b->d_solo : member_off(b, 1),
                                                b->fused ? b->tot_solo_rot : b->tot_slots, n, st));
    } else {
        fs = fork(b, st);
        if (fs != SC_OK) return fs;
        for (size_t g = 0; g < b->members.size(); ++g) {
            sc_ctx *c = b->members[g];
            sc_status s = sc_internal::rotate_fields(c, b->aux[g % sc_batch::kAux]);
            if (s != SC_OK) return berr(b, s, c->err);
        }
        fs = join(b, st);
        if (fs != SC_OK) return fs;
    }
    if (b->classes.size() > (size_t)sc_batch::kMaxClasses)
        return berr(b, SC_ESTATE, "more energies-per-lane classes than work counters");
    BCK(cudaMemsetAsync(b->d_counter, 0, sc_batch::kMaxClasses * sizeof(int32_t), st));
    BCK(cudaEventRecordWithFlags(b->ev[0], st, ev_flags));
    for (size_t k = 0; k < b->classes.size(); ++k) {
        const sc_batch::Class &c = b->classes[k];
        BCK(cudaEventRecordWithFlags(b->cev[k], st, ev_flags));
        scd::SweepLaunch a{};
        a.grains = b->d_grains;
        a.items = b->d_items + c.first;
        a.n_items = c.n;
        a.counter = b->d_counter + k;
        a.scratch = b->d_scratch;
        a.scratch_stride = b->stride;
        a.scratch_elems = (int64_t)(b->scratch_bytes / (2 * (b->fp64 ? 8 : 4)));
        a.n_grains = b->n_gs;
        a.energies_per_lane = c.ept;
        a.first_sweep = b->have_boundary ? 0 : 1;
        a.parity = b->parity;
        a.retarded = 0;
        a.grid_blocks = c.grid_blocks;
        a.block_threads = 128;
        a.stepper = b->stepper;
        a.weighted = b->weighted ? 1 : 0;
        a.blocked = c.blocked;
        if (c.side_n > 0) {  // with the lattice transfers of other members as work items
            a.side_members = b->d_members;
            a.side = b->d_side + c.side_first;
            a.n_side = (int32_t)c.side_n;
            a.n_side_members = n;
            BCK(scd::launch_sweep_side_f32(a, st));
        } else {
            BCK(scd::launch_sweep(b->fp64, a, st));
        }
    }
    BCK(cudaEventRecordWithFlags(b->cev[b->classes.size()], st, ev_flags));
    for (size_t g = 0; g < b->members.size(); ++g) {
        if (b->member_blocks[g] > 1)  // the energy blocks' images, added in block order
            BCK(scd::launch_block_sum(b->fp64, b->member_plan[g]->d_img_blocks, b->member_blocks[g],
                                      b->members[g]->geo.n_slots, b->members[g]->d_img_out, st));
        if (b->member_parts[g] > 1)  // the two energy parts' images, first part first
            BCK(scd::launch_block_sum(false, b->part_img[g], 2, b->members[g]->geo.n_slots,
                                      b->members[g]->d_img_out, st));
    }
    // the sweep's time: the class launches and the sums that complete the images
    BCK(cudaEventRecordWithFlags(b->ev[1], st, ev_flags));
    b->timed = true;
    if (!b->fp64) {
        // the Fermi-surface averages of every member: one launch per component count
        // (with transfer items, of the one-component members no class launch rotates back)
        for (int k = 0; k < 4; ++k) {
            const bool solo = b->fused && k == 0;
            BCK(scd::launch_batch_rotate_back_f32(b->d_members, solo ? b->d_solo + (n + 1) : member_off(b, 2 + k),
                                                  solo ? b->tot_solo_back : b->tot_back[k], k + 1, n, st));
        }
    } else {
        fs = fork(b, st);
        if (fs != SC_OK) return fs;
        for (size_t g = 0; g < b->members.size(); ++g) {
            sc_status s = sc_internal::rotate_back(b->members[g], b->aux[g % sc_batch::kAux]);
            if (s != SC_OK) return berr(b, s, b->members[g]->err);
        }
        fs = join(b, st);
        if (fs != SC_OK) return fs;
    }
    BCK(cudaEventRecordWithFlags(b->iev[1], st, ev_flags));
    for (sc_ctx *c : b->members) {
        c->cur = b->parity ^ 1;
        c->have_boundary = true;
        c->have_sweep = true;
        c->have_outputs = false;
        ++c->sweeps;
    }
    b->parity ^= 1;
    b->have_boundary = true;
    return SC_OK;
}

// one batch iteration (sweep, and optionally every member's outputs) on stream st
static sc_status iteration(sc_batch *b, int with_outputs, cudaStream_t st) {
    sc_status s = sc_batch_sweep(b, st);
    if (s != SC_OK) return s;
    if (with_outputs) {
        // Delta_new, j, F and the grid sums of every member in two launches
        BCK(scd::launch_batch_outputs(b->d_members, member_off(b, 6), b->tot_out, (int)b->members.size(), st));
        for (sc_ctx *c : b->members) c->have_outputs = true;
    }
    return SC_OK;
}

sc_status sc_batch_set_energy_parts(sc_batch *b, int32_t on) {
    if (!b) return SC_EINVAL;
    if (b->failed) return SC_ESTATE;
    if (on && b->fp64) return berr(b, SC_EINVAL, "energy parts are an FP32 layout");
    BCK(cudaSetDevice(b->device));
    b->split = on != 0;
    return build(b, b->ept);
}

sc_status sc_batch_set_fused_transfers(sc_batch *b, int32_t on) {
    if (!b) return SC_EINVAL;
    if (b->failed) return SC_ESTATE;
    if (on && b->fp64) return berr(b, SC_EINVAL, "transfer items are an FP32 layout");
    BCK(cudaSetDevice(b->device));
    b->fuse = on != 0;
    return build(b, b->ept);
}

sc_status sc_batch_reset_boundary(sc_batch *b) {
    if (!b) return SC_EINVAL;
    if (b->failed) return SC_ESTATE;
    b->have_boundary = false;
    for (sc_ctx *c : b->members) c->have_boundary = false;
    return SC_OK;
}

sc_status sc_batch_run(sc_batch *b, int32_t n_sweeps, int32_t with_outputs, void *stream) {
    if (!b || n_sweeps < 0) return SC_EINVAL;
    if (b->failed) return SC_ESTATE;
    BCK(cudaSetDevice(b->device));
    cudaStream_t user = (cudaStream_t)stream;
    if (!b->gstream) {
        BCK(cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking));
        BCK(cudaEventCreateWithFlags(&b->sync_ev[0], cudaEventDisableTiming));
        BCK(cudaEventCreateWithFlags(&b->sync_ev[1], cudaEventDisableTiming));
    }
    // the first sweep from fresh boundary values runs eagerly (different launch arguments)
    int done = 0;
    BCK(cudaEventRecord(b->sync_ev[0], user));
    BCK(cudaStreamWaitEvent(b->gstream, b->sync_ev[0], 0));
    if (!b->have_boundary && n_sweeps > 0) {
        sc_status s = iteration(b, with_outputs, b->gstream);
        if (s != SC_OK) return s;
        done = 1;
    }
    if (done < n_sweeps && (b->graph_outputs != (with_outputs ? 1 : 0) || b->graph_ept != b->ept || !b->graph[0])) {
        free_graphs(b);
        // capture one iteration per parity; the host state advances as if they ran,
        // so after capturing both it is back where it started (the members' sweep
        // counts, which only advance, are put back)
        std::vector<int64_t> swept(b->members.size());
        for (size_t g = 0; g < b->members.size(); ++g) swept[g] = b->members[g]->sweeps;
        for (int k = 0; k < 2; ++k) {
            const int par = b->parity;
            cudaGraph_t g = nullptr;
            BCK(cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal));
            sc_status s = iteration(b, with_outputs, b->gstream);
            cudaError_t e = cudaStreamEndCapture(b->gstream, &g);
            if (s != SC_OK) {
                if (g) cudaGraphDestroy(g);
                return s;
            }
            if (e != cudaSuccess) return berr(b, SC_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
            e = cudaGraphInstantiate(&b->graph[par], g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return berr(b, SC_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
        }
        b->graph_outputs = with_outputs ? 1 : 0;
        b->graph_ept = b->ept;
        for (size_t g = 0; g < b->members.size(); ++g) b->members[g]->sweeps = swept[g];
    }
    for (; done < n_sweeps; ++done) {
        BCK(cudaGraphLaunch(b->graph[b->parity], b->gstream));
        // host mirror of what the graph did
        for (sc_ctx *c : b->members) {
            c->cur = b->parity ^ 1;
            c->have_boundary = true;
            c->have_sweep = true;
            c->have_outputs = with_outputs != 0;
            ++c->sweeps;
        }
        b->parity ^= 1;
    }
    BCK(cudaEventRecord(b->sync_ev[1], b->gstream));
    BCK(cudaStreamWaitEvent(user, b->sync_ev[1], 0));
    return SC_OK;
}

sc_status sc_batch_autotune(sc_batch *b, int32_t *energies_per_lane, void *stream) {
    if (!b) return SC_EINVAL;
    if (b->failed) return SC_ESTATE;
    int max_ne = 0;
    for (sc_ctx *c : b->members) max_ne = std::max(max_ne, c->n_e);
    int best = b->ept;
    float best_ms = 1e30f;
    b->bps_choice.clear();  // grids at occupancy while the layout is chosen
    b->min_lanes = 2;
    for (int ept = 2; ept <= (b->fp64 ? 8 : 10); ++ept) {
        if (max_ne > 32 * ept) continue;
        sc_status s = build(b, ept);
        if (s != SC_OK) return s;
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {  // the second sweep is the one timed
            s = sc_batch_sweep(b, stream);
            if (s != SC_OK) return s;
            BCK(cudaEventSynchronize(b->iev[1]));
            BCK(cudaEventElapsedTime(&ms, b->iev[0], b->iev[1]));
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = ept;
        }
    }
    // the fewest lanes per line (the most lines per warp): a warp steps all its lines
    // as long as its longest, so more lines per warp trade padding for idle lanes
    int best_min = b->min_lanes;
    best_ms = 1e30f;
    for (int ml : {2, 4, 8, 16}) {
        b->min_lanes = ml;
        sc_status s = build(b, best);
        if (s != SC_OK) return s;
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
            s = sc_batch_sweep(b, stream);
            if (s != SC_OK) return s;
            BCK(cudaEventSynchronize(b->iev[1]));
            BCK(cudaEventElapsedTime(&ms, b->iev[0], b->iev[1]));
        }
        if (ms < best_ms) {
            best_ms = ms;
            best_min = ml;
        }
    }
    b->min_lanes = best_min;
    // FP32: members in two energy parts (each in its own layout) or in one
    if (!b->fp64) {
        float t[2] = {0.f, 0.f};  // with, without
        for (int v = 0; v < 2; ++v) {
            b->split = v == 0;
            sc_status s = build(b, best);
            if (s != SC_OK) return s;
            for (int rep = 0; rep < 3; ++rep) {  // the second and third sweeps are timed
                s = sc_batch_sweep(b, stream);
                if (s != SC_OK) return s;
                BCK(cudaEventSynchronize(b->iev[1]));
                float ms = 0.f;
                BCK(cudaEventElapsedTime(&ms, b->iev[0], b->iev[1]));
                if (rep > 0) t[v] += ms;
            }
        }
        const float ms_on = 0.5f * t[0], ms_off = 0.5f * t[1];
        b->split = ms_on < 0.99f * ms_off;  // parts only where they are clearly faster
        b->split_ms[0] = ms_on;
        b->split_ms[1] = ms_off;
        // the members' lattice transfers as work items of the class launches, or
        // in their own launches
        float u[2] = {0.f, 0.f};  // with, without
        for (int v = 0; v < 2; ++v) {
            b->fuse = v == 0;
            sc_status s = build(b, best);
            if (s != SC_OK) return s;
            for (int rep = 0; rep < 3; ++rep) {  // the second and third sweeps are timed
                s = sc_batch_sweep(b, stream);
                if (s != SC_OK) return s;
                BCK(cudaEventSynchronize(b->iev[1]));
                float ms = 0.f;
                BCK(cudaEventElapsedTime(&ms, b->iev[0], b->iev[1]));
                if (rep > 0) u[v] += ms;
            }
        }
        b->fuse_ms[0] = 0.5f * u[0];
        b->fuse_ms[1] = 0.5f * u[1];
        b->fuse = b->fuse_ms[0] < 0.99f * b->fuse_ms[1];
    }
    b->bps_choice.clear();
    sc_status s = build(b, best);
    if (s != SC_OK) return s;
    // per class: the persistent grid sized for occupancy, occupancy - 1, occupancy - 2
    // resident blocks per SM; each class keeps its fastest
    const size_t nc = b->classes.size();
    constexpr size_t kE = 11;  // energies per lane 1..10
    std::vector<int> pick(kE, 0);
    std::vector<float> pick_ms(kE, 1e30f);
    for (int d = 0; d <= 2; ++d) {
        b->bps_choice.assign(kE, 0);
        bool any = false;
        for (size_t k = 0; k < nc; ++k) {
            const int occ = b->classes[k].occ;
            b->bps_choice[b->classes[k].ept] = std::max(1, occ - d);
            any = any || occ - d >= 1;
        }
        if (!any) break;
        s = build(b, best);
        if (s != SC_OK) return s;
        for (int rep = 0; rep < 2; ++rep) {  // the second sweep is the one timed
            s = sc_batch_sweep(b, stream);
            if (s != SC_OK) return s;
        }
        BCK(cudaEventSynchronize(b->cev[nc]));
        for (size_t k = 0; k < nc; ++k) {
            float ms = 0.f;
            BCK(cudaEventElapsedTime(&ms, b->cev[k], b->cev[k + 1]));
            const int e = b->classes[k].ept;
            if (ms < pick_ms[e]) {
                pick_ms[e] = ms;
                pick[e] = b->bps_choice[e];
            }
        }
    }
    b->bps_choice = pick;
    s = build(b, best);
    if (s != SC_OK) return s;
    if (energies_per_lane) *energies_per_lane = best;
    return SC_OK;
}

sc_status sc_batch_set_fields(sc_batch *b, const double *delta_all, int on_device, void *stream) {
    if (!b || !delta_all) return SC_EINVAL;
    if (b->failed) return SC_ESTATE;
    BCK(cudaSetDevice(b->device));
    cudaStream_t st = (cudaStream_t)stream;
    const double *src = delta_all;
    if (!on_device) {
        if (!b->d_stage_in) BCK(cudaMalloc(&b->d_stage_in, 2 * (size_t)b->tot_cplx * sizeof(double)));
        BCK(cudaMemcpyAsync(b->d_stage_in, delta_all, 2 * (size_t)b->tot_cplx * sizeof(double),
                            cudaMemcpyHostToDevice, st));
        src = b->d_stage_in;
    }
    BCK(scd::launch_batch_set_fields(b->d_members, member_off(b, 6), b->tot_out, b->d_pt, (int)b->members.size(),
                                     src, st));
    if (!on_device) BCK(cudaStreamSynchronize(st));
    for (sc_ctx *c : b->members) {
        c->have_aind = false;
        c->have_sweep = false;
        c->have_outputs = false;
        c->acc_kind = -1;
    }
    return SC_OK;
}

sc_status sc_batch_get_outputs(sc_batch *b, double *delta_new_all, double *j_all, double *F_all, int on_device,
                               void *stream) {
    if (!b) return SC_EINVAL;
    if (b->failed) return SC_ESTATE;
    for (sc_ctx *c : b->members)
        if (!c->have_outputs) return berr(b, SC_ESTATE, "a member has no outputs of its last sweep");
    BCK(cudaSetDevice(b->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int n = (int)b->members.size();
    if (on_device) {
        BCK(scd::launch_batch_get_outputs(b->d_members, member_off(b, 6), b->tot_out, b->d_pt, n, delta_new_all,
                                          j_all, F_all, st));
        return SC_OK;
    }
    const size_t nd = 2 * (size_t)b->tot_cplx, nj = 2 * (size_t)b->tot_pts, nf = (size_t)b->tot_pts;
    if (!b->d_stage_out) BCK(cudaMalloc(&b->d_stage_out, (nd + nj + nf) * sizeof(double)));
    double *sd = b->d_stage_out, *sj = sd + nd, *sf = sj + nj;
    BCK(scd::launch_batch_get_outputs(b->d_members, member_off(b, 6), b->tot_out, b->d_pt, n,
                                      delta_new_all ? sd : nullptr, j_all ? sj : nullptr, F_all ? sf : nullptr, st));
    if (delta_new_all) BCK(cudaMemcpyAsync(delta_new_all, sd, nd * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (j_all) BCK(cudaMemcpyAsync(j_all, sj, nj * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (F_all) BCK(cudaMemcpyAsync(F_all, sf, nf * sizeof(double), cudaMemcpyDeviceToHost, st));
    BCK(cudaStreamSynchronize(st));
    return SC_OK;
}

sc_status sc_batch_get_info(const sc_batch *b, sc_batch_info *info) {
    if (!b || !info) return SC_EINVAL;
    std::memset(info, 0, sizeof *info);
    info->n_grains = (int32_t)b->members.size();
    info->n_items = b->n_items;
    info->energies_per_lane = b->ept;
    info->steps_per_sweep = b->steps_per_sweep;
    info->lane_steps_per_sweep = b->lane_steps_per_sweep;
    info->sweep_launches = (int32_t)b->classes.size();
    info->scratch_bytes = (int64_t)b->scratch_bytes;
    info->min_lanes_per_line = b->min_lanes;
    // the launches sc_batch_sweep and the outputs of iteration() make
    int32_t nl = (int32_t)b->classes.size() + 2;  // sweep classes; outputs and their final sums
    for (int nbk : b->member_blocks) nl += nbk > 1 ? 1 : 0;  // energy-block sums
    for (int np : b->member_parts) nl += np > 1 ? 1 : 0;     // sums of two energy parts
    if (!b->fp64) {
        nl += (b->tot_pad > 0) + ((b->fused ? b->tot_solo_rot : b->tot_slots) > 0);
        for (int k = 0; k < 4; ++k) nl += (b->fused && k == 0 ? b->tot_solo_back : b->tot_back[k]) > 0;
    } else {
        nl += 2 * (int32_t)b->members.size();  // rotate and rotate-back per member
    }
    info->launches_per_iteration = nl;
    info->split_ms_on = b->split_ms[0];
    info->split_ms_off = b->split_ms[1];
    info->fused_transfers = b->fused ? 1 : 0;
    info->transfer_items = b->n_side;
    info->fuse_ms_on = b->fuse_ms[0];
    info->fuse_ms_off = b->fuse_ms[1];
    info->split_members = 0;
    for (int np : b->member_parts) info->split_members += np > 1 ? 1 : 0;
    static_assert(sc_batch::kMaxClasses <= 16, "sc_batch_info holds 16 classes");
    for (size_t k = 0; k < b->classes.size(); ++k) {
        info->class_ept[k] = b->classes[k].ept;
        info->class_blocks_per_sm[k] = b->classes[k].bps;
    }
    if (b->timed) {
        const size_t nc = b->classes.size();
        for (size_t k = 0; k < nc; ++k) {
            float cms = 0.f;
            if (cudaEventSynchronize(b->cev[nc]) == cudaSuccess &&
                cudaEventElapsedTime(&cms, b->cev[k], b->cev[k + 1]) == cudaSuccess)
                info->class_ms[k] = cms;
            else
                (void)cudaGetLastError();
        }
        float ms = 0.f;
        if (cudaEventSynchronize(b->ev[1]) == cudaSuccess && cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]) == cudaSuccess)
            info->ms_sweep = ms;
        else
            (void)cudaGetLastError();  // a failed query must not linger as the thread's last error
        if (cudaEventSynchronize(b->iev[1]) == cudaSuccess &&
            cudaEventElapsedTime(&ms, b->iev[0], b->iev[1]) == cudaSuccess)
            info->ms_iteration = ms;
        else
            (void)cudaGetLastError();
    }
    return SC_OK;
}

}  // extern "C"
