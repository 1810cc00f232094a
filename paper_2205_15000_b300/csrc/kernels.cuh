// Device data layouts and kernel launchers of the Riccati sweep.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "bounds.cuh"

namespace scd {

// One trajectory line of an angle pair, as the sweep kernel reads it.
struct LineDev {
    int32_t ns;          // lattice samples on the line (0: one slot holds the chord midpoint)
    int32_t slot0;       // first image slot of the line
    int32_t exit_f;      // exit slot of angle p (at smax)
    int32_t exit_b;      // exit slot of angle p + P (at smin)
    double lead;         // smin -> first sample (chord length when ns == 0)
    double tail;         // last sample -> smax (chord length when ns == 0)
    int32_t tap_f[4];    // entry link of angle p: exit slots
    int32_t tap_b[4];    // entry link of angle p + P
    double w_f[4];
    double w_b[4];
};

// Where the rotate kernel finds the position of every image slot.
struct LineGeo {
    int32_t pair, l, m0, ns, slot0, pad;
    double smid;         // chord midpoint (position of the single slot when ns == 0)
};

// Per angle pair, for the rotate-back kernel.
struct PairDev {
    double ex, ey;       // e_par
    double u0, v0;       // lattice coordinates (line, sample) of grid point (0, 0), units of h
    double eta;          // basis function of the pair (component 0)
    double wa, wb;       // quadrature weights of angle p and of angle p + P
    int32_t l_lo, l_hi, lat0, pad;  // lattice lines l_lo..l_hi; their BackLine records from lat0
    double eta_c[4];     // basis function of each order-parameter component
};

// Per lattice line, for the rotate-back kernels: the sampled chord (m0, ns,
// slot0) of the nearest lattice line that has one.  When that line has several
// sampled chords (composite grains), `more` indexes a list of them further on
// in the same table (each entry's `more` holding the list length), and the
// chord nearest to the grid point along the line is taken; else more = -1.
struct BackLine {
    int32_t more, m0, ns, slot0;
};

// Distance, along the line, from lattice coordinate iv + fv (units of h,
// 0 <= fv < 1) to the samples m0 .. m0 + ns - 1 of a chord.
template <typename F>
__device__ __forceinline__ F chord_distance(const BackLine &c, int iv, F fv) {
    const int m1 = c.m0 + c.ns - 1;
    if (iv < c.m0) return (F)(c.m0 - iv) - fv;
    if (iv > m1 || (iv == m1 && fv > F(0))) return (F)(iv - m1) + fv;
    return F(0);
}

// The chord a rotate-back tap takes on lattice-line record L: the only one,
// or the listed chord nearest to the point (ties to the chord of lower s).
template <typename F>
__device__ __forceinline__ BackLine back_chord(const BackLine *__restrict__ bl, BackLine L, int iv, F fv) {
    if (L.more < 0) return L;
    const int first = L.more;
    BackLine best = bl[first];
    F bd = chord_distance(best, iv, fv);
    const int n = best.more;
    for (int k = 1; k < n; ++k) {
        const BackLine c = bl[first + k];
        const F d = chord_distance(c, iv, fv);
        if (d < bd) {
            bd = d;
            best = c;
        }
    }
    return best;
}

// back_chord of record idx of the rotate-back table (n_back records); in the
// bounds-checked build an index outside the table gives the first record
template <typename F>
__device__ __forceinline__ BackLine back_chord_at(const BackLine *__restrict__ bl, int32_t n_back, int64_t idx, int iv,
                                                  F fv) {
    if (!in_bounds(idx, n_back)) idx = 0;
    const BackLine L = bl[idx];
    if (L.more >= 0 && !(in_bounds(L.more, n_back) && in_bounds((int64_t)L.more + bl[L.more].more - 1, n_back)))
        return bl[0];
    return back_chord(bl, L, iv, fv);
}

struct GridDev {
    int32_t nx, ny;
    double h, x0, y0, ox, oy;
    double bfield;       // external field, units of B0 (symmetric and landau gauges)
    double gx, gy;       // gauge origin
    double flux;         // flux quanta alpha (solenoid gauge)
    int64_t gfx, gfy;    // gauge origin in fixed-point grid coordinates (FP32 path)
    int32_t gauge;       // sc_gauge
    int32_t charge_sign;
    int32_t n_comp;      // order-parameter components; Delta is [n_comp][ny][nx] complex
    // table sizes (the bounds-checked build compares indices with them)
    int64_t n_slots;     // image slots
    int32_t n_lines;     // chords (lines of the sweep)
    int32_t n_pairs;     // angle pairs
    int32_t n_back;      // rotate-back records
};

// FP32 production path: lattice coordinates in fixed point (2^-40 grid units),
// so that floor and fraction are exact and no FP64 arithmetic is needed.
constexpr int kFixBits = 40;

struct LineF32 {
    int64_t gx0, gy0;    // grid coordinates (x - x0)/h - 1/2 of the first slot's point
    float aext;          // sigma v.A_ext in the symmetric gauge (constant along a line); 0 otherwise
    int32_t pair, ns, slot0;
    int32_t m0;          // lattice index (along the line, units of h) of the first slot's point
};

// The FP32 rotate-back takes a grid in tiles of 8 x 4 points, one point per lane
// of a warp, tiles along x first: the tile's points fall on at most about nine
// lattice lines and nine samples per line at any angle.
__host__ __device__ inline int64_t back_tiles(int64_t nx, int64_t ny) { return ((nx + 7) / 8) * ((ny + 3) / 4); }

// The fields the rotate-back reads for every (grid point, pair) come first, in
// 16-byte groups that it loads as vectors (five loads per pair instead of one per
// field).
struct alignas(16) PairF32 {
    int64_t ui, uj, u0, vi, vj, v0; // u = i ui + j uj + u0, v = i vi + j vj + v0
    int32_t l_lo, l_hi, lat0, pad;  // lattice lines l_lo..l_hi; their BackLine records from lat0
    float w_eta, w_ex, w_ey, w_sum; // (w_p + w_{p+P}) times eta, e_x, e_y, 1
    float w_eta_c[4];               // per order-parameter component: (w_p + w_{p+P}) eta_c
    int64_t dx, dy;                 // e_par in grid units per sample
    float eta;                      // basis function (component 0)
    float wa, wb;                   // w_p, w_{p+P}
    float ex_f, ey_f;               // e_par in FP32
    float eta_c[4];                 // per order-parameter component: eta_c
};
static_assert(offsetof(PairF32, l_lo) == 48 && offsetof(PairF32, w_eta) == 64 && offsetof(PairF32, w_eta_c) == 80 &&
                  alignof(PairF32) == 16,
              "the rotate-back loads PairF32 as 16-byte groups");

// Everything the sweep needs of one grain (one context, or one member of a batch).
struct GrainSweep {
    const LineDev *lines;
    const int32_t *groups;     // [n_groups][lines_per_warp] line indices, -1 padded
    const void *image_in;      // T4 per slot
    void *image_out;           // T4 per slot (retarded mode: n_e values per slot)
    void *exits[2];            // complex T [2 n_lines][n_e]; a sweep reads exits[parity]
                               // (previous sweep) and writes exits[parity ^ 1]
    const double *energies;    // retarded mode: n_e real energies, symmetric about zero
    const double *mats_eps;    // Matsubara mode: positive energies (nullptr: eps_n = t (n + 1/2))
    const double *mats_w;      // Matsubara mode: weights of the energy sums (nullptr: 1)
    double t;                  // Matsubara energies eps_n = t (n + 1/2)
    double h;                  // lattice spacing
    double broadening;         // retarded mode: z = eps + i broadening
    int32_t n_e;
    int32_t lanes;             // energy lanes per line, Lw (lines_per_warp * Lw = 32)
    int32_t lines_per_warp;
    int32_t ne_pad;            // Lw * ept
    int32_t max_ns;            // longest line of the grain
    int32_t ept;               // energies per lane (equals the launch's EPT)
    int32_t n_blocks;          // energy blocks of ne_pad energies: work item y of the grain is
                               // line group y / n_blocks with the energies of block y % n_blocks
    int64_t n_slots;           // image slots; a blocked sweep's block k writes its sums at
                               // image_out + k n_slots
    int32_t n_lines;           // lines of the grain (exit rows: 2 n_lines)
    int32_t n_groups;          // line groups (groups holds n_groups x lines_per_warp entries)
    int32_t e_first, e_count;  // a part of the grain's energies, [e_first, e_first + e_count),
                               // in its own layout and image (e_count 0: all n_e energies)
};

struct MemberDev;

// One persistent launch over the work items (grain, line group) of any number
// of grains; items are taken from an atomic counter, longest first.
struct SweepLaunch {
    const GrainSweep *grains;
    const int2 *items;         // (grain, group)
    int32_t n_items;
    int32_t *counter;
    void *scratch;             // per-warp slab of parked gammas
    int64_t scratch_stride;    // complex T elements per warp (>= G * max_ns * ne_pad of every grain)
    int64_t scratch_elems;     // complex T elements of the whole scratch
    int32_t n_grains;          // entries of grains
    int32_t energies_per_lane; // EPT (template)
    int32_t first_sweep;       // start every line from the homogeneous solution
    int32_t parity;            // which exit buffer holds the previous sweep's values
    int32_t retarded;          // LDOS mode
    int32_t grid_blocks, block_threads;
    int32_t stepper;           // 0 closed-form step, 1 implicit midpoint rule
    int32_t weighted;          // Matsubara mode: weighted energy sums (grains carry mats_w)
    int32_t blocked;           // some grain splits its energies into blocks (each block writes its
                               // own partial image; launch_block_sum adds them in block order)
    // FP32 batch (launch_sweep_side_f32 only): lattice transfers of other members
    // as work items of the launch, spread evenly among the sweep items.  side[s] =
    // (2 member + kind, index): kind 0 rotates lines 4 index .. 4 index + 3 of the
    // member, kind 1 rotates back its tile `index` of 8 x 4 grid points (members of
    // one order-parameter component).
    const MemberDev *side_members;
    const int2 *side;
    int32_t n_side;
    int32_t n_side_members;
};

// launchers (return cudaError_t)
cudaError_t launch_rotate(bool fp64, const LineGeo *geo, const int32_t *slot_line, int64_t n_slots,
                          const PairDev *pairs, const GridDev &grid, const int32_t *ghost,
                          const double *delta, const double *aind, void *image_in,
                          cudaStream_t s);
cudaError_t launch_sweep(bool fp64, const SweepLaunch &a, cudaStream_t s);
// Image of a blocked sweep: out[s] = sum over k = 0 .. nb-1, in this order, of
// blocks[k n_slots + s] (four values per slot, FP64 or FP32), so the result does
// not depend on the order in which the blocks' work items ran.
cudaError_t launch_block_sum(bool fp64, const void *blocks, int nb, int64_t n_slots, void *out, cudaStream_t st);
// the FP64 device reciprocal and reciprocal square root of the sweep on n values
cudaError_t launch_fp64_math(const double *x, int64_t n, double *rcp, double *rsqrt, cudaStream_t s);
// lane fused multiply-adds per second of a launch of eight blocks of 256 threads per SM,
// eight independent chains per thread (scalar, or two-wide when packed)
cudaError_t measure_fma_rate(bool packed, int sm_count, double *lane_ops_per_s, cudaStream_t st);
// FP32 production path
// FP32 fields on the ghost-padded grid: every padded point takes the values of its
// nearest grain point (ghost map), zero where it has none
cudaError_t launch_fields_f32(const GridDev &grid, const int32_t *ghost, const double *delta, const double *aind,
                              float4 *pad0, float2 *padc, cudaStream_t s);
cudaError_t launch_rotate_f32(const LineF32 *lines, const int32_t *slot_line, int64_t n_slots,
                              const PairF32 *pairs, const GridDev &grid, const int32_t *ghost,
                              const float4 *pad0, const float2 *padc, float4 *image_in,
                              cudaStream_t s);
cudaError_t launch_rotate_back_f32(const PairF32 *pairs, int32_t n_pairs, const BackLine *bl,
                                   const GridDev &grid, const uint8_t *mask, const float4 *image_out,
                                   double *acc, cudaStream_t s);
int sweep_occupancy(bool fp64, int ept, int block_threads, int stepper, bool weighted);
// per-precision instantiations (sweep_f32.cu, sweep_f64.cu)
cudaError_t launch_sweep_f32(const SweepLaunch &a, cudaStream_t s);
// the FP32 batch sweep with lattice transfers as work items (a.n_side > 0;
// Matsubara or Ozaki sums, no energy blocks, not retarded)
cudaError_t launch_sweep_side_f32(const SweepLaunch &a, cudaStream_t s);
int sweep_side_occupancy_f32(int ept, int block_threads, int stepper, bool weighted);
cudaError_t launch_sweep_f64(const SweepLaunch &a, cudaStream_t s);
int sweep_occupancy_f32(int ept, int block_threads, int stepper, bool weighted);
int sweep_occupancy_f64(int ept, int block_threads, int stepper, bool weighted);
cudaError_t launch_rotate_back(bool fp64, const PairDev *pairs, int32_t n_pairs,
                               const BackLine *bl, const GridDev &grid, const uint8_t *mask,
                               const void *image_out, double *acc, cudaStream_t s);
// Reductions over the grid finish in a fixed order (per-block partials, then
// one block): the sums do not depend on scheduling.  partials: reduce_blocks(npts)
// x 4 doubles of scratch.
int reduce_blocks(int64_t npts);
// Accumulator planes: <eta_0 Sf> (2), <v Sg> (2), <SF>, then <eta_c Sf> (2 per
// component c >= 1): 3 + 2 n_comp planes of nx*ny doubles.
// normD_c: the gap-equation normalisation of each component, D - ln(T_c^c/T_c).
struct CompNorm {
    double D[4];
    double kD[4];  // t / (2 pi D[c]): Delta_c = kD[c] <eta_c Sf> (Eq. gapeq_fixpoint)
};

// One batch member's tables and buffers for the per-member kernels of a batch
// iteration (FP32 lattice transfers, outputs), so that one launch serves every
// member.  aind always points at the member's induced potential (zero while
// none is set); kappa is 0 when the member has no magnetic energy term.
struct MemberDev {
    GridDev grid;
    const int32_t *ghost;
    const uint8_t *mask;
    const double *delta, *aind;
    float4 *pad0;
    float2 *padc;
    const LineF32 *lines;
    const int32_t *slot_line;
    const PairF32 *pairs;
    int32_t n_pairs;
    const BackLine *back;
    float4 *image_in;
    const float4 *image_out;
    double *acc;
    double t, kappa;
    CompNorm norms;
    double *dnew, *j, *F, *sums, *partials;
    int64_t n_slots, n_pad;  // image slots; padded grid points (nx + 2)(ny + 2)
};

#ifdef __CUDACC__
// A block's member of a batch: the member whose block range [off[g], off[g + 1])
// holds the block (bisection over the n + 1 offsets; empty ranges are skipped),
// its table copied to the shared `sh` by the block's threads.  Returns the
// block's index within the member.  All threads of the block must call it.
__device__ __forceinline__ int64_t batch_member(const MemberDev *__restrict__ m, const int64_t *__restrict__ off,
                                                int n, MemberDev &sh) {
    __shared__ int g_sh;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n;  // off[lo] <= b < off[hi]
        const int64_t b = blockIdx.x;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (off[mid] <= b) lo = mid;
            else hi = mid;
        }
        g_sh = lo;
    }
    __syncthreads();
    const int g = g_sh;
    constexpr int words = (int)(sizeof(MemberDev) / sizeof(int));
    static_assert(sizeof(MemberDev) % sizeof(int) == 0, "MemberDev is copied as words");
    const int *src = (const int *)(m + g);
    int *dst = (int *)&sh;
    for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
    __syncthreads();
    return (int64_t)blockIdx.x - off[g];
}
#endif

// Batch iterations: every member's FP32 field conversion and rotation (off_*:
// prefix sums over the members, n + 1 entries, of their blocks of 256 padded
// points and of 16 lines), rotate-back of the members with nc components
// (off_blocks: prefix of tiles of 8 x 4 grid points, back_tiles, zero for other members), and
// outputs (off_blocks: prefix of reduction blocks of 256 grid points).  Each
// block serves one member and holds its table in shared memory.
cudaError_t launch_batch_fields_rotate_f32(const MemberDev *members, const int64_t *off_pad, int64_t pad_blocks,
                                           const int64_t *off_lines, int64_t line_blocks, int n, cudaStream_t st);
cudaError_t launch_batch_rotate_back_f32(const MemberDev *members, const int64_t *off_blocks, int64_t n_blocks,
                                         int nc, int n, cudaStream_t st);
cudaError_t launch_batch_outputs(const MemberDev *members, const int64_t *off_blocks, int64_t n_blocks, int n,
                                 cudaStream_t st);
// Members' fields from / outputs to arrays of all members one after another
// (off_blocks: prefix of blocks of 256 grid points; pt_off: prefix of grid points).
// set: Delta (n_comp planes) from delta_all, A_ind zeroed.  get: Delta_new, j, F
// into the arrays that are not null.
cudaError_t launch_batch_set_fields(const MemberDev *members, const int64_t *off_blocks, int64_t n_blocks,
                                    const int64_t *pt_off, int n, const double *delta_all, cudaStream_t st);
cudaError_t launch_batch_get_outputs(const MemberDev *members, const int64_t *off_blocks, int64_t n_blocks,
                                     const int64_t *pt_off, int n, double *dnew_all, double *j_all, double *F_all,
                                     cudaStream_t st);


cudaError_t launch_outputs(const GridDev &grid, const uint8_t *mask, const double *acc,
                           const double *delta, const double *aind, double t, const CompNorm &normD,
                           double kappa, double *delta_new, double *j, double *F,
                           double *sums /* [4]: num, den, Fsum, nonfinite */, double *partials,
                           cudaStream_t s);
cudaError_t launch_mean_current(const GridDev &grid, const uint8_t *mask, const double *j,
                                double *sums /* [2] */, double *partials, cudaStream_t s);
cudaError_t launch_vector_potential(const GridDev &grid, const uint8_t *mask, const double *j,
                                    const double *jsum, double n_in, const double *G, int W,
                                    double inv_k2, double *aind, cudaStream_t s);
cudaError_t launch_copy_delta(int64_t n, const double *src, double *dst, cudaStream_t s);
cudaError_t launch_max_diff(int64_t n, const void *a, const void *b, bool fp64, double *out,
                            cudaStream_t s);
cudaError_t launch_ldos_back(bool fp64, const PairDev *pairs, int32_t n_pairs,
                             const BackLine *bl, const GridDev &grid, const uint8_t *mask,
                             const void *ldos_img, int32_t n_e, double *out, cudaStream_t s);

}  // namespace scd
