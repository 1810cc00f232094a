/*
 * sc.h -- C ABI of the B300-native Riccati sweep (quasiclassical Eilenberger
 * method of Holmvall et al., "SuperConga", arXiv 2205.15000).
 *
 * One context = one 2D grain on the current CUDA device.  The context owns all
 * of its device memory (allocated in sc_create, freed in sc_destroy).  Every
 * pointer argument is owned by the caller and never retained after the call.
 * Device pointers (on_device = 1) must live on the context's device; `stream`
 * is a cudaStream_t (NULL = legacy default stream).  Calls are asynchronous on
 * `stream` unless they return a host scalar.  One context must not be used
 * from two threads at once.
 *
 * Units (Table units): lengths xi0 = hbar vF / 2 pi kB Tc, energies
 * 2 pi kB Tc, vector potential Phi0/(pi xi0), current j0, free energy
 * Omega_A = (2 pi kB Tc)^2 N_F A.
 *
 * Layouts: grids are row-major [ny][nx]; grid point (i, j) sits at
 * (x0 + (i + 1/2) h, y0 + (j + 1/2) h).  Complex grids interleave (re, im) as
 * two doubles per point; vector grids interleave (x, y).
 *
 * Errors: every call returns an sc_status.  Nothing aborts or exits.  A CUDA
 * error puts the context into a failed state; later calls return SC_ESTATE.
 * sc_last_error(ctx) (or sc_last_error(NULL) for sc_create) gives the message.
 * For tests of the error paths, the environment variable SC_TEST_FAIL_ALLOC_AT=N
 * (read by sc_create) makes the N-th device allocation of that context fail as
 * if the device were out of memory; nothing is allocated for it.
 */
#ifndef SC_H
#define SC_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sc_ctx sc_ctx;

typedef enum {
    SC_OK = 0,
    SC_EINVAL = 1,    /* invalid argument or parameter */
    SC_ENOMEM = 2,    /* device or host allocation failed */
    SC_ECUDA = 3,     /* CUDA runtime error */
    SC_ETIMEOUT = 4,  /* a bounded device wait gave up */
    SC_ENUMERIC = 5,  /* NaN / Inf detected in a result */
    SC_ESTATE = 6,    /* context unusable after an earlier failure, or wrong call order */
    SC_ENOTCONV = 7   /* iteration limit reached without convergence */
} sc_status;

typedef enum { SC_PAIR_S = 0, SC_PAIR_DX2Y2 = 1, SC_PAIR_DXY = 2, SC_PAIR_G = 3 } sc_pairing;
typedef enum { SC_PREC_FP64 = 0, SC_PREC_FP32 = 1 } sc_precision;
/* Integrator of Eq. riccati along a line (App. C).  CLOSED: the exact solution
   for coefficients held constant on each segment (half-step values, linear
   interpolation between samples).  MIDPOINT: the implicit midpoint rule with the
   same half-step values, g1 = g0 + ell f((g0 + g1)/2), solved as a quadratic
   (Eq. riccati_midpoint; the paper's production method). */
typedef enum { SC_STEP_CLOSED = 0, SC_STEP_MIDPOINT = 1 } sc_stepper;
/* Energy sums (Sec. 3.1).  MATSUBARA: eps_n = t (n + 1/2), n < n_energies, unit
   weights, D = ln t + 2 sum 1/(2n + 1).  OZAKI: the continued-fraction poles of
   the Fermi function (Ozaki 2007; the sum the paper uses): eps_p = t z_p / (2 pi)
   with weights R_p (sc_ozaki_poles), and D = ln t + t sum_p R_p / eps_p; the
   first poles coincide with Matsubara energies (R_p = 1), the later ones spread
   out with larger weights, so far fewer energies reach a given cutoff. */
typedef enum { SC_SUM_MATSUBARA = 0, SC_SUM_OZAKI = 1 } sc_energy_sum;

/* External vector potential (App. B, "gauge"), about the gauge origin
   (gauge_cx, gauge_cy):
     SC_GAUGE_SYMMETRIC  A = B/2 (-(y - yg), x - xg)               (Sec. 5.1.2)
     SC_GAUGE_LANDAU     A = B (-(y - yg), 0)
     SC_GAUGE_SOLENOID   A = alpha / (2 r) phi^ = alpha/(2 r^2) (-(y - yg), x - xg)
                         (Eq. solenoid_gauge: the flux alpha Phi0 threads a line
                         at the origin, which must lie outside the grain, e.g. in
                         the hole of an annulus)
   with B = pi alpha / area (units B0 = Phi0/(pi xi0^2), area of the grain), alpha =
   flux_quanta, A in units A0 = Phi0/(pi xi0). */
typedef enum { SC_GAUGE_SYMMETRIC = 0, SC_GAUGE_LANDAU = 1, SC_GAUGE_SOLENOID = 2 } sc_gauge;

/* Shape kinds: a disc, a convex polygon, or a composite of parts. */
typedef enum { SC_SHAPE_DISC = 0, SC_SHAPE_POLYGON = 1, SC_SHAPE_COMPOSITE = 2 } sc_shape;

/* One part of a composite grain (Sec. 4 and App. B, composite geometries):
   a disc or a convex polygon whose area is added to, or removed from, the
   grain made of the parts before it, in the listed order.  A grain with a
   hole is a disc or polygon followed by a removed part; regular polygons are
   given by their vertices. */
typedef struct {
    int32_t kind;            /* 0 = disc, 1 = convex polygon (counter-clockwise) */
    int32_t add;             /* 1 = add the area, 0 = remove it */
    double cx, cy, r;        /* disc centre and radius (xi0) */
    int32_t n_vert;          /* polygon vertex count (>= 3) */
    const double *vx, *vy;   /* polygon vertices (copied by sc_create) */
} sc_part;

/*
 * Problem statement of one grain (configuration appendix of the paper:
 * physics, geometry, numerics).  Call sc_params_default() first.
 */
typedef struct {
    int32_t nx, ny;          /* grid points */
    double h, x0, y0;        /* spacing and lower-left corner of the grid box (xi0) */
    int32_t shape_kind;      /* sc_shape: 0 = disc, 1 = convex polygon (counter-clockwise),
                                2 = composite (n_parts, parts below) */
    double disc_cx, disc_cy, disc_r;
    int32_t n_vert;          /* polygon vertex count (>= 3) */
    const double *vx, *vy;   /* polygon vertices (copied by sc_create) */
    int32_t pairing;         /* sc_pairing (Table basis_functions) */
    double crystal_rotation; /* crystal a-axis rotation, units of 2 pi */
    double t;                /* temperature T/Tc, 0 < t <= 1 */
    double flux_quanta;      /* alpha: symmetric and landau gauges, B_ext * area / Phi0;
                                solenoid gauge, the flux through the hole / Phi0 */
    double gauge_cx, gauge_cy; /* gauge origin */
    double kappa;            /* penetration depth lambda0/xi0; <= 0 or inf: no induced A */
    int32_t charge_sign;     /* sign of the carrier charge, +1 or -1 */
    int32_t n_angles;        /* Fermi-surface angles, even */
    int32_t n_energies;      /* positive Matsubara energies eps_n = t (n + 1/2), at most 4096
                                (more than 256 run as energy blocks); 0 = from eps_cut */
    double lattice_ox, lattice_oy; /* origin of the rotated lattices relative to the
                                      grid-box centre, units of h (default 0.1, 0.2) */
    int32_t precision;       /* sc_precision: FP64 plain sweep or FP32 production sweep */
    int32_t lanes_per_line;  /* 0 = automatic; else 2, 4, 8, 16 or 32 energy lanes per line
                                (the energies per lane then follow: at most 8, or 10 for an
                                FP32 sweep on 2, 16 or 32 lanes; the adjoint takes at most 8).
                                A warp holds 32 / lanes_per_line lines of one angle pair,
                                taken longest first. */
    int32_t host_only;       /* 1 = build the geometry tables only (no device memory); every
                                call that computes then returns SC_ESTATE.  For inspecting
                                the discretisation on a machine without a GPU. */
    int32_t record_timings;  /* 1 = time the three kernels of every sweep with CUDA events on
                                the sweep's stream (reported by sc_get_info) */
    int32_t stepper;         /* sc_stepper: how each segment of a line is integrated
                                (App. C); every sweep, burn-in, LDOS and adjoint of the
                                context uses it */
    int32_t energy_sum;      /* sc_energy_sum: which energies and weights the Matsubara
                                sums use; with SC_SUM_OZAKI, n_energies is the number of
                                Ozaki poles (at most 1024) */
    int32_t n_components;    /* order-parameter components Delta_Gamma (Eq. order_parameter,
                                Delta(p, R) = sum_Gamma Delta_Gamma(R) eta_Gamma(p)): 0 or 1
                                = one component (`pairing`), at most 4.  Delta (sc_set_fields)
                                and Delta_new (sc_gap_update) are then
                                [n_components][ny][nx] complex. */
    int32_t pairings[4];     /* sc_pairing of components 1 .. n_components-1 (component 0
                                uses `pairing`) */
    double tc_ratios[4];     /* T_c^Gamma / T_c per component (Eq. gapeq_regularized);
                                0 means 1 */
    int32_t n_parts;         /* composite grain: parts applied in order (copied by
                                sc_create); every added part must lie inside the grid box */
    const sc_part *parts;
    int32_t gauge;           /* sc_gauge of the external vector potential */
    double eps_cut;          /* energy cutoff (units 2 pi kB Tc), used when n_energies = 0:
                                Matsubara, the energies t (n + 1/2) below it; Ozaki, the
                                fewest poles whose largest energy t z_max / 2 pi reaches it */
    const uint8_t *mask;     /* optional [ny][nx] grain mask (1 = inside) that the caller
                                expects; sc_create returns SC_EINVAL unless it equals the
                                mask built from the shape (copied, not retained) */
    int32_t adjoint_checkpoint; /* storage of the forward gamma in the adjoint sweep:
                                0 (default) parks it at every sample; k >= 2 keeps it at
                                every k-th sample only and recomputes the k - 1 samples
                                after each when the reverse pass reaches them (one more
                                forward step per sample); k >= 2 needs precision FP32 and
                                the closed-form stepper */
} sc_params;

typedef struct {
    int32_t n_pairs;         /* angle pairs (phi, phi + pi) = n_angles / 2 */
    int32_t n_lines;         /* trajectories (lines) summed over angle pairs */
    int64_t n_samples;       /* lattice samples summed over angle pairs */
    int64_t n_in;            /* grid points inside the grain */
    int64_t steps_per_sweep; /* closed-form Riccati steps per sweep:
                                n_energies * sum_pairs sum_lines 2 (n_samples + 1) */
    int64_t points_per_sweep;/* (angle, energy, sample) points where g is formed */
    double area;             /* exact grain area (xi0^2) */
    double norm_D;           /* gap-equation normalisation ln t + 2 sum 1/(2n+1) */
    int32_t lanes_per_line, energies_per_lane, lines_per_warp; /* the sweep's lane layout:
                                energies per lane 1..8, or 9..10 for the FP32 sweep on 16
                                or 32 lanes per line */
    int64_t scratch_bytes;   /* device scratch used by the sweep */
    double ms_rotate, ms_sweep, ms_rotate_back; /* last sweep's kernel times when
                                record_timings = 1 (sc_get_info then waits for that sweep) */
    double ms_adjoint;       /* last adjoint sweep kernel, when record_timings = 1 */
} sc_info;

/* Ozaki's poles (host only, no context): z[p] ascending and residues R[p] of
   the n-pole continued-fraction representation 1/(1 + e^x) =
   1/2 - sum_p R_p [1/(x - i z_p) + 1/(x + i z_p)], 1 <= n <= 1024. */
sc_status sc_ozaki_poles(int32_t n, double *z, double *R);
/* The fewest Ozaki poles whose largest energy t z_max / 2 pi reaches eps_cut
   (units 2 pi kB Tc; host only), or 0 when 1024 poles do not reach it or the
   arguments are not positive. */
int32_t sc_ozaki_poles_for_cutoff(double t, double eps_cut);
/* The context's positive energies (units of 2 pi kB Tc) and their weights in
   the energy sums (n_energies each). */
sc_status sc_energy_grid(const sc_ctx *ctx, double *eps, double *weights);

/* Fill defaults: 64x64 unit grid, s-wave disc, t = 0.5, 32 angles, 16 energies,
   charge -1, lattice offset (0.1, 0.2), FP32. */
sc_status sc_params_default(sc_params *p);

/* Validate the parameters, build the geometry (mask, rotated lattices, chords,
   specular boundary links; Sec. 3.1) and allocate device memory.
   SC_EINVAL: odd n_angles, t outside (0,1], shape outside the grid box, empty
   grain, non-convex polygon.  SC_ENOMEM / SC_ECUDA on device failures. */
sc_status sc_create(const sc_params *p, sc_ctx **out);
sc_status sc_destroy(sc_ctx *ctx);
sc_status sc_get_info(const sc_ctx *ctx, sc_info *info);
/* Grain mask (nx*ny bytes, 1 = inside), host pointer. */
sc_status sc_get_mask(const sc_ctx *ctx, uint8_t *mask);

/* Set the order-parameter amplitude Delta(R) (complex, nx*ny) and the induced
   vector potential A_ind (vector, nx*ny; NULL = zero).  Eq. order_parameter:
   Delta(p, R) = Delta(R) eta(p).  Values outside the grain are ignored. */
sc_status sc_set_fields(sc_ctx *ctx, const double *delta, const double *a_ind, int on_device,
                        void *stream);
/* Copy the context's current fields out: Delta ([n_components][ny][nx]
   complex) and the induced vector potential A_ind ([ny][nx][2]; zero when none
   was set or computed), e.g. after sc_picard_step or sc_accelerate.  Either
   pointer may be NULL; on_device = 1: device pointers (ordered on `stream`),
   0: host pointers (the call waits for the copies). */
sc_status sc_get_fields(sc_ctx *ctx, double *delta, double *a_ind, int on_device, void *stream);
/* Forget the boundary coherence functions: the next sweep starts every
   trajectory from the local homogeneous solution. */
sc_status sc_reset_boundary(sc_ctx *ctx);

/* One Riccati sweep (Algorithm 1 inner loop): for every angle pair, line and
   positive Matsubara energy integrate gamma (Eq. riccati) along and gamma~
   (Eq. riccati_tilde) against the Fermi velocity with the closed-form
   constant-coefficient step, starting from the boundary values of the
   previous sweep (specular condition, Fig. riccati_fig_A); form the propagator
   (Eq. riccati_parameterization), sum over energies and Fermi-surface angles
   and keep the sums for sc_gap_update / sc_current / sc_free_energy.  The
   exit values become the next sweep's boundary values. */
sc_status sc_riccati_sweep(sc_ctx *ctx, void *stream);

/* Sweeps with Delta and A frozen until the boundary values change by less
   than tol (max abs) or max_sweeps is reached (burn-in, Sec. 3.1).  Returns
   SC_ENOTCONV if tol was not met; the sweeps are done either way. */
sc_status sc_burnin(sc_ctx *ctx, int32_t max_sweeps, double tol, void *stream);

/* Gap equation in fixed-point form (Eq. gapeq_fixpoint):
   Delta_new(R) = T sum_n <eta f> / (ln t + pi T sum_n 1/|eps_n|), complex nx*ny
   (zero outside the grain).  eps_G (host, may be NULL) = ||Delta_new - Delta||_2 /
   ||Delta||_2 over the grain (Eq. global_error, p = 2); asking for it
   synchronises the stream.  Requires a preceding sc_riccati_sweep. */
sc_status sc_gap_update(sc_ctx *ctx, double *delta_out, double *eps_G, int on_device,
                        void *stream);
/* Residual history (the per-iteration record of the self-consistency loop,
   Algorithm 1): one record per residual eps_G (Eq. global_error) that
   sc_gap_update computed -- every residual check of sc_self_consistency
   included -- oldest first, each with the number of sweeps the context (or its
   batch) had run at that point; the newest 65536 are kept.  *n: in, the
   capacity of `sweeps` and `eps_G` (0 with NULL arrays to ask for the count);
   out, the number of records held (the first min(capacity, count) are
   written).  SC_EINVAL for a NULL context or n, a negative capacity, or a
   positive capacity with a NULL array.  sc_clear_history forgets them. */
sc_status sc_get_history(const sc_ctx *ctx, int32_t *n, int64_t *sweeps, double *eps_G);
sc_status sc_clear_history(sc_ctx *ctx);
/* Charge-current density j(R) = 2 e N_F T sum_n <v_F g> (Eq. current_density),
   vector nx*ny in units of j0. */
sc_status sc_current(sc_ctx *ctx, double *j_out, int on_device, void *stream);
/* Free energy (Eq. qcLWFE with the Eilenberger form of I(R)): density F(R)
   (nx*ny, may be NULL) and F_total = mean over the grain in units of
   Omega_A/area (host, may be NULL; synchronises).  Includes
   (kappa^2/2)|B_ind|^2 when kappa > 0. */
sc_status sc_free_energy(sc_ctx *ctx, double *F_total, double *density_out, int on_device,
                         void *stream);
/* Induced vector potential from the current of the last sweep (App. D):
   A_ind = -(1/kappa^2) sum G (j - <j>), full correlation; becomes the
   context's A_ind.  No-op when kappa <= 0. */
sc_status sc_update_vector_potential(sc_ctx *ctx, void *stream);
/* One Picard step of Algorithm 1 (App. E, alpha = 1): Delta <- Delta_new,
   A_ind <- from j (when kappa > 0). */
sc_status sc_picard_step(sc_ctx *ctx, void *stream);

/* ---- self-consistency accelerators (App. E) ----------------------------
   The unknowns x = (Re Delta, Im Delta, kappa^2 A_x, kappa^2 A_y) (Eq. x_concat;
   Re and Im of every order-parameter component): Delta over the grain's grid
   points, A_ind over the whole grid (only when kappa > 0 is finite).  g(x) = (Delta_new, kappa^2 A from j) of the last sweep,
   d = g(x) - x (Eq. difference).  Each call of sc_accelerate takes one step:
     PICARD            x += alpha d                                  (Eq. picard)
     POLYAK            v = (1 - beta) v + alpha d, x += v; v starts at 0
     BARZILAI_BORWEIN  alpha *= BB1 (odd iterations) or BB2 (even), clamped to
                       [step_size_min, step_size_max]; x += alpha d; the first
                       iteration uses alpha = step_size
     CONGACC           per component c: s = cos(m_c, d_c); alpha_c *= k^s
                       (clamped); w_c = w* with cos(w* m_c + (1-w*) d_c, d_c) =
                       s_min when s < s_min; m_c = w_c m_c + (1 - w_c) d_c;
                       x_c += alpha_c m_c; the first iteration takes m_c = d_c
   The history (velocity, previous d, moving averages, step sizes) lives in the
   context; it restarts when the kind changes, after sc_set_fields and after
   sc_accel_reset.  BB and CongAcc read dot products back to the host, so their
   steps synchronise the stream. */
typedef enum {
    SC_ACC_PICARD = 0,
    SC_ACC_POLYAK = 1,
    SC_ACC_BARZILAI_BORWEIN = 2,
    SC_ACC_CONGACC = 3
} sc_accel_kind;

typedef struct {
    int32_t kind;               /* sc_accel_kind */
    double step_size;           /* alpha (Picard, Polyak); initial alpha (BB, CongAcc); > 0 */
    double drag;                /* Polyak beta, 0 < beta <= 1 */
    double step_size_factor;    /* CongAcc k > 0 */
    double cos_similarity_min;  /* CongAcc s_min in [-1, 1] */
    double step_size_max, step_size_min;  /* BB and CongAcc clamps, 0 < min <= max */
} sc_accel_params;

/* The paper's listing defaults for `kind`: Picard 1.0; Polyak 2.0, drag 0.5;
   BB 1.0 in [0.001, 100]; CongAcc 0.5, k = 1.234, s_min = 0.7, [0.001, 100]. */
sc_status sc_accel_params_default(int32_t kind, sc_accel_params *p);
/* One accelerator step after a sweep; Delta and A_ind of the context are
   replaced by x_{i+1} (the next sweep reads them). */
sc_status sc_accelerate(sc_ctx *ctx, const sc_accel_params *p, void *stream);
/* The self-consistency loop of Algorithm 1 run natively: per iteration a
   sweep, then (every check_every iterations, and at max_iter) the residual
   eps_G of Delta (Eq. global_error, l2) read back and compared with tol, then
   the accelerator step (which updates A_ind when kappa is finite).  Stops
   after the sweep whose residual is below tol (the context then holds those
   fields, their boundary values and outputs) or after max_iter sweeps (no step
   after the last).  iterations and eps_G (may be NULL) receive the sweeps run
   and the last residual read.  Returns SC_OK when converged, SC_ENOTCONV
   otherwise.  Only the residual checks wait for the device. */
sc_status sc_self_consistency(sc_ctx *ctx, const sc_accel_params *p, int32_t max_iter, double tol,
                              int32_t check_every, int32_t *iterations, double *eps_G, void *stream);
sc_status sc_accel_reset(sc_ctx *ctx);
/* Accelerator history: steps taken, step sizes (BB/Picard/Polyak: alpha in
   [0]; CongAcc: alpha_c for c = Re Delta_0, Im Delta_0, ..., Re Delta_{C-1},
   Im Delta_{C-1}, A_x, A_y, i.e. 2 n_components + 2 entries) and CongAcc's
   weights w_c (same layout); alpha and w may be NULL. */
sc_status sc_accel_get_state(const sc_ctx *ctx, int32_t *iterations, double *alpha, double *w);

/* Local density of states N(R, eps)/N_F = -<Im g^R(eps + i broadening)>/pi
   (Sec. 2).  energies: host array of n_e <= 256 real energies that must be symmetric
   about zero (eps_k = -eps_{n_e-1-k}), because gamma~ at eps is taken from
   gamma at -eps (Eq. symmetries).  Boundary values are burnt in with Delta, A
   frozen for up to n_burnin sweeps.  ldos_out: n_e * nx * ny doubles. */
sc_status sc_ldos(sc_ctx *ctx, const double *energies, int32_t n_e, double broadening,
                  int32_t n_burnin, double *ldos_out, int on_device, void *stream);

/* Adjoint of the last sweep (the differentiable form; the paper computes no
   gradients).  Given the cotangents of that sweep's outputs -- dL/dDelta_new
   (complex grid), dL/dj (vector grid), dL/dF(R) (grid), each NULL for zero,
   and the scalar dL/d(F_total) -- it returns dL/dDelta(R) (complex grid) and
   dL/dA_ind(R) (vector grid; may be NULL), with the boundary entry values of
   the differentiated sweep held fixed.  Reverse mode through the closed-form
   steps: per line the forward coherence functions are recomputed and parked
   in device scratch, and the two adjoint chains run against their chains.
   Requires a sweep of the current fields. */
sc_status sc_sweep_adjoint(sc_ctx *ctx, const double *g_delta_new, const double *g_j,
                           const double *g_F, double g_Ftotal, double *dL_ddelta,
                           double *dL_daind, int on_device, void *stream);

/* Adjoint of sc_ldos for an LDOS-map loss: runs the same n_burnin retarded
   sweeps as sc_ldos (boundary values converged with Delta, A frozen), then
   differentiates the last one with its entry values held fixed.  g_ldos:
   dL/dN(R, eps) with the layout of ldos_out (n_e * nx * ny).  Returns
   dL/dDelta(R) (complex grid) and dL/dA_ind(R) (vector grid; may be NULL). */
sc_status sc_ldos_adjoint(sc_ctx *ctx, const double *energies, int32_t n_e, double broadening,
                          int32_t n_burnin, const double *g_ldos, double *dL_ddelta,
                          double *dL_daind, int on_device, void *stream);

/* ---- batched form: many grains in one persistent launch ---------------- */
typedef struct sc_batch sc_batch;
typedef struct {
    int32_t n_grains;
    int32_t n_items;           /* (grain, line group) work items of one sweep */
    int32_t energies_per_lane; /* bound on any member's energies per lane */
    int64_t steps_per_sweep;   /* closed-form steps of one batch sweep, all grains */
    int64_t scratch_bytes;
    double ms_sweep;           /* last batch sweep: its class launches and the sums of energy
                                  blocks and parts (CUDA events on its stream) */
    int64_t lane_steps_per_sweep; /* steps the lanes execute, padded energy slots included */
    int32_t sweep_launches;    /* uniform sweep launches per batch sweep (one per layout class) */
    int32_t class_ept[16];     /* per launch (class, sweep_launches of them): its energies per lane */
    int32_t class_blocks_per_sm[16]; /* per launch: resident blocks per SM its grid is sized for */
    double class_ms[16];       /* per launch: its duration in the last batch sweep */
    int32_t min_lanes_per_line; /* fewest energy lanes per line a member may take */
    int32_t launches_per_iteration; /* kernel launches of one batch iteration with outputs
                                       (sc_batch_run with with_outputs = 1) */
    int32_t split_members;      /* members whose energies run as two parts in their own layouts */
    double split_ms_on, split_ms_off; /* sc_batch_autotune's iteration times with and without
                                         two-part members (0 before it runs) */
    int32_t fused_transfers;    /* 1: the class launches also run the members' rotations and
                                   rotate-backs as work items (sc_batch_set_fused_transfers) */
    int64_t transfer_items;     /* those work items (4 lines, or a tile of 8 x 4 grid points, each) */
    double fuse_ms_on, fuse_ms_off; /* sc_batch_autotune's iteration times with and without them */
    double ms_iteration;        /* last batch sweep from its rotation to its rotate-back (CUDA events) */
} sc_batch_info;

/* Create n member contexts (params[0..n-1], same precision; each validated as
   in sc_create) and one work list over all their (line group) items, longest
   first.  energies_per_lane (1..8; FP32 batches 1..10) bounds the energies
   one lane carries; 0 picks a default; sc_batch_autotune chooses by timing.
   Each member takes the lanes per line (2, 4, 8, 16, 32; at least the batch's
   fewest, 2 unless sc_batch_autotune raises it) and energies per lane (<= the
   bound; 9 and 10 only without energy blocks) with the fewest padded lane
   slots, then the most energies per lane.  After sc_batch_autotune has found
   it faster, an FP32 member whose layout pads its energies runs them as two
   parts, [0, n1) and [n1, n_e), each in its own layout and image (added in
   order after the sweep), where the padded lane slots weighted by the measured
   cost of a lane-step at each energies-per-lane count fall by at least 5 % and
   both parts keep 5 or more energies per lane (132 energies: 2 x 10 and 16 x 7
   instead of 16 x 9).  Members with
   equal energies per lane share one persistent launch; a batch sweep runs
   these launches back to back.  The members are owned by the batch. */
sc_status sc_batch_create(const sc_params *params, int32_t n, int32_t energies_per_lane,
                          sc_batch **out);
sc_status sc_batch_destroy(sc_batch *b);
/* Member context i: set its fields and read its outputs with the sc_* calls
   above; sweeping it alone returns SC_ESTATE (its boundary values are the
   batch's). */
sc_status sc_batch_member(sc_batch *b, int32_t i, sc_ctx **out);
/* One sweep of every member (rotate per member, the persistent sweep launches,
   rotate-back per member); equivalent to sc_riccati_sweep on each member. */
sc_status sc_batch_sweep(sc_batch *b, void *stream);
/* n_sweeps batch sweeps (with_outputs = 1: plus every member's gap update,
   current and free energy on the device), replayed as captured CUDA graphs --
   one graph per iteration parity -- on an internal stream ordered after and
   before `stream`.  The first sweep from fresh boundary values runs uncaptured. */
sc_status sc_batch_run(sc_batch *b, int32_t n_sweeps, int32_t with_outputs, void *stream);
/* FP32 batches: on = 1 lets padded members run their energies as two parts
   (the rule above), 0 keeps every member in one layout; the work list is laid
   out again (captured graphs are dropped).  SC_EINVAL for an FP64 batch with
   on = 1. */
sc_status sc_batch_set_energy_parts(sc_batch *b, int32_t on);
/* FP32 batches: on = 1 runs the members' lattice transfers (Sec. 3.1) inside the
   sweep's class launches: each one-part member's rotation as work items (four
   lines each) of a launch before its own class and its rotate-back (one
   component; tiles of 8 x 4 grid points) of a launch after it, spread evenly
   among that launch's sweep items, so that these gathers, bound by the L1 data
   pipe, share the SMs with the sweep, bound by FP32 arithmetic and its
   latency.  Transfers go to the eligible launch with the least transfer work
   relative to its sweep work, largest first, and never more than that launch's
   sweep work; the rest (and every transfer while some member has energy blocks)
   run in their own launches before and after the sweep.  Results are bit for
   bit those of on = 0 (the same arithmetic in the same order).  The work list
   is laid out again (captured graphs are dropped).  SC_EINVAL for an FP64 batch
   with on = 1. */
sc_status sc_batch_set_fused_transfers(sc_batch *b, int32_t on);
/* Forget every member's boundary coherence functions: the next batch sweep
   starts every trajectory from the local homogeneous solution, as the first
   sweep after sc_batch_create does.  The layout (energies per lane, lanes per
   line, blocks per SM) is kept. */
sc_status sc_batch_reset_boundary(sc_batch *b);
/* Time one batch sweep (rotation to rotate-back) per candidate bound on
   energies per lane (2..8; FP32 2..10) and keep the fastest; then the fewest lanes per line a member may take (2, 4, 8, 16:
   at most 16, 8, 4, 2 lines per warp, which a warp steps as long as its longest);
   then (FP32) the members in two energy parts where that is more than 1 %
   faster, else all in one; then (FP32) the lattice transfers inside the class
   launches (sc_batch_set_fused_transfers) where that is more than 1 % faster;
   then, for that layout, size every class launch's persistent
   grid for each of its occupancy, occupancy - 1 and occupancy - 2 resident blocks
   per SM and keep, per class, the fastest (each class launch timed by its own
   CUDA events).  The timing sweeps are real sweeps (boundary values advance). */
sc_status sc_batch_autotune(sc_batch *b, int32_t *energies_per_lane, void *stream);
sc_status sc_batch_get_info(const sc_batch *b, sc_batch_info *info);
/* Every member's Delta at once (the batch form of sc_set_fields without A_ind):
   delta_all holds the members' complex Delta one after another, member g's
   n_components x ny x nx values (doubles re, im) at the offset of the members
   before it.  on_device = 1: a device pointer, read by one kernel on `stream`;
   0: a host pointer, copied to a device buffer of the batch (allocated on the
   first such call) and the call waits for the copy.  Every member's induced
   vector potential is set to zero.  SC_EINVAL for NULL, SC_ESTATE after a
   failure, SC_ECUDA on a CUDA error. */
sc_status sc_batch_set_fields(sc_batch *b, const double *delta_all, int on_device, void *stream);
/* Every member's Delta_new, j and F(R) of the last batch iteration with outputs
   (sc_batch_run with with_outputs = 1), one after another in the layout of
   sc_batch_set_fields (Delta_new: n_components x ny x nx complex; j: ny x nx x 2;
   F: ny x nx); any of the three may be NULL.  on_device = 1: device pointers,
   filled by one kernel on `stream`; 0: host pointers, through a device buffer of
   the batch (allocated on the first such call), and the call waits.  SC_ESTATE
   when a member has no outputs of its last sweep. */
sc_status sc_batch_get_outputs(sc_batch *b, double *delta_new_all, double *j_all, double *F_all, int on_device,
                               void *stream);

/* ---- inspection (tests and tools) -------------------------------------
 * A "line" is one chord: a maximal piece of a lattice line inside the grain,
 * ordered by pair, lattice line l, then s.  Convex grains have one chord per
 * lattice line; composite grains can have several or none. */
/* per pair l_lo, l_hi (n_pairs each); per line smin, smax, m0, m1 (n_lines) */
sc_status sc_debug_lines(const sc_ctx *ctx, int32_t *l_lo, int32_t *l_hi, double *smin,
                         double *smax, int32_t *m0, int32_t *m1);
/* per line: its pair and lattice line index l (n_lines each; either may be NULL) */
sc_status sc_debug_chords(const sc_ctx *ctx, int32_t *pair, int32_t *l);
/* padded (nx+2)*(ny+2) nearest-grain-point map, -1 where unused */
sc_status sc_debug_ghost(const sc_ctx *ctx, int32_t *ghost);
/* entry links of gamma for every angle k and line (k-major, lines of pair k mod
   n_pairs): 4 taps of (angle, lattice line l of the tapped line, the tapped
   line's index within its pair, weight); any pointer may be NULL */
sc_status sc_debug_links(const sc_ctx *ctx, int32_t *tap_angle, int32_t *tap_line,
                         int32_t *tap_chord, double *tap_w);
/* boundary exit values after the last sweep: complex [angle][line][energy] */
sc_status sc_debug_exits(sc_ctx *ctx, double *exits);
/* per-sample energy sums of the last sweep: [pair][sample][4] = (Re Sf, Im Sf,
   Sg, SF) for angle p (angle p + N/2 follows by symmetry) */
sc_status sc_debug_images(sc_ctx *ctx, double *images);
/* The FP64 reciprocal and reciprocal square root the sweep uses on the device
   (Newton-Raphson iteration from the FP32 approximations, about 1 ulp; arguments
   outside the float range take the IEEE operations), evaluated on n values: x,
   rcp and rsqrt are device pointers to n doubles (caller-owned); the call waits
   for the stream.  SC_EINVAL for n < 0 or a null pointer with n > 0, SC_ECUDA
   for a failed launch (message in sc_last_error(NULL)). */
sc_status sc_debug_fp64_math(const double *x, int64_t n, double *rcp, double *rsqrt, void *stream);
/* Measured FP32 fused multiply-add rate of this GPU (no counterpart in the paper;
   the measured side of the sweep's roofline): lane operations per second of a
   launch of 8 blocks of 256 threads per SM, each thread running eight independent
   chains of 100000 FMAs -- scalar (packed = 0) or two-wide fma.rn.f32x2, two lane
   operations per instruction (packed != 0).  Allocates and frees a small output
   buffer and waits for the stream.  SC_EINVAL for a NULL pointer, SC_ECUDA on a
   CUDA error (message in sc_last_error(NULL)). */
sc_status sc_debug_fma_rate(int32_t packed, double *lane_ops_per_s, void *stream);

/* ---- index checks ------------------------------------------------------
 * Engineering aids with no counterpart in the paper (the checks that stand in
 * for a memory checker).
 *
 * sc_debug_validate_tables: checks, on the host, every index of the context's
 * sweep tables against the size of the table it points into -- each line's
 * image slots and its rows of the exit buffers, the exit slots of its 4 + 4
 * boundary taps, each pair's lines and lattice-line records, the lattice
 * lines' chord ranges -- and stores the number of bad entries in *n_bad (0 for
 * every table sc_create builds; sc_create itself refuses a context whose
 * tables fail).  Works on host_only contexts.  SC_EINVAL for NULL arguments.
 *
 * sc_debug_corrupt_table: for tests of that validation only, and only on a
 * host_only context (whose tables never reach a GPU): makes one index of the
 * host tables out of range -- which = 0 a line's first image slot, 1 a
 * boundary tap's exit slot, 2 a pair's first lattice-line record.  SC_ESTATE
 * on a context with device memory, SC_EINVAL for another `which`.
 *
 * sc_debug_bounds: the kernels' index-check violations on the current device
 * since the last reset (reset != 0 clears them after reading) and, in
 * *checked_build, 1 when this library was compiled with the checks
 * (libsc_checked.so, -DSC_DEBUG_BOUNDS; a failed check skips the access and
 * counts), 0 for the regular build, whose count is always 0.  Waits for the
 * device.  SC_EINVAL for NULL pointers, SC_ECUDA when the counters cannot be
 * read (message in sc_last_error(NULL)). */
sc_status sc_debug_validate_tables(const sc_ctx *ctx, int64_t *n_bad);
sc_status sc_debug_corrupt_table(sc_ctx *ctx, int32_t which);
sc_status sc_debug_bounds(uint64_t *violations, int32_t *checked_build, int32_t reset);

/* ---- allocation-free line sweep ---------------------------------------
 * No counterpart in the paper: an engineering entry point for callers that
 * must not allocate device memory when they run a sweep -- code whose device
 * heap is owned by another allocator or memory pool, real-time loops that
 * cannot afford the implicit synchronisation of cudaMalloc/cudaFree, or hosts
 * that reserve all device memory up front.  It needs no sc_ctx and allocates
 * nothing: the caller passes every input and output as a device pointer, and
 * the only scratch (the forward coherence functions parked between the two
 * passes of a line) lives in a static 32 MiB device array inside the library,
 * which every GPU that loads the library holds until the process exits.
 *
 * FP32 sweep of n_lines independent lines, both directions, at the positive
 * Matsubara energies eps_n = t (n + 1/2), n < n_e (the same step, propagator
 * and energy sums as sc_riccati_sweep; one warp per line, energies on lanes).
 *   samples     [n_slots][4] floats: Re(Delta eta), Im(Delta eta), a = sigma v.A
 *               at each lattice sample, lines stored one after another
 *               (a line with no sample has one slot: the chord-midpoint value)
 *   line_slot0  [n_lines] first slot of each line;  line_ns [n_lines] samples
 *               on the line (0 <= line_ns <= max_ns; longer lines are skipped and
 *               their exits set to NaN)
 *   line_len    [n_lines][2] floats: lengths from the chord start to the first
 *               sample and from the last sample to the chord end (both the chord
 *               length when line_ns = 0)
 *   entry       [2][n_lines][n_e] complex floats: gamma entering at the chord
 *               start (+ direction) and at the chord end (- direction); NULL =
 *               start from the local homogeneous solution
 *   images out  [n_slots][4] floats per sample: (Re Sf, Im Sf, Sg, SF) of the +
 *               direction, as sc_debug_images reports them
 *   exits out   [2][n_lines][n_e] complex floats: gamma leaving at the chord end
 *               (+) and at the chord start (-)
 * Limits: n_e <= 256 and max(max_ns, 1) * 32 * ceil(n_e / 32) <= 4 Mi
 * (SC_EINVAL otherwise, with the reason in sc_last_error(NULL)).
 * The first call on each device looks up the device address of the static
 * array (cudaGetSymbolAddress) and loads the kernels of all eight energy
 * layouts (ceil(n_e / 32) = 1..8), so that no later call loads code or
 * allocates, whatever its n_e; make that first call before any stream capture.
 * Every call uses the same array and leaves its contents behind; nothing in it
 * needs to start at zero.  Calls whose kernels overlap on the GPU (different
 * streams, or several host threads) race on the array: serialise them.
 * SC_ECUDA without a launch when a CUDA error from earlier work is already
 * pending on the calling thread (the error is left for its owner). */
sc_status sc_sweep_lines_noalloc(const float *samples, const int32_t *line_slot0,
                                 const int32_t *line_ns, const float *line_len,
                                 const float *entry, int32_t n_lines, int32_t max_ns,
                                 int32_t n_e, double t, double h, float *images,
                                 float *exits, void *stream);

const char *sc_last_error(const sc_ctx *ctx);
const char *sc_version(void);

#ifdef __cplusplus
}
#endif
#endif
