/*
 * Plain FP64 CPU oracle of the quasiclassical Riccati sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library includes, links or
 * calls this code; only the tests, the package's smoke() check and the CPU
 * baseline leg of bench.py use it.  It shares no code with the CUDA path.
 *
 * Every function follows the paper (Holmvall et al., "SuperConga", arXiv
 * 2205.15000) step by step in plain double-precision C:
 *   - order parameter Delta(p,R) = Delta(R) eta(p)             (Eq. order_parameter)
 *   - Fermi-surface quadrature by Boole / Simpson 3/8 / 1/3 / trapezoid
 *                                                              (Sec. 3.1, main algorithm)
 *   - Riccati equations for gamma and gamma~                   (Eqs. riccati, riccati_tilde)
 *     integrated with the closed-form step for piecewise-constant
 *     coefficients (the "stepping method" of App. C) or with the
 *     implicit midpoint rule                                    (App. C, Eq. riccati_midpoint)
 *   - propagator from the coherence functions                  (Eq. riccati_parameterization)
 *   - gap equation in fixed-point form                         (Eq. gapeq_fixpoint)
 *   - current density                                          (Eq. current_density)
 *   - Eilenberger free-energy functional                       (Eq. qcLWFE, Eilenberger form)
 *   - induced vector potential via the 2D Green's function     (App. D)
 *   - local density of states                                  (Sec. 2, LDOS definition)
 * Units: lengths xi0, energies 2 pi kB Tc, A in Phi0/(pi xi0), j in j0.
 * Grid arrays are row-major [ny][nx]; complex and 2-vector grids interleave
 * their two components per point.  With several order-parameter components,
 * Delta and Delta_new are [n_components][ny][nx] complex, and the mode-0
 * accumulators gain two planes per component beyond the first.
 */
#ifndef SC_ORACLE_H
#define SC_ORACLE_H
#include <stdint.h>

/* One part of a composite grain (Sec. 4, composite geometries): a disc or a
   convex polygon whose area is added to, or removed from, the grain built by
   the parts before it. */
typedef struct {
    int32_t kind;            /* 0 = disc, 1 = convex polygon (CCW vertices) */
    int32_t add;             /* 1 = add the area, 0 = remove it */
    double cx, cy, r;        /* disc centre and radius */
    int32_t n_vert;
    const double *vx, *vy;
} or_part;

typedef struct {
    int32_t nx, ny;          /* grid points; point (i,j) at (x0+(i+.5)h, y0+(j+.5)h) */
    double h, x0, y0;
    int32_t shape_kind;      /* 0 = disc, 1 = convex polygon (CCW vertices),
                                2 = composite: the parts below, in order */
    double disc_cx, disc_cy, disc_r;
    int32_t n_vert;
    const double *vx, *vy;
    int32_t pairing;         /* 0 s, 1 d_{x2-y2}, 2 d_xy, 3 g */
    double crystal_rotation; /* units of 2 pi */
    double t;                /* T / Tc */
    double flux_quanta;      /* alpha: symmetric / landau gauge, B_ext * area / Phi0;
                                solenoid gauge, flux threading the hole / Phi0 */
    double gauge_cx, gauge_cy; /* gauge origin (solenoid: the flux line) */
    double kappa;            /* <= 0 : no induced A */
    int32_t charge_sign;     /* +1 / -1 */
    int32_t n_angles;        /* even */
    int32_t n_energies;      /* positive Matsubara energies */
    double lattice_ox, lattice_oy; /* lattice origin offset from the grid centre, units of h */
    int32_t stepper;         /* 0 = closed-form step for piecewise-constant coefficients,
                                1 = implicit midpoint rule (App. C, Eq. riccati_midpoint) */
    int32_t n_components;    /* order-parameter components Delta_Gamma (Eq. order_parameter):
                                0 or 1 = one (`pairing`), at most 4 */
    int32_t pairings[4];     /* basis of component c >= 1 (component 0 uses `pairing`) */
    double tc_ratios[4];     /* T_c^Gamma / T_c of each component (0 means 1) */
    int32_t n_parts;         /* composite grain (shape_kind 2) */
    const or_part *parts;
    int32_t gauge;           /* external vector potential: 0 symmetric B/2 (-y, x),
                                1 landau B (-y, 0), 2 solenoid alpha/(2 r^2) (-y, x)
                                (Eq. solenoid_gauge), all about the gauge origin */
} or_params;

typedef struct or_geom or_geom;

const char *or_last_error(void);

or_geom *or_geom_create(const or_params *p);
void or_geom_free(or_geom *g);

/* info[0]=n_pairs info[1]=total chords over pairs info[2]=total samples over pairs
   info[3]=n_in (mask points) info[4]=total lines over all angles (= 2*info[1])
   info[5]=total samples over all angles (= 2*info[2]) */
int or_geom_info(const or_geom *g, int64_t *info);
double or_geom_area(const or_geom *g);
int or_geom_mask(const or_geom *g, uint8_t *mask);
int or_geom_ghost(const or_geom *g, int32_t *ghost);  /* (nx+2)*(ny+2), -1 where unused */
/* A "line" below is one chord: a maximal piece of a lattice line inside the
   grain.  Convex grains have one chord per lattice line; composite grains can
   have several (ordered by s) or none.
   per pair: l_lo, l_hi; per chord (pair-major, then l, then s): smin, smax, m0, m1 */
int or_geom_lines(const or_geom *g, int32_t *l_lo, int32_t *l_hi, double *smin,
                  double *smax, int32_t *m0, int32_t *m1);
/* per chord: its pair and lattice line index l */
int or_geom_chords(const or_geom *g, int32_t *pair, int32_t *l);
/* entry links of gamma, [angle][chord][4]: tap angle, lattice line l of the tapped
   chord, the tapped chord's index within its pair, weight */
int or_geom_links(const or_geom *g, int32_t *tap_angle, int32_t *tap_line, int32_t *tap_chord,
                  double *tap_w);
/* external vector potential of the gauge at n points (xy: [n][2], A: [n][2]) */
int or_external_a(const or_geom *g, int n, const double *xy, double *A);
int or_geom_quadrature(const or_geom *g, double *w, double *vhat, double *eta);

/* Closed-form step of d gamma/ds = i (P g^2 + 2 Q g + R) over a length ell. */
void or_step(const double *P, const double *Q, const double *R, double ell,
             const double *ga, double *gb);

/* Implicit midpoint step (App. C) of the same equation over a length ell:
   gb = ga + ell i (P m^2 + 2 Q m + R) with m = (ga + gb)/2, solved as a quadratic. */
void or_step_midpoint(const double *P, const double *Q, const double *R, double ell,
                      const double *ga, double *gb);

/* Fields sampled on the rotated lattice of one pair: delta (complex, without eta)
   and A_total (vector) at every sample, canonical order (line, m). */
int or_sample_fields(const or_geom *g, const double *delta, const double *aind, int pair,
                     double *delta_s, double *a_vec_s);

/* One sweep over all angles, lines and energies.
   z: complex energies (2*n_e doubles), without the vector-potential term.
   mode 0 (Matsubara sums, z = i eps_n): images [angle][sample][4] = (Re Sf, Im Sf, Sg, SF)
   mode 1 (retarded, LDOS): images [angle][sample][n_e] = -Im g / pi
   exit_in: NULL (fresh boundary) or [2][angle][line][n_e] complex from the previous sweep
   exit_out: same layout; [0] gamma at the exit end, [1] gamma~ at the entry end.
   gam_out (optional, may be NULL): [2][angle][sample][n_e] complex gamma, gamma~ at samples. */
int or_sweep(const or_geom *g, const double *delta, const double *aind, const double *z,
             int n_e, int mode, const double *exit_in, double *exit_out, double *images,
             double *gam_out);

/* Rotate the per-angle images back to the reference grid and take the FS average.
   mode 0: acc [5][nx*ny] = sum_k w_k {eta_k Re Sf, eta_k Im Sf, vx_k Sg, vy_k Sg, SF}
   mode 1: acc [n_e][nx*ny] = sum_k w_k X_k   (X from the n_e per-sample values) */
int or_rotate_back(const or_geom *g, const double *images, int mode, int n_e, double *acc);

double or_norm_D(double t, int n_e);
/* Weighted energy sums (Ozaki's poles, Sec. 3.1): the mode-0 images sum
   w[n] * (terms of energy n) and the outputs use normD as the gap-equation
   normalisation; w = NULL restores unit weights and the Matsubara D. */
int or_geom_set_energy_weights(or_geom *g, const double *w, int n_e, double normD);

/* Outputs from the mode-0 accumulators. delta_new: complex grid; j: [nx*ny][2];
   F: density grid; scalars[0]=F/Omega_A (mean over mask), scalars[1]=eps_G (l2). */
int or_outputs(const or_geom *g, const double *acc, const double *delta, const double *aind,
               double *delta_new, double *j, double *F, double *scalars);

/* First sweep (homogeneous entries) for the listed angles only; images are
   packed [selected angle][samples of its pair][4] (mode-0 sums). */
int or_sweep_subset(const or_geom *g, const double *delta, const double *aind, const double *z,
                    int n_e, const int *angles, int n_sel, double *images);

double or_greens(int m, int n, double h);
/* A_ind = -(1/kappa^2) sum G (j - mean_mask j); direct double sum. j, aind: [nx*ny][2]. */
int or_vector_potential(const or_geom *g, const double *j, double *aind);
/* Bulk gap from the truncated regularised gap equation (bisection). */
double or_bulk_gap(int pairing, double t, int n_e, int n_angles);
double or_quad_weight(int k, int n);
#endif
