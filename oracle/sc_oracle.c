/*
 * Plain FP64 CPU oracle of the quasiclassical Riccati sweep (SuperConga,
 * arXiv 2205.15000).  TEST INFRASTRUCTURE ONLY: only tests/, the package's
 * smoke() check and bench.py's CPU-baseline leg may load it.  It shares no
 * code, header, table or constant generator with the CUDA path.
 *
 * The code is deliberately plain: loops in the order the method states them,
 * C99 complex doubles, no blocking or fusion.  OpenMP only splits independent
 * (angle, line) work and grid points.
 *
 * Discretisation (the paper leaves the details open; each reading is listed in
 * the repository's design notes and repeated here where it is applied):
 *   grid       point (i,j) at (x0+(i+1/2)h, y0+(j+1/2)h); mask = centre inside
 *              the shape, with points on the boundary counted inside.
 *   angles     phi_k = 2 pi k / N; pair p < N/2 owns a rotated square lattice
 *              with spacing h (Sec. 3.1): line l is O + l h e_perp + s e_par,
 *              samples at s = m h.  Angle p+N/2 uses the same lines, run in
 *              the opposite direction (its direction vector is exactly -e_par).
 *   chord      exact intersection with the disc / convex polygon; samples
 *              ceil(smin/h) .. floor(smax/h).
 *   segments   end segments take the nearest sample's value, interior segments
 *              the mean of their two samples (App. C: linear interpolation to
 *              the half step, nearest-neighbour extrapolation at the boundary).
 *   step       exact solution of the Riccati equation with constant
 *              coefficients over each segment (the stepping method, App. C).
 *   boundary   specular: the entry value is the exit value of the reflected
 *              incoming trajectory, bilinear in (angle, line coordinate)
 *              (Sec. 3.1 and Fig. riccati_fig_A).
 *   average    per-angle images are interpolated back to the grid (bilinear)
 *              and summed with the quadrature weights (Sec. 3.1).
 */
#define _GNU_SOURCE
#include "sc_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* Tolerance (units of h) for the robust geometric decisions of the
   discretisation: inside test, chord existence, sample inclusion and the
   choice of the active polygon edge. */
#define TAU 1e-9

static __thread char g_err[512];
const char *or_last_error(void) { return g_err; }
static int fail(const char *msg) {
    snprintf(g_err, sizeof g_err, "%s", msg);
    return -1;
}

/* One part of the grain: a disc or a convex polygon, added or removed. */
typedef struct {
    int kind, add;          /* 0 disc, 1 convex polygon; 1 add, 0 remove */
    double cx, cy, r;       /* disc */
    int nv;                 /* polygon: CCW vertices and unit outward edge normals */
    double *vx, *vy, *nx, *ny;
} o_part;

/* A chord end lies on the boundary of one part: the part, its polygon edge
   (-1 for a disc), and +1 if the grain lies on the inner side of that
   boundary (an added part) or -1 if on its outer side (a removed part). */
typedef struct {
    int part, edge, sign;
} o_tag;

struct or_geom {
    or_params P;
    int nparts;
    o_part *parts;          /* a lone disc or polygon is one added part */
    uint8_t *mask;
    int32_t *ghost;         /* padded (nx+2)*(ny+2) */
    int64_t n_in;
    double area;
    double Ox, Oy;
    int npair, N;
    double *w;              /* [N] quadrature weights */
    double *vh;             /* [N][2] Fermi velocity directions */
    double *eta;            /* [N] basis function of component 0 (= eta_c) */
    double *eta_c;          /* [C][N] basis functions of the components */
    int C;                  /* order-parameter components */
    double tcr[4];          /* T_c^Gamma / T_c */
    double *ewt;            /* [n_energies] weights of the energy sums, NULL = 1 (Matsubara) */
    double normD;           /* gap-equation normalisation when ewt is set */
    /* per pair: lattice lines l_lo..l_hi; chords line_off[p]..line_off[p+1]-1;
       lattice-line records lat_off[p]..; samples samp_off[p].. */
    int *l_lo, *l_hi, *line_off, *samp_off, *lat_off;
    /* per lattice line: its chords lat_c0 .. lat_c0+lat_nc-1 (ascending s), the
       nearest lattice line of the pair that has a chord (lat_chorded) and one
       that has a chord with samples (lat_near), as line indices l */
    int *lat_c0, *lat_nc, *lat_chorded, *lat_near;
    /* per chord (pair-major, then l, then s) */
    int *ch_pair, *ch_l;
    double *smin, *smax;
    o_tag *tag_lo, *tag_hi;
    int *m0, *m1, *ns, *soff; /* soff: sample offset within the pair */
    /* links per angle: [N][chords of the pair][4]: tap angle, tap chord (global index) */
    int *lk_g_angle, *lk_g_line;
    double *lk_g_w;
    int *lk_t_angle, *lk_t_line;
    double *lk_t_w;
    int64_t *ang_line_off;   /* [N+1] cumulative chord counts over angles */
    int64_t *ang_samp_off;   /* [N+1] cumulative sample counts over angles */
};

/* ---------------------------------------------------------------------- */
/* Fermi surface: quadrature weights (Sec. 3.1: Boole, Simpson 3/8,       */
/* Simpson 1/3 or trapezoid by divisibility of N by 4, 3, 2, else),       */
/* composite rule closed on the periodic grid and normalised to sum 1.    */
/* ---------------------------------------------------------------------- */
double or_quad_weight(int k, int n) {
    if (n % 4 == 0) {
        static const double c[4] = {14.0, 32.0, 12.0, 32.0}; /* Boole 7,32,12,32,7 */
        return 2.0 * c[k % 4] / (45.0 * n);
    } else if (n % 3 == 0) {
        static const double c[3] = {2.0, 3.0, 3.0};          /* Simpson 3/8: 1,3,3,1 */
        return 3.0 * c[k % 3] / (8.0 * n);
    } else if (n % 2 == 0) {
        static const double c[2] = {2.0, 4.0};               /* Simpson 1/3: 1,4,1 */
        return c[k % 2] / (3.0 * n);
    }
    return 1.0 / n;
}

/* Basis functions of Table basis_functions for a circular Fermi surface,
   evaluated at the direction (c, s) rotated by -2 pi * crystal_rotation. */
static double basis_eta(int pairing, double rot, double c, double s) {
    double th = 2.0 * M_PI * rot;
    double cr = c * cos(th) + s * sin(th);
    double sr = -c * sin(th) + s * cos(th);
    double c2 = cr * cr - sr * sr;  /* cos 2 phi */
    double s2 = 2.0 * cr * sr;      /* sin 2 phi */
    switch (pairing) {
    case 0: return 1.0;
    case 1: return sqrt(2.0) * c2;
    case 2: return sqrt(2.0) * s2;
    case 3: return sqrt(2.0) * 2.0 * s2 * c2; /* sin 4 phi */
    }
    return 0.0;
}

/* Normalisation of the fixed-point gap equation (Eq. gapeq_fixpoint), in
   units of 2 pi kB Tc with eps_n = t (n + 1/2):  ln t + pi T sum_n 1/|eps_n|
   = ln t + 2 sum_{n<Ne} 1/(2n+1). */
int or_geom_set_energy_weights(or_geom *g, const double *w, int n_e, double normD) {
    if (!g || n_e != g->P.n_energies) return 1;
    free(g->ewt);
    g->ewt = NULL;
    if (w) {
        g->ewt = malloc(sizeof(double) * n_e);
        for (int n = 0; n < n_e; ++n) g->ewt[n] = w[n];
        g->normD = normD;
    }
    return 0;
}

double or_norm_D(double t, int n_e) {
    double s = 0.0;
    for (int n = 0; n < n_e; ++n) s += 1.0 / (2.0 * n + 1.0);
    return log(t) + 2.0 * s;
}

/* ---------------------------------------------------------------------- */
/* Geometry.  A grain is built by adding and removing discs and convex    */
/* polygons in the listed order (Sec. 4 and App. B, composite             */
/* geometries); a lone disc or polygon is the composite of one added part. */
/* ---------------------------------------------------------------------- */
/* signed distance of one part (negative inside) */
static double part_sdist(const o_part *q, double x, double y) {
    if (q->kind == 0) {
        double dx = x - q->cx, dy = y - q->cy;
        return sqrt(dx * dx + dy * dy) - q->r;
    }
    double d = -INFINITY;
    for (int e = 0; e < q->nv; ++e) {
        double v = (x - q->vx[e]) * q->nx[e] + (y - q->vy[e]) * q->ny[e];
        if (v > d) d = v;
    }
    return d;
}

/* signed distance of the grain: the union takes the minimum, the removal of
   a part the maximum with the part's negated distance */
static double sdist(const or_geom *g, double x, double y) {
    double d = INFINITY;
    for (int k = 0; k < g->nparts; ++k) {
        double dk = part_sdist(&g->parts[k], x, y);
        if (g->parts[k].add) {
            if (dk < d) d = dk;
        } else if (-dk > d) {
            d = -dk;
        }
    }
    return d;
}

/* Interval of the line B + s*e inside one part: returns 0 if it is empty or
   not longer than tol.  For a polygon, e0/e1 are the entering / leaving
   edges: the lowest index whose bound is within tol of the extremum. */
static int part_chord(const o_part *q, double bx, double by, double ex, double ey, double tol,
                      double *smin, double *smax, int *elo, int *ehi) {
    *elo = *ehi = -1;
    if (q->kind == 0) {
        double dx = bx - q->cx, dy = by - q->cy;
        double b = dx * ex + dy * ey;
        double c = dx * dx + dy * dy - q->r * q->r;
        double disc = b * b - c;
        if (disc <= 0.0) return 0;
        double r = sqrt(disc);
        *smin = -b - r;
        *smax = -b + r;
    } else {
        double lo = -INFINITY, hi = INFINITY;
        int n = q->nv;
        double *bound = malloc(sizeof(double) * n);
        int *kind = malloc(sizeof(int) * n);
        for (int e = 0; e < n; ++e) {
            double f0 = (bx - q->vx[e]) * q->nx[e] + (by - q->vy[e]) * q->ny[e];
            double ge = ex * q->nx[e] + ey * q->ny[e];
            kind[e] = 0;
            if (ge > 0.0) {           /* leaving through edge e at s = -f0/ge */
                bound[e] = -f0 / ge;
                kind[e] = 1;
                if (bound[e] < hi) hi = bound[e];
            } else if (ge < 0.0) {    /* entering through edge e */
                bound[e] = -f0 / ge;
                kind[e] = -1;
                if (bound[e] > lo) lo = bound[e];
            } else if (f0 > 0.0) {    /* parallel and outside */
                free(bound);
                free(kind);
                return 0;
            }
        }
        for (int e = 0; e < n && *elo < 0; ++e)
            if (kind[e] == -1 && bound[e] >= lo - tol) *elo = e;
        for (int e = 0; e < n && *ehi < 0; ++e)
            if (kind[e] == 1 && bound[e] <= hi + tol) *ehi = e;
        free(bound);
        free(kind);
        *smin = lo;
        *smax = hi;
    }
    return (*smax - *smin) > tol;
}

/* The chords of the line B + s*e: the maximal intervals of s inside the
   grain, ascending, built part by part in order (union with an added part's
   interval, difference with a removed part's).  Part intervals not longer
   than tol are ignored; intervals that overlap or touch within tol merge; a
   difference leaves only pieces longer than tol, and a removed interval that
   overlaps a chord by no more than tol leaves it whole.  On equal ends the
   earlier part keeps the end.  Arrays hold 2 * nparts + 1 entries. */
static int comp_chords(const or_geom *g, double bx, double by, double ex, double ey, double tol,
                       double *lo, double *hi, o_tag *tlo, o_tag *thi) {
    int n = 0;
    for (int k = 0; k < g->nparts; ++k) {
        const o_part *q = &g->parts[k];
        double a, b;
        int ea, eb;
        if (!part_chord(q, bx, by, ex, ey, tol, &a, &b, &ea, &eb)) continue;
        o_tag ta = {k, ea, q->add ? 1 : -1}, tb = {k, eb, q->add ? 1 : -1};
        if (q->add) {
            int first = -1, last = -1;
            for (int i = 0; i < n; ++i)
                if (lo[i] <= b + tol && hi[i] >= a - tol) {
                    if (first < 0) first = i;
                    last = i;
                }
            if (first < 0) {
                int pos = 0;
                while (pos < n && lo[pos] < a) ++pos;
                for (int i = n; i > pos; --i) {
                    lo[i] = lo[i - 1];
                    hi[i] = hi[i - 1];
                    tlo[i] = tlo[i - 1];
                    thi[i] = thi[i - 1];
                }
                lo[pos] = a;
                hi[pos] = b;
                tlo[pos] = ta;
                thi[pos] = tb;
                ++n;
            } else {
                if (a < lo[first]) {
                    lo[first] = a;
                    tlo[first] = ta;
                }
                if (b > hi[last]) {
                    hi[first] = b;
                    thi[first] = tb;
                } else {
                    hi[first] = hi[last];
                    thi[first] = thi[last];
                }
                int gone = last - first;
                for (int i = first + 1; i + gone < n; ++i) {
                    lo[i] = lo[i + gone];
                    hi[i] = hi[i + gone];
                    tlo[i] = tlo[i + gone];
                    thi[i] = thi[i + gone];
                }
                n -= gone;
            }
        } else {
            double nlo[n + 1], nhi[n + 1];
            o_tag ntl[n + 1], nth[n + 1];
            int m = 0;
            for (int i = 0; i < n; ++i) {
                if (hi[i] <= a + tol || lo[i] >= b - tol) {
                    nlo[m] = lo[i];
                    nhi[m] = hi[i];
                    ntl[m] = tlo[i];
                    nth[m] = thi[i];
                    ++m;
                    continue;
                }
                if (a - lo[i] > tol) {
                    nlo[m] = lo[i];
                    nhi[m] = a;
                    ntl[m] = tlo[i];
                    nth[m] = ta;
                    ++m;
                }
                if (hi[i] - b > tol) {
                    nlo[m] = b;
                    nhi[m] = hi[i];
                    ntl[m] = tb;
                    nth[m] = thi[i];
                    ++m;
                }
            }
            for (int i = 0; i < m; ++i) {
                lo[i] = nlo[i];
                hi[i] = nhi[i];
                tlo[i] = ntl[i];
                thi[i] = nth[i];
            }
            n = m;
        }
    }
    return n;
}

/* outward normal of the grain at a chord end */
static void end_normal(const or_geom *g, o_tag t, double px, double py, double *nx, double *ny) {
    const o_part *q = &g->parts[t.part];
    if (q->kind == 0) {
        double dx = px - q->cx, dy = py - q->cy;
        double r = sqrt(dx * dx + dy * dy);
        *nx = t.sign * dx / r;
        *ny = t.sign * dy / r;
    } else {
        *nx = t.sign * q->nx[t.edge];
        *ny = t.sign * q->ny[t.edge];
    }
}

/* lattice-line record of line l of pair p */
static inline int glat(const or_geom *g, int p, int l) { return g->lat_off[p] + (l - g->l_lo[p]); }

/* Bilinear link: boundary values of the angles bracketing direction (ux,uy),
   on the lattice lines bracketing point (px,py), which lies on the boundary
   of part `part`.  The value is taken at each tapped chord's exit end (in
   that angle's direction of travel) for gamma, which runs along the travel,
   and at its entry end for gamma~ (at_entry = 1), which runs against it.  A
   line index outside the pair's range is clamped; a line without chords is
   replaced by the nearest one with chords.  On each line the candidates are
   the chords whose end of interest lies on the same part, and the one whose
   end lies nearest to the point along the line is taken; a line without a
   candidate (it passes the part, e.g. beside a hole) gives its weight to the
   other line's chord, and when neither line has one the nearest end of any
   part is taken.  Writes 4 taps (angle, global chord index, weight). */
static void make_link(const or_geom *g, double px, double py, double ux, double uy, int part,
                      int at_entry, int *ta, int *tl, double *tw) {
    int N = g->N;
    double psi = atan2(uy, ux);
    if (psi < 0.0) psi += 2.0 * M_PI;
    double u = psi * N / (2.0 * M_PI);
    int j0 = (int)floor(u);
    double wa = u - j0;
    if (j0 >= N) j0 -= N;
    if (j0 < 0) j0 += N;
    int js[2] = {j0, (j0 + 1) % N};
    double was[2] = {1.0 - wa, wa};
    for (int a = 0; a < 2; ++a) {
        int j = js[a];
        int p = j % g->npair;
        double epx = -g->vh[2 * p + 1], epy = g->vh[2 * p]; /* e_perp of the pair */
        double c = ((px - g->Ox) * epx + (py - g->Oy) * epy) / g->P.h;
        double sp = (px - g->Ox) * g->vh[2 * p] + (py - g->Oy) * g->vh[2 * p + 1];
        int i0 = (int)floor(c);
        double wl = c - i0;
        int ls[2] = {i0, i0 + 1};
        double wls[2] = {1.0 - wl, wl};
        int pick[2], same[2];
        for (int b = 0; b < 2; ++b) {
            int l = ls[b];
            if (l < g->l_lo[p]) l = g->l_lo[p];
            if (l > g->l_hi[p]) l = g->l_hi[p];
            l = g->lat_chorded[glat(g, p, l)];
            int lat = glat(g, p, l);
            int best_any = -1, best_same = -1;
            double d_any = INFINITY, d_same = INFINITY;
            for (int q = 0; q < g->lat_nc[lat]; ++q) {
                int L = g->lat_c0[lat] + q;
                int hi_end = (j < g->npair) != (at_entry != 0);  /* the end at smax? */
                double se = hi_end ? g->smax[L] : g->smin[L];
                int ep = hi_end ? g->tag_hi[L].part : g->tag_lo[L].part;
                double d = fabs(se - sp);
                if (d < d_any) {
                    d_any = d;
                    best_any = L;
                }
                if (ep == part && d < d_same) {
                    d_same = d;
                    best_same = L;
                }
            }
            same[b] = best_same >= 0;
            pick[b] = same[b] ? best_same : best_any;
        }
        if (same[0] && !same[1]) pick[1] = pick[0];
        if (same[1] && !same[0]) pick[0] = pick[1];
        for (int b = 0; b < 2; ++b) {
            ta[2 * a + b] = j;
            tl[2 * a + b] = pick[b];
            tw[2 * a + b] = was[a] * wls[b];
        }
    }
}

/* the chord with samples of lattice record `lat` nearest to the lattice
   coordinate v (units of h) along the line: distance from v to [m0, m1];
   ties to the chord of lower s */
static int pick_sampled_chord(const or_geom *g, int lat, double v) {
    int best = -1;
    double bd = INFINITY;
    for (int q = 0; q < g->lat_nc[lat]; ++q) {
        int L = g->lat_c0[lat] + q;
        if (g->ns[L] < 1) continue;
        double d = 0.0;
        if (v < g->m0[L]) d = g->m0[L] - v;
        else if (v > g->m1[L]) d = v - g->m1[L];
        if (d < bd) {
            bd = d;
            best = L;
        }
    }
    return best;
}

static double polygon_area(int n, const double *x, const double *y) {
    double s = 0.0;
    for (int e = 0; e < n; ++e) {
        int f = (e + 1) % n;
        s += x[e] * y[f] - x[f] * y[e];
    }
    return 0.5 * s;
}

/* y of the points where the boundaries of parts a and b cross (appended) */
static int crossings_y(const o_part *a, const o_part *b, double *ys) {
    int n = 0;
    if (a->kind == 0 && b->kind == 0) {
        double dx = b->cx - a->cx, dy = b->cy - a->cy, d = sqrt(dx * dx + dy * dy);
        if (d == 0.0 || d > a->r + b->r || d < fabs(a->r - b->r)) return 0;
        double s = (a->r * a->r - b->r * b->r + d * d) / (2.0 * d);
        double hh = a->r * a->r - s * s;
        hh = hh > 0.0 ? sqrt(hh) : 0.0;
        ys[n++] = a->cy + s * dy / d + hh * dx / d;
        ys[n++] = a->cy + s * dy / d - hh * dx / d;
        return n;
    }
    if (a->kind == 1 && b->kind == 0) return crossings_y(b, a, ys);
    if (a->kind == 0) { /* circle a, polygon b: |P0 + t D - c|^2 = r^2 on each edge */
        for (int e = 0; e < b->nv; ++e) {
            int f = (e + 1) % b->nv;
            double Dx = b->vx[f] - b->vx[e], Dy = b->vy[f] - b->vy[e];
            double fx = b->vx[e] - a->cx, fy = b->vy[e] - a->cy;
            double A = Dx * Dx + Dy * Dy, B = 2.0 * (fx * Dx + fy * Dy), C = fx * fx + fy * fy - a->r * a->r;
            double disc = B * B - 4.0 * A * C;
            if (disc < 0.0) continue;
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                double t = (-B + sgn * sqrt(disc)) / (2.0 * A);
                if (t >= 0.0 && t <= 1.0) ys[n++] = b->vy[e] + t * Dy;
            }
        }
        return n;
    }
    for (int e = 0; e < a->nv; ++e) { /* two polygons: edge against edge */
        int f = (e + 1) % a->nv;
        double rx = a->vx[f] - a->vx[e], ry = a->vy[f] - a->vy[e];
        for (int k = 0; k < b->nv; ++k) {
            int m = (k + 1) % b->nv;
            double sx = b->vx[m] - b->vx[k], sy = b->vy[m] - b->vy[k];
            double den = rx * sy - ry * sx;
            if (den == 0.0) continue;
            double qx = b->vx[k] - a->vx[e], qy = b->vy[k] - a->vy[e];
            double t = (qx * sy - qy * sx) / den, u = (qx * ry - qy * rx) / den;
            if (t >= 0.0 && t <= 1.0 && u >= 0.0 && u <= 1.0) ys[n++] = a->vy[e] + t * ry;
        }
    }
    return n;
}

static int cmp_double(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return x < y ? -1 : x > y;
}

/* Area of a composite grain: the integral over y of the total length of the
   grain's horizontal chords.  Between consecutive breakpoints (top and bottom
   of every disc, every polygon vertex, every crossing of two part boundaries)
   each chord end stays on one disc half or one polygon edge, so the slab's
   integral is exact: int sqrt(r^2 - u^2) du = (u sqrt(r^2 - u^2) + r^2 asin(u/r))/2
   for a disc end, the midpoint value times the height for an edge end. */
static double composite_area(const or_geom *g) {
    int cap = 4;
    for (int k = 0; k < g->nparts; ++k) cap += g->parts[k].kind == 0 ? 2 : g->parts[k].nv;
    int maxv = 2;
    for (int k = 0; k < g->nparts; ++k)
        if (g->parts[k].kind == 1 && g->parts[k].nv > maxv) maxv = g->parts[k].nv;
    cap += g->nparts * g->nparts * 2 * maxv * maxv;
    double *ys = malloc(sizeof(double) * cap);
    int ny = 0;
    for (int k = 0; k < g->nparts; ++k) {
        const o_part *q = &g->parts[k];
        if (q->kind == 0) {
            ys[ny++] = q->cy - q->r;
            ys[ny++] = q->cy + q->r;
        } else {
            for (int e = 0; e < q->nv; ++e) ys[ny++] = q->vy[e];
        }
        for (int k2 = 0; k2 < k; ++k2) ny += crossings_y(&g->parts[k2], q, ys + ny);
    }
    qsort(ys, ny, sizeof(double), cmp_double);
    int nc = 2 * g->nparts + 1;
    double *lo = malloc(sizeof(double) * nc), *hi = malloc(sizeof(double) * nc);
    o_tag *tlo = malloc(sizeof(o_tag) * nc), *thi = malloc(sizeof(o_tag) * nc);
    double area = 0.0;
    for (int s = 0; s + 1 < ny; ++s) {
        double ya = ys[s], yb = ys[s + 1];
        if (!(yb > ya)) continue;
        double ym = 0.5 * (ya + yb);
        int n = comp_chords(g, 0.0, ym, 1.0, 0.0, 0.0, lo, hi, tlo, thi);
        for (int i = 0; i < n; ++i) {
            for (int end = 0; end < 2; ++end) {
                o_tag t = end ? thi[i] : tlo[i];
                double xm = end ? hi[i] : lo[i];
                const o_part *q = &g->parts[t.part];
                double integ;
                if (q->kind == 0) {
                    double r = q->r, sg = xm >= q->cx ? 1.0 : -1.0;
                    double ua = fmax(-r, fmin(r, ya - q->cy)), ub = fmax(-r, fmin(r, yb - q->cy));
                    double Fa = 0.5 * (ua * sqrt(fmax(0.0, r * r - ua * ua)) + r * r * asin(ua / r));
                    double Fb = 0.5 * (ub * sqrt(fmax(0.0, r * r - ub * ub)) + r * r * asin(ub / r));
                    integ = q->cx * (yb - ya) + sg * (Fb - Fa);
                } else {
                    integ = xm * (yb - ya);  /* linear along the slab: exact at the midpoint */
                }
                area += end ? integ : -integ;
            }
        }
    }
    free(ys);
    free(lo);
    free(hi);
    free(tlo);
    free(thi);
    return area;
}

void or_geom_free(or_geom *g) {
    if (!g) return;
    for (int k = 0; k < g->nparts && g->parts; ++k) {
        free(g->parts[k].vx);
        free(g->parts[k].vy);
        free(g->parts[k].nx);
        free(g->parts[k].ny);
    }
    void *ptrs[] = {g->parts, g->mask, g->ghost, g->w, g->vh, /* eta is eta_c */
                    g->l_lo, g->l_hi, g->line_off, g->samp_off, g->lat_off, g->lat_c0, g->lat_nc,
                    g->lat_chorded, g->lat_near, g->ch_pair, g->ch_l, g->smin, g->smax, g->tag_lo,
                    g->tag_hi, g->m0, g->m1, g->ns, g->soff,
                    g->lk_g_angle, g->lk_g_line, g->lk_g_w, g->lk_t_angle, g->lk_t_line,
                    g->lk_t_w, g->ang_line_off, g->ang_samp_off, g->ewt, g->eta_c};
    for (size_t i = 0; i < sizeof ptrs / sizeof ptrs[0]; ++i) free(ptrs[i]);
    free(g);
}

/* copy one part; returns 0 or fails */
static int load_part(o_part *q, int kind, int add, double cx, double cy, double r, int nv,
                     const double *vx, const double *vy) {
    memset(q, 0, sizeof *q);
    q->kind = kind;
    q->add = add ? 1 : 0;
    if (kind == 0) {
        if (!(r > 0)) return fail("disc radius must be > 0");
        q->cx = cx;
        q->cy = cy;
        q->r = r;
        return 0;
    }
    if (kind != 1) return fail("unknown part kind");
    if (nv < 3 || !vx || !vy) return fail("polygon needs >= 3 vertices");
    q->nv = nv;
    q->vx = malloc(sizeof(double) * nv);
    q->vy = malloc(sizeof(double) * nv);
    q->nx = malloc(sizeof(double) * nv);
    q->ny = malloc(sizeof(double) * nv);
    memcpy(q->vx, vx, sizeof(double) * nv);
    memcpy(q->vy, vy, sizeof(double) * nv);
    for (int e = 0; e < nv; ++e) {
        int f = (e + 1) % nv;
        double dx = q->vx[f] - q->vx[e], dy = q->vy[f] - q->vy[e];
        double len = sqrt(dx * dx + dy * dy);
        if (!(len > 0)) return fail("polygon has a repeated vertex");
        q->nx[e] = dy / len;   /* outward for counter-clockwise order */
        q->ny[e] = -dx / len;
    }
    if (!(polygon_area(nv, q->vx, q->vy) > 0)) return fail("polygon must be counter-clockwise");
    return 0;
}

or_geom *or_geom_create(const or_params *prm) {
    if (!prm) { fail("null params"); return NULL; }
    if (prm->nx < 2 || prm->ny < 2 || !(prm->h > 0)) { fail("bad grid"); return NULL; }
    if (prm->n_angles < 2 || prm->n_angles % 2) { fail("n_angles must be even"); return NULL; }
    if (prm->n_energies < 1) { fail("n_energies < 1"); return NULL; }
    if (prm->stepper != 0 && prm->stepper != 1) { fail("stepper must be 0 or 1"); return NULL; }
    if (prm->n_components < 0 || prm->n_components > 4) { fail("1 to 4 components"); return NULL; }
    if (!(prm->t > 0 && prm->t <= 1)) { fail("t out of (0,1]"); return NULL; }
    if (prm->gauge < 0 || prm->gauge > 2) { fail("gauge must be 0, 1 or 2"); return NULL; }
    or_geom *g = calloc(1, sizeof *g);
    g->P = *prm;
    int nx = prm->nx, ny = prm->ny;
    double h = prm->h;

    /* parts */
    if (prm->shape_kind == 0 || prm->shape_kind == 1) {
        g->nparts = 1;
        g->parts = calloc(1, sizeof(o_part));
        if (load_part(&g->parts[0], prm->shape_kind, 1, prm->disc_cx, prm->disc_cy, prm->disc_r,
                      prm->n_vert, prm->vx, prm->vy)) {
            or_geom_free(g);
            return NULL;
        }
        const o_part *q = &g->parts[0];
        g->area = q->kind == 0 ? M_PI * q->r * q->r : polygon_area(q->nv, q->vx, q->vy);
    } else if (prm->shape_kind == 2) {
        if (prm->n_parts < 1 || !prm->parts) { fail("composite grain needs parts"); or_geom_free(g); return NULL; }
        g->nparts = prm->n_parts;
        g->parts = calloc(prm->n_parts, sizeof(o_part));
        for (int k = 0; k < prm->n_parts; ++k) {
            const or_part *s = &prm->parts[k];
            if (load_part(&g->parts[k], s->kind, s->add, s->cx, s->cy, s->r, s->n_vert, s->vx, s->vy)) {
                or_geom_free(g);
                return NULL;
            }
        }
        g->area = composite_area(g);
        if (!(g->area > 0)) { fail("composite grain has no area"); or_geom_free(g); return NULL; }
    } else {
        fail("unknown shape_kind");
        or_geom_free(g);
        return NULL;
    }
    g->P.vx = g->P.vy = NULL;
    g->P.parts = NULL;

    /* every added part lies inside the grid box */
    {
        double xlo = prm->x0, xhi = prm->x0 + nx * h, ylo = prm->y0, yhi = prm->y0 + ny * h;
        int ok = 1;
        for (int k = 0; k < g->nparts; ++k) {
            const o_part *q = &g->parts[k];
            if (!q->add) continue;
            if (q->kind == 0) {
                ok = ok && q->cx - q->r >= xlo && q->cx + q->r <= xhi && q->cy - q->r >= ylo &&
                     q->cy + q->r <= yhi;
            } else {
                for (int e = 0; e < q->nv; ++e)
                    ok = ok && q->vx[e] >= xlo && q->vx[e] <= xhi && q->vy[e] >= ylo && q->vy[e] <= yhi;
            }
        }
        if (!ok) { fail("shape extends outside the grid box"); or_geom_free(g); return NULL; }
    }
    /* the solenoid gauge's flux line must lie outside the grain */
    if (prm->gauge == 2 && !(sdist(g, prm->gauge_cx, prm->gauge_cy) > TAU * h)) {
        fail("solenoid gauge: the flux line must lie outside the grain");
        or_geom_free(g);
        return NULL;
    }

    /* mask: grid point centre inside (boundary counts as inside) */
    g->mask = calloc((size_t)nx * ny, 1);
    g->n_in = 0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double x = prm->x0 + (i + 0.5) * h, y = prm->y0 + (j + 0.5) * h;
            if (sdist(g, x, y) <= TAU * h) {
                g->mask[(size_t)j * nx + i] = 1;
                g->n_in++;
            }
        }
    if (g->n_in == 0) { fail("empty mask"); or_geom_free(g); return NULL; }

    /* ghost map on the padded index range [-1,nx] x [-1,ny]: every index whose
       centre is within 1.5 h of the shape maps to the nearest in-mask grid point
       (integer squared distance; ties -> lowest row-major index). Brute force. */
    int px = nx + 2, py = ny + 2;
    g->ghost = malloc(sizeof(int32_t) * (size_t)px * py);
#pragma omp parallel for schedule(dynamic, 4)
    for (int jj = 0; jj < py; ++jj) {
        for (int ii = 0; ii < px; ++ii) {
            int i = ii - 1, j = jj - 1;
            int32_t *out = &g->ghost[(size_t)jj * px + ii];
            *out = -1;
            if (i >= 0 && i < nx && j >= 0 && j < ny && g->mask[(size_t)j * nx + i]) {
                *out = j * nx + i;
                continue;
            }
            double x = prm->x0 + (i + 0.5) * h, y = prm->y0 + (j + 0.5) * h;
            if (sdist(g, x, y) > 1.5 * h) continue;
            long best = -1;
            long bestd = 0;
            for (int j2 = 0; j2 < ny; ++j2)
                for (int i2 = 0; i2 < nx; ++i2) {
                    if (!g->mask[(size_t)j2 * nx + i2]) continue;
                    long d = (long)(i - i2) * (i - i2) + (long)(j - j2) * (j - j2);
                    if (best < 0 || d < bestd) {
                        best = (long)j2 * nx + i2;
                        bestd = d;
                    }
                }
            *out = (int32_t)best;
        }
    }

    /* angles */
    int N = prm->n_angles, np = N / 2;
    g->N = N;
    g->npair = np;
    g->w = malloc(sizeof(double) * N);
    g->vh = malloc(sizeof(double) * 2 * N);
    g->C = prm->n_components > 1 ? prm->n_components : 1;
    g->eta_c = malloc(sizeof(double) * N * g->C);
    g->eta = g->eta_c;
    for (int c = 0; c < g->C; ++c) g->tcr[c] = prm->tc_ratios[c] > 0 ? prm->tc_ratios[c] : 1.0;
    for (int k = 0; k < np; ++k) {
        double phi = 2.0 * M_PI * k / N;
        g->vh[2 * k] = cos(phi);
        g->vh[2 * k + 1] = sin(phi);
        g->vh[2 * (k + np)] = -g->vh[2 * k];   /* exactly opposite */
        g->vh[2 * (k + np) + 1] = -g->vh[2 * k + 1];
    }
    for (int k = 0; k < N; ++k) {
        g->w[k] = or_quad_weight(k, N);
        for (int c = 0; c < g->C; ++c)
            g->eta_c[(size_t)c * N + k] = basis_eta(c == 0 ? prm->pairing : prm->pairings[c], prm->crystal_rotation,
                                                    g->vh[2 * k], g->vh[2 * k + 1]);
    }

    /* lattice origin: grid-box centre plus the offset (units of h) */
    g->Ox = prm->x0 + 0.5 * nx * h + prm->lattice_ox * h;
    g->Oy = prm->y0 + 0.5 * ny * h + prm->lattice_oy * h;
    double rext = 0.0;
    for (int k = 0; k < g->nparts; ++k) {
        const o_part *q = &g->parts[k];
        if (!q->add) continue;
        if (q->kind == 0) {
            double d = hypot(q->cx - g->Ox, q->cy - g->Oy) + q->r;
            if (d > rext) rext = d;
        } else {
            for (int e = 0; e < q->nv; ++e) {
                double d = hypot(q->vx[e] - g->Ox, q->vy[e] - g->Oy);
                if (d > rext) rext = d;
            }
        }
    }
    int Lmax = (int)ceil(rext / h) + 1;

    /* chords of every lattice line of every pair */
    int nc = 2 * g->nparts + 1;
    double *clo = malloc(sizeof(double) * nc), *chi = malloc(sizeof(double) * nc);
    o_tag *ctl = malloc(sizeof(o_tag) * nc), *cth = malloc(sizeof(o_tag) * nc);
    g->l_lo = malloc(sizeof(int) * np);
    g->l_hi = malloc(sizeof(int) * np);
    g->line_off = malloc(sizeof(int) * (np + 1));
    g->samp_off = malloc(sizeof(int) * (np + 1));
    g->lat_off = malloc(sizeof(int) * (np + 1));
    int nch = 0, cap_ch = 0, nlat = 0, cap_lat = 0;
    g->line_off[0] = g->samp_off[0] = g->lat_off[0] = 0;
    for (int p = 0; p < np; ++p) {
        double ex = g->vh[2 * p], ey = g->vh[2 * p + 1];
        double qx = -ey, qy = ex;
        int lo = 1 << 30, hi = -(1 << 30);
        for (int l = -Lmax; l <= Lmax; ++l)
            if (comp_chords(g, g->Ox + l * h * qx, g->Oy + l * h * qy, ex, ey, TAU * h, clo, chi, ctl, cth) > 0) {
                if (l < lo) lo = l;
                if (l > hi) hi = l;
            }
        if (lo > hi) { fail("pair without lines"); goto bad; }
        g->l_lo[p] = lo;
        g->l_hi[p] = hi;
        int cnt = 0;
        for (int l = lo; l <= hi; ++l) {
            int n = comp_chords(g, g->Ox + l * h * qx, g->Oy + l * h * qy, ex, ey, TAU * h, clo, chi, ctl, cth);
            if (nlat >= cap_lat) {
                cap_lat = cap_lat ? 2 * cap_lat : 256;
                g->lat_c0 = realloc(g->lat_c0, sizeof(int) * cap_lat);
                g->lat_nc = realloc(g->lat_nc, sizeof(int) * cap_lat);
            }
            g->lat_c0[nlat] = nch;
            g->lat_nc[nlat] = n;
            ++nlat;
            for (int i = 0; i < n; ++i) {
                if (nch >= cap_ch) {
                    cap_ch = cap_ch ? 2 * cap_ch : 256;
                    g->ch_pair = realloc(g->ch_pair, sizeof(int) * cap_ch);
                    g->ch_l = realloc(g->ch_l, sizeof(int) * cap_ch);
                    g->smin = realloc(g->smin, sizeof(double) * cap_ch);
                    g->smax = realloc(g->smax, sizeof(double) * cap_ch);
                    g->tag_lo = realloc(g->tag_lo, sizeof(o_tag) * cap_ch);
                    g->tag_hi = realloc(g->tag_hi, sizeof(o_tag) * cap_ch);
                    g->m0 = realloc(g->m0, sizeof(int) * cap_ch);
                    g->m1 = realloc(g->m1, sizeof(int) * cap_ch);
                    g->ns = realloc(g->ns, sizeof(int) * cap_ch);
                    g->soff = realloc(g->soff, sizeof(int) * cap_ch);
                }
                int L = nch++;
                g->ch_pair[L] = p;
                g->ch_l[L] = l;
                g->smin[L] = clo[i];
                g->smax[L] = chi[i];
                g->tag_lo[L] = ctl[i];
                g->tag_hi[L] = cth[i];
                g->m0[L] = (int)ceil(clo[i] / h - TAU);
                g->m1[L] = (int)floor(chi[i] / h + TAU);
                g->ns[L] = g->m1[L] - g->m0[L] + 1;
                if (g->ns[L] < 0) g->ns[L] = 0;
                g->soff[L] = cnt;
                cnt += g->ns[L];
            }
        }
        g->line_off[p + 1] = nch;
        g->samp_off[p + 1] = g->samp_off[p] + cnt;
        g->lat_off[p + 1] = nlat;
    }
    g->lat_chorded = malloc(sizeof(int) * (nlat > 0 ? nlat : 1));
    g->lat_near = malloc(sizeof(int) * (nlat > 0 ? nlat : 1));
    for (int p = 0; p < np; ++p) {
        /* nearest lattice line with a chord, and with a chord that has samples
           (ties -> lower index) */
        int any = 0;
        for (int l = g->l_lo[p]; l <= g->l_hi[p]; ++l) {
            int lat = glat(g, p, l);
            for (int q = 0; q < g->lat_nc[lat]; ++q) any = any || g->ns[g->lat_c0[lat] + q] > 0;
        }
        if (!any) { fail("pair without samples"); goto bad; }
        for (int l = g->l_lo[p]; l <= g->l_hi[p]; ++l) {
            int bc = 0, dc = 1 << 30, bs = 0, ds = 1 << 30;
            for (int l2 = g->l_lo[p]; l2 <= g->l_hi[p]; ++l2) {
                int lat2 = glat(g, p, l2), d = abs(l2 - l);
                int sampled = 0;
                for (int q = 0; q < g->lat_nc[lat2]; ++q) sampled = sampled || g->ns[g->lat_c0[lat2] + q] > 0;
                if (g->lat_nc[lat2] > 0 && d < dc) { dc = d; bc = l2; }
                if (sampled && d < ds) { ds = d; bs = l2; }
            }
            g->lat_chorded[glat(g, p, l)] = bc;
            g->lat_near[glat(g, p, l)] = bs;
        }
    }

    /* per-angle offsets */
    g->ang_line_off = malloc(sizeof(int64_t) * (N + 1));
    g->ang_samp_off = malloc(sizeof(int64_t) * (N + 1));
    g->ang_line_off[0] = g->ang_samp_off[0] = 0;
    for (int k = 0; k < N; ++k) {
        int p = k % np;
        g->ang_line_off[k + 1] = g->ang_line_off[k] + (g->line_off[p + 1] - g->line_off[p]);
        g->ang_samp_off[k + 1] = g->ang_samp_off[k] + (g->samp_off[p + 1] - g->samp_off[p]);
    }

    /* boundary links, Sec. 3.1 and Fig. riccati_fig_A: entry of gamma for
       angle k on a chord takes the exit value of the specularly reflected
       incoming direction; gamma~ starts from the gamma~ value that leaves
       along the reflected outgoing direction.  The normal is the grain's
       outward normal where the chord ends (for an end on a removed part, the
       part's inward normal). */
    int64_t NL = g->ang_line_off[N];
    g->lk_g_angle = malloc(sizeof(int) * 4 * NL);
    g->lk_g_line = malloc(sizeof(int) * 4 * NL);
    g->lk_g_w = malloc(sizeof(double) * 4 * NL);
    g->lk_t_angle = malloc(sizeof(int) * 4 * NL);
    g->lk_t_line = malloc(sizeof(int) * 4 * NL);
    g->lk_t_w = malloc(sizeof(double) * 4 * NL);
    for (int k = 0; k < N; ++k) {
        int p = k % np;
        int sg = k < np ? 1 : -1;
        double ex = g->vh[2 * p], ey = g->vh[2 * p + 1];
        double qx = -ey, qy = ex;
        double vx = g->vh[2 * k], vy = g->vh[2 * k + 1];
        for (int L = g->line_off[p]; L < g->line_off[p + 1]; ++L) {
            int l = g->ch_l[L];
            int64_t A = g->ang_line_off[k] + (L - g->line_off[p]);
            double bx = g->Ox + l * h * qx, by = g->Oy + l * h * qy;
            /* entry end and exit end of the chord in the direction of travel */
            double s_in = sg > 0 ? g->smin[L] : g->smax[L];
            double s_out = sg > 0 ? g->smax[L] : g->smin[L];
            o_tag t_in = sg > 0 ? g->tag_lo[L] : g->tag_hi[L];
            o_tag t_out = sg > 0 ? g->tag_hi[L] : g->tag_lo[L];
            double pex = bx + s_in * ex, pey = by + s_in * ey;
            double nnx, nny;
            end_normal(g, t_in, pex, pey, &nnx, &nny);
            double vn = vx * nnx + vy * nny;
            double uix = vx - 2.0 * vn * nnx, uiy = vy - 2.0 * vn * nny;
            make_link(g, pex, pey, uix, uiy, t_in.part, 0, &g->lk_g_angle[4 * A], &g->lk_g_line[4 * A],
                      &g->lk_g_w[4 * A]);
            double pxx = bx + s_out * ex, pxy = by + s_out * ey;
            end_normal(g, t_out, pxx, pxy, &nnx, &nny);
            vn = vx * nnx + vy * nny;
            double uox = vx - 2.0 * vn * nnx, uoy = vy - 2.0 * vn * nny;
            make_link(g, pxx, pxy, uox, uoy, t_out.part, 1, &g->lk_t_angle[4 * A], &g->lk_t_line[4 * A],
                      &g->lk_t_w[4 * A]);
        }
    }
    free(clo);
    free(chi);
    free(ctl);
    free(cth);
    return g;
bad:
    free(clo);
    free(chi);
    free(ctl);
    free(cth);
    or_geom_free(g);
    return NULL;
}

int or_geom_info(const or_geom *g, int64_t *info) {
    info[0] = g->npair;
    info[1] = g->line_off[g->npair];
    info[2] = g->samp_off[g->npair];
    info[3] = g->n_in;
    info[4] = g->ang_line_off[g->N];
    info[5] = g->ang_samp_off[g->N];
    return 0;
}
double or_geom_area(const or_geom *g) { return g->area; }
int or_geom_mask(const or_geom *g, uint8_t *m) {
    memcpy(m, g->mask, (size_t)g->P.nx * g->P.ny);
    return 0;
}
int or_geom_ghost(const or_geom *g, int32_t *o) {
    memcpy(o, g->ghost, sizeof(int32_t) * (size_t)(g->P.nx + 2) * (g->P.ny + 2));
    return 0;
}
int or_geom_lines(const or_geom *g, int32_t *l_lo, int32_t *l_hi, double *smin, double *smax,
                  int32_t *m0, int32_t *m1) {
    for (int p = 0; p < g->npair; ++p) {
        l_lo[p] = g->l_lo[p];
        l_hi[p] = g->l_hi[p];
    }
    int nl = g->line_off[g->npair];
    for (int L = 0; L < nl; ++L) {
        smin[L] = g->smin[L];
        smax[L] = g->smax[L];
        m0[L] = g->m0[L];
        m1[L] = g->m1[L];
    }
    return 0;
}
int or_geom_chords(const or_geom *g, int32_t *pair, int32_t *l) {
    for (int L = 0; L < g->line_off[g->npair]; ++L) {
        pair[L] = g->ch_pair[L];
        l[L] = g->ch_l[L];
    }
    return 0;
}
int or_geom_links(const or_geom *g, int32_t *ta, int32_t *tl, int32_t *tc, double *tw) {
    int64_t n = 4 * g->ang_line_off[g->N];
    for (int64_t i = 0; i < n; ++i) {
        int L = g->lk_g_line[i];
        ta[i] = g->lk_g_angle[i];
        tl[i] = g->ch_l[L];
        tc[i] = L - g->line_off[g->ch_pair[L]];
        tw[i] = g->lk_g_w[i];
    }
    return 0;
}
int or_geom_quadrature(const or_geom *g, double *w, double *vh, double *eta) {
    for (int k = 0; k < g->N; ++k) {
        w[k] = g->w[k];
        vh[2 * k] = g->vh[2 * k];
        vh[2 * k + 1] = g->vh[2 * k + 1];
        eta[k] = g->eta[k];
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Fields on the rotated lattice (Sec. 3.1: bilinear interpolation from   */
/* the reference grid; grid points outside the grain take the value of    */
/* the nearest grain point).                                              */
/* ---------------------------------------------------------------------- */
static int interp2(const or_geom *g, const double *f, double x, double y, double out[2]) {
    int nx = g->P.nx, ny = g->P.ny;
    double gx = (x - g->P.x0) / g->P.h - 0.5, gy = (y - g->P.y0) / g->P.h - 0.5;
    int i0 = (int)floor(gx), j0 = (int)floor(gy);
    double fx = gx - i0, fy = gy - j0;
    out[0] = out[1] = 0.0;
    if (i0 < -1 || i0 > nx - 1 || j0 < -1 || j0 > ny - 1) return -1;
    for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
            double wgt = (a ? fx : 1.0 - fx) * (b ? fy : 1.0 - fy);
            int src = g->ghost[(size_t)(j0 + b + 1) * (nx + 2) + (i0 + a + 1)];
            if (src < 0) {
                if (wgt != 0.0) return -1;
                continue;
            }
            out[0] += wgt * f[2 * (size_t)src];
            out[1] += wgt * f[2 * (size_t)src + 1];
        }
    return 0;
}

/* Total vector potential at a point: the external part of the gauge,
   analytic, plus the interpolated induced part.  Symmetric gauge
   A = B/2 (-(y-yg), x-xg) and landau gauge A = B (-(y-yg), 0) with
   B = pi alpha / area (units B0; Sec. 5.1.2); solenoid gauge
   A = alpha/(2 r) phi^ = alpha/(2 r^2) (-(y-yg), x-xg) (Eq. solenoid_gauge
   with Phi_ext = alpha Phi0, units A0 = Phi0/(pi xi0)). */
static int a_total(const or_geom *g, const double *aind, double x, double y, double A[2]) {
    double dx = x - g->P.gauge_cx, dy = y - g->P.gauge_cy;
    if (g->P.gauge == 2) {
        double r2 = dx * dx + dy * dy;
        if (!(r2 > 0.0)) return -1;
        A[0] = -0.5 * g->P.flux_quanta * dy / r2;
        A[1] = 0.5 * g->P.flux_quanta * dx / r2;
    } else {
        double B = M_PI * g->P.flux_quanta / g->area;
        if (g->P.gauge == 1) {
            A[0] = -B * dy;
            A[1] = 0.0;
        } else {
            A[0] = -0.5 * B * dy;
            A[1] = 0.5 * B * dx;
        }
    }
    if (aind) {
        double ai[2];
        if (interp2(g, aind, x, y, ai)) return -1;
        A[0] += ai[0];
        A[1] += ai[1];
    }
    return 0;
}

int or_external_a(const or_geom *g, int n, const double *xy, double *A) {
    for (int i = 0; i < n; ++i)
        if (a_total(g, NULL, xy[2 * i], xy[2 * i + 1], &A[2 * i])) return fail("gauge singular at a point");
    return 0;
}

int or_sample_fields(const or_geom *g, const double *delta, const double *aind, int p,
                     double *ds, double *as) {
    double h = g->P.h;
    double ex = g->vh[2 * p], ey = g->vh[2 * p + 1], qx = -ey, qy = ex;
    for (int L = g->line_off[p]; L < g->line_off[p + 1]; ++L) {
        int l = g->ch_l[L];
        for (int m = g->m0[L]; m <= g->m1[L]; ++m) {
            int idx = g->soff[L] + (m - g->m0[L]);
            double x = g->Ox + l * h * qx + m * h * ex, y = g->Oy + l * h * qy + m * h * ey;
            if (interp2(g, delta, x, y, &ds[2 * idx])) return fail("sample outside grid");
            if (a_total(g, aind, x, y, &as[2 * idx])) return fail("sample outside grid");
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Closed-form Riccati step.  For d gamma/ds = i (P g^2 + 2 Q g + R) with  */
/* constant coefficients, gamma_h = -R/(Q + i Om), Om = sqrt(PR - Q^2)    */
/* (principal branch), is the fixed point that is stable along s; with    */
/* delta = gamma - gamma_h the equation is of Bernoulli type and          */
/*   delta(ell) = delta E / (1 - i P delta (1-E)/(2 Om)),  E = e^{-2 Om ell}.*/
/* ---------------------------------------------------------------------- */
static cplx one_minus_exp_over(cplx Om, double ell) {
    /* (1 - exp(-2 Om ell)) / (2 Om), with the series near Om ell = 0 */
    cplx x = 2.0 * Om * ell;
    if (cabs(x) < 1e-2) {
        cplx s = 0.0, term = 1.0;
        for (int k = 0; k < 8; ++k) { /* sum_k (-x)^k/(k+1)! */
            double fact = 1.0;
            for (int q = 2; q <= k + 1; ++q) fact *= q;
            s += term / fact;
            term *= -x;
        }
        return ell * s;
    }
    return (1.0 - cexp(-x)) / (2.0 * Om);
}

static cplx riccati_fixed_point(cplx P, cplx Q, cplx R) {
    cplx Om = csqrt(P * R - Q * Q);
    return -R / (Q + I * Om);
}

static cplx riccati_step(cplx P, cplx Q, cplx R, double ell, cplx ga) {
    cplx Om = csqrt(P * R - Q * Q);
    cplx gh = -R / (Q + I * Om);
    cplx E = cexp(-2.0 * Om * ell);
    cplx c = one_minus_exp_over(Om, ell);
    cplx d = ga - gh;
    return gh + d * E / (1.0 - I * P * d * c);
}

/* Implicit midpoint rule (App. C): g1 = g0 + ell f((g0 + g1)/2) with
   f(g) = i (P g^2 + 2 Q g + R).  Collecting powers of g1 gives
   c2 g1^2 + c1 g1 + c0 = 0 with
     c2 = i ell P / 4,
     c1 = 2 c2 g0 + i ell Q - 1,
     c0 = (c1 - c2 g0 + 2) g0 + i ell R
   (for R = conj P, as for gamma and gamma~, i ell R = -4 conj(c2): the paper's
   form), and the root that tends to -c0/c1 as P -> 0 is
     g1 = 2 c0 / (-c1 + sqrt(c1^2 - 4 c2 c0))      (principal square root;
   Re c1 < 0 whenever ell |P| < 2 and Im Q > 0, so the denominator is near -2 c1). */
static cplx riccati_midpoint(cplx P, cplx Q, cplx R, double ell, cplx g0) {
    cplx c2 = I * ell * P / 4.0;
    cplx c1 = 2.0 * c2 * g0 + I * ell * Q - 1.0;
    cplx c0 = (c1 - c2 * g0 + 2.0) * g0 + I * ell * R;
    return 2.0 * c0 / (-c1 + csqrt(c1 * c1 - 4.0 * c2 * c0));
}

/* the step of the configured method */
static cplx riccati_advance(const or_geom *g, cplx P, cplx Q, cplx R, double ell, cplx ga) {
    return g->P.stepper == 1 ? riccati_midpoint(P, Q, R, ell, ga) : riccati_step(P, Q, R, ell, ga);
}

void or_step_midpoint(const double *P, const double *Q, const double *R, double ell,
                      const double *ga, double *gb) {
    cplx r = riccati_midpoint(P[0] + I * P[1], Q[0] + I * Q[1], R[0] + I * R[1], ell, ga[0] + I * ga[1]);
    gb[0] = creal(r);
    gb[1] = cimag(r);
}

void or_step(const double *P, const double *Q, const double *R, double ell, const double *ga,
             double *gb) {
    cplx r = riccati_step(P[0] + I * P[1], Q[0] + I * Q[1], R[0] + I * R[1], ell, ga[0] + I * ga[1]);
    gb[0] = creal(r);
    gb[1] = cimag(r);
}

/* Delta(p, R) = sum_c eta_c(p) Delta_c(R) on the grid (complex, npts). */
static double *combined_field(const or_geom *g, const double *delta, int p) {
    size_t npts = (size_t)g->P.nx * g->P.ny;
    double *f = calloc(2 * npts, sizeof(double));
    for (int c = 0; c < g->C; ++c) {
        double e = g->eta_c[(size_t)c * g->N + p];
        const double *dc = delta + 2 * npts * c;
        for (size_t i = 0; i < 2 * npts; ++i) f[i] += e * dc[i];
    }
    return f;
}

/* ---------------------------------------------------------------------- */
/* Sweep                                                                  */
/* ---------------------------------------------------------------------- */
int or_sweep(const or_geom *g, const double *delta, const double *aind, const double *z,
             int n_e, int mode, const double *exit_in, double *exit_out, double *images,
             double *gam_out) {
    int N = g->N, np = g->npair;
    double h = g->P.h;
    int64_t NLA = g->ang_line_off[N];
    int64_t NSA = g->ang_samp_off[N];
    int sgc = g->P.charge_sign;
    int err = 0;

    /* sample fields of every pair; with several components the sampled field is
       Delta(p, R) = sum_c eta_c(p) Delta_c(R) (Eq. order_parameter; the basis
       functions are even, eta(p + pi) = eta(p)), formed on the grid first since
       bilinear sampling is linear */
    double **dS = malloc(sizeof(double *) * np), **aS = malloc(sizeof(double *) * np);
    double **comb = calloc(np, sizeof(double *));
    for (int p = 0; p < np; ++p) {
        int ns = g->samp_off[p + 1] - g->samp_off[p];
        dS[p] = malloc(sizeof(double) * 2 * (ns > 0 ? ns : 1));
        aS[p] = malloc(sizeof(double) * 2 * (ns > 0 ? ns : 1));
        if (g->C > 1) {
            comb[p] = combined_field(g, delta, p);
            if (or_sample_fields(g, comb[p], aind, p, dS[p], aS[p])) err = 1;
        } else if (or_sample_fields(g, delta, aind, p, dS[p], aS[p])) {
            err = 1;
        }
    }
    if (err) goto done;

#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t A = 0; A < NLA; ++A) {
        {
            int k = 0;
            while (g->ang_line_off[k + 1] <= A) ++k;
            int p = k % np;
            int L = g->line_off[p] + (int)(A - g->ang_line_off[k]);
            int l = g->ch_l[L];
            int sg = k < np ? 1 : -1;
            double vx = g->vh[2 * k], vy = g->vh[2 * k + 1];
            double eta = g->C > 1 ? 1.0 : g->eta[k];  /* combined fields already carry eta */
            const double *dfield = g->C > 1 ? comb[p] : delta;
            int ns = g->ns[L];
            int m0 = g->m0[L], m1 = g->m1[L];
            /* coefficient of each segment in travel order: Delta(p,R) and a = sigma v.A */
            int nseg = ns + 1;
            cplx *dseg = malloc(sizeof(cplx) * nseg);
            double *aseg = malloc(sizeof(double) * nseg);
            double *lseg = malloc(sizeof(double) * nseg);
            cplx *dsm = malloc(sizeof(cplx) * (ns > 0 ? ns : 1)); /* sample values, travel order */
            double *asm_ = malloc(sizeof(double) * (ns > 0 ? ns : 1));
            int *sidx = malloc(sizeof(int) * (ns > 0 ? ns : 1));   /* canonical sample index */
            for (int q = 0; q < ns; ++q) {
                int m = sg > 0 ? m0 + q : m1 - q;
                int idx = g->soff[L] + (m - m0);
                sidx[q] = idx;
                dsm[q] = eta * (dS[p][2 * idx] + I * dS[p][2 * idx + 1]);
                asm_[q] = sgc * (vx * aS[p][2 * idx] + vy * aS[p][2 * idx + 1]);
            }
            if (ns == 0) {
                double ex = g->vh[2 * p], ey = g->vh[2 * p + 1];
                double smid = 0.5 * (g->smin[L] + g->smax[L]);
                double x = g->Ox - l * h * ey + smid * ex, y = g->Oy + l * h * ex + smid * ey;
                double dd[2] = {0.0, 0.0}, AA[2] = {0.0, 0.0};
                if (interp2(g, dfield, x, y, dd) || a_total(g, aind, x, y, AA)) {
#pragma omp atomic write
                    err = 1;
                }
                dseg[0] = eta * (dd[0] + I * dd[1]);
                aseg[0] = sgc * (vx * AA[0] + vy * AA[1]);
                lseg[0] = g->smax[L] - g->smin[L];
            } else {
                double lead = sg > 0 ? m0 * h - g->smin[L] : g->smax[L] - m1 * h;
                double tail = sg > 0 ? g->smax[L] - m1 * h : m0 * h - g->smin[L];
                dseg[0] = dsm[0];
                aseg[0] = asm_[0];
                lseg[0] = lead > 0.0 ? lead : 0.0;
                for (int q = 1; q < ns; ++q) {
                    dseg[q] = 0.5 * (dsm[q - 1] + dsm[q]);
                    aseg[q] = 0.5 * (asm_[q - 1] + asm_[q]);
                    lseg[q] = h;
                }
                dseg[ns] = dsm[ns - 1];
                aseg[ns] = asm_[ns - 1];
                lseg[ns] = tail > 0.0 ? tail : 0.0;
            }
            cplx *gam = malloc(sizeof(cplx) * (ns > 0 ? ns : 1));
            cplx *gat = malloc(sizeof(cplx) * (ns > 0 ? ns : 1));
            for (int n = 0; n < n_e; ++n) {
                cplx zn = z[2 * n] + I * z[2 * n + 1];
                /* gamma along the direction of travel (Eq. riccati):
                   d gamma/ds = i (Delta* gamma^2 + 2 z gamma + Delta) */
                cplx gm;
                if (exit_in) {
                    gm = 0.0;
                    for (int q = 0; q < 4; ++q) {
                        int ja = g->lk_g_angle[4 * A + q];
                        int jc = g->lk_g_line[4 * A + q];
                        int64_t B = g->ang_line_off[ja] + (jc - g->line_off[ja % np]);
                        gm += g->lk_g_w[4 * A + q] *
                              (exit_in[2 * (B * n_e + n)] + I * exit_in[2 * (B * n_e + n) + 1]);
                    }
                } else {
                    gm = riccati_fixed_point(conj(dseg[0]), zn + aseg[0], dseg[0]);
                }
                for (int q = 0; q < nseg; ++q) {
                    gm = riccati_advance(g, conj(dseg[q]), zn + aseg[q], dseg[q], lseg[q], gm);
                    if (q < ns) gam[q] = gm;
                }
                int64_t oi = 2 * (A * n_e + n);
                exit_out[oi] = creal(gm);
                exit_out[oi + 1] = cimag(gm);
                /* gamma~ against the direction of travel (Eq. riccati_tilde):
                   d gamma~/ds = i (Delta gamma~^2 - 2 z gamma~ + Delta*); with u = -s
                   d gamma~/du = i (-Delta gamma~^2 + 2 z gamma~ - Delta*) */
                cplx gt;
                if (exit_in) {
                    gt = 0.0;
                    for (int q = 0; q < 4; ++q) {
                        int ja = g->lk_t_angle[4 * A + q];
                        int jc = g->lk_t_line[4 * A + q];
                        int64_t B = g->ang_line_off[ja] + (jc - g->line_off[ja % np]);
                        int64_t ii = 2 * (NLA * n_e + B * n_e + n);
                        gt += g->lk_t_w[4 * A + q] * (exit_in[ii] + I * exit_in[ii + 1]);
                    }
                } else {
                    gt = riccati_fixed_point(-dseg[ns], zn + aseg[ns], -conj(dseg[ns]));
                }
                for (int q = ns; q >= 0; --q) {
                    gt = riccati_advance(g, -dseg[q], zn + aseg[q], -conj(dseg[q]), lseg[q], gt);
                    if (q > 0) gat[q - 1] = gt;
                }
                int64_t ti = 2 * (NLA * n_e + A * n_e + n);
                exit_out[ti] = creal(gt);
                exit_out[ti + 1] = cimag(gt);
                /* propagator at each sample (Eq. riccati_parameterization) */
                for (int q = 0; q < ns; ++q) {
                    cplx ga = gam[q], gb = gat[q];
                    cplx den = 1.0 + ga * gb;
                    cplx gg = -I * M_PI * (1.0 - ga * gb) / den;
                    cplx ff = -2.0 * I * M_PI * ga / den;
                    cplx ft = 2.0 * I * M_PI * gb / den;
                    int64_t si = g->ang_samp_off[k] + sidx[q];
                    if (gam_out) {
                        int64_t gi = 2 * (si * n_e + n);
                        gam_out[gi] = creal(ga);
                        gam_out[gi + 1] = cimag(ga);
                        gam_out[2 * NSA * n_e + gi] = creal(gb);
                        gam_out[2 * NSA * n_e + gi + 1] = cimag(gb);
                    }
                    if (mode == 0) {
                        /* positive Matsubara energies; the negative ones follow from
                           g(-e) = g(e)*, f(-e) = f~(e)* (Eq. symmetries) */
                        cplx dl = dsm[q];
                        cplx In = (conj(dl) * ff + dl * ft) / (M_PI + I * gg);
                        double *im = &images[4 * si];
                        if (n == 0) im[0] = im[1] = im[2] = im[3] = 0.0;
                        cplx sf = ff + conj(ft);
                        double wn = g->ewt ? g->ewt[n] : 1.0;
                        im[0] += wn * creal(sf);
                        im[1] += wn * cimag(sf);
                        im[2] += wn * 2.0 * creal(gg);
                        im[3] += wn * 2.0 * creal(In);
                    } else {
                        images[si * n_e + n] = -cimag(gg) / M_PI;
                    }
                }
            }
            free(gam);
            free(gat);
            free(dseg);
            free(aseg);
            free(lseg);
            free(dsm);
            free(asm_);
            free(sidx);
        }
    }
done:
    for (int p = 0; p < np; ++p) {
        free(dS[p]);
        free(aS[p]);
        free(comb[p]);
    }
    free(comb);
    free(dS);
    free(aS);
    if (err) return fail("sample outside grid");
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Rotate back + FS average (Sec. 3.1).                                   */
/* ---------------------------------------------------------------------- */
int or_rotate_back(const or_geom *g, const double *images, int mode, int n_e, double *acc) {
    int nx = g->P.nx, ny = g->P.ny, N = g->N, np = g->npair;
    double h = g->P.h;
    int nv = mode == 0 ? 4 : n_e;
    int nout = mode == 0 ? 3 + 2 * g->C : n_e;
    size_t npts = (size_t)nx * ny;
    memset(acc, 0, sizeof(double) * nout * npts);
#pragma omp parallel for schedule(dynamic, 16)
    for (size_t idx = 0; idx < npts; ++idx) {
        if (!g->mask[idx]) continue;
        int i = (int)(idx % nx), j = (int)(idx / nx);
        double x = g->P.x0 + (i + 0.5) * h, y = g->P.y0 + (j + 0.5) * h;
        double *X = malloc(sizeof(double) * nv);
        for (int k = 0; k < N; ++k) {
            int p = k % np;
            double ex = g->vh[2 * p], ey = g->vh[2 * p + 1], qx = -ey, qy = ex;
            double u = ((x - g->Ox) * qx + (y - g->Oy) * qy) / h;
            double v = ((x - g->Ox) * ex + (y - g->Oy) * ey) / h;
            int iu = (int)floor(u), iv = (int)floor(v);
            double wu = u - iu, wv = v - iv;
            for (int c = 0; c < nv; ++c) X[c] = 0.0;
            for (int b = 0; b < 2; ++b) {
                int l = iu + b;
                if (l < g->l_lo[p]) l = g->l_lo[p];
                if (l > g->l_hi[p]) l = g->l_hi[p];
                /* the nearest line with samples, and on it the sampled chord
                   nearest to the point along the line */
                int L = pick_sampled_chord(g, glat(g, p, g->lat_near[glat(g, p, l)]), v);
                for (int a = 0; a < 2; ++a) {
                    int m = iv + a;
                    if (m < g->m0[L]) m = g->m0[L];
                    if (m > g->m1[L]) m = g->m1[L];
                    int64_t si = g->ang_samp_off[k] + g->soff[L] + (m - g->m0[L]);
                    double wgt = (b ? wu : 1.0 - wu) * (a ? wv : 1.0 - wv);
                    for (int c = 0; c < nv; ++c) X[c] += wgt * images[si * nv + c];
                }
            }
            double wk = g->w[k];
            if (mode == 0) {
                /* planes: <eta_0 Sf> (2), <v Sg> (2), <SF>, then <eta_c Sf> (2 per c >= 1) */
                acc[0 * npts + idx] += wk * g->eta[k] * X[0];
                acc[1 * npts + idx] += wk * g->eta[k] * X[1];
                acc[2 * npts + idx] += wk * g->vh[2 * k] * X[2];
                acc[3 * npts + idx] += wk * g->vh[2 * k + 1] * X[2];
                acc[4 * npts + idx] += wk * X[3];
                for (int c = 1; c < g->C; ++c) {
                    double e = g->eta_c[(size_t)c * N + k];
                    acc[(3 + 2 * c) * npts + idx] += wk * e * X[0];
                    acc[(4 + 2 * c) * npts + idx] += wk * e * X[1];
                }
            } else {
                for (int c = 0; c < n_e; ++c) acc[c * npts + idx] += wk * X[c];
            }
        }
        free(X);
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Outputs: gap equation (Eq. gapeq_fixpoint), current (Eq.               */
/* current_density), Eilenberger free energy (Eq. qcLWFE with the         */
/* Eilenberger form of I(R)), global error (Eq. global_error, p = 2).     */
/* ---------------------------------------------------------------------- */
int or_outputs(const or_geom *g, const double *acc, const double *delta, const double *aind,
               double *delta_new, double *jout, double *F, double *scalars) {
    int nx = g->P.nx, ny = g->P.ny;
    double h = g->P.h, t = g->P.t;
    size_t npts = (size_t)nx * ny;
    double D = g->ewt ? g->normD : or_norm_D(t, g->P.n_energies);
    double sgc = g->P.charge_sign;
    int magn = g->P.kappa > 0 && isfinite(g->P.kappa) && aind;
    double k2 = magn ? g->P.kappa * g->P.kappa : 0.0;
    double Fsum = 0.0, num = 0.0, den = 0.0;
    for (size_t idx = 0; idx < npts; ++idx) {
        if (!g->mask[idx]) {
            for (int c = 0; c < g->C; ++c) delta_new[2 * (c * npts + idx)] = delta_new[2 * (c * npts + idx) + 1] = 0.0;
            jout[2 * idx] = jout[2 * idx + 1] = 0.0;
            F[idx] = 0.0;
            continue;
        }
        int i = (int)(idx % nx), j = (int)(idx / nx);
        /* component c (Eq. gapeq_fixpoint): Delta_c = T sum_n <eta_c f> / D_c,
           D_c = ln(T/T_c^c) + pi T sum 1/|eps_n| = D - ln(T_c^c/T_c), T = t/(2 pi) */
        double f = -0.5 * t * acc[4 * npts + idx];
        for (int c = 0; c < g->C; ++c) {
            double Dc = D - log(g->tcr[c]);
            size_t pr = c == 0 ? 0 : (size_t)(3 + 2 * c), pi_ = c == 0 ? 1 : (size_t)(4 + 2 * c);
            double dr = t / (2.0 * M_PI) * acc[pr * npts + idx] / Dc;
            double di = t / (2.0 * M_PI) * acc[pi_ * npts + idx] / Dc;
            size_t o = 2 * (c * npts + idx);
            delta_new[o] = dr;
            delta_new[o + 1] = di;
            /* F(R) = sum_c |Delta_c|^2 D_c - (t/2) <SF> + (kappa^2/2) |B_ind|^2 */
            double d2 = delta[o] * delta[o] + delta[o + 1] * delta[o + 1];
            f += d2 * Dc;
            double er = dr - delta[o], ei = di - delta[o + 1];
            num += er * er + ei * ei;
            den += d2;
        }
        /* j = 2 e N_F T sum_n <v g>  ->  sigma (t/pi) <v Sg> in units of j0 */
        jout[2 * idx] = sgc * t / M_PI * acc[2 * npts + idx];
        jout[2 * idx + 1] = sgc * t / M_PI * acc[3 * npts + idx];
        if (magn) {
            /* B_ind = dAy/dx - dAx/dy, central differences (one-sided at the grid edge) */
            int ia = i > 0 ? i - 1 : i, ib = i < nx - 1 ? i + 1 : i;
            int ja = j > 0 ? j - 1 : j, jb = j < ny - 1 ? j + 1 : j;
            double dAy = (aind[2 * ((size_t)j * nx + ib) + 1] - aind[2 * ((size_t)j * nx + ia) + 1]) /
                         ((ib - ia) * h);
            double dAx = (aind[2 * ((size_t)jb * nx + i)] - aind[2 * ((size_t)ja * nx + i)]) /
                         ((jb - ja) * h);
            double B = dAy - dAx;
            f += 0.5 * k2 * B * B;
        }
        F[idx] = f;
        Fsum += f;
    }
    scalars[0] = Fsum / (double)g->n_in;
    scalars[1] = den > 0 ? sqrt(num / den) : 0.0;
    return 0;
}

/* ---------------------------------------------------------------------- */
/* App. D: cell-integrated Green's function of the 2D Laplacian and the   */
/* induced vector potential (full correlation, the tolerance-zero case).  */
/* ---------------------------------------------------------------------- */
static double gf_alpha(double m, double n) {
    return (1.0 + 2.0 * m) * (1.0 + 2.0 * n) *
           log(0.5 * (1.0 + 2.0 * m) * (1.0 + 2.0 * m) + 0.5 * (1.0 + 2.0 * n) * (1.0 + 2.0 * n));
}
static double gf_beta(double m, double n) {
    return (-2.0 * m * m + 2.0 * n * n + 4.0 * n + 1.0) * atan((1.0 + 2.0 * m) / (1.0 + 2.0 * n));
}
static double gf_Gamma(double m, double n) { return gf_alpha(m, n) + gf_beta(m, n) + gf_beta(n, m); }

double or_greens(int m, int n, double h) {
    double s = 0.0;
    for (int a = -1; a <= 1; a += 2)
        for (int b = -1; b <= 1; b += 2) s += gf_Gamma(a * (double)m, b * (double)n);
    return h * h / (4.0 * M_PI) * (2.0 * log(h) - log(2.0) - 3.0 + 0.25 * s);
}

int or_vector_potential(const or_geom *g, const double *j, double *aind) {
    int nx = g->P.nx, ny = g->P.ny;
    size_t npts = (size_t)nx * ny;
    if (!(g->P.kappa > 0) || !isfinite(g->P.kappa)) {
        memset(aind, 0, sizeof(double) * 2 * npts);
        return 0;
    }
    double k2 = g->P.kappa * g->P.kappa;
    /* subtract the mean current over the grain (App. D, last paragraph) */
    double mx = 0.0, my = 0.0;
    for (size_t i = 0; i < npts; ++i)
        if (g->mask[i]) { mx += j[2 * i]; my += j[2 * i + 1]; }
    mx /= g->n_in;
    my /= g->n_in;
    int W = nx > ny ? nx : ny;
    double *G = malloc(sizeof(double) * (size_t)W * W);
    for (int a = 0; a < W; ++a)
        for (int b = 0; b < W; ++b) G[(size_t)a * W + b] = or_greens(a, b, g->P.h);
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < npts; ++i) {
        int xi = (int)(i % nx), yi = (int)(i / nx);
        double sx = 0.0, sy = 0.0;
        for (size_t q = 0; q < npts; ++q) {
            if (!g->mask[q]) continue;
            int xq = (int)(q % nx), yq = (int)(q / nx);
            double Gv = G[(size_t)abs(xq - xi) * W + abs(yq - yi)];
            sx += Gv * (j[2 * q] - mx);
            sy += Gv * (j[2 * q + 1] - my);
        }
        aind[2 * i] = -sx / k2;
        aind[2 * i + 1] = -sy / k2;
    }
    free(G);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Bulk gap: root of  D = t sum_{n<Ne} <eta^2 / sqrt(eta^2 Delta^2 + eps_n^2)> */
/* (homogeneous limit of Eq. gapeq_fixpoint, f = pi Delta eta / Omega).   */
/* ---------------------------------------------------------------------- */
static double bulk_rhs(int pairing, double t, int n_e, int N, double d) {
    double s = 0.0;
    for (int k = 0; k < N; ++k) {
        double phi = 2.0 * M_PI * k / N;
        double eta = basis_eta(pairing, 0.0, cos(phi), sin(phi));
        double w = or_quad_weight(k, N);
        double sk = 0.0;
        for (int n = 0; n < n_e; ++n) {
            double e = t * (n + 0.5);
            sk += eta * eta / sqrt(eta * eta * d * d + e * e);
        }
        s += w * sk;
    }
    return t * s;
}

double or_bulk_gap(int pairing, double t, int n_e, int N) {
    double D = or_norm_D(t, n_e);
    if (bulk_rhs(pairing, t, n_e, N, 0.0) <= D) return 0.0;
    double lo = 0.0, hi = 2.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (bulk_rhs(pairing, t, n_e, N, mid) > D) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* ---------------------------------------------------------------------- */
/* First sweep (homogeneous entry values) for a chosen subset of angles:  */
/* the same per-line integration as or_sweep, restricted so that a large  */
/* grain can be checked angle by angle.  images: [n_sel][samples of the   */
/* angle's pair][4] (mode-0 sums).                                        */
/* ---------------------------------------------------------------------- */
int or_sweep_subset(const or_geom *g, const double *delta, const double *aind, const double *z,
                    int n_e, const int *angles, int n_sel, double *images) {
    int np = g->npair;
    double h = g->P.h;
    int sgc = g->P.charge_sign;
    int64_t out_off = 0;
    for (int si = 0; si < n_sel; ++si) {
        int k = angles[si];
        if (k < 0 || k >= g->N) return fail("angle out of range");
        int p = k % np;
        int sg = k < np ? 1 : -1;
        int nsp = g->samp_off[p + 1] - g->samp_off[p];
        double *dS = malloc(sizeof(double) * 2 * (nsp > 0 ? nsp : 1));
        double *aS = malloc(sizeof(double) * 2 * (nsp > 0 ? nsp : 1));
        double *comb = g->C > 1 ? combined_field(g, delta, p) : NULL;
        int bad = or_sample_fields(g, comb ? comb : delta, aind, p, dS, aS);
        free(comb);
        if (bad) {
            free(dS);
            free(aS);
            return -1;
        }
        double vx = g->vh[2 * k], vy = g->vh[2 * k + 1], eta = g->C > 1 ? 1.0 : g->eta[k];
        int nl = g->line_off[p + 1] - g->line_off[p];
#pragma omp parallel for schedule(dynamic, 1)
        for (int li = 0; li < nl; ++li) {
            int L = g->line_off[p] + li;
            int ns = g->ns[L], m0 = g->m0[L], m1 = g->m1[L];
            if (ns == 0) continue;
            cplx *dseg = malloc(sizeof(cplx) * (ns + 1));
            double *aseg = malloc(sizeof(double) * (ns + 1));
            double *lseg = malloc(sizeof(double) * (ns + 1));
            cplx *dsm = malloc(sizeof(cplx) * ns);
            double *asm_ = malloc(sizeof(double) * ns);
            int *sidx = malloc(sizeof(int) * ns);
            for (int q = 0; q < ns; ++q) {
                int m = sg > 0 ? m0 + q : m1 - q;
                int idx = g->soff[L] + (m - m0);
                sidx[q] = idx;
                dsm[q] = eta * (dS[2 * idx] + I * dS[2 * idx + 1]);
                asm_[q] = sgc * (vx * aS[2 * idx] + vy * aS[2 * idx + 1]);
            }
            double lead = sg > 0 ? m0 * h - g->smin[L] : g->smax[L] - m1 * h;
            double tail = sg > 0 ? g->smax[L] - m1 * h : m0 * h - g->smin[L];
            dseg[0] = dsm[0];
            aseg[0] = asm_[0];
            lseg[0] = lead > 0.0 ? lead : 0.0;
            for (int q = 1; q < ns; ++q) {
                dseg[q] = 0.5 * (dsm[q - 1] + dsm[q]);
                aseg[q] = 0.5 * (asm_[q - 1] + asm_[q]);
                lseg[q] = h;
            }
            dseg[ns] = dsm[ns - 1];
            aseg[ns] = asm_[ns - 1];
            lseg[ns] = tail > 0.0 ? tail : 0.0;
            cplx *gam = malloc(sizeof(cplx) * ns), *gat = malloc(sizeof(cplx) * ns);
            for (int q = 0; q < ns; ++q) {
                double *im = &images[4 * (out_off + sidx[q])];
                im[0] = im[1] = im[2] = im[3] = 0.0;
            }
            for (int n = 0; n < n_e; ++n) {
                cplx zn = z[2 * n] + I * z[2 * n + 1];
                cplx gm = riccati_fixed_point(conj(dseg[0]), zn + aseg[0], dseg[0]);
                for (int q = 0; q <= ns; ++q) {
                    gm = riccati_advance(g, conj(dseg[q]), zn + aseg[q], dseg[q], lseg[q], gm);
                    if (q < ns) gam[q] = gm;
                }
                cplx gt = riccati_fixed_point(-dseg[ns], zn + aseg[ns], -conj(dseg[ns]));
                for (int q = ns; q >= 0; --q) {
                    gt = riccati_advance(g, -dseg[q], zn + aseg[q], -conj(dseg[q]), lseg[q], gt);
                    if (q > 0) gat[q - 1] = gt;
                }
                for (int q = 0; q < ns; ++q) {
                    cplx ga = gam[q], gb = gat[q];
                    cplx den = 1.0 + ga * gb;
                    cplx gg = -I * M_PI * (1.0 - ga * gb) / den;
                    cplx ff = -2.0 * I * M_PI * ga / den;
                    cplx ft = 2.0 * I * M_PI * gb / den;
                    cplx In = (conj(dsm[q]) * ff + dsm[q] * ft) / (M_PI + I * gg);
                    double *im = &images[4 * (out_off + sidx[q])];
                    cplx sf = ff + conj(ft);
                    double wn = g->ewt ? g->ewt[n] : 1.0;
                    im[0] += wn * creal(sf);
                    im[1] += wn * cimag(sf);
                    im[2] += wn * 2.0 * creal(gg);
                    im[3] += wn * 2.0 * creal(In);
                }
            }
            free(gam);
            free(gat);
            free(dseg);
            free(aseg);
            free(lseg);
            free(dsm);
            free(asm_);
            free(sidx);
        }
        free(dS);
        free(aS);
        out_off += nsp;
    }
    return 0;
}

