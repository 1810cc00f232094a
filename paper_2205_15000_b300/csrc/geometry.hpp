// Host-side grain geometry for the Riccati sweep: mask, nearest-grain-point
// map, one rotated square lattice per angle pair, chords and the specular
// boundary links.  Built once per grain on the CPU (Sec. 3.1 of the paper:
// square reference grid with spacing h; per Fermi angle a rotated square
// lattice with the same spacing; bilinear interpolation between the two;
// boundary values interpolated in angle and boundary coordinate).  A grain is
// a list of discs and convex polygons, each added to or removed from the
// grain made of those before it (Sec. 4 and App. B, composite geometries).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "sc.h"

namespace scg {

// Geometric decisions (inside test, chord existence, sample inclusion, active
// polygon edge, merging of touching chords) are taken with this tolerance in
// units of h, so that points that lie on a boundary up to rounding are treated
// as on it.
constexpr double kTol = 1e-9;

// One part of the grain.
struct Part {
    int kind = 0;                       // 0 disc, 1 convex polygon
    bool add = true;                    // added or removed
    double cx = 0, cy = 0, r = 0;       // disc
    std::vector<double> vx, vy, nx, ny; // polygon: CCW vertices, unit outward edge normals

    double sdist(double x, double y) const;  // signed distance, negative inside
    // Interval [s0, s1] of the line B + s e inside the part, longer than tol;
    // e0 / e1: entering / leaving polygon edge (lowest index within tol of the
    // extremum), -1 for a disc.
    bool chord(double bx, double by, double ex, double ey, double tol, double &s0, double &s1, int &e0,
               int &e1) const;
};

// Where a chord ends: on the boundary of part `part` (polygon edge `edge`,
// -1 for a disc); side +1 when the grain lies on the part's inner side (an
// added part), -1 on its outer side (a removed part).
struct End {
    int32_t part = 0, edge = -1, side = 1;
};

struct Tap {
    int32_t slot;   // exit slot: angle k < P -> line index; k >= P -> n_lines + line index
    double w;
};

// One chord ("line" of the sweep): a maximal piece of a lattice line inside
// the grain.  Chords are ordered by pair, lattice line l, then s.
struct LineInfo {
    int32_t pair, l;        // pair index and lattice line index
    double smin, smax;      // chord along e_par
    int32_t m0, m1, ns;     // samples m0..m1 (ns = m1 - m0 + 1, may be 0)
    int32_t slot0;          // first image slot (each chord owns max(ns, 1) slots)
    End lo, hi;             // boundary at smin / smax
    Tap fwd[4], bwd[4];     // entry links of angle p (at smin) and p + P (at smax)
    int32_t dbg_fwd_angle[4], dbg_fwd_line[4], dbg_fwd_chord[4];
    int32_t dbg_bwd_angle[4], dbg_bwd_line[4], dbg_bwd_chord[4];
};

// The chords of one lattice line of a pair.
struct LatticeLine {
    int32_t c0, nc;         // chords c0 .. c0 + nc - 1 (ascending s)
    int32_t chorded;        // nearest lattice line l of the pair with a chord
    int32_t sampled;        // nearest lattice line l of the pair with a sampled chord
};

struct PairInfo {
    double ex, ey;          // e_par = (cos phi_p, sin phi_p); e_perp = (-ey, ex)
    double eta;             // basis function at phi_p (= at phi_p + pi), component 0
    double eta_c[4];        // basis function of each order-parameter component
    double wsum;            // quadrature weight of phi_p plus that of phi_p + pi
    int32_t l_lo, l_hi;     // lattice lines with chords lie in l_lo .. l_hi
    int32_t line0, n_lines; // chords line0 .. line0 + n_lines - 1
    int32_t lat0;           // lattice-line records lat0 .. lat0 + (l_hi - l_lo)
};

class Geometry {
public:
    // Returns an empty string on success, else the reason.
    std::string build(const sc_params &p);

    sc_params prm{};
    std::vector<Part> parts;
    double area = 0.0;
    double ox = 0.0, oy = 0.0;             // lattice origin
    int32_t nx = 0, ny = 0, n_angles = 0, n_pairs = 0;
    int32_t n_comp = 1;                    // order-parameter components
    double tc_ratio[4] = {1, 1, 1, 1};     // T_c^Gamma / T_c
    int64_t n_in = 0;
    std::vector<uint8_t> mask;
    std::vector<int32_t> ghost;            // (nx+2)*(ny+2)
    std::vector<double> weight;            // per angle
    std::vector<PairInfo> pairs;
    std::vector<LineInfo> lines;           // chords
    std::vector<LatticeLine> lats;
    int64_t n_slots = 0, n_samples = 0;
    int32_t max_ns = 0;

    double signed_distance(double x, double y) const;
    const LatticeLine &lat(int pair, int l) const { return lats[pairs[pair].lat0 + (l - pairs[pair].l_lo)]; }

private:
    struct Seg {
        double a, b;
        End ea, eb;
    };
    void chords(double bx, double by, double ex, double ey, std::vector<Seg> &out) const;
    void outward_normal(const End &e, double px, double py, double &nx_, double &ny_) const;
    void link(double px, double py, double ux, double uy, int part, Tap *taps, int32_t *dbg_angle,
              int32_t *dbg_line, int32_t *dbg_chord) const;
    int32_t exit_slot(int angle, int line_index) const;
    double composite_area() const;
};

double basis_function(int pairing, double crystal_rotation, double c, double s);
double quadrature_weight(int k, int n);

}  // namespace scg
