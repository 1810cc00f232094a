// Host-side grain geometry for the Riccati sweep: mask, nearest-grain-point
// map, one rotated square lattice per angle pair, chords and the specular
// boundary links.  Built once per grain on the CPU (Sec. 3.1 of the paper:
// square reference grid with spacing h; per Fermi angle a rotated square
// lattice with the same spacing; bilinear interpolation between the two;
// boundary values interpolated in angle and boundary coordinate).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "sc.h"

namespace scg {

// Geometric decisions (inside test, chord existence, sample inclusion, active
// polygon edge) are taken with this tolerance in units of h, so that points
// that lie on a boundary up to rounding are treated as on it.
constexpr double kTol = 1e-9;

struct Tap {
    int32_t slot;   // exit slot: angle k < P -> line index; k >= P -> n_lines + line index
    double w;
};

struct LineInfo {
    int32_t pair, l;        // pair index and lattice line index
    double smin, smax;      // chord along e_par
    int32_t m0, m1, ns;     // samples m0..m1 (ns = m1 - m0 + 1, may be 0)
    int32_t slot0;          // first image slot (each line owns max(ns, 1) slots)
    int32_t edge_lo, edge_hi;  // polygon edges at smin / smax (-1 for a disc)
    int32_t nearest;        // nearest line of the same pair that has samples
    Tap fwd[4], bwd[4];     // entry links of angle p (at smin) and p + P (at smax)
    int32_t dbg_fwd_angle[4], dbg_fwd_line[4], dbg_bwd_angle[4], dbg_bwd_line[4];
};

struct PairInfo {
    double ex, ey;          // e_par = (cos phi_p, sin phi_p); e_perp = (-ey, ex)
    double eta;             // basis function at phi_p (= at phi_p + pi), component 0
    double eta_c[4];        // basis function of each order-parameter component
    double wsum;            // quadrature weight of phi_p plus that of phi_p + pi
    int32_t l_lo, l_hi, line0;
};

class Geometry {
public:
    // Returns an empty string on success, else the reason.
    std::string build(const sc_params &p);

    sc_params prm{};
    std::vector<double> vx, vy, enx, eny;  // polygon vertices, unit outward edge normals
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
    std::vector<LineInfo> lines;
    int64_t n_slots = 0, n_samples = 0;
    int32_t max_ns = 0;

    double signed_distance(double x, double y) const;

private:
    bool intersect(double bx, double by, double ex, double ey, double &s0, double &s1, int &e0,
                   int &e1) const;
    void outward_normal(double px, double py, int edge, double &nx_, double &ny_) const;
    void link(double px, double py, double ux, double uy, Tap *taps, int32_t *dbg_angle,
              int32_t *dbg_line) const;
    int32_t exit_slot(int angle, int line_index) const;
};

double basis_function(int pairing, double crystal_rotation, double c, double s);
double quadrature_weight(int k, int n);

}  // namespace scg
