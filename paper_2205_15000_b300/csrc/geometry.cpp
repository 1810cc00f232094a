// Grain geometry for the Riccati sweep (host side, built once per grain).
//
// Conventions (Sec. 3.1 of the paper fixes the idea, these fix the details):
//  * grid point (i, j) at (x0 + (i + 1/2) h, y0 + (j + 1/2) h); it belongs to
//    the grain if its signed distance to the shape is <= kTol * h;
//  * angle pair p (0 <= p < P = N/2) owns the lattice O + l h e_perp + s e_par,
//    samples at s = m h; angle p travels along +e_par, angle p + P along -e_par
//    on the same lines;
//  * lines whose chord is longer than kTol * h are kept; samples are
//    ceil(smin/h - kTol) .. floor(smax/h + kTol);
//  * the entry value of a line is the bilinear combination, in angle and in
//    line coordinate, of exit values of the directions that reflect specularly
//    into it (outward normal of the disc, or of the active polygon edge).
#include "geometry.hpp"

#include <algorithm>
#include <cmath>
#include <limits>

namespace scg {

double quadrature_weight(int k, int n) {
    // Boole / Simpson 3/8 / Simpson 1/3 / trapezoid chosen by divisibility of n by
    // 4 / 3 / 2, closed on the periodic angle grid, normalised to sum 1.
    if (n % 4 == 0) {
        const double pattern[4] = {14.0, 32.0, 12.0, 32.0};
        return pattern[k % 4] * 2.0 / (45.0 * n);
    }
    if (n % 3 == 0) {
        const double pattern[3] = {2.0, 3.0, 3.0};
        return pattern[k % 3] * 3.0 / (8.0 * n);
    }
    if (n % 2 == 0) {
        const double pattern[2] = {2.0, 4.0};
        return pattern[k % 2] / (3.0 * n);
    }
    return 1.0 / n;
}

double basis_function(int pairing, double crystal_rotation, double c, double s) {
    // Table basis_functions for a circular Fermi surface, in the crystal frame.
    const double th = 2.0 * M_PI * crystal_rotation;
    const double cc = c * std::cos(th) + s * std::sin(th);
    const double ss = s * std::cos(th) - c * std::sin(th);
    const double cos2 = cc * cc - ss * ss, sin2 = 2.0 * cc * ss;
    const double r2 = std::sqrt(2.0);
    switch (pairing) {
        case SC_PAIR_S: return 1.0;
        case SC_PAIR_DX2Y2: return r2 * cos2;
        case SC_PAIR_DXY: return r2 * sin2;
        case SC_PAIR_G: return r2 * 2.0 * sin2 * cos2;
        default: return 0.0;
    }
}

double Geometry::signed_distance(double x, double y) const {
    if (prm.shape_kind == 0) return std::hypot(x - prm.disc_cx, y - prm.disc_cy) - prm.disc_r;
    double d = -std::numeric_limits<double>::infinity();
    for (size_t e = 0; e < vx.size(); ++e)
        d = std::max(d, (x - vx[e]) * enx[e] + (y - vy[e]) * eny[e]);
    return d;
}

bool Geometry::intersect(double bx, double by, double ex, double ey, double &s0, double &s1,
                         int &e0, int &e1) const {
    const double tol = kTol * prm.h;
    e0 = e1 = -1;
    if (prm.shape_kind == 0) {
        const double dx = bx - prm.disc_cx, dy = by - prm.disc_cy;
        const double b = dx * ex + dy * ey;
        const double disc = b * b - (dx * dx + dy * dy - prm.disc_r * prm.disc_r);
        if (!(disc > 0.0)) return false;
        const double r = std::sqrt(disc);
        s0 = -b - r;
        s1 = -b + r;
        return s1 - s0 > tol;
    }
    // clip the line against each half-plane (P - V_e) . n_e <= 0
    const size_t n = vx.size();
    std::vector<double> lim(n, 0.0);
    std::vector<int> side(n, 0);
    double lo = -std::numeric_limits<double>::infinity();
    double hi = std::numeric_limits<double>::infinity();
    for (size_t e = 0; e < n; ++e) {
        const double f0 = (bx - vx[e]) * enx[e] + (by - vy[e]) * eny[e];
        const double rate = ex * enx[e] + ey * eny[e];
        if (rate == 0.0) {
            if (f0 > 0.0) return false;
            continue;
        }
        lim[e] = -f0 / rate;
        side[e] = rate > 0.0 ? +1 : -1;
        if (rate > 0.0) hi = std::min(hi, lim[e]);
        else lo = std::max(lo, lim[e]);
    }
    for (size_t e = 0; e < n; ++e) {
        if (e0 < 0 && side[e] < 0 && lim[e] >= lo - tol) e0 = (int)e;
        if (e1 < 0 && side[e] > 0 && lim[e] <= hi + tol) e1 = (int)e;
    }
    s0 = lo;
    s1 = hi;
    return s1 - s0 > tol;
}

void Geometry::outward_normal(double px, double py, int edge, double &nx_, double &ny_) const {
    if (prm.shape_kind == 0) {
        const double dx = px - prm.disc_cx, dy = py - prm.disc_cy;
        const double r = std::hypot(dx, dy);
        nx_ = dx / r;
        ny_ = dy / r;
    } else {
        nx_ = enx[edge];
        ny_ = eny[edge];
    }
}

int32_t Geometry::exit_slot(int angle, int line_index) const {
    return angle < n_pairs ? line_index : (int32_t)lines.size() + line_index;
}

void Geometry::link(double px, double py, double ux, double uy, Tap *taps, int32_t *dbg_angle,
                    int32_t *dbg_line) const {
    // angle coordinate of the incoming direction on the discrete Fermi surface
    double psi = std::atan2(uy, ux);
    if (psi < 0.0) psi += 2.0 * M_PI;
    const double ua = psi * n_angles / (2.0 * M_PI);
    int a0 = (int)std::floor(ua);
    const double fa = ua - a0;
    a0 = ((a0 % n_angles) + n_angles) % n_angles;
    const int angles[2] = {a0, (a0 + 1) % n_angles};
    const double wa[2] = {1.0 - fa, fa};
    int q = 0;
    for (int ia = 0; ia < 2; ++ia) {
        const int k = angles[ia];
        const PairInfo &pp = pairs[k % n_pairs];
        // line coordinate of the point in that pair's lattice
        const double c = ((px - ox) * (-pp.ey) + (py - oy) * pp.ex) / prm.h;
        const int l0 = (int)std::floor(c);
        const double fl = c - l0;
        for (int il = 0; il < 2; ++il) {
            const int l = std::min(std::max(l0 + il, pp.l_lo), pp.l_hi);
            const int li = pp.line0 + (l - pp.l_lo);
            taps[q].slot = exit_slot(k, li);
            taps[q].w = wa[ia] * (il ? fl : 1.0 - fl);
            dbg_angle[q] = k;
            dbg_line[q] = l;
            ++q;
        }
    }
}

std::string Geometry::build(const sc_params &p) {
    prm = p;
    nx = p.nx;
    ny = p.ny;
    n_angles = p.n_angles;
    const double h = p.h;
    if (nx < 2 || ny < 2 || !(h > 0.0)) return "grid needs nx, ny >= 2 and h > 0";
    if ((int64_t)nx * ny > (int64_t)1 << 28) return "grid too large";
    if (n_angles < 2 || n_angles % 2) return "n_angles must be even and >= 2";
    if (n_angles > 8192) return "n_angles too large";
    if (p.n_energies < 1 || p.n_energies > 4096) return "n_energies must be in [1, 4096]";
    if (!(p.t > 0.0 && p.t <= 1.0)) return "t must be in (0, 1]";
    if (p.charge_sign != 1 && p.charge_sign != -1) return "charge_sign must be +1 or -1";
    if (p.pairing < 0 || p.pairing > 3) return "unknown pairing";
    if (p.n_components < 0 || p.n_components > 4) return "n_components must be 0 to 4";
    n_comp = p.n_components > 1 ? p.n_components : 1;
    for (int c = 0; c < n_comp; ++c) {
        const int pc = c == 0 ? p.pairing : p.pairings[c];
        if (pc < 0 || pc > 3) return "unknown pairing of a component";
        if (!(p.tc_ratios[c] >= 0.0) || !std::isfinite(p.tc_ratios[c])) return "tc_ratios must be >= 0";
        tc_ratio[c] = p.tc_ratios[c] > 0.0 ? p.tc_ratios[c] : 1.0;
    }
    n_pairs = n_angles / 2;

    if (p.shape_kind == 1) {
        if (p.n_vert < 3 || !p.vx || !p.vy) return "polygon needs >= 3 vertices";
        vx.assign(p.vx, p.vx + p.n_vert);
        vy.assign(p.vy, p.vy + p.n_vert);
        const int n = p.n_vert;
        enx.resize(n);
        eny.resize(n);
        double twice_area = 0.0;
        for (int e = 0; e < n; ++e) {
            const int f = (e + 1) % n;
            const double dx = vx[f] - vx[e], dy = vy[f] - vy[e];
            const double len = std::hypot(dx, dy);
            if (!(len > 0.0)) return "polygon has a repeated vertex";
            enx[e] = dy / len;
            eny[e] = -dx / len;
            twice_area += vx[e] * vy[f] - vx[f] * vy[e];
            // convexity: the next vertex must not lie to the right of edge e
            const int g = (f + 1) % n;
            const double cross = dx * (vy[g] - vy[f]) - dy * (vx[g] - vx[f]);
            if (cross < 0.0) return "polygon must be convex and counter-clockwise";
        }
        area = 0.5 * twice_area;
        if (!(area > 0.0)) return "polygon must be counter-clockwise";
    } else if (p.shape_kind == 0) {
        if (!(p.disc_r > 0.0)) return "disc radius must be > 0";
        area = M_PI * p.disc_r * p.disc_r;
    } else {
        return "unknown shape_kind";
    }
    prm.vx = vx.empty() ? nullptr : vx.data();
    prm.vy = vy.empty() ? nullptr : vy.data();

    // the grid box must contain the shape
    const double X0 = p.x0, X1 = p.x0 + nx * h, Y0 = p.y0, Y1 = p.y0 + ny * h;
    if (p.shape_kind == 0) {
        if (p.disc_cx - p.disc_r < X0 || p.disc_cx + p.disc_r > X1 || p.disc_cy - p.disc_r < Y0 ||
            p.disc_cy + p.disc_r > Y1)
            return "shape extends outside the grid box";
    } else {
        for (size_t e = 0; e < vx.size(); ++e)
            if (vx[e] < X0 || vx[e] > X1 || vy[e] < Y0 || vy[e] > Y1)
                return "shape extends outside the grid box";
    }

    // mask
    mask.assign((size_t)nx * ny, 0);
    n_in = 0;
    for (int j = 0; j < ny; ++j) {
        const double y = p.y0 + (j + 0.5) * h;
        for (int i = 0; i < nx; ++i) {
            const double x = p.x0 + (i + 0.5) * h;
            if (signed_distance(x, y) <= kTol * h) {
                mask[(size_t)j * nx + i] = 1;
                ++n_in;
            }
        }
    }
    if (n_in == 0) return "no grid point inside the grain";

    // nearest grain point for padded indices within 1.5 h of the shape: expanding
    // square rings; exact integer distances, ties to the lowest row-major index
    const int px = nx + 2, py = ny + 2;
    ghost.assign((size_t)px * py, -1);
    for (int jj = 0; jj < py; ++jj) {
        for (int ii = 0; ii < px; ++ii) {
            const int i = ii - 1, j = jj - 1;
            const bool in_grid = i >= 0 && i < nx && j >= 0 && j < ny;
            if (in_grid && mask[(size_t)j * nx + i]) {
                ghost[(size_t)jj * px + ii] = j * nx + i;
                continue;
            }
            if (signed_distance(p.x0 + (i + 0.5) * h, p.y0 + (j + 0.5) * h) > 1.5 * h) continue;
            int64_t best_d = -1, best_idx = -1;
            const int rmax = std::max(nx, ny) + 2;
            for (int r = 1; r <= rmax; ++r) {
                for (int dj = -r; dj <= r; ++dj) {
                    const int jq = j + dj;
                    if (jq < 0 || jq >= ny) continue;
                    const int step = (dj == -r || dj == r) ? 1 : 2 * r;
                    for (int di = -r; di <= r; di += step) {
                        const int iq = i + di;
                        if (iq < 0 || iq >= nx || !mask[(size_t)jq * nx + iq]) continue;
                        const int64_t d = (int64_t)di * di + (int64_t)dj * dj;
                        const int64_t idx = (int64_t)jq * nx + iq;
                        if (best_d < 0 || d < best_d || (d == best_d && idx < best_idx)) {
                            best_d = d;
                            best_idx = idx;
                        }
                    }
                }
                if (best_d >= 0 && best_d <= (int64_t)r * r) break;
            }
            ghost[(size_t)jj * px + ii] = (int32_t)best_idx;
        }
    }

    // Fermi surface: angle p + P is exactly opposite to angle p
    weight.resize(n_angles);
    for (int k = 0; k < n_angles; ++k) weight[k] = quadrature_weight(k, n_angles);
    pairs.resize(n_pairs);
    for (int q = 0; q < n_pairs; ++q) {
        const double phi = 2.0 * M_PI * q / n_angles;
        pairs[q].ex = std::cos(phi);
        pairs[q].ey = std::sin(phi);
        for (int c = 0; c < 4; ++c)
            pairs[q].eta_c[c] = c < n_comp ? basis_function(c == 0 ? p.pairing : p.pairings[c], p.crystal_rotation,
                                                            pairs[q].ex, pairs[q].ey)
                                           : 0.0;
        pairs[q].eta = pairs[q].eta_c[0];
        pairs[q].wsum = weight[q] + weight[q + n_pairs];
    }

    // lattices
    ox = p.x0 + 0.5 * nx * h + p.lattice_ox * h;
    oy = p.y0 + 0.5 * ny * h + p.lattice_oy * h;
    double reach = 0.0;
    if (p.shape_kind == 0) {
        reach = std::hypot(p.disc_cx - ox, p.disc_cy - oy) + p.disc_r;
    } else {
        for (size_t e = 0; e < vx.size(); ++e) reach = std::max(reach, std::hypot(vx[e] - ox, vy[e] - oy));
    }
    const int lmax = (int)std::ceil(reach / h) + 1;
    lines.clear();
    n_slots = 0;
    n_samples = 0;
    max_ns = 0;
    for (int q = 0; q < n_pairs; ++q) {
        PairInfo &pp = pairs[q];
        const double qx = -pp.ey, qy = pp.ex;
        pp.l_lo = std::numeric_limits<int>::max();
        pp.l_hi = std::numeric_limits<int>::min();
        pp.line0 = (int32_t)lines.size();
        for (int l = -lmax; l <= lmax; ++l) {
            double s0, s1;
            int e0, e1;
            const double bx = ox + l * h * qx, by = oy + l * h * qy;
            const bool hit = intersect(bx, by, pp.ex, pp.ey, s0, s1, e0, e1);
            if (!hit) {
                if (pp.l_lo <= pp.l_hi) {
                    // a convex shape has one contiguous run of lines
                    double t0, t1;
                    int f0, f1;
                    for (int l2 = l + 1; l2 <= lmax; ++l2)
                        if (intersect(ox + l2 * h * qx, oy + l2 * h * qy, pp.ex, pp.ey, t0, t1, f0, f1))
                            return "line range not contiguous (shape not convex?)";
                    break;
                }
                continue;
            }
            pp.l_lo = std::min(pp.l_lo, l);
            pp.l_hi = std::max(pp.l_hi, l);
            LineInfo li{};
            li.pair = q;
            li.l = l;
            li.smin = s0;
            li.smax = s1;
            li.edge_lo = e0;
            li.edge_hi = e1;
            li.m0 = (int)std::ceil(s0 / h - kTol);
            li.m1 = (int)std::floor(s1 / h + kTol);
            li.ns = std::max(0, li.m1 - li.m0 + 1);
            li.slot0 = (int32_t)n_slots;
            n_slots += std::max(li.ns, 1);
            n_samples += li.ns;
            max_ns = std::max(max_ns, li.ns);
            lines.push_back(li);
        }
        if (pp.l_lo > pp.l_hi) return "an angle pair has no line through the grain";
        // nearest line with samples
        bool any = false;
        for (int l = pp.l_lo; l <= pp.l_hi; ++l) any = any || lines[pp.line0 + l - pp.l_lo].ns > 0;
        if (!any) return "an angle pair has no lattice sample in the grain";
        for (int l = pp.l_lo; l <= pp.l_hi; ++l) {
            // line indices can be negative: search outward with an explicit flag
            int best = l;
            bool found = false;
            for (int d = 0; !found; ++d) {
                if (l - d >= pp.l_lo && lines[pp.line0 + l - d - pp.l_lo].ns > 0) {
                    best = l - d;
                    found = true;
                } else if (l + d <= pp.l_hi && lines[pp.line0 + l + d - pp.l_lo].ns > 0) {
                    best = l + d;
                    found = true;
                }
            }
            lines[pp.line0 + l - pp.l_lo].nearest = pp.line0 + best - pp.l_lo;
        }
    }

    // specular links; angle p enters at smin, angle p + P at smax
    for (size_t L = 0; L < lines.size(); ++L) {
        LineInfo &li = lines[L];
        const PairInfo &pp = pairs[li.pair];
        const double bx = ox + li.l * h * (-pp.ey), by = oy + li.l * h * pp.ex;
        for (int dir = 0; dir < 2; ++dir) {
            const double s = dir == 0 ? li.smin : li.smax;
            const int edge = dir == 0 ? li.edge_lo : li.edge_hi;
            const double vx_ = dir == 0 ? pp.ex : -pp.ex, vy_ = dir == 0 ? pp.ey : -pp.ey;
            const double px_ = bx + s * pp.ex, py_ = by + s * pp.ey;
            double nx_, ny_;
            outward_normal(px_, py_, edge, nx_, ny_);
            const double vn = vx_ * nx_ + vy_ * ny_;
            // the trajectory that arrives at the point and reflects into v
            const double ux = vx_ - 2.0 * vn * nx_, uy = vy_ - 2.0 * vn * ny_;
            if (dir == 0) link(px_, py_, ux, uy, li.fwd, li.dbg_fwd_angle, li.dbg_fwd_line);
            else link(px_, py_, ux, uy, li.bwd, li.dbg_bwd_angle, li.dbg_bwd_line);
        }
    }
    return std::string();
}

}  // namespace scg
