// Grain geometry for the Riccati sweep (host side, built once per grain).
//
// Conventions (Sec. 3.1 of the paper fixes the idea, these fix the details):
//  * the grain is built from its parts in order: union with an added part,
//    difference with a removed one; its signed distance is the minimum with an
//    added part's and the maximum with a removed part's negated distance;
//  * grid point (i, j) at (x0 + (i + 1/2) h, y0 + (j + 1/2) h); it belongs to
//    the grain if its signed distance is <= kTol * h;
//  * angle pair p (0 <= p < P = N/2) owns the lattice O + l h e_perp + s e_par,
//    samples at s = m h; angle p travels along +e_par, angle p + P along -e_par
//    on the same lines;
//  * the chords of a lattice line are the maximal pieces inside the grain,
//    longer than kTol * h (pieces that touch within kTol * h merge); samples are
//    ceil(smin/h - kTol) .. floor(smax/h + kTol);
//  * the entry value of a chord is the bilinear combination, in angle and in
//    line coordinate, of exit values of the directions that reflect specularly
//    into it (the grain's outward normal where the chord starts); on each
//    tapped lattice line the chord is the one whose exit lies on the same part,
//    nearest to the reflection point.
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

double Part::sdist(double x, double y) const {
    if (kind == 0) return std::hypot(x - cx, y - cy) - r;
    double d = -std::numeric_limits<double>::infinity();
    for (size_t e = 0; e < vx.size(); ++e) d = std::max(d, (x - vx[e]) * nx[e] + (y - vy[e]) * ny[e]);
    return d;
}

bool Part::chord(double bx, double by, double ex, double ey, double tol, double &s0, double &s1, int &e0,
                 int &e1) const {
    e0 = e1 = -1;
    if (kind == 0) {
        const double dx = bx - cx, dy = by - cy;
        const double b = dx * ex + dy * ey;
        const double disc = b * b - (dx * dx + dy * dy - r * r);
        if (!(disc > 0.0)) return false;
        const double q = std::sqrt(disc);
        s0 = -b - q;
        s1 = -b + q;
        return s1 - s0 > tol;
    }
    // clip the line against each half-plane (P - V_e) . n_e <= 0
    const size_t n = vx.size();
    std::vector<double> lim(n, 0.0);
    std::vector<int> side(n, 0);
    double lo = -std::numeric_limits<double>::infinity();
    double hi = std::numeric_limits<double>::infinity();
    for (size_t e = 0; e < n; ++e) {
        const double f0 = (bx - vx[e]) * nx[e] + (by - vy[e]) * ny[e];
        const double rate = ex * nx[e] + ey * ny[e];
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

double Geometry::signed_distance(double x, double y) const {
    double d = std::numeric_limits<double>::infinity();
    for (const Part &q : parts) d = q.add ? std::min(d, q.sdist(x, y)) : std::max(d, -q.sdist(x, y));
    return d;
}

void Geometry::chords(double bx, double by, double ex, double ey, std::vector<Seg> &out) const {
    const double tol = kTol * prm.h;
    out.clear();
    std::vector<Seg> next;
    for (size_t k = 0; k < parts.size(); ++k) {
        const Part &q = parts[k];
        double a, b;
        int e0, e1;
        if (!q.chord(bx, by, ex, ey, tol, a, b, e0, e1)) continue;
        const int32_t side = q.add ? 1 : -1;
        Seg s{a, b, End{(int32_t)k, e0, side}, End{(int32_t)k, e1, side}};
        next.clear();
        if (q.add) {
            // union: absorb every chord that overlaps or touches; on equal ends
            // the earlier part keeps the end
            bool placed = false;
            for (const Seg &c : out) {
                if (c.b < s.a - tol) {
                    next.push_back(c);
                } else if (c.a > s.b + tol) {
                    if (!placed) next.push_back(s);
                    placed = true;
                    next.push_back(c);
                } else {
                    if (c.a <= s.a) {
                        s.a = c.a;
                        s.ea = c.ea;
                    }
                    if (c.b >= s.b) {
                        s.b = c.b;
                        s.eb = c.eb;
                    }
                }
            }
            if (!placed) next.push_back(s);
        } else {
            // difference: a chord overlapped by more than tol loses the overlap;
            // pieces not longer than tol disappear
            for (const Seg &c : out) {
                if (c.b <= s.a + tol || c.a >= s.b - tol) {
                    next.push_back(c);
                    continue;
                }
                if (s.a - c.a > tol) next.push_back(Seg{c.a, s.a, c.ea, s.ea});
                if (c.b - s.b > tol) next.push_back(Seg{s.b, c.b, s.eb, c.eb});
            }
        }
        out.swap(next);
    }
}

void Geometry::outward_normal(const End &e, double px, double py, double &nx_, double &ny_) const {
    const Part &q = parts[e.part];
    if (q.kind == 0) {
        const double dx = px - q.cx, dy = py - q.cy;
        const double r = std::hypot(dx, dy);
        nx_ = e.side * dx / r;
        ny_ = e.side * dy / r;
    } else {
        nx_ = e.side * q.nx[e.edge];
        ny_ = e.side * q.ny[e.edge];
    }
}

int32_t Geometry::exit_slot(int angle, int line_index) const {
    return angle < n_pairs ? line_index : (int32_t)lines.size() + line_index;
}

void Geometry::link(double px, double py, double ux, double uy, int part, Tap *taps, int32_t *dbg_angle,
                    int32_t *dbg_line, int32_t *dbg_chord) const {
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
        const bool forward = k < n_pairs;  // exits at smax
        const PairInfo &pp = pairs[k % n_pairs];
        // line coordinate of the point in that pair's lattice, and its position along the lines
        const double c = ((px - ox) * (-pp.ey) + (py - oy) * pp.ex) / prm.h;
        const double sp = (px - ox) * pp.ex + (py - oy) * pp.ey;
        const int l0 = (int)std::floor(c);
        const double fl = c - l0;
        int pick[2];
        bool on_part[2];
        for (int il = 0; il < 2; ++il) {
            const int l = std::min(std::max(l0 + il, pp.l_lo), pp.l_hi);
            const LatticeLine &lt = lat(k % n_pairs, lat(k % n_pairs, l).chorded);
            // the chord whose exit lies on the same part nearest to the point,
            // else the nearest exit of any part
            int best = -1, best_same = -1;
            double d_best = 0.0, d_same = 0.0;
            for (int ci = lt.c0; ci < lt.c0 + lt.nc; ++ci) {
                const LineInfo &li = lines[ci];
                const double d = std::fabs((forward ? li.smax : li.smin) - sp);
                const int32_t ep = forward ? li.hi.part : li.lo.part;
                if (best < 0 || d < d_best) {
                    best = ci;
                    d_best = d;
                }
                if (ep == part && (best_same < 0 || d < d_same)) {
                    best_same = ci;
                    d_same = d;
                }
            }
            on_part[il] = best_same >= 0;
            pick[il] = on_part[il] ? best_same : best;
        }
        // a lattice line that passes the part (beside a hole) lends its weight
        // to the other line's chord
        if (on_part[0] != on_part[1]) pick[0] = pick[1] = on_part[0] ? pick[0] : pick[1];
        for (int il = 0; il < 2; ++il) {
            taps[q].slot = exit_slot(k, pick[il]);
            taps[q].w = wa[ia] * (il ? fl : 1.0 - fl);
            dbg_angle[q] = k;
            dbg_line[q] = lines[pick[il]].l;
            dbg_chord[q] = pick[il] - pp.line0;
            ++q;
        }
    }
}

// Area of a composite grain by Green's theorem, A = (1/2) \oint (x dy - y dx)
// over its boundary.  Every part's boundary (circle, or polygon edges) is cut
// where another part's boundary crosses it or one of its vertices lies on it;
// a piece belongs to the grain's boundary when the grain lies on exactly one
// side of it (tested a small distance either side of its midpoint) and then
// contributes its line integral in the part's counter-clockwise sense, with
// the sign of the side the grain is on.  A piece on an earlier part's boundary
// is left to that part.
double Geometry::composite_area() const {
    double ext = 0.0;
    for (const Part &q : parts) {
        if (q.kind == 0) ext = std::max(ext, std::fabs(q.cx) + std::fabs(q.cy) + q.r);
        for (size_t e = 0; e < q.vx.size(); ++e) ext = std::max(ext, std::fabs(q.vx[e]) + std::fabs(q.vy[e]));
    }
    const double probe = 1e-9 * std::max(ext, 1.0);
    auto inside = [&](double x, double y) { return signed_distance(x, y) <= 0.0; };
    auto on_earlier = [&](size_t k, double x, double y) {
        for (size_t j = 0; j < k; ++j)
            if (std::fabs(parts[j].sdist(x, y)) < 16 * probe) {
                // a polygon's sdist vanishes on the lines of its edges: check the segment
                const Part &q = parts[j];
                if (q.kind == 0) return true;
                for (size_t e = 0; e < q.vx.size(); ++e) {
                    const size_t f = (e + 1) % q.vx.size();
                    const double dx = q.vx[f] - q.vx[e], dy = q.vy[f] - q.vy[e];
                    const double t = ((x - q.vx[e]) * dx + (y - q.vy[e]) * dy) / (dx * dx + dy * dy);
                    if (t < -1e-12 || t > 1 + 1e-12) continue;
                    if (std::hypot(q.vx[e] + t * dx - x, q.vy[e] + t * dy - y) < 16 * probe) return true;
                }
            }
        return false;
    };
    // crossings of a segment P0 + t D (0 <= t <= 1) with part j's boundary: parameters t
    auto cut_segment = [&](const Part &o, double x0, double y0, double dx, double dy, std::vector<double> &ts) {
        if (o.kind == 0) {
            const double fx = x0 - o.cx, fy = y0 - o.cy;
            const double A = dx * dx + dy * dy, B = 2 * (fx * dx + fy * dy), C = fx * fx + fy * fy - o.r * o.r;
            const double disc = B * B - 4 * A * C;
            if (disc < 0) return;
            const double sq = std::sqrt(disc);
            for (double t : {(-B - sq) / (2 * A), (-B + sq) / (2 * A)})
                if (t > 0 && t < 1) ts.push_back(t);
            return;
        }
        const size_t n = o.vx.size();
        for (size_t e = 0; e < n; ++e) {
            const size_t f = (e + 1) % n;
            const double sx = o.vx[f] - o.vx[e], sy = o.vy[f] - o.vy[e];
            const double den = dx * sy - dy * sx;
            const double qx = o.vx[e] - x0, qy = o.vy[e] - y0;
            if (den != 0.0) {
                const double t = (qx * sy - qy * sx) / den, u = (qx * dy - qy * dx) / den;
                if (t > 0 && t < 1 && u >= 0 && u <= 1) ts.push_back(t);
            }
            // a vertex of the other part on the segment
            const double L2 = dx * dx + dy * dy;
            const double t = (qx * dx + qy * dy) / L2;
            if (t > 0 && t < 1 && std::fabs(qx * dy - qy * dx) / std::sqrt(L2) < probe) ts.push_back(t);
        }
    };
    double A2 = 0.0;  // twice the area
    for (size_t k = 0; k < parts.size(); ++k) {
        const Part &q = parts[k];
        if (q.kind == 0) {
            std::vector<double> th;
            for (size_t j = 0; j < parts.size(); ++j) {
                if (j == k) continue;
                const Part &o = parts[j];
                if (o.kind == 0) {
                    const double dx = o.cx - q.cx, dy = o.cy - q.cy, d = std::hypot(dx, dy);
                    if (d == 0.0 || d > q.r + o.r || d < std::fabs(q.r - o.r)) continue;
                    const double a = std::acos(std::max(-1.0, std::min(1.0, (q.r * q.r + d * d - o.r * o.r) / (2 * q.r * d))));
                    const double base = std::atan2(dy, dx);
                    th.push_back(base - a);
                    th.push_back(base + a);
                } else {
                    const size_t n = o.vx.size();
                    for (size_t e = 0; e < n; ++e) {
                        const size_t f = (e + 1) % n;
                        std::vector<double> ts;
                        const double dx = o.vx[f] - o.vx[e], dy = o.vy[f] - o.vy[e];
                        // circle crossings of the edge, and its end points on the circle
                        Part c = q;
                        cut_segment(c, o.vx[e], o.vy[e], dx, dy, ts);
                        ts.push_back(0.0);
                        for (double t : ts) {
                            const double x = o.vx[e] + t * dx, y = o.vy[e] + t * dy;
                            if (std::fabs(std::hypot(x - q.cx, y - q.cy) - q.r) < 16 * probe)
                                th.push_back(std::atan2(y - q.cy, x - q.cx));
                        }
                    }
                }
            }
            for (double &a : th) a = std::fmod(std::fmod(a, 2 * M_PI) + 2 * M_PI, 2 * M_PI);
            std::sort(th.begin(), th.end());
            if (th.empty()) th.push_back(0.0);
            for (size_t i = 0; i < th.size(); ++i) {
                const double t0 = th[i], t1 = i + 1 < th.size() ? th[i + 1] : th[0] + 2 * M_PI;
                if (!(t1 - t0 > 1e-15)) continue;
                const double tm = 0.5 * (t0 + t1), c = std::cos(tm), s = std::sin(tm);
                const double mx = q.cx + q.r * c, my = q.cy + q.r * s;
                const bool in_in = inside(mx - probe * c, my - probe * s);
                const bool in_out = inside(mx + probe * c, my + probe * s);
                if (in_in == in_out || on_earlier(k, mx, my)) continue;
                // int (x dy - y dx) over the arc t0 -> t1
                const double w = q.r * q.cx * (std::sin(t1) - std::sin(t0)) - q.r * q.cy * (std::cos(t1) - std::cos(t0)) +
                                 q.r * q.r * (t1 - t0);
                A2 += in_in ? w : -w;
            }
        } else {
            const size_t n = q.vx.size();
            for (size_t e = 0; e < n; ++e) {
                const size_t f = (e + 1) % n;
                const double x0 = q.vx[e], y0 = q.vy[e], dx = q.vx[f] - x0, dy = q.vy[f] - y0;
                std::vector<double> ts{0.0, 1.0};
                for (size_t j = 0; j < parts.size(); ++j)
                    if (j != k) cut_segment(parts[j], x0, y0, dx, dy, ts);
                std::sort(ts.begin(), ts.end());
                for (size_t i = 0; i + 1 < ts.size(); ++i) {
                    const double ta = ts[i], tb = ts[i + 1];
                    if (!(tb - ta > 1e-15)) continue;
                    const double tm = 0.5 * (ta + tb);
                    const double mx = x0 + tm * dx, my = y0 + tm * dy;
                    const bool in_in = inside(mx - probe * q.nx[e], my - probe * q.ny[e]);
                    const bool in_out = inside(mx + probe * q.nx[e], my + probe * q.ny[e]);
                    if (in_in == in_out || on_earlier(k, mx, my)) continue;
                    const double ax = x0 + ta * dx, ay = y0 + ta * dy, bx = x0 + tb * dx, by = y0 + tb * dy;
                    const double w = ax * by - bx * ay;
                    A2 += in_in ? w : -w;
                }
            }
        }
    }
    return 0.5 * A2;
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
    if (p.gauge < 0 || p.gauge > 2) return "unknown gauge";
    if (p.n_components < 0 || p.n_components > 4) return "n_components must be 0 to 4";
    n_comp = p.n_components > 1 ? p.n_components : 1;
    for (int c = 0; c < n_comp; ++c) {
        const int pc = c == 0 ? p.pairing : p.pairings[c];
        if (pc < 0 || pc > 3) return "unknown pairing of a component";
        if (!(p.tc_ratios[c] >= 0.0) || !std::isfinite(p.tc_ratios[c])) return "tc_ratios must be >= 0";
        tc_ratio[c] = p.tc_ratios[c] > 0.0 ? p.tc_ratios[c] : 1.0;
    }
    n_pairs = n_angles / 2;

    // parts
    auto load = [&](int kind, bool add, double cx, double cy, double r, int nv, const double *vx,
                    const double *vy) -> std::string {
        Part q;
        q.kind = kind;
        q.add = add;
        if (kind == 0) {
            if (!(r > 0.0)) return "disc radius must be > 0";
            q.cx = cx;
            q.cy = cy;
            q.r = r;
        } else if (kind == 1) {
            if (nv < 3 || !vx || !vy) return "polygon needs >= 3 vertices";
            q.vx.assign(vx, vx + nv);
            q.vy.assign(vy, vy + nv);
            q.nx.resize(nv);
            q.ny.resize(nv);
            double twice_area = 0.0;
            for (int e = 0; e < nv; ++e) {
                const int f = (e + 1) % nv, g = (f + 1) % nv;
                const double dx = q.vx[f] - q.vx[e], dy = q.vy[f] - q.vy[e];
                const double len = std::hypot(dx, dy);
                if (!(len > 0.0)) return "polygon has a repeated vertex";
                q.nx[e] = dy / len;
                q.ny[e] = -dx / len;
                twice_area += q.vx[e] * q.vy[f] - q.vx[f] * q.vy[e];
                // convexity: the next vertex must not lie to the right of edge e
                if (dx * (q.vy[g] - q.vy[f]) - dy * (q.vx[g] - q.vx[f]) < 0.0)
                    return "polygon must be convex and counter-clockwise";
            }
            if (!(twice_area > 0.0)) return "polygon must be counter-clockwise";
        } else {
            return "unknown part kind";
        }
        parts.push_back(std::move(q));
        return std::string();
    };
    parts.clear();
    if (p.shape_kind == SC_SHAPE_DISC || p.shape_kind == SC_SHAPE_POLYGON) {
        std::string why = load(p.shape_kind, true, p.disc_cx, p.disc_cy, p.disc_r, p.n_vert, p.vx, p.vy);
        if (!why.empty()) return why;
        const Part &q = parts[0];
        if (q.kind == 0) {
            area = M_PI * q.r * q.r;
        } else {
            double a2 = 0.0;
            for (size_t e = 0; e < q.vx.size(); ++e) {
                const size_t f = (e + 1) % q.vx.size();
                a2 += q.vx[e] * q.vy[f] - q.vx[f] * q.vy[e];
            }
            area = 0.5 * a2;
        }
    } else if (p.shape_kind == SC_SHAPE_COMPOSITE) {
        if (p.n_parts < 1 || !p.parts) return "a composite grain needs parts";
        if (p.n_parts > 4096) return "too many parts";
        for (int k = 0; k < p.n_parts; ++k) {
            const sc_part &s = p.parts[k];
            std::string why = load(s.kind, s.add != 0, s.cx, s.cy, s.r, s.n_vert, s.vx, s.vy);
            if (!why.empty()) return "part " + std::to_string(k) + ": " + why;
        }
        area = composite_area();
        if (!(area > 0.0)) return "the composite grain has no area";
    } else {
        return "unknown shape_kind";
    }
    prm.vx = prm.vy = nullptr;
    prm.parts = nullptr;
    prm.mask = nullptr;

    // the grid box must contain every added part
    const double X0 = p.x0, X1 = p.x0 + nx * h, Y0 = p.y0, Y1 = p.y0 + ny * h;
    for (const Part &q : parts) {
        if (!q.add) continue;
        if (q.kind == 0) {
            if (q.cx - q.r < X0 || q.cx + q.r > X1 || q.cy - q.r < Y0 || q.cy + q.r > Y1)
                return "shape extends outside the grid box";
        } else {
            for (size_t e = 0; e < q.vx.size(); ++e)
                if (q.vx[e] < X0 || q.vx[e] > X1 || q.vy[e] < Y0 || q.vy[e] > Y1)
                    return "shape extends outside the grid box";
        }
    }
    if (p.gauge == SC_GAUGE_SOLENOID && !(signed_distance(p.gauge_cx, p.gauge_cy) > kTol * h))
        return "solenoid gauge: the flux line (gauge origin) must lie outside the grain";

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
    for (const Part &q : parts) {
        if (!q.add) continue;
        if (q.kind == 0) reach = std::max(reach, std::hypot(q.cx - ox, q.cy - oy) + q.r);
        for (size_t e = 0; e < q.vx.size(); ++e) reach = std::max(reach, std::hypot(q.vx[e] - ox, q.vy[e] - oy));
    }
    const int lmax = (int)std::ceil(reach / h) + 1;
    lines.clear();
    lats.clear();
    n_slots = 0;
    n_samples = 0;
    max_ns = 0;
    std::vector<Seg> segs;
    std::vector<std::vector<Seg>> per_l(2 * lmax + 1);
    for (int q = 0; q < n_pairs; ++q) {
        PairInfo &pp = pairs[q];
        const double qx = -pp.ey, qy = pp.ex;
        pp.l_lo = std::numeric_limits<int>::max();
        pp.l_hi = std::numeric_limits<int>::min();
        for (int l = -lmax; l <= lmax; ++l) {
            chords(ox + l * h * qx, oy + l * h * qy, pp.ex, pp.ey, per_l[l + lmax]);
            if (!per_l[l + lmax].empty()) {
                pp.l_lo = std::min(pp.l_lo, l);
                pp.l_hi = std::max(pp.l_hi, l);
            }
        }
        if (pp.l_lo > pp.l_hi) return "an angle pair has no line through the grain";
        pp.line0 = (int32_t)lines.size();
        pp.lat0 = (int32_t)lats.size();
        for (int l = pp.l_lo; l <= pp.l_hi; ++l) {
            LatticeLine lt{};
            lt.c0 = (int32_t)lines.size();
            for (const Seg &s : per_l[l + lmax]) {
                LineInfo li{};
                li.pair = q;
                li.l = l;
                li.smin = s.a;
                li.smax = s.b;
                li.lo = s.ea;
                li.hi = s.eb;
                li.m0 = (int)std::ceil(s.a / h - kTol);
                li.m1 = (int)std::floor(s.b / h + kTol);
                li.ns = std::max(0, li.m1 - li.m0 + 1);
                li.slot0 = (int32_t)n_slots;
                n_slots += std::max(li.ns, 1);
                n_samples += li.ns;
                max_ns = std::max(max_ns, li.ns);
                lines.push_back(li);
            }
            lt.nc = (int32_t)lines.size() - lt.c0;
            lats.push_back(lt);
        }
        pp.n_lines = (int32_t)lines.size() - pp.line0;
        // nearest lattice line with a chord, and with a sampled chord (ties to
        // the lower index); line indices can be negative
        auto sampled = [&](int l) {
            const LatticeLine &lt = lats[pp.lat0 + (l - pp.l_lo)];
            for (int c = lt.c0; c < lt.c0 + lt.nc; ++c)
                if (lines[c].ns > 0) return true;
            return false;
        };
        bool any = false;
        for (int l = pp.l_lo; l <= pp.l_hi; ++l) any = any || sampled(l);
        if (!any) return "an angle pair has no lattice sample in the grain";
        for (int l = pp.l_lo; l <= pp.l_hi; ++l) {
            LatticeLine &lt = lats[pp.lat0 + (l - pp.l_lo)];
            int best_c = l, best_s = l;
            bool fc = false, fs = false;
            for (int d = 0; !(fc && fs); ++d) {
                for (int cand : {l - d, l + d}) {
                    if (cand < pp.l_lo || cand > pp.l_hi) continue;
                    if (!fc && lats[pp.lat0 + (cand - pp.l_lo)].nc > 0) {
                        best_c = cand;
                        fc = true;
                    }
                    if (!fs && sampled(cand)) {
                        best_s = cand;
                        fs = true;
                    }
                }
            }
            lt.chorded = best_c;
            lt.sampled = best_s;
        }
    }

    // specular links; angle p enters at smin, angle p + P at smax
    for (size_t L = 0; L < lines.size(); ++L) {
        LineInfo &li = lines[L];
        const PairInfo &pp = pairs[li.pair];
        const double bx = ox + li.l * h * (-pp.ey), by = oy + li.l * h * pp.ex;
        for (int dir = 0; dir < 2; ++dir) {
            const double s = dir == 0 ? li.smin : li.smax;
            const End &end = dir == 0 ? li.lo : li.hi;
            const double vx_ = dir == 0 ? pp.ex : -pp.ex, vy_ = dir == 0 ? pp.ey : -pp.ey;
            const double px_ = bx + s * pp.ex, py_ = by + s * pp.ey;
            double nx_, ny_;
            outward_normal(end, px_, py_, nx_, ny_);
            const double vn = vx_ * nx_ + vy_ * ny_;
            // the trajectory that arrives at the point and reflects into v
            const double ux = vx_ - 2.0 * vn * nx_, uy = vy_ - 2.0 * vn * ny_;
            if (dir == 0) link(px_, py_, ux, uy, end.part, li.fwd, li.dbg_fwd_angle, li.dbg_fwd_line, li.dbg_fwd_chord);
            else link(px_, py_, ux, uy, end.part, li.bwd, li.dbg_bwd_angle, li.dbg_bwd_line, li.dbg_bwd_chord);
        }
    }
    return std::string();
}

}  // namespace scg
