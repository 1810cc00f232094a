// Ozaki's continued-fraction poles of the Fermi function (Ozaki, Phys. Rev. B
// 75, 035123 (2007)), the energy sum the paper uses instead of plain Matsubara
// sums (Sec. 3.1).  With the 2N x 2N symmetric tridiagonal matrix B (zero
// diagonal, B[m-1][m] = B[m][m-1] = 1/(2 sqrt((2m-1)(2m+1))), m = 1 .. 2N-1)
// and its positive eigenvalues b_p with normalised eigenvectors v_p,
//   1/(1 + e^x) = 1/2 - sum_p R_p [1/(x - i z_p) + 1/(x + i z_p)],
//   z_p = 1/b_p,  R_p = v_p[0]^2 / (4 b_p^2).
// A Matsubara sum T sum_n F(i eps_n) becomes sum_p R_p T [F(i T z_p) + F(-i T z_p)]:
// energies z_p T (the first N/2 or so equal pi T (2n+1) with R_p = 1) and
// weights R_p.
//
// Eigenvalues by bisection on Sturm counts, first eigenvector components by
// inverse iteration (tridiagonal LU with partial pivoting).
#include <cmath>
#include <vector>

#include "sc.h"

namespace {

// number of eigenvalues of the zero-diagonal tridiagonal matrix below x
int sturm_count(const std::vector<double> &off, double x) {
    const int M = (int)off.size() + 1;
    int neg = 0;
    double q = -x;
    if (q < 0.0) ++neg;
    for (int i = 1; i < M; ++i) {
        const double qq = q != 0.0 ? q : 1e-300;
        q = -x - off[i - 1] * off[i - 1] / qq;
        if (q < 0.0) ++neg;
    }
    return neg;
}

// solve (B - s I) y = r for the tridiagonal B (zero diagonal), partial pivoting
void tri_solve(const std::vector<double> &off, double s, std::vector<double> &r) {
    const int M = (int)r.size();
    // bands of U (u0 diagonal, u1, u2 super-diagonals) and multipliers
    std::vector<double> u0(M), u1(M, 0.0), u2(M, 0.0), lm(M, 0.0);
    std::vector<char> sw(M, 0);
    // working rows: row i = [sub, diag, sup]
    double a_d = -s, a_u = M > 1 ? off[0] : 0.0, a_u2 = 0.0;
    for (int i = 0; i < M; ++i) {
        if (i == M - 1) {
            u0[i] = a_d != 0.0 ? a_d : 1e-300;
            u1[i] = 0.0;
            break;
        }
        const double b_l = off[i], b_d = -s, b_u = i + 1 < M - 1 ? off[i + 1] : 0.0;
        if (std::fabs(b_l) > std::fabs(a_d)) {  // swap rows i and i+1
            sw[i] = 1;
            u0[i] = b_l;
            u1[i] = b_d;
            u2[i] = b_u;
            const double m = a_d / b_l;
            lm[i] = m;
            a_d = a_u - m * b_d;
            a_u = a_u2 - m * b_u;
            a_u2 = 0.0;
        } else {
            const double piv = a_d != 0.0 ? a_d : 1e-300;
            u0[i] = piv;
            u1[i] = a_u;
            u2[i] = a_u2;
            const double m = b_l / piv;
            lm[i] = m;
            a_d = b_d - m * a_u;
            a_u = b_u - m * a_u2;
            a_u2 = 0.0;
        }
    }
    // forward: apply the row swaps and eliminations to r
    for (int i = 0; i < M - 1; ++i) {
        if (sw[i]) std::swap(r[i], r[i + 1]);
        r[i + 1] -= lm[i] * r[i];
    }
    // back substitution
    for (int i = M - 1; i >= 0; --i) {
        double v = r[i];
        if (i + 1 < M) v -= u1[i] * r[i + 1];
        if (i + 2 < M) v -= u2[i] * r[i + 2];
        r[i] = v / u0[i];
    }
}

}  // namespace

extern "C" sc_status sc_ozaki_poles(int32_t n, double *z, double *R) {
    if (n < 1 || n > 1024 || !z || !R) return SC_EINVAL;
    const int M = 2 * n;
    std::vector<double> off(M - 1);
    for (int m = 1; m < M; ++m) off[m - 1] = 1.0 / (2.0 * std::sqrt((2.0 * m - 1.0) * (2.0 * m + 1.0)));
    // spectrum symmetric about 0 and inside [-1, 1] (Gershgorin: rows sum < 1)
    for (int k = 0; k < n; ++k) {
        // k-th largest positive eigenvalue: the (M - 1 - k)-th in ascending order
        const int idx = M - 1 - k;
        double lo = 0.0, hi = 1.0;
        for (int it = 0; it < 200 && hi - lo > 1e-17 * hi; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (sturm_count(off, mid) > idx)
                hi = mid;
            else
                lo = mid;
        }
        const double b = 0.5 * (lo + hi);
        // inverse iteration for the eigenvector
        std::vector<double> v(M);
        for (int i = 0; i < M; ++i) v[i] = 1.0 / std::sqrt((double)M) * (1.0 + 0.1 * std::sin(1.0 + i));
        const double shift = b * (1.0 + 1e-13);
        for (int it = 0; it < 3; ++it) {
            tri_solve(off, shift, v);
            double nrm = 0.0;
            for (double x : v) nrm += x * x;
            nrm = std::sqrt(nrm);
            for (double &x : v) x /= nrm;
        }
        // poles in ascending z = 1/b: the largest b gives the smallest z
        z[k] = 1.0 / b;
        R[k] = v[0] * v[0] / (4.0 * b * b);
    }
    return SC_OK;
}

extern "C" int32_t sc_ozaki_poles_for_cutoff(double t, double eps_cut) {
    if (!(t > 0.0) || !(eps_cut > 0.0)) return 0;
    for (int n = 1; n <= 1024; ++n) {
        // smallest positive eigenvalue b_min (ascending index n of 2n): z_max = 1/b_min
        const int M = 2 * n;
        std::vector<double> off(M - 1);
        for (int m = 1; m < M; ++m) off[m - 1] = 1.0 / (2.0 * std::sqrt((2.0 * m - 1.0) * (2.0 * m + 1.0)));
        double lo = 0.0, hi = 1.0;
        for (int it = 0; it < 200 && hi - lo > 1e-17 * hi; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (sturm_count(off, mid) > n)
                hi = mid;
            else
                lo = mid;
        }
        if (t / (0.5 * (lo + hi)) / (2.0 * M_PI) >= eps_cut) return n;
    }
    return 0;
}
