// Cell-integrated Green's tensor to second order in kd (the igt_so
// interaction and polarizability named in Sec. S5 of the paper).
//
// A dipole stands for its cubic cell uniformly polarised, so the field it
// makes at another dipole is the Green's tensor (Eq. 5) averaged over the
// source cell.  With rho = R - s (s in the cell), G~(rho) = exp(ik rho)
// [k^2 A - B + ik C], A = (I - rr)/rho, B = (I - 3 rr)/rho^3,
// C = (I - 3 rr)/rho^2; expanding exp(ik rho) = exp(ikR)(1 + ik delta -
// k^2 delta^2 / 2), delta = rho - R, and keeping terms up to k^2:
//   G_so(R) = exp(ikR) [ -<B> + ik <C - delta B> + k^2 <A - delta C + delta^2 B / 2> ],
// <.> the average over the cell, here by 24^3-point Gauss-Legendre cubature
// in lattice units (lengths in d), for every lattice offset of max-norm
// <= IGT_NEAR.  The D-hat build (k_green) uses these for near offsets and
// the point tensor beyond.  The self term of the cell to the same order is
// (2/3)(c1 kappa^2 + i kappa^3), c1 = 3 ln(2 + sqrt 3) - pi/2 (energy_params).
#include <cmath>
#include <mutex>
#include <vector>

#include "kernels.h"

namespace eels {

namespace {

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on the
// Legendre recurrence from the usual cosine first guesses).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            // p1 = P_n(z), p0 = P_{n-1}(z)
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

void build_tables(std::vector<double>& tab) {
    const int n = 24, L = IGT_NEAR, side = 2 * L + 1;
    std::vector<double> gx, gw;
    gauss_legendre(n, gx, gw);
    tab.assign((size_t)side * side * side * 18, 0.0);
    const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {0, 1, 2, 1, 2, 2};
    for (int oz = -L; oz <= L; ++oz)
        for (int oy = -L; oy <= L; ++oy)
            for (int ox = -L; ox <= L; ++ox) {
                if (ox == 0 && oy == 0 && oz == 0) continue;
                const double R[3] = {(double)ox, (double)oy, (double)oz};
                const double Rn = std::sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
                double t0[6] = {0}, t1[6] = {0}, t2[6] = {0};
                for (int a = 0; a < n; ++a)
                    for (int b = 0; b < n; ++b)
                        for (int c = 0; c < n; ++c) {
                            const double wq = 0.125 * gw[a] * gw[b] * gw[c];   // nodes on [-1/2, 1/2]^3
                            const double rho[3] = {R[0] - 0.5 * gx[a], R[1] - 0.5 * gx[b], R[2] - 0.5 * gx[c]};
                            const double r2 = rho[0] * rho[0] + rho[1] * rho[1] + rho[2] * rho[2];
                            const double r = std::sqrt(r2);
                            const double h[3] = {rho[0] / r, rho[1] / r, rho[2] / r};
                            const double del = r - Rn;
                            for (int q = 0; q < 6; ++q) {
                                const double hh = h[pa[q]] * h[pb[q]];
                                const double id = pa[q] == pb[q] ? 1.0 : 0.0;
                                const double A = (id - hh) / r;
                                const double B = (id - 3.0 * hh) / (r2 * r);
                                const double C = (id - 3.0 * hh) / r2;
                                t0[q] += wq * B;
                                t1[q] += wq * (C - del * B);
                                t2[q] += wq * (A - del * C + 0.5 * del * del * B);
                            }
                        }
                double* o = tab.data() + ((size_t)((oz + L) * side + (oy + L)) * side + (ox + L)) * 18;
                for (int q = 0; q < 6; ++q) {
                    o[q] = t0[q];
                    o[6 + q] = t1[q];
                    o[12 + q] = t2[q];
                }
            }
}

}  // namespace

const std::vector<double>& igt_tables() {
    static std::vector<double> tab;
    static std::once_flag once;
    std::call_once(once, [] { build_tables(tab); });
    return tab;
}

}  // namespace eels
