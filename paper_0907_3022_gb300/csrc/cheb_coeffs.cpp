// Host FP64 expansion coefficients of the Chebyshev propagator (Sec. 2.2, Eqs. U_1, c_k).
//
// c_k(z) = (-i)^k J_k(z).  J_k is computed for all k at once by Miller's backward
// recurrence (J. C. P. Miller 1952; see Abramowitz & Stegun, Handbook, Sec. 9.12):
// starting far above both z and the largest wanted order with J_{K+1} = 0, J_K = tiny,
// J_{k-1} = (2k/z) J_k - J_{k+1} runs down to k = 0 and converges to a multiple of the
// minimal solution J_k(z).  The multiple is fixed by the identity
// J_0^2 + 2 sum_{k>=1} J_k^2 = 1 (a sum of squares, so no cancellation), with the sign
// taken from J_0 + 2 sum_{k>=1} J_{2k} = 1.
#include <algorithm>
#include <cmath>
#include <vector>

#include "cheb_internal.cuh"

namespace cheb {

int bessel_j_seq(double z, int kmax, std::vector<double>& J)
{
    J.assign((size_t)kmax + 1, 0.0);
    if (!(z >= 0.0) || !std::isfinite(z)) return -1;
    if (z == 0.0) {
        J[0] = 1.0;
        return 0;
    }
    // Start well past the turning point k ~ z: there J_k(z) decays like exp(-c (k-z)^{3/2}
    // / z^{1/2}), so K = z + 40 + 25 z^{1/3} puts the start below 1e-50 of the peak.
    long K = (long)std::ceil(z + 40.0 + 25.0 * std::cbrt(z));
    if (K < kmax + 20) K = kmax + 20;
    std::vector<double> t((size_t)K + 1, 0.0);
    double jp1 = 0.0, j = 1e-300;
    t[(size_t)K] = j;
    for (long k = K; k >= 1; --k) {
        double jm1 = (2.0 * (double)k / z) * j - jp1;
        jp1 = j;
        j = jm1;
        t[(size_t)(k - 1)] = j;
        if (std::fabs(j) > 1e100) {  // rescale everything computed so far (keeps t^2 finite)
            for (long m = k - 1; m <= K; ++m) t[(size_t)m] *= 1e-100;
            j *= 1e-100;
            jp1 *= 1e-100;
        }
    }
    // bring the largest value near 1 by a power of two (exact) so that the squares neither
    // overflow nor underflow, then normalise
    double mx = 0.0;
    for (long k = 0; k <= K; ++k) mx = std::max(mx, std::fabs(t[(size_t)k]));
    if (!(mx > 0.0) || !std::isfinite(mx)) return -2;
    int ex = 0;
    std::frexp(mx, &ex);
    for (long k = 0; k <= K; ++k) t[(size_t)k] = std::ldexp(t[(size_t)k], -ex);
    double sq = t[0] * t[0], lin = t[0];
    for (long k = 1; k <= K; ++k) {
        sq += 2.0 * t[(size_t)k] * t[(size_t)k];
        if ((k & 1) == 0) lin += 2.0 * t[(size_t)k];
    }
    if (!(sq > 0.0) || !std::isfinite(sq)) return -2;
    double scale = (lin < 0.0 ? -1.0 : 1.0) / std::sqrt(sq);
    for (int k = 0; k <= kmax; ++k) J[(size_t)k] = t[(size_t)k] * scale;
    return 0;
}

}  // namespace cheb

using namespace cheb;

extern "C" int cheb_rescale(double emin, double emax, double alpha, double* a, double* b)
{
    if (!a || !b) return fail(CHEB_ERR_INVALID, "cheb_rescale: NULL output");
    if (!(emax >= emin) || !(alpha >= 0.0) || !std::isfinite(emin) || !std::isfinite(emax))
        return fail(CHEB_ERR_INVALID, "cheb_rescale: need emin <= emax and alpha >= 0");
    *b = 0.5 * (emax + emin);
    *a = 0.5 * (emax - emin) * (1.0 + alpha);
    if (!(*a > 0.0)) return fail(CHEB_ERR_INVALID, "cheb_rescale: a = 0 (emin == emax, alpha == 0)");
    return CHEB_OK;
}

extern "C" int cheb_coeffs(double a, double b, double dt, double tol, int max_order, double* c_re,
                           double* c_im, int* M_out)
{
    if (!c_re || !c_im || !M_out) return fail(CHEB_ERR_INVALID, "cheb_coeffs: NULL pointer");
    if (!(a > 0.0) || !(dt >= 0.0) || !(tol > 0.0) || max_order < 2 || !std::isfinite(b))
        return fail(CHEB_ERR_INVALID, "cheb_coeffs: need a > 0, dt >= 0, tol > 0, max_order >= 2");
    const double z = a * dt;
    // Past k ~ z + 60 + 20 z^{1/3} every |C_k| is far below any tolerance >= 1e-300.
    long natural = (long)std::ceil(z + 60.0 + 20.0 * std::cbrt(z));
    int kmax = (int)std::min<long>((long)max_order, natural);
    std::vector<double> J;
    if (bessel_j_seq(z, kmax, J) != 0) return fail(CHEB_ERR_INVALID, "cheb_coeffs: Bessel recurrence failed");
    const double pr = std::cos(b * dt), pi = -std::sin(b * dt);  // e^{-i b dt}
    int M = 0;
    for (int k = 0; k <= kmax; ++k) {
        double g = (k == 0 ? 1.0 : 2.0) * J[(size_t)k];
        // (-i)^k g
        double re = 0.0, im = 0.0;
        switch (k & 3) {
            case 0: re = g; break;
            case 1: im = -g; break;
            case 2: re = -g; break;
            default: im = g; break;
        }
        c_re[k] = pr * re - pi * im;
        c_im[k] = pr * im + pi * re;
        if (std::fabs(g) >= tol) M = k;
    }
    if (M == kmax && kmax < natural)
        return fail(CHEB_ERR_ORDER, "cheb_coeffs: |c_k| >= tol at max_order; raise max_order");
    if (M < 2) {
        M = 2;  // the fused kernels need at least two recurrence steps; C_2 is kept exactly
    }
    *M_out = M;
    return CHEB_OK;
}
