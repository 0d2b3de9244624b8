// Upper bounds of |phi| from the plan's tables, for choosing the leading-digit
// grids of the split operand images without a pass over the points.
//
// phi = u(d)/d^(l+1) N_lm Q_lm(x, y, z) with Q homogeneous of degree l, so
// |phi| <= |u(d)/d| * max over the unit sphere of |Y_lm|.  The radial factor
// is bounded per knot interval and turned into a suffix maximum, so that one
// lookup at any distance d' <= d gives a bound valid at every r >= d'.
// Pure C++: the host builds the tables, the kernels only read them.
#pragma once
#include <cmath>
#include <limits>
#include <utility>

namespace fgi {

// Entries of the |Y_lm| table: index l*l + l + m, l <= 3.
constexpr int kYlmMaxEntries = 16;

// max over the unit sphere of |Y_lm| for the real harmonics of the basis
// (unit-normalised, no Condon-Shortley phase), exact values:
//   l = 0: 1/(2 sqrt(pi));  l = 1: sqrt(3/(4 pi)) for every m
//   l = 2: xy, yz, xz: a/2;  3z^2 - 1: 2b at the poles;  x^2 - y^2: c
//   l = 3: y(3x^2 - y^2), x(x^2 - 3y^2): c3 (on the equator)
//          xyz and z(x^2 - y^2): 1/(3 sqrt 3) at |x| = |y| = |z|, resp.
//          z = 1/sqrt 3 on the x axis
//          y(4z^2 - x^2 - y^2), x(...): sqrt(256/135) at rho^2 = 4/15
//          z(5z^2 - 3): 2 at the poles
// with a = sqrt(15/pi)/2, b = sqrt(5/pi)/4, c = sqrt(15/pi)/4,
// c3 = sqrt(35/(2 pi))/4, c2 = sqrt(105/pi)/2, c1 = sqrt(21/(2 pi))/4,
// c0 = sqrt(7/pi)/4, c2b = sqrt(105/pi)/4, each times (1 + 2^-10).
inline void ylm_abs_max(float out[kYlmMaxEntries])
{
    const double pi = 3.14159265358979323846;
    const double a = std::sqrt(15.0 / pi) / 2.0, b = std::sqrt(5.0 / pi) / 4.0, c = std::sqrt(15.0 / pi) / 4.0;
    const double c3 = std::sqrt(35.0 / (2.0 * pi)) / 4.0, c2 = std::sqrt(105.0 / pi) / 2.0;
    const double c1 = std::sqrt(21.0 / (2.0 * pi)) / 4.0, c0 = std::sqrt(7.0 / pi) / 4.0;
    const double c2b = std::sqrt(105.0 / pi) / 4.0;
    const double s3 = 1.0 / (3.0 * std::sqrt(3.0)), q = std::sqrt(256.0 / 135.0);
    const double v[kYlmMaxEntries] = {
        0.5 / std::sqrt(pi),                                                   // l = 0
        std::sqrt(3.0 / (4.0 * pi)), std::sqrt(3.0 / (4.0 * pi)), std::sqrt(3.0 / (4.0 * pi)),
        a / 2.0, a / 2.0, 2.0 * b, a / 2.0, c,                                 // l = 2
        c3, c2 * s3, c1 * q, 2.0 * c0, c1 * q, 2.0 * c2b * s3, c3};             // l = 3
    for (int i = 0; i < kYlmMaxEntries; i++) out[i] = (float)(v[i] * (1.0 + 1.0 / 1024.0));
}

// Roots in (0, 1) of the quadratic a t^2 + b t + c, ascending; returns the count.
inline int quadratic_roots01(double a, double b, double c, double *r)
{
    int n = 0;
    double t[2];
    if (a == 0.0) {
        if (b != 0.0) t[n++] = -c / b;
    } else {
        const double disc = b * b - 4.0 * a * c;
        if (disc >= 0.0) {
            const double sq = std::sqrt(disc);
            const double q = -0.5 * (b + (b >= 0.0 ? sq : -sq));
            if (q != 0.0) {
                t[n++] = q / a;
                t[n++] = c / q;
            } else {
                t[n++] = 0.0;   // b = 0 and c = 0: the double root t = 0
            }
        }
    }
    int m = 0;
    for (int i = 0; i < n; i++)
        if (t[i] > 0.0 && t[i] < 1.0) r[m++] = t[i];
    if (m == 2 && r[0] > r[1]) std::swap(r[0], r[1]);
    return m;
}

// max |u(r)/r| over knot interval j of a radial spline with coefficients cf
// (u = c0 + t (c1 + t (c2 + t c3)), r = h (j + t), t in [0, 1]).
// j >= 1: g(t) = u/(h (j + t)) is stationary where
//   N(t) = 2 c3 t^3 + (3 j c3 + c2) t^2 + 2 j c2 t + (j c1 - c0) = 0;
// the roots of N' = 6 c3 t^2 + 2 (3 j c3 + c2) t + 2 j c2 cut [0, 1] into
// pieces on which N is monotone, and each sign change is bisected to double
// precision; the maximum is at an end point or one of those roots.
// j = 0 (u(0) = c0 = 0): u/r = (c1 + c2 t + c3 t^2)/h, a quadratic: end
// points and vertex.  u(0) != 0 makes u/r unbounded: +infinity.
inline double interval_ratio_max(const double *cf, int j, double h)
{
    if (j == 0) {
        if (cf[0] != 0.0) return std::numeric_limits<double>::infinity();
        auto q = [&](double t) { return std::fabs(cf[1] + t * (cf[2] + t * cf[3])) / h; };
        double m = std::fmax(q(0.0), q(1.0));
        if (cf[3] != 0.0) {
            const double tv = -cf[2] / (2.0 * cf[3]);
            if (tv > 0.0 && tv < 1.0) m = std::fmax(m, q(tv));
        }
        return m;
    }
    const double jj = (double)j;
    auto g = [&](double t) { return std::fabs(cf[0] + t * (cf[1] + t * (cf[2] + t * cf[3]))) / (h * (jj + t)); };
    auto N = [&](double t) {
        return ((2.0 * cf[3] * t + (3.0 * jj * cf[3] + cf[2])) * t + 2.0 * jj * cf[2]) * t + (jj * cf[1] - cf[0]);
    };
    double cuts[4];
    int nc = 0;
    cuts[nc++] = 0.0;
    double r[2];
    const int nr = quadratic_roots01(6.0 * cf[3], 2.0 * (3.0 * jj * cf[3] + cf[2]), 2.0 * jj * cf[2], r);
    for (int i = 0; i < nr; i++) cuts[nc++] = r[i];
    cuts[nc++] = 1.0;
    double m = std::fmax(g(0.0), g(1.0));
    for (int i = 0; i + 1 < nc; i++) {
        double a = cuts[i], b = cuts[i + 1];
        double fa = N(a), fb = N(b);
        if (fa == 0.0) m = std::fmax(m, g(a));
        if (fb == 0.0) m = std::fmax(m, g(b));
        if ((fa < 0.0) == (fb < 0.0)) continue;
        for (int it = 0; it < 100 && b - a > 0.0; it++) {
            const double c = 0.5 * (a + b);
            if (c <= a || c >= b) break;
            const double fc = N(c);
            if ((fc < 0.0) == (fa < 0.0)) {
                a = c;
                fa = fc;
            } else {
                b = c;
            }
        }
        m = std::fmax(m, std::fmax(g(a), g(b)));
    }
    return m;
}

// The smallest float >= x (x >= 0).
inline float round_up_float(double x)
{
    float f = (float)x;
    if ((double)f < x) f = std::nextafter(f, std::numeric_limits<float>::infinity());
    return f;
}

// out[k] >= max |u(r)/r| over r >= k h, for k = 0 .. n_int-1, non-increasing
// in k (beyond the last knot u = 0): the suffix maxima of the exact
// per-interval maxima, times (1 + 1e-12) against rounding, rounded up to
// FP32.  Entry 0 is +infinity when u(0) != 0 (the caller then keeps the
// pass over the points).
inline void radial_over_r_bounds(const double *coef, int n_int, double h, float *out)
{
    double run = 0.0;
    for (int j = n_int - 1; j >= 0; j--) {
        run = std::fmax(run, interval_ratio_max(coef + 4 * j, j, h) * (1.0 + 1e-12));
        out[j] = std::isinf(run) ? std::numeric_limits<float>::infinity() : round_up_float(run);
    }
}

}  // namespace fgi
