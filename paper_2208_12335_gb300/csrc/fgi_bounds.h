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

// max |c0 + c1 t + c2 t^2 + c3 t^3| over t in [0, 1]: the end points and the
// stationary points inside the interval.
inline double cubic_abs_max(const double *cf)
{
    auto u = [&](double t) { return cf[0] + t * (cf[1] + t * (cf[2] + t * cf[3])); };
    double m = std::fmax(std::fabs(u(0.0)), std::fabs(u(1.0)));
    // u'(t) = c1 + 2 c2 t + 3 c3 t^2
    const double A = 3.0 * cf[3], B = 2.0 * cf[2], C = cf[1];
    double roots[2];
    int nr = 0;
    if (A == 0.0) {
        if (B != 0.0) roots[nr++] = -C / B;
    } else {
        const double disc = B * B - 4.0 * A * C;
        if (disc >= 0.0) {
            const double sq = std::sqrt(disc);
            const double qq = -0.5 * (B + (B >= 0.0 ? sq : -sq));
            roots[nr++] = qq / A;
            if (qq != 0.0) roots[nr++] = C / qq;
        }
    }
    for (int i = 0; i < nr; i++)
        if (roots[i] > 0.0 && roots[i] < 1.0) m = std::fmax(m, std::fabs(u(roots[i])));
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
// in k (beyond the last knot u = 0).  Interval j >= 1: max |u| / (j h) (r >= j h
// there).  Interval 0: u(r)/r = (c1 + c2 t + c3 t^2)/h when c0 = u(0) = 0, so
// (|c1| + |c2| + |c3|)/h; when u(0) != 0 the ratio is unbounded near r = 0 and
// the entry is +infinity (the caller then keeps the pass over the points).
// A magnitude of 1e-15 and more on |u| in an interval is rounded up by 1e-12
// relative against the rounding of the cubic's evaluation.
inline void radial_over_r_bounds(const double *coef, int n_int, double h, float *out)
{
    double run = 0.0;
    for (int j = n_int - 1; j >= 0; j--) {
        const double *cf = coef + 4 * j;
        double b;
        if (j > 0) {
            b = cubic_abs_max(cf) / (j * h);
        } else if (cf[0] == 0.0) {
            b = (std::fabs(cf[1]) + std::fabs(cf[2]) + std::fabs(cf[3])) / h;
        } else {
            b = std::numeric_limits<double>::infinity();
        }
        run = std::fmax(run, b * (1.0 + 1e-12));
        out[j] = std::isinf(run) ? std::numeric_limits<float>::infinity() : round_up_float(run);
    }
}

}  // namespace fgi
