// Real spherical harmonics of any degree up to kHartreeLmax, for the
// multipole expansion of the Hartree potential (host and device).
//
// Associated Legendre functions without the Condon-Shortley phase by the
// standard three-term recurrences in l, written for Pbar_l^m = P_l^m /
// sin^m(theta), a polynomial in z = cos(theta):
//   Pbar_m^m = (2m-1)!!,  Pbar_{m+1}^m = (2m+1) z Pbar_m^m,
//   (l-m) Pbar_l^m = (2l-1) z Pbar_{l-1}^m - (l+m-1) Pbar_{l-2}^m,
// and sin^m(theta) (cos m phi, sin m phi) = (Re, Im) (x + i y)^m for a unit
// vector (x, y, z), so no division by sin(theta) is needed at the poles.
//   Y_l0 = K_l0 Pbar_l^0,  Y_l,+m = sqrt2 K_lm Pbar_l^m Re(x+iy)^m,
//   Y_l,-m = sqrt2 K_lm Pbar_l^m Im(x+iy)^m,
//   K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),  index l*l + l + m.
// Any orthonormal real basis of each l gives the same Hartree potential
// (the addition theorem), so the sign convention is immaterial there.
#pragma once
#include <cmath>

#ifndef __CUDACC__
#define FGI_HD
#else
#define FGI_HD __host__ __device__
#endif

namespace fgi {

constexpr int kHartreeLmax = 6;

template <int LMAX>
FGI_HD inline void real_ylm_all(double x, double y, double z, double *Y)
{
    // (x + i y)^m
    double cm[LMAX + 1], sm[LMAX + 1];
    cm[0] = 1.0;
    sm[0] = 0.0;
#pragma unroll
    for (int m = 1; m <= LMAX; m++) {
        cm[m] = cm[m - 1] * x - sm[m - 1] * y;
        sm[m] = cm[m - 1] * y + sm[m - 1] * x;
    }
    const double inv4pi = 0.079577471545947667884;     // 1/(4 pi)
    double pmm = 1.0;                                    // Pbar_m^m
#pragma unroll
    for (int m = 0; m <= LMAX; m++) {
        if (m > 0) pmm *= (double)(2 * m - 1);
        double p2 = 0.0, p1 = pmm;                       // Pbar_{l-2}^m, Pbar_{l-1}^m along l
        // K_lm^2 = (2l+1)/(4 pi) (l-m)!/(l+m)!, advanced along l
        double ratio = 1.0;                              // (l-m)!/(l+m)! at l = m: 1/(2m)!
        for (int q = 2; q <= 2 * m; q++) ratio /= (double)q;
#pragma unroll
        for (int l = m; l <= LMAX; l++) {
            double p;
            if (l == m) {
                p = pmm;
            } else if (l == m + 1) {
                p = (double)(2 * m + 1) * z * pmm;
            } else {
                p = ((double)(2 * l - 1) * z * p1 - (double)(l + m - 1) * p2) / (double)(l - m);
            }
            if (l > m) {
                ratio *= (double)(l - m) / (double)(l + m);   // (l-m)!/(l+m)! from its value at l-1
                p2 = p1;
                p1 = p;
            }
            const double K = sqrt((2.0 * l + 1.0) * inv4pi * ratio);
            if (m == 0) {
                Y[l * l + l] = K * p;
            } else {
                const double s2K = 1.4142135623730951 * K * p;
                Y[l * l + l + m] = s2K * cm[m];
                Y[l * l + l - m] = s2K * sm[m];
            }
        }
    }
}

}  // namespace fgi
