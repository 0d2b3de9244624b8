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
// The multipole kernels work with the unnormalised A_lm (the same without
// K_lm) and fold K_lm^2 into their radial tables.
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

// The unnormalised real harmonics A_lm = Pbar_l^|m|(z) Re/Im (x + i y)^|m|
// (index l*l + l + m; cos for m > 0, sin for m < 0) of a unit vector, in T.
// The recurrence multiplies by 1/(l-m) (a constant) instead of dividing.
template <int LMAX, typename T>
FGI_HD inline void ylm_unnormalised(T x, T y, T z, T *A)
{
    T cm[LMAX + 1], sm[LMAX + 1];
    cm[0] = T(1);
    sm[0] = T(0);
#pragma unroll
    for (int m = 1; m <= LMAX; m++) {
        cm[m] = cm[m - 1] * x - sm[m - 1] * y;
        sm[m] = cm[m - 1] * y + sm[m - 1] * x;
    }
    T pmm = T(1);                                        // Pbar_m^m
#pragma unroll
    for (int m = 0; m <= LMAX; m++) {
        if (m > 0) pmm *= T(2 * m - 1);
        T p2 = T(0), p1 = pmm;                           // Pbar_{l-2}^m, Pbar_{l-1}^m along l
#pragma unroll
        for (int l = m; l <= LMAX; l++) {
            T p;
            if (l == m) {
                p = pmm;
            } else if (l == m + 1) {
                p = T(2 * m + 1) * z * pmm;
            } else {
                p = (T(2 * l - 1) * z * p1 - T(l + m - 1) * p2) * T(1.0 / (double)(l - m));
            }
            if (l > m) {
                p2 = p1;
                p1 = p;
            }
            if (m == 0) {
                A[l * l + l] = p;
            } else {
                A[l * l + l + m] = p * cm[m];
                A[l * l + l - m] = p * sm[m];
            }
        }
    }
}

// the square of the factor that makes A_lm unit-normalised:
// K_lm^2 (x 2 for m != 0) = (2l+1)/(4 pi) (l-|m|)!/(l+|m|)! (x 2)
FGI_HD inline double ylm_norm2(int l, int m)
{
    const int am = m < 0 ? -m : m;
    double ratio = 1.0;
    for (int q = l - am + 1; q <= l + am; q++) ratio /= (double)q;
    return (2.0 * l + 1.0) * 0.079577471545947667884 * ratio * (am ? 2.0 : 1.0);
}

// unit-normalised real harmonics Y_lm = sqrt(ylm_norm2) A_lm, in FP64
template <int LMAX>
FGI_HD inline void real_ylm_all(double x, double y, double z, double *Y)
{
    ylm_unnormalised<LMAX, double>(x, y, z, Y);
#pragma unroll
    for (int l = 0; l <= LMAX; l++)
#pragma unroll
        for (int m = -l; m <= l; m++) Y[l * l + l + m] *= sqrt(ylm_norm2(l, m));
}

}  // namespace fgi
