// Device-side basis-function evaluation: phi = u(d)/d * Y_lm(d/|d|).
//
// The numeric atom-centred orbitals of the method (paper, "Development
// Priorities"): a radial function u tabulated as a uniform cubic spline times
// a real spherical harmonic (unit-normalised, no Condon-Shortley phase,
// m = -l..l).  Templated on the arithmetic type: FP64 for the reference GPU
// path, FP32 for the tensor-core path.
#pragma once
#include "fgi_internal.h"

namespace fgi {

// Real spherical harmonics of the unit vector (x, y, z) for one l, m = -l..l.
template <typename T>
__device__ __forceinline__ void ylm_unit(int l, T x, T y, T z, T *Y)
{
    if (l == 0) {
        Y[0] = T(0.28209479177387814);
    } else if (l == 1) {
        const T c = T(0.4886025119029199);
        Y[0] = c * y; Y[1] = c * z; Y[2] = c * x;
    } else if (l == 2) {
        const T a = T(1.0925484305920792), b = T(0.31539156525252005), c = T(0.5462742152960396);
        Y[0] = a * x * y;
        Y[1] = a * y * z;
        Y[2] = b * (T(2) * z * z - x * x - y * y);
        Y[3] = a * x * z;
        Y[4] = c * (x * x - y * y);
    } else {
        const T c3 = T(0.5900435899266435), c2 = T(2.890611442640554), c1 = T(0.4570457994644658),
                c0 = T(0.3731763325901154), c2b = T(1.445305721320277);
        const T q = T(4) * z * z - x * x - y * y;
        Y[0] = c3 * y * (T(3) * x * x - y * y);
        Y[1] = c2 * x * y * z;
        Y[2] = c1 * y * q;
        Y[3] = c0 * z * (T(2) * z * z - T(3) * x * x - T(3) * y * y);
        Y[4] = c1 * x * q;
        Y[5] = c2b * z * (x * x - y * y);
        Y[6] = c3 * x * (x * x - T(3) * y * y);
    }
}

// Gradient (with respect to the Cartesian components) of the homogeneous
// polynomial r^l Y_lm, evaluated at the unit vector (x, y, z): G[m][3].
template <typename T>
__device__ __forceinline__ void ylm_poly_grad(int l, T x, T y, T z, T (*G)[3])
{
    if (l == 0) {
        G[0][0] = G[0][1] = G[0][2] = T(0);
    } else if (l == 1) {
        const T c = T(0.4886025119029199);
        G[0][0] = 0; G[0][1] = c; G[0][2] = 0;
        G[1][0] = 0; G[1][1] = 0; G[1][2] = c;
        G[2][0] = c; G[2][1] = 0; G[2][2] = 0;
    } else if (l == 2) {
        const T a = T(1.0925484305920792), b = T(0.31539156525252005), c = T(0.5462742152960396);
        G[0][0] = a * y; G[0][1] = a * x; G[0][2] = 0;
        G[1][0] = 0; G[1][1] = a * z; G[1][2] = a * y;
        G[2][0] = -T(2) * b * x; G[2][1] = -T(2) * b * y; G[2][2] = T(4) * b * z;
        G[3][0] = a * z; G[3][1] = 0; G[3][2] = a * x;
        G[4][0] = T(2) * c * x; G[4][1] = -T(2) * c * y; G[4][2] = 0;
    } else {
        const T c3 = T(0.5900435899266435), c2 = T(2.890611442640554), c1 = T(0.4570457994644658),
                c0 = T(0.3731763325901154), c2b = T(1.445305721320277);
        G[0][0] = T(6) * c3 * x * y; G[0][1] = T(3) * c3 * (x * x - y * y); G[0][2] = 0;
        G[1][0] = c2 * y * z; G[1][1] = c2 * x * z; G[1][2] = c2 * x * y;
        G[2][0] = -T(2) * c1 * x * y; G[2][1] = c1 * (T(4) * z * z - x * x - T(3) * y * y);
        G[2][2] = T(8) * c1 * y * z;
        G[3][0] = -T(6) * c0 * x * z; G[3][1] = -T(6) * c0 * y * z;
        G[3][2] = c0 * (T(6) * z * z - T(3) * x * x - T(3) * y * y);
        G[4][0] = c1 * (T(4) * z * z - T(3) * x * x - y * y); G[4][1] = -T(2) * c1 * x * y;
        G[4][2] = T(8) * c1 * x * z;
        G[5][0] = T(2) * c2b * x * z; G[5][1] = -T(2) * c2b * y * z; G[5][2] = c2b * (x * x - y * y);
        G[6][0] = T(3) * c3 * (x * x - y * y); G[6][1] = -T(6) * c3 * x * y; G[6][2] = 0;
    }
}

// u(d)/d for one radial function (FP64).  Zero at and beyond the cutoff;
// for d < 1e-12 the l = 0 limit u'(0) = c1/h, else 0.
__device__ __forceinline__ double radial_over_d_f64(const DevRadial &R, const double *coef,
                                                    double d, double *du_out = nullptr)
{
    if (d >= R.rcut) {
        if (du_out) *du_out = 0.0;
        return 0.0;
    }
    const double *c0 = coef + 4 * R.coef_off;
    if (d < 1e-12) {
        if (du_out) *du_out = 0.0;
        return R.l == 0 ? c0[1] * R.inv_h : 0.0;
    }
    double s = d * R.inv_h;
    int k = (int)s;
    if (k > R.nk - 2) k = R.nk - 2;
    double t = s - (double)k;
    const double2 *c = reinterpret_cast<const double2 *>(c0 + 4 * (long long)k);
    double2 a = __ldg(c), b = __ldg(c + 1);
    double u = a.x + t * (a.y + t * (b.x + t * b.y));
    if (du_out) *du_out = (a.y + t * (2.0 * b.x + t * 3.0 * b.y)) * R.inv_h;
    return u / d;
}

}  // namespace fgi
