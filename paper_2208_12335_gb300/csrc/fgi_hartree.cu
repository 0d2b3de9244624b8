// The step upstream of the grid integration: the Hartree potential of the
// density on the grid, v_H(r) = int n(r') / |r - r'| dr', by the multipole
// method of Becke & Dickson (1988) and Delley (1990), which the NAO method
// uses for the electrostatic potential (the paper's Fig. 4 caption notes that
// this potential was not yet accelerated on GPUs).
//
//  1. k_hartree_moments (FP64): per point p on atom a's radial shell k,
//       rho~_a,lm(r_k) += (w_p / (r_k^3 ln q)) n_p A_lm(rhat_p)
//     (w_p / (r_k^3 ln q) is the partitioned angular weight; A_lm = Y_lm / K_lm
//     the unnormalised harmonics), FP64 atomics.
//  2. k_hartree_radial (FP64): per (atom, l, m) the radial Poisson equation
//       V(r) = 4 pi/(2l+1) [r^-(l+1) int_0^r rho r'^(l+2) dr' + r^l int_r^inf rho r'^(1-l) dr']
//     with the partial integrals in x = ln r interval by interval, each by the
//     integral of the cubic through its four nearest shells, plus
//     rho(r_0) r_0^(l+3)/(l+3) inside the first shell; Q_lm = the whole inner
//     integral (the exterior multipole moments).  Stored with K_lm^2 folded in
//     (Y_lm Y_lm-weighted sums become A_lm sums): l = 0 in FP64 (V) and as a
//     double-float (Q, in a packed per-atom record with the atom's position),
//     l >= 1 in FP32.
//  3. k_hartree_eval: per point, over the atoms of its system, V_a,lm at the
//     distance times Y_lm of the direction: 4-point Lagrange interpolation in
//     the fractional shell index inside the grid (l = 0 as a double-float:
//     the interpolating cubic of each interval stored in f = x - k, and
//     f = ln(d / r_k) / ln q from an atanh series; FP64 for coarse grids),
//     4 pi/(2l+1) Q_lm / d^(l+1) beyond the last shell (l = 0 as a
//     double-float: offset, distance and 1/d from the double-float point and
//     atom positions), V(r_0) (d/r_0)^l inside the first shell.  The l >= 1
//     terms (angular functions, their coefficients and sums) are FP32: each
//     carries a relative error of a few FP32 roundings of the l >= 1 part,
//     against the FP64 pipe's 1/64 rate on GB300.  The sum over atoms is a
//     double-float.
#include "fgi_dd.cuh"
#include "fgi_hartree.h"
#include "fgi_ylm.cuh"

namespace fgi {

namespace {

constexpr int kL = (kHartreeLmax + 1) * (kHartreeLmax + 1);  // stride of the FP64 moment rows
constexpr int kLf = kL - 1;                                     // stride of the FP32 l >= 1 rows
// 2/3 and 2/5 as double-floats (compile-time)
constexpr float kTwoThirdHi = (float)(2.0 / 3.0), kTwoThirdLo = (float)(2.0 / 3.0 - (double)kTwoThirdHi);
constexpr float kTwoFifthHi = (float)(2.0 / 5.0), kTwoFifthLo = (float)(2.0 / 5.0 - (double)kTwoFifthHi);

struct HartreeTabs {
    double *rho;      // [n_shells][kL]    unnormalised moments
    double *Vd;       // [n_shells][kL]    scratch: inner part of V
    double *F;        // [n_shells][kL]    scratch: inner integrand
    float4 *rec;      // [n_atoms][3]      position (double-float), (last radius)^2, 4 pi K_00^2 Q_00
    float4 *rk;       // [n_shells]        r_k and 1/r_k as double-floats
    float4 *c0;       // [n_shells][2]     V_00 on interval k as a cubic in f (double-floats a0..a3)
    double *V0;       // [n_shells]        K_00^2 V_00
    float *Vf;        // [n_shells][kLf]   K_lm^2 V_lm, l >= 1
    float *Qf;        // [n_atoms][kLf]    4 pi/(2l+1) K_lm^2 Q_lm, l >= 1
};

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

HartreeTabs carve(const HartreeDev &H, void *ws)
{
    char *b = (char *)ws;
    HartreeTabs T;
    T.rho = (double *)b;
    b += al256(sizeof(double) * kL * (size_t)H.n_shells);
    T.Vd = (double *)b;
    b += al256(sizeof(double) * kL * (size_t)H.n_shells);
    T.F = (double *)b;
    b += al256(sizeof(double) * kL * (size_t)H.n_shells);
    T.rec = (float4 *)b;
    b += al256(sizeof(float4) * 3 * (size_t)H.n_atoms);
    T.rk = (float4 *)b;
    b += al256(sizeof(float4) * (size_t)H.n_shells);
    T.c0 = (float4 *)b;
    b += al256(sizeof(float4) * 2 * (size_t)H.n_shells);
    T.V0 = (double *)b;
    b += al256(sizeof(double) * (size_t)H.n_shells);
    T.Vf = (float *)b;
    b += al256(sizeof(float) * kLf * (size_t)H.n_shells);
    T.Qf = (float *)b;
    return T;
}

__device__ __forceinline__ df dfa(df a, df b)      // sum of two double-floats (absolute accuracy)
{
    df s = df_two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df dfa_f(df a, float b)
{
    df s = df_two_sum(a.hi, b);
    s.lo += a.lo;
    return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_sqr(df a)
{
    df p = df_two_prod(a.hi, a.hi);
    p.lo = fmaf(2.0f * a.hi, a.lo, p.lo);
    return df_fast_two_sum(p.hi, p.lo);
}

// 1/sqrt(a) from y ~ rsqrtf(a.hi) by one Newton step with a double-float residual
__device__ __forceinline__ df df_rsqrt(df a, float y)
{
    const df ay2 = df_mul(a, df_two_prod(y, y));   // ~ 1
    const float e = (1.0f - ay2.hi) - ay2.lo;
    return df_fast_two_sum(y, y * (0.5f * e));
}

template <int LMAX>
__global__ void __launch_bounds__(256) k_hartree_moments(DevPlan P, HartreeDev H, long long n_pts, const double *n,
                                                         double *rho)
{
    constexpr int L = (LMAX + 1) * (LMAX + 1);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n_pts;
         p += (long long)gridDim.x * blockDim.x) {
        const int a = H.owner[p];
        if (a < 0) continue;
        const int k = H.shell[p];
        const HartreeRad g = H.rad[a];
        const double dx = P.px[p] - P.atom_xyz[3 * a], dy = P.py[p] - P.atom_xyz[3 * a + 1],
                     dz = P.pz[p] - P.atom_xyz[3 * a + 2];
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        if (!(r > 0.0)) continue;
        const double rk = g.r0 * exp(g.lnq * (double)k);
        const double val = P.pw[p] / (rk * rk * rk * g.lnq) * n[p];
        const double ir = 1.0 / r;
        double A[L];
        ylm_unnormalised<LMAX, double>(dx * ir, dy * ir, dz * ir, A);
        double *dst = rho + (H.rad_off[a] + k) * kL;
#pragma unroll
        for (int q = 0; q < L; q++) atomicAdd(dst + q, val * A[q]);
    }
}

__device__ __forceinline__ double ipow(double r, int n)      // r^n, 0 <= n <= 9
{
    double p = 1.0;
    for (int i = 0; i < n; i++) p *= r;
    return p;
}

// one thread per (atom, lm); the thread with lm = 0 also packs the atom's
// record for the evaluation
__global__ void __launch_bounds__(32) k_hartree_radial(DevPlan P, HartreeDev H, int l_max, HartreeTabs T)
{
    const int L = (l_max + 1) * (l_max + 1);
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)H.n_atoms * L) return;
    const int a = (int)(t / L), lm = (int)(t % L);
    int l = 0;
    while ((l + 1) * (l + 1) <= lm) l++;
    const HartreeRad g = H.rad[a];
    const int n = g.nrad;
    const long long o = H.rad_off[a];
    const double h = g.lnq;
    double *rho = T.rho + o * kL + lm, *F = T.F + o * kL + lm, *Vin = T.Vd + o * kL + lm;
    auto rk = [&](int k) { return g.r0 * exp(h * (double)k); };
    // the integrands per dx = dr / r: f = rho r^(l+3) (inner), g = rho r^(2-l) (outer, over rho)
    for (int k = 0; k < n; k++) {
        const double r = rk(k), rr = rho[(long long)k * kL];
        F[(long long)k * kL] = rr * ipow(r, l + 3);
        rho[(long long)k * kL] = l <= 2 ? rr * ipow(r, 2 - l) : rr / ipow(r, l - 2);
    }
    // integral over interval [k, k+1] of the cubic through the nearest four samples (n >= 4)
    auto seg = [&](const double *fn, int k) {
        auto v = [&](int j) { return fn[(long long)j * kL]; };
        if (k == 0) return h * (9.0 * v(0) + 19.0 * v(1) - 5.0 * v(2) + v(3)) / 24.0;
        if (k == n - 2) return h * (v(n - 4) - 5.0 * v(n - 3) + 19.0 * v(n - 2) + 9.0 * v(n - 1)) / 24.0;
        return h * (-v(k - 1) + 13.0 * v(k) + 13.0 * v(k + 1) - v(k + 2)) / 24.0;
    };
    // 4 pi/(2l+1), times K_lm^2 for the two unnormalised harmonics (moment, evaluation)
    const double pref = 4.0 * 3.14159265358979323846 / (2.0 * l + 1.0) * ylm_norm2(l, lm - l * l - l);
    // inner integrals, forward: the inner part of V in FP64 scratch
    double iin = F[0] / (double)(l + 3);
    for (int k = 0; k < n; k++) {
        if (k > 0) iin += seg(F, k - 1);
        Vin[(long long)k * kL] = pref * iin / ipow(rk(k), l + 1);
    }
    if (lm == 0) {
        const float *aa = P.atom_dd + 6 * a;
        const df q = df_from_double(pref * iin);
        T.rec[3 * a] = make_float4(aa[0], aa[1], aa[2], aa[3]);
        T.rec[3 * a + 1] = make_float4(aa[4], aa[5], g.rmax2_hi, g.rmax2_lo);
        T.rec[3 * a + 2] = make_float4(q.hi, q.lo, 0.f, 0.f);
    } else {
        T.Qf[(long long)a * kLf + lm - 1] = (float)(pref * iin);
    }
    // outer integrals, backward; V = inner + outer part, stored once
    double iout = 0.0;
    for (int k = n - 1; k >= 0; k--) {
        if (k < n - 1) iout += seg(rho, k);
        const double v = Vin[(long long)k * kL] + pref * iout * ipow(rk(k), l);
        if (lm == 0) T.V0[o + k] = v;
        else T.Vf[(o + k) * kLf + lm - 1] = (float)v;
    }
    if (lm != 0) return;
    // the shells' radii, and V_00 on each interval k as the cubic through
    // shells i0 .. i0+3 (i0 = k - 1 clamped to [0, n-4]) in f = x - k,
    // x = ln(r / r_0) / ln q: a_m = p^(m)(o) / m! with o = k - i0 and
    // p(t) = V_i0 + t D1 + t(t-1)/2 D2 + t(t-1)(t-2)/6 D3 (forward differences)
    for (int k = 0; k < n; k++) {
        const double r = rk(k);
        const df rh = df_from_double(r), ri = df_from_double(1.0 / r);
        T.rk[o + k] = make_float4(rh.hi, rh.lo, ri.hi, ri.lo);
    }
    for (int k = 0; k + 1 < n; k++) {
        const int i0 = k - 1 < 0 ? 0 : (k - 1 > n - 4 ? n - 4 : k - 1);
        const double t = (double)(k - i0);
        const double *v = T.V0 + o + i0;
        const double D1 = v[1] - v[0], D2 = v[2] - 2.0 * v[1] + v[0], D3 = v[3] - 3.0 * v[2] + 3.0 * v[1] - v[0];
        const df a0 = df_from_double(v[k - i0]);
        const df a1 = df_from_double(D1 + (2.0 * t - 1.0) * 0.5 * D2 + (3.0 * t * t - 6.0 * t + 2.0) * (1.0 / 6.0) * D3);
        const df a2 = df_from_double(0.5 * (D2 + (t - 1.0) * D3));
        const df a3 = df_from_double(D3 * (1.0 / 6.0));
        T.c0[2 * (o + k)] = make_float4(a0.hi, a0.lo, a1.hi, a1.lo);
        T.c0[2 * (o + k) + 1] = make_float4(a2.hi, a2.lo, a3.hi, a3.lo);
    }
}

// CTA per batch, thread per point; the atoms of the batch's system
template <int LMAX>
__global__ void __launch_bounds__(128) k_hartree_eval(DevPlan P, HartreeDev H, HartreeTabs T, double *vh)
{
    constexpr int L = (LMAX + 1) * (LMAX + 1);
    const DevBatch B = P.batches[blockIdx.x];
    const long long a0 = H.sys_atom0[B.sys], a1 = H.sys_atom0[B.sys + 1];
    for (int i = threadIdx.x; i < B.np; i += blockDim.x) {
        const long long p = B.pt0 + i;
        const float *pp = P.pts_dd + 6 * p;
        const df px{pp[0], pp[1]}, py{pp[2], pp[3]}, pz{pp[4], pp[5]};
        df acc{0.f, 0.f};
        for (long long a = a0; a < a1; a++) {
            const float4 r0 = T.rec[3 * a], r1 = T.rec[3 * a + 1];
            const df dx = dfa(px, df{-r0.x, -r0.y}), dy = dfa(py, df{-r0.z, -r0.w}), dz = dfa(pz, df{-r1.x, -r1.y});
            const df d2 = dfa(dfa(df_sqr(dx), df_sqr(dy)), df_sqr(dz));
            const float ri = d2.hi > 0.f ? rsqrtf(d2.hi) : 0.f;
            float A[L];
            if constexpr (LMAX > 0) ylm_unnormalised<LMAX, float>(dx.hi * ri, dy.hi * ri, dz.hi * ri, A);
            float part = 0.f;
            if (d2.hi > r1.z || (d2.hi == r1.z && d2.lo >= r1.w)) {
                // beyond the last shell: the exterior multipoles
                const float4 r2 = T.rec[3 * a + 2];
                acc = dfa(acc, df_mul(df{r2.x, r2.y}, df_rsqrt(d2, ri)));
                if constexpr (LMAX > 0) {
                    constexpr int NQ4 = (L - 1 + 3) / 4;
                    float q[NQ4 * 4];
                    const float4 *q4 = reinterpret_cast<const float4 *>(T.Qf + a * kLf);
#pragma unroll
                    for (int j = 0; j < NQ4; j++) {
                        const float4 u = q4[j];
                        q[4 * j] = u.x;
                        q[4 * j + 1] = u.y;
                        q[4 * j + 2] = u.z;
                        q[4 * j + 3] = u.w;
                    }
                    float rl = ri * ri;                              // 1/d^(l+1), l = 1
#pragma unroll
                    for (int l = 1; l <= LMAX; l++) {
                        float s = 0.f;
#pragma unroll
                        for (int m = -l; m <= l; m++) s = fmaf(q[l * l + l + m - 1], A[l * l + l + m], s);
                        part = fmaf(s, rl, part);
                        rl *= ri;
                    }
                }
            } else {
                const HartreeRad g = H.rad[a];
                const long long o = H.rad_off[a];
                const float4 R0 = T.rk[o];
                const df r02 = df_sqr(df{R0.x, R0.y});
                if (d2.hi < r02.hi || (d2.hi == r02.hi && d2.lo <= r02.lo)) {
                    // inside the first shell: V(r_0) (d / r_0)^l
                    acc = dfa(acc, df_from_double(T.V0[o]));
                    if constexpr (LMAX > 0) {
                        const float sr = d2.hi * ri * g.inv_r0;
                        const float *vf = T.Vf + o * kLf;
                        float sl = sr;
#pragma unroll
                        for (int l = 1; l <= LMAX; l++) {
                            float s = 0.f;
#pragma unroll
                            for (int m = -l; m <= l; m++) s = fmaf(vf[l * l + l + m - 1], A[l * l + l + m], s);
                            part = fmaf(s, sl, part);
                            sl *= sr;
                        }
                    }
                } else {
                    // between shells: interval k (r_k <= d < r_k+1), f = ln(d / r_k) / ln q
                    int k, i0;
                    float t;
                    if (g.df_log) {
                        // double-float: k from an FP32 estimate of x = ln(d / r_0) / ln q,
                        // corrected against the radii; ln(d / r_k) = 2 atanh(s),
                        // s = u / (2 + u), u = d / r_k - 1 < q - 1:
                        // 2 s + s z (2/3 + z (2/5 + z R(z))), z = s^2, with the terms
                        // to s^5 as double-floats and R = 2/7 + 2/9 z + ... + 2/19 z^6
                        // in FP32 (ln q <= 0.6 keeps s <= 0.3; the FP32 part's rounding
                        // and the first dropped term, 2 s^21 / 21, together stay below
                        // 6e-12 in ln(d / r_k))
                        const df d = df_sqrt(d2);
                        k = (int)floorf((__logf(d.hi) - g.ln_r0_f) * g.inv_lnq_f);
                        k = k < 0 ? 0 : (k > g.nrad - 2 ? g.nrad - 2 : k);
                        float4 Rk = T.rk[o + k];
                        if (k > 0 && (d.hi < Rk.x || (d.hi == Rk.x && d.lo < Rk.y))) {
                            k--;
                            Rk = T.rk[o + k];
                        } else if (k < g.nrad - 2) {
                            const float4 R1 = T.rk[o + k + 1];
                            if (!(d.hi < R1.x || (d.hi == R1.x && d.lo < R1.y))) {
                                k++;
                                Rk = R1;
                            }
                        }
                        const df u = dfa(df_mul(d, df{Rk.z, Rk.w}), df{-1.f, 0.f});
                        const df sv = df_mul(u, df_rcp(dfa(u, df{2.f, 0.f})));
                        const df z = df_sqr(sv);
                        float rz = 2.f / 19.f;
                        rz = fmaf(rz, z.hi, 2.f / 17.f);
                        rz = fmaf(rz, z.hi, 2.f / 15.f);
                        rz = fmaf(rz, z.hi, 2.f / 13.f);
                        rz = fmaf(rz, z.hi, 2.f / 11.f);
                        rz = fmaf(rz, z.hi, 2.f / 9.f);
                        rz = fmaf(rz, z.hi, 2.f / 7.f);
                        df ser = dfa_f(df{kTwoFifthHi, kTwoFifthLo}, z.hi * rz);     // 2/5 + z R
                        ser = dfa(df{kTwoThirdHi, kTwoThirdLo}, df_mul(z, ser));     // 2/3 + z (...)
                        const df ln1p = dfa(df{2.f * sv.hi, 2.f * sv.lo}, df_mul(sv, df_mul(z, ser)));
                        const df f = df_mul(ln1p, df{g.inv_lnq_hi, g.inv_lnq_lo});
                        // V_00 = a0 + f (a1 + f (a2 + f a3)) on interval k
                        const float4 c01 = T.c0[2 * (o + k)], c23 = T.c0[2 * (o + k) + 1];
                        df pv = dfa(df{c23.x, c23.y}, df_mul(f, df{c23.z, c23.w}));
                        pv = dfa(df{c01.z, c01.w}, df_mul(f, pv));
                        pv = dfa(df{c01.x, c01.y}, df_mul(f, pv));
                        acc = dfa(acc, pv);
                        i0 = k - 1 < 0 ? 0 : (k - 1 > g.nrad - 4 ? g.nrad - 4 : k - 1);
                        t = (float)(k - i0) + f.hi;
                    } else {
                        // coarse radial grids: FP64 logarithm and Lagrange weights
                        const double dd2 = (double)d2.hi + (double)d2.lo;
                        const double *v0 = T.V0 + o;
                        const double x = (0.5 * log(dd2) - g.ln_r0) * g.inv_lnq;
                        i0 = (int)floor(x) - 1;
                        i0 = i0 < 0 ? 0 : (i0 > g.nrad - 4 ? g.nrad - 4 : i0);
                        const double td = x - (double)i0;
                        const double w0 = -(td - 1.0) * (td - 2.0) * (td - 3.0) * (1.0 / 6.0);
                        const double w1 = td * (td - 2.0) * (td - 3.0) * 0.5;
                        const double w2 = -td * (td - 1.0) * (td - 3.0) * 0.5;
                        const double w3 = td * (td - 1.0) * (td - 2.0) * (1.0 / 6.0);
                        acc = dfa(acc, df_from_double(w0 * v0[i0] + w1 * v0[i0 + 1] + w2 * v0[i0 + 2] + w3 * v0[i0 + 3]));
                        t = (float)td;
                        k = 0;
                    }
                    (void)k;
                    if constexpr (LMAX > 0) {
                        // l >= 1: Lagrange weights at nodes t = 0, 1, 2, 3 (shells i0 .. i0+3), FP32
                        const float f0 = -(t - 1.f) * (t - 2.f) * (t - 3.f) * (1.f / 6.f);
                        const float f1 = t * (t - 2.f) * (t - 3.f) * 0.5f;
                        const float f2 = -t * (t - 1.f) * (t - 3.f) * 0.5f;
                        const float f3 = t * (t - 1.f) * (t - 2.f) * (1.f / 6.f);
                        const float *vf = T.Vf + (o + i0) * kLf;
#pragma unroll
                        for (int q = 1; q < L; q++)
                            part = fmaf(f0 * vf[q - 1] + f1 * vf[kLf + q - 1] + f2 * vf[2 * kLf + q - 1] +
                                            f3 * vf[3 * kLf + q - 1],
                                        A[q], part);
                    }
                }
            }
            acc = dfa_f(acc, part);
        }
        vh[p] = (double)acc.hi + (double)acc.lo;
    }
}

}  // namespace

HartreeRad hartree_rad(double r_min, double ln_q, int n_rad)
{
    HartreeRad g{};
    g.r0 = r_min;
    g.lnq = ln_q;
    g.inv_lnq = 1.0 / ln_q;
    g.ln_r0 = std::log(r_min);
    const double rmax = r_min * std::exp(ln_q * (double)(n_rad - 1));
    const double r2 = rmax * rmax;
    const df d = df_from_double(r2);
    // a normalised pair: hi the nearest float, lo the remainder rounded
    g.rmax2_hi = d.hi;
    g.rmax2_lo = d.lo;
    g.inv_r0 = (float)(1.0 / r_min);
    g.nrad = n_rad;
    const df il = df_from_double(1.0 / ln_q);
    g.inv_lnq_hi = il.hi;
    g.inv_lnq_lo = il.lo;
    g.ln_r0_f = (float)std::log(r_min);
    g.inv_lnq_f = (float)(1.0 / ln_q);
    g.df_log = ln_q <= 0.6 ? 1 : 0;
    return g;
}

size_t hartree_ws_bytes(const HartreeDev &H)
{
    return 3 * al256(sizeof(double) * kL * (size_t)H.n_shells) + al256(sizeof(float4) * 3 * (size_t)H.n_atoms) +
           al256(sizeof(float4) * (size_t)H.n_shells) + al256(sizeof(float4) * 2 * (size_t)H.n_shells) +
           al256(sizeof(double) * (size_t)H.n_shells) +
           al256(sizeof(float) * kLf * (size_t)H.n_shells) +
           al256(sizeof(float) * kLf * (size_t)H.n_atoms);
}

cudaError_t launch_hartree(const DevPlan &P, const HartreeDev &H, int n_batch, long long n_pts, int l_max,
                           const double *n, double *vh, double *ws, cudaStream_t s)
{
    const HartreeTabs T = carve(H, ws);
    cudaError_t e = cudaMemsetAsync(T.rho, 0, sizeof(double) * kL * (size_t)H.n_shells, s);
    if (e != cudaSuccess) return e;
    if (n_pts > 0) {
        const unsigned grid = (unsigned)std::min<long long>((n_pts + 255) / 256, 4864);
        switch (l_max) {
        case 0: k_hartree_moments<0><<<grid, 256, 0, s>>>(P, H, n_pts, n, T.rho); break;
        case 1: k_hartree_moments<1><<<grid, 256, 0, s>>>(P, H, n_pts, n, T.rho); break;
        case 2: k_hartree_moments<2><<<grid, 256, 0, s>>>(P, H, n_pts, n, T.rho); break;
        case 3: k_hartree_moments<3><<<grid, 256, 0, s>>>(P, H, n_pts, n, T.rho); break;
        case 4: k_hartree_moments<4><<<grid, 256, 0, s>>>(P, H, n_pts, n, T.rho); break;
        case 5: k_hartree_moments<5><<<grid, 256, 0, s>>>(P, H, n_pts, n, T.rho); break;
        default: k_hartree_moments<6><<<grid, 256, 0, s>>>(P, H, n_pts, n, T.rho); break;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const long long nt = (long long)H.n_atoms * (l_max + 1) * (l_max + 1);
    if (nt > 0) {
        k_hartree_radial<<<(unsigned)((nt + 31) / 32), 32, 0, s>>>(P, H, l_max, T);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (n_batch > 0) {
        switch (l_max) {
        case 0: k_hartree_eval<0><<<n_batch, 128, 0, s>>>(P, H, T, vh); break;
        case 1: k_hartree_eval<1><<<n_batch, 128, 0, s>>>(P, H, T, vh); break;
        case 2: k_hartree_eval<2><<<n_batch, 128, 0, s>>>(P, H, T, vh); break;
        case 3: k_hartree_eval<3><<<n_batch, 128, 0, s>>>(P, H, T, vh); break;
        case 4: k_hartree_eval<4><<<n_batch, 128, 0, s>>>(P, H, T, vh); break;
        case 5: k_hartree_eval<5><<<n_batch, 128, 0, s>>>(P, H, T, vh); break;
        default: k_hartree_eval<6><<<n_batch, 128, 0, s>>>(P, H, T, vh); break;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace fgi
