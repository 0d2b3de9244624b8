// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers (about 48 significant bits).  Built from the error-free
// transformations of Dekker (1971) and Knuth (TAOCP vol. 2): the exact
// rounding error of a sum from six additions, of a product from one FMA.
// Used where FP32 rounding would be systematic across many grid points
// (the radial spline and its normalisation), at a fraction of the cost of
// GB300's FP64 pipe.  Relies on IEEE FP32 without reassociation (nvcc's
// default; explicit fmaf where an FMA is meant).
#pragma once
#include <cuda_runtime.h>

namespace fgi {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ df df_fast_two_sum(float a, float b)   // |a| >= |b|
{
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ df df_two_prod(float a, float b)
{
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ df df_add(df a, df b)
{
    df s = df_two_sum(a.hi, b.hi);
    const df t = df_two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = df_fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df{-b.hi, -b.lo}); }

// Sum with one error-free transformation (the high parts) and a rounded sum
// of the low parts: error within about 2^-48 (|a| + |b|) instead of
// 2^-48 |a + b|.  Exact enough for sums of one sign, and for differences of
// grid coordinates, whose rounding differs from point to point.
__device__ __forceinline__ df df_add_sloppy(df a, df b)
{
    const df s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ df df_sub_sloppy(df a, df b) { return df_add_sloppy(a, df{-b.hi, -b.lo}); }

__device__ __forceinline__ df df_mul(df a, df b)
{
    df p = df_two_prod(a.hi, b.hi);
    p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
    return df_fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df df_mul_f(df a, float b)
{
    df p = df_two_prod(a.hi, b);
    p.lo = fmaf(a.lo, b, p.lo);
    return df_fast_two_sum(p.hi, p.lo);
}

// The same product without the final renormalisation: hi = fl(a.hi b) and
// lo the rest, |lo| up to about two ulps of hi.  For consumers that use the
// pair only as the sum hi + lo (the split into BF16 terms).
__device__ __forceinline__ df df_mul_f_raw(df a, float b)
{
    const float p = a.hi * b;
    return {p, fmaf(a.lo, b, fmaf(a.hi, b, -p))};
}

// sqrt by one Newton correction of the FP32 root (IEEE sqrtf)
__device__ __forceinline__ df df_sqrt(df a)
{
    if (a.hi <= 0.f) return {0.f, 0.f};
    const float r = sqrtf(a.hi);
    const float e = fmaf(-r, r, a.hi) + a.lo;
    return df_fast_two_sum(r, e * (0.5f / r));
}

// 1/a by one Newton correction of the FP32 reciprocal
__device__ __forceinline__ df df_rcp(df a)
{
    const float r = 1.0f / a.hi;
    float e = fmaf(-a.hi, r, 1.0f);
    e = fmaf(-a.lo, r, e);
    return df_fast_two_sum(r, e * r);
}

// 1/sqrt(a) from an approximation y (relative error up to ~2^-20): with
// rho = 1 - a y^2 (from exact products, to about 2^-46 absolute),
// 1/sqrt(a) = y (1 - rho)^(-1/2) = y (1 + rho/2 + 3 rho^2/8 + O(rho^3)).
// Host-callable so that tests can check it against FP64 with a perturbed y.
__host__ __device__ __forceinline__ df df_rsqrt_refine(df a, float y)
{
    const float y2h = y * y;
    const float y2l = fmaf(y, y, -y2h);
    const float ph = a.hi * y2h;
    const float pl = fmaf(a.hi, y2h, -ph);
    // 1 - ph is exact (ph is within a factor two of 1)
    const float rho = ((1.f - ph) - pl) - fmaf(a.hi, y2l, a.lo * y2h);
    const float c = y * (rho * fmaf(0.375f, rho, 0.5f));
    const float s = y + c;
    return {s, c - (s - y)};
}

#if defined(__CUDACC__)
// 1/sqrt(a) for a > 0 (a.hi a normal FP32 number): the FP32 approximation
// rsqrtf refined once
__device__ __forceinline__ df df_rsqrt(df a) { return df_rsqrt_refine(a, rsqrtf(a.hi)); }
#endif

__host__ __device__ __forceinline__ df df_from_double(double x)
{
    const float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}

}  // namespace fgi
