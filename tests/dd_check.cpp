// Host driver for the double-float reciprocal square root of the basis
// kernels (fgi_dd.cuh, df_rsqrt_refine): for seeded positive values a (as
// double-floats) and starting approximations y = (1 + delta)/sqrt(a.hi)
// with |delta| up to 2^-20, prints the largest relative error of the
// refined 1/sqrt(a) against long double for |delta| <= 2^-22 and for all
// delta, and that of a * (1/sqrt(a)) = sqrt(a) evaluated the way the
// kernels do (a double-float product).
#include <cmath>
#include <cstdint>
#include <cstdio>

#include "fgi_dd.cuh"

int main()
{
    uint64_t s = 0x9e3779b97f4a7c15ull;
    auto next = [&]() {                      // splitmix64
        uint64_t z = (s += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return z ^ (z >> 31);
    };
    // rsqrtf is within 2 ulp (|delta| < 2^-22); 2^-20 is a pessimistic case
    const double deltas[] = {-0x1p-20, -0x1p-22, -0x1p-23, 0.0, 0x1p-23, 0x1p-22, 0x1p-20};
    long double worst_r = 0, worst_s = 0, worst_r2 = 0;
    for (int i = 0; i < 200000; i++) {
        const double u = (double)(next() >> 11) * 0x1p-53;
        const double a = std::exp(std::log(1e-20) + u * (std::log(1e6) - std::log(1e-20)));
        const fgi::df ad = fgi::df_from_double(a);
        const long double ref = 1.0L / std::sqrt((long double)ad.hi + (long double)ad.lo);
        for (double dl : deltas) {
            const float y = (float)((1.0 + dl) / std::sqrt((double)ad.hi));
            const fgi::df r = fgi::df_rsqrt_refine(ad, y);
            const long double er = std::fabs(((long double)r.hi + (long double)r.lo) / ref - 1.0L);
            if (std::fabs(dl) < 0x1p-21 && er > worst_r2) worst_r2 = er;
            if (er > worst_r) worst_r = er;
            // sqrt(a) = a * (1/sqrt(a)) as a double-float product
            const float ph = ad.hi * r.hi;
            const float pl = std::fma(ad.hi, r.lo, std::fma(ad.lo, r.hi, std::fma(ad.hi, r.hi, -ph)));
            const long double sq = (long double)ph + (long double)pl;
            const long double es = std::fabs(sq * ref - 1.0L);
            if (es > worst_s) worst_s = es;
        }
    }
    std::printf("%.6Le %.6Le %.6Le\n", worst_r2, worst_r, worst_s);
    return 0;
}
