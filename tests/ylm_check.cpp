// Host driver for the library's real spherical harmonics (fgi_ylm.cuh):
// reads unit vectors "x y z" from stdin, prints Y_lm, l <= 6, one line each.
#include <cstdio>

#include "fgi_ylm.cuh"

int main()
{
    double x, y, z;
    double Y[(fgi::kHartreeLmax + 1) * (fgi::kHartreeLmax + 1)];
    while (std::scanf("%lf %lf %lf", &x, &y, &z) == 3) {
        fgi::real_ylm_all<fgi::kHartreeLmax>(x, y, z, Y);
        for (double v : Y) std::printf("%.17g ", v);
        std::printf("\n");
    }
    return 0;
}
