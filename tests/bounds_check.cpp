// Prints the table bounds of paper_2208_12335_gb300/csrc/fgi_bounds.h for
// tests/test_bounds_host.py:
//   bounds_check ylm            -> the 16 entries of max |Y_lm|
//   bounds_check radial < in    -> in: "n_int h" then 4 n_int coefficients;
//                                  out: the n_int suffix bounds of |u(r)/r|
#include <cstdio>
#include <cstring>
#include <vector>

#include "fgi_bounds.h"

int main(int argc, char **argv)
{
    if (argc == 2 && std::strcmp(argv[1], "ylm") == 0) {
        float y[fgi::kYlmMaxEntries];
        fgi::ylm_abs_max(y);
        for (int i = 0; i < fgi::kYlmMaxEntries; i++) std::printf("%.9g\n", (double)y[i]);
        return 0;
    }
    if (argc == 2 && std::strcmp(argv[1], "radial") == 0) {
        int n = 0;
        double h = 0.0;
        if (std::scanf("%d %lf", &n, &h) != 2 || n <= 0) return 2;
        std::vector<double> coef(4 * (size_t)n);
        for (double &c : coef)
            if (std::scanf("%lf", &c) != 1) return 2;
        std::vector<float> out(n);
        fgi::radial_over_r_bounds(coef.data(), n, h, out.data());
        for (float v : out) std::printf("%.9g\n", (double)v);
        return 0;
    }
    return 1;
}
