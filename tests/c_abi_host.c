/*
 * A plain C99 caller of the library's C ABI, host-only (no GPU): it builds a
 * three-atom problem from C arrays, plans it in a host-only context and
 * checks the sizes, the sparsity pattern, the per-batch work, the schedule
 * and the error paths.  tests/test_c_abi.py compiles it with gcc against
 * include/fgi.h and libfgi.so and runs it.  Exit status 0 and "C ABI OK"
 * on success; otherwise the failing check is printed.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "fgi.h"

static int failures = 0;

#define CHECK(cond)                                                          \
    do {                                                                     \
        if (!(cond)) {                                                       \
            fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #cond); \
            failures++;                                                      \
        }                                                                    \
    } while (0)

/* piecewise-linear spline of u(r) = r^(l+1) exp(-a r^2) on n_knots knots */
static void linear_spline(int l, double a, double h, int n_knots, double *coef)
{
    for (int k = 0; k < n_knots - 1; k++) {
        const double r0 = k * h, r1 = (k + 1) * h;
        const double u0 = pow(r0, l + 1) * exp(-a * r0 * r0);
        const double u1 = pow(r1, l + 1) * exp(-a * r1 * r1);
        coef[4 * k + 0] = u0;
        coef[4 * k + 1] = u1 - u0;
        coef[4 * k + 2] = 0.0;
        coef[4 * k + 3] = 0.0;
    }
}

int main(void)
{
    enum { NK = 101 };
    const double h = 0.05; /* cutoff (NK - 1) h = 5 Bohr */
    static double coef_s[4 * (NK - 1)], coef_p[4 * (NK - 1)];
    linear_spline(0, 0.8, h, NK, coef_s);
    linear_spline(1, 0.6, h, NK, coef_p);

    fgi_ctx *ctx = NULL;
    CHECK(fgi_create(&ctx, -1) == FGI_OK && ctx != NULL);
    CHECK(strcmp(fgi_last_error(ctx), "") == 0);

    /* out-of-order and bad-argument calls */
    CHECK(fgi_plan(ctx, FGI_FP64, NULL) == FGI_ERR_STATE);
    CHECK(strlen(fgi_last_error(ctx)) > 0);
    int bad_id = -1;
    CHECK(fgi_add_radial(ctx, 9, h, NK, coef_s, &bad_id) < 0);

    int rs = -1, rp = -1, sp = -1;
    CHECK(fgi_add_radial(ctx, 0, h, NK, coef_s, &rs) == FGI_OK);
    CHECK(fgi_add_radial(ctx, 1, h, NK, coef_p, &rp) == FGI_OK);
    const int shells[2] = {rs, rp};
    CHECK(fgi_add_species(ctx, 1.0, 2, shells, &sp) == FGI_OK); /* s + p: 4 functions */

    /* atoms A and B 1.4 Bohr apart (neighbours), C 30 Bohr away (alone) */
    const int64_t atom_off[2] = {0, 3};
    const int species[3] = {sp, sp, sp};
    const double xyz[9] = {0.0, 0.0, 0.0, 1.4, 0.0, 0.0, 30.0, 0.0, 0.0};
    CHECK(fgi_set_systems(ctx, 1, atom_off, species, xyz) == FGI_OK);

    /* batch 0: 12 points between A and B; batch 1: 6 points around C;
       batch 2: empty; batch 3: 2 points 50 Bohr from every atom */
    enum { NP = 20, NB = 4 };
    double pts[3 * NP], w[NP];
    for (int p = 0; p < 12; p++) {
        pts[3 * p] = -1.0 + 0.3 * p;
        pts[3 * p + 1] = 0.2;
        pts[3 * p + 2] = -0.1;
    }
    for (int p = 12; p < 18; p++) {
        pts[3 * p] = 30.0 + 0.5 * (p - 15);
        pts[3 * p + 1] = 0.3;
        pts[3 * p + 2] = 0.0;
    }
    for (int p = 18; p < NP; p++) {
        pts[3 * p] = 0.0;
        pts[3 * p + 1] = 50.0 + p;
        pts[3 * p + 2] = 0.0;
    }
    for (int p = 0; p < NP; p++) w[p] = 0.1;
    const int64_t batch_off[NB + 1] = {0, 12, 18, 18, NP};
    const int batch_sys[NB] = {0, 0, 0, 0};
    CHECK(fgi_set_grid(ctx, NP, pts, w, NB, batch_off, batch_sys) == FGI_OK);

    /* a non-finite point is refused */
    pts[5] = NAN;
    CHECK(fgi_set_grid(ctx, NP, pts, w, NB, batch_off, batch_sys) == FGI_ERR_NONFINITE);
    pts[5] = -0.1;
    CHECK(fgi_set_grid(ctx, NP, pts, w, NB, batch_off, batch_sys) == FGI_OK);

    CHECK(fgi_plan(ctx, FGI_SPLIT_BF16, NULL) == FGI_OK);

    int64_t n_fn = 0, nnz = 0, n_pts = 0, n_atoms = 0;
    CHECK(fgi_get_sizes(ctx, &n_fn, &nnz, &n_pts, &n_atoms) == FGI_OK);
    CHECK(n_fn == 12 && n_pts == NP && n_atoms == 3);
    /* upper triangle: the A-B block pair (8 x 8: 36 values) and C alone (10) */
    CHECK(nnz == 36 + 10);

    int64_t fn0 = -1, sn = -1, val0 = -1, snnz = -1;
    CHECK(fgi_get_system(ctx, 0, &fn0, &sn, &val0, &snnz) == FGI_OK);
    CHECK(fn0 == 0 && sn == 12 && val0 == 0 && snnz == nnz);

    int64_t pnnz = 0;
    const int64_t *rowptr = NULL;
    const int *col = NULL;
    CHECK(fgi_get_pattern(ctx, 0, &pnnz, &rowptr, &col) == FGI_OK);
    CHECK(pnnz == nnz && rowptr[0] == 0 && rowptr[12] == nnz);
    for (int i = 0; i < 12; i++) {
        const int expect = i < 8 ? 8 - i : 12 - i; /* columns i..last of the row's block group */
        CHECK(rowptr[i + 1] - rowptr[i] == expect);
        CHECK(col[rowptr[i]] == i);                 /* the diagonal comes first */
        for (int64_t k = rowptr[i] + 1; k < rowptr[i + 1]; k++) CHECK(col[k] > col[k - 1]);
    }

    int64_t bp[NB];
    int32_t bf[NB];
    CHECK(fgi_get_batch_work(ctx, NB, bp, bf) == FGI_OK);
    CHECK(bp[0] == 12 && bp[1] == 6 && bp[2] == 0 && bp[3] == 2);
    CHECK(bf[0] == 8 && bf[1] == 4 && bf[2] == 0 && bf[3] == 0);
    CHECK(fgi_get_batch_work(ctx, NB + 1, bp, bf) == FGI_ERR_ARG);

    int64_t n_super = 0, n_waves = 0;
    CHECK(fgi_get_schedule(ctx, 1, &n_super, &n_waves, NULL, NULL, NULL, NULL, NULL) == FGI_OK);
    CHECK(n_super >= 1 && n_super <= NB && n_waves == 1);
    int64_t *first = malloc(sizeof(int64_t) * (size_t)(n_super + 1));
    int64_t wave_first[2];
    CHECK(fgi_get_schedule(ctx, 1, &n_super, &n_waves, first, NULL, NULL, wave_first, NULL) == FGI_OK);
    CHECK(first[0] == 0 && first[n_super] == NB && wave_first[0] == 0 && wave_first[1] == n_super);
    free(first);

    size_t ws = 0;
    CHECK(fgi_workspace_size(ctx, &ws) == FGI_OK && ws > 0);

    /* compute calls need a device context */
    CHECK(fgi_integrate_h(ctx, NULL, NULL, 0, NULL, 0, NULL) == FGI_ERR_STATE);
    CHECK(fgi_sync(ctx, NULL) == FGI_ERR_STATE);

    CHECK(fgi_destroy(ctx) == FGI_OK);
    CHECK(fgi_destroy(NULL) == FGI_OK);

    if (failures) {
        fprintf(stderr, "%d checks failed\n", failures);
        return 1;
    }
    printf("C ABI OK\n");
    return 0;
}
