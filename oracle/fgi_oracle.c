/*
 * Plain FP64 CPU oracle for NAO real-space grid integration.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this file's library; the product path
 * never does.  It shares no code with the CUDA library.
 *
 * What it computes (the paper, "Development Priorities", names numeric
 * atom-centred orbitals integrated on real-space grids as the numerical core
 * of the method; the formulas are the textbook definitions of that method):
 *
 *   phi_i(r) = u_i(d)/d * Y_{l_i m_i}(d/|d|),  d = r - R_{atom(i)},  d = |d|
 *              u_i a piecewise cubic on a uniform radial grid, 0 for d >= r_cut
 *   H_ij = sum_p w_p v_p phi_i(r_p) phi_j(r_p)        (S_ij: the same, v = 1)
 *   n(r_p) = sum_ij phi_i(r_p) D_ij phi_j(r_p)
 *   adjoint of L = sum_ij G_ij H_ij with the grid held fixed:
 *     dL/dv_p = w_p sum_ij G_ij phi_i phi_j
 *     dL/dR_a = -2 sum_p w_p v_p sum_{i in a} grad phi_i(r_p) * sum_j G_ij phi_j(r_p)
 *
 * Readings where the method leaves a choice:
 *   - Y_lm are real, unit-normalised, without the Condon-Shortley phase,
 *     m ordered -l..l; l = 0..3 are supported.
 *   - interval k = min(floor(d/h), n_knots-2), t = d/h - k.
 *   - for d < 1e-12 Bohr, phi = (c1/h) Y_00 for l = 0 (the limit u'(0)), else 0,
 *     and grad phi = 0.
 *
 * Every matrix is computed in full (both triangles), with no use of symmetry
 * and no blocking; the only thing skipped is a term that is exactly zero
 * because d >= r_cut.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int n_atoms;
    const double *atom_xyz;    /* [n_atoms][3] */
    int n_fn;
    const int *fn_atom;        /* per fn: atom index */
    const int *fn_rad;         /* per fn: radial index */
    const int *fn_m;           /* per fn: m in -l..l */
    int n_rad;
    const int *rad_l;          /* per radial */
    const int *rad_nk;         /* knots per radial */
    const double *rad_h;       /* knot spacing per radial */
    const int64_t *rad_off;    /* offset of the radial's coefficients (in units of 4 doubles) */
    const double *coef;        /* [sum(nk-1)][4] */
} orc_basis;

/* real solid harmonics P_lm(x,y,z) (homogeneous of degree l) such that
   Y_lm(d) = P_lm(d)/|d|^l, and their Cartesian gradients */
static double solid_harmonic(int l, int m, double x, double y, double z, double g[3])
{
    const double c00 = 0.28209479177387814;   /* 1/(2 sqrt(pi)) */
    const double c1 = 0.4886025119029199;     /* sqrt(3/(4 pi)) */
    const double c2a = 1.0925484305920792;    /* sqrt(15/pi)/2 */
    const double c20 = 0.31539156525252005;   /* sqrt(5/pi)/4 */
    const double c22 = 0.5462742152960396;    /* sqrt(15/pi)/4 */
    const double c33 = 0.5900435899266435;    /* sqrt(35/(2 pi))/4 */
    const double c32 = 2.890611442640554;     /* sqrt(105/pi)/2 */
    const double c31 = 0.4570457994644658;    /* sqrt(21/(2 pi))/4 */
    const double c30 = 0.3731763325901154;    /* sqrt(7/pi)/4 */
    const double c32b = 1.445305721320277;    /* sqrt(105/pi)/4 */
    g[0] = g[1] = g[2] = 0.0;
    switch (l * 10 + (m + 3)) {
    case 3: return c00;                                   /* l0 m0 */
    case 12: g[1] = c1; return c1 * y;                    /* l1 m-1 */
    case 13: g[2] = c1; return c1 * z;                    /* l1 m0 */
    case 14: g[0] = c1; return c1 * x;                    /* l1 m1 */
    case 21: g[0] = c2a * y; g[1] = c2a * x; return c2a * x * y;          /* l2 m-2 */
    case 22: g[1] = c2a * z; g[2] = c2a * y; return c2a * y * z;          /* l2 m-1 */
    case 23: g[0] = -2 * c20 * x; g[1] = -2 * c20 * y; g[2] = 4 * c20 * z;
             return c20 * (2 * z * z - x * x - y * y);                    /* l2 m0 */
    case 24: g[0] = c2a * z; g[2] = c2a * x; return c2a * x * z;          /* l2 m1 */
    case 25: g[0] = 2 * c22 * x; g[1] = -2 * c22 * y; return c22 * (x * x - y * y); /* l2 m2 */
    case 30: g[0] = 6 * c33 * x * y; g[1] = c33 * (3 * x * x - 3 * y * y);
             return c33 * y * (3 * x * x - y * y);                        /* l3 m-3 */
    case 31: g[0] = c32 * y * z; g[1] = c32 * x * z; g[2] = c32 * x * y;
             return c32 * x * y * z;                                      /* l3 m-2 */
    case 32: g[0] = -2 * c31 * x * y; g[1] = c31 * (4 * z * z - x * x - 3 * y * y);
             g[2] = 8 * c31 * y * z;
             return c31 * y * (4 * z * z - x * x - y * y);                /* l3 m-1 */
    case 33: g[0] = -6 * c30 * x * z; g[1] = -6 * c30 * y * z;
             g[2] = c30 * (6 * z * z - 3 * x * x - 3 * y * y);
             return c30 * z * (2 * z * z - 3 * x * x - 3 * y * y);        /* l3 m0 */
    case 34: g[0] = c31 * (4 * z * z - 3 * x * x - y * y); g[1] = -2 * c31 * x * y;
             g[2] = 8 * c31 * x * z;
             return c31 * x * (4 * z * z - x * x - y * y);                /* l3 m1 */
    case 35: g[0] = 2 * c32b * x * z; g[1] = -2 * c32b * y * z; g[2] = c32b * (x * x - y * y);
             return c32b * z * (x * x - y * y);                           /* l3 m2 */
    case 36: g[0] = c33 * (3 * x * x - 3 * y * y); g[1] = -6 * c33 * x * y;
             return c33 * x * (x * x - 3 * y * y);                        /* l3 m3 */
    default: return 0.0;
    }
}

/* u(d) and du/dd from the radial spline; zero at and beyond the cutoff */
static void radial_u(const orc_basis *B, int rad, double d, double *u, double *du)
{
    int nk = B->rad_nk[rad];
    double h = B->rad_h[rad];
    *u = 0.0;
    *du = 0.0;
    if (d >= h * (nk - 1)) return;
    double s = d / h;
    int k = (int)floor(s);
    if (k > nk - 2) k = nk - 2;
    double t = s - k;
    const double *c = B->coef + 4 * (B->rad_off[rad] + k);
    *u = c[0] + t * (c[1] + t * (c[2] + t * c[3]));
    *du = (c[1] + t * (2.0 * c[2] + t * 3.0 * c[3])) / h;
}

/* phi_i at point r; optional gradient */
static double phi_fn(const orc_basis *B, int i, const double r[3], double grad[3])
{
    int a = B->fn_atom[i];
    int rad = B->fn_rad[i];
    int l = B->rad_l[rad];
    int m = B->fn_m[i];
    double x = r[0] - B->atom_xyz[3 * a + 0];
    double y = r[1] - B->atom_xyz[3 * a + 1];
    double z = r[2] - B->atom_xyz[3 * a + 2];
    double d = sqrt(x * x + y * y + z * z);
    if (grad) grad[0] = grad[1] = grad[2] = 0.0;
    double cut = B->rad_h[rad] * (B->rad_nk[rad] - 1);
    if (d >= cut) return 0.0;
    if (d < 1e-12) {
        if (l == 0) return B->coef[4 * B->rad_off[rad] + 1] / B->rad_h[rad] * 0.28209479177387814;
        return 0.0;
    }
    double u, du, gP[3];
    radial_u(B, rad, d, &u, &du);
    double P = solid_harmonic(l, m, x, y, z, gP);
    /* phi = u(d) P(x,y,z) / d^(l+1) */
    double dl1 = pow(d, l + 1);
    double val = u * P / dl1;
    if (grad) {
        /* d/dr [u/d^(l+1)] = (u' - (l+1) u/d)/d^(l+1), times r/d */
        double f = (du - (l + 1) * u / d) / dl1 * P / d;
        double q = u / dl1;
        grad[0] = f * x + q * gP[0];
        grad[1] = f * y + q * gP[1];
        grad[2] = f * z + q * gP[2];
    }
    return val;
}

/* non-zero basis functions at r (those of atoms within their cutoff) */
static int phi_nonzero(const orc_basis *B, int n_sub, const int *sub, const double r[3],
                       int *idx, double *val, double *grad)
{
    int cnt = 0;
    for (int s = 0; s < n_sub; s++) {
        int i = sub[s];
        double g[3];
        double v = phi_fn(B, i, r, grad ? g : NULL);
        int nz = (v != 0.0);
        if (grad) nz = nz || g[0] != 0.0 || g[1] != 0.0 || g[2] != 0.0;
        if (nz) {
            idx[cnt] = s;
            val[cnt] = v;
            if (grad) { grad[3 * cnt] = g[0]; grad[3 * cnt + 1] = g[1]; grad[3 * cnt + 2] = g[2]; }
            cnt++;
        }
    }
    return cnt;
}

/* phi[p][s] for all points and the subset of functions */
void orc_phi(const orc_basis *B, int64_t n_pts, const double *pts, int n_sub, const int *sub,
             double *phi, double *grad /* may be NULL: [n_pts][n_sub][3] */)
{
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n_pts; p++) {
        for (int s = 0; s < n_sub; s++) {
            double g[3];
            phi[p * n_sub + s] = phi_fn(B, sub[s], pts + 3 * p, grad ? g : NULL);
            if (grad) {
                grad[(p * n_sub + s) * 3 + 0] = g[0];
                grad[(p * n_sub + s) * 3 + 1] = g[1];
                grad[(p * n_sub + s) * 3 + 2] = g[2];
            }
        }
    }
}

/* H[s][t] = sum_p w_p v_p phi_s(r_p) phi_t(r_p) over the subset (v == NULL: v = 1) */
int orc_h(const orc_basis *B, int64_t n_pts, const double *pts, const double *w, const double *v,
          int n_sub, const int *sub, double *H)
{
    size_t nn = (size_t)n_sub * n_sub;
    memset(H, 0, nn * sizeof(double));
    int fail = 0;
#pragma omp parallel
    {
        double *Ht = (double *)calloc(nn, sizeof(double));
        int *idx = (int *)malloc(sizeof(int) * (n_sub > 0 ? n_sub : 1));
        double *val = (double *)malloc(sizeof(double) * (n_sub > 0 ? n_sub : 1));
        if (!Ht || !idx || !val) {
#pragma omp atomic write
            fail = 1;
        } else {
#pragma omp for schedule(dynamic, 256)
            for (int64_t p = 0; p < n_pts; p++) {
                int cnt = phi_nonzero(B, n_sub, sub, pts + 3 * p, idx, val, NULL);
                double f = w[p] * (v ? v[p] : 1.0);
                for (int a = 0; a < cnt; a++) {
                    double fa = f * val[a];
                    double *row = Ht + (size_t)idx[a] * n_sub;
                    for (int b = 0; b < cnt; b++) row[idx[b]] += fa * val[b];
                }
            }
#pragma omp critical
            for (size_t k = 0; k < nn; k++) H[k] += Ht[k];
        }
        free(Ht);
        free(idx);
        free(val);
    }
    return fail ? -1 : 0;
}

/* H values for listed pairs (subset indices are global fn indices here) */
void orc_h_pairs(const orc_basis *B, int64_t n_pts, const double *pts, const double *w,
                 const double *v, int64_t n_pairs, const int *pi, const int *pj, double *out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < n_pairs; k++) {
        double acc = 0.0;
        for (int64_t p = 0; p < n_pts; p++) {
            double a = phi_fn(B, pi[k], pts + 3 * p, NULL);
            if (a == 0.0) continue;
            double b = phi_fn(B, pj[k], pts + 3 * p, NULL);
            acc += w[p] * (v ? v[p] : 1.0) * a * b;
        }
        out[k] = acc;
    }
}

/* n_p = sum_st phi_s D[s][t] phi_t */
int orc_density(const orc_basis *B, int64_t n_pts, const double *pts, int n_sub, const int *sub,
                const double *D, double *n_out)
{
    int fail = 0;
#pragma omp parallel
    {
        int *idx = (int *)malloc(sizeof(int) * (n_sub > 0 ? n_sub : 1));
        double *val = (double *)malloc(sizeof(double) * (n_sub > 0 ? n_sub : 1));
        if (!idx || !val) {
#pragma omp atomic write
            fail = 1;
        } else {
#pragma omp for schedule(dynamic, 256)
            for (int64_t p = 0; p < n_pts; p++) {
                int cnt = phi_nonzero(B, n_sub, sub, pts + 3 * p, idx, val, NULL);
                double n = 0.0;
                for (int a = 0; a < cnt; a++)
                    for (int b = 0; b < cnt; b++)
                        n += val[a] * D[(size_t)idx[a] * n_sub + idx[b]] * val[b];
                n_out[p] = n;
            }
        }
        free(idx);
        free(val);
    }
    return fail ? -1 : 0;
}

/* adjoint of L = sum_st G[s][t] H[s][t] (G symmetric, over the subset):
   dv[p] = w_p sum_st G phi_s phi_t;  dR[a] = -2 sum_p w_p v_p sum_{s in a} grad phi_s * (G phi)_s */
int orc_adjoint(const orc_basis *B, int64_t n_pts, const double *pts, const double *w,
                const double *v, int n_sub, const int *sub, const double *G, double *dv,
                double *dR)
{
    int n_at = B->n_atoms;
    memset(dR, 0, sizeof(double) * 3 * n_at);
    int fail = 0;
#pragma omp parallel
    {
        int *idx = (int *)malloc(sizeof(int) * (n_sub > 0 ? n_sub : 1));
        double *val = (double *)malloc(sizeof(double) * (n_sub > 0 ? n_sub : 1));
        double *grd = (double *)malloc(sizeof(double) * 3 * (n_sub > 0 ? n_sub : 1));
        double *dRt = (double *)calloc(3 * (size_t)n_at, sizeof(double));
        if (!idx || !val || !grd || !dRt) {
#pragma omp atomic write
            fail = 1;
        } else {
#pragma omp for schedule(dynamic, 256)
            for (int64_t p = 0; p < n_pts; p++) {
                int cnt = phi_nonzero(B, n_sub, sub, pts + 3 * p, idx, val, grd);
                double q = 0.0;
                for (int a = 0; a < cnt; a++) {
                    double gphi = 0.0;   /* (G phi)_a */
                    for (int b = 0; b < cnt; b++) gphi += G[(size_t)idx[a] * n_sub + idx[b]] * val[b];
                    q += val[a] * gphi;
                    int at = B->fn_atom[sub[idx[a]]];
                    double f = -2.0 * w[p] * v[p] * gphi;
                    dRt[3 * at + 0] += f * grd[3 * a + 0];
                    dRt[3 * at + 1] += f * grd[3 * a + 1];
                    dRt[3 * at + 2] += f * grd[3 * a + 2];
                }
                dv[p] = w[p] * q;
            }
#pragma omp critical
            for (int k = 0; k < 3 * n_at; k++) dR[k] += dRt[k];
        }
        free(idx);
        free(val);
        free(grd);
        free(dRt);
    }
    return fail ? -1 : 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* threads of the later parallel loops (the single-core baseline) */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
