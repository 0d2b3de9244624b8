// The step upstream of the grid integration: the Hartree potential of the
// density on the grid, v_H(r) = int n(r') / |r - r'| dr', by the multipole
// method of Becke & Dickson (1988) and Delley (1990), which the NAO method
// uses for the electrostatic potential (the paper's Fig. 4 caption notes that
// this potential was not yet accelerated on GPUs).  FP64 throughout.
//
//  1. k_hartree_moments: per point p on atom a's radial shell k,
//       rho_a,lm(r_k) += (w_p / (r_k^3 ln q)) n_p Y_lm(rhat_p)
//     (w_p / (r_k^3 ln q) is the partitioned angular weight), FP64 atomics.
//  2. k_hartree_radial: per (atom, l, m) the radial Poisson equation
//       V(r) = 4 pi/(2l+1) [r^-(l+1) int_0^r rho r'^(l+2) dr' + r^l int_r^inf rho r'^(1-l) dr']
//     with the partial integrals in x = ln r interval by interval, each by the
//     integral of the cubic through its four nearest shells, plus
//     rho(r_0) r_0^(l+3)/(l+3) inside the first shell; Q_lm = the whole inner
//     integral (the exterior multipole moments).
//  3. k_hartree_eval: per point, over the atoms of its system, V_a,lm at the
//     distance (4-point Lagrange interpolation in the fractional shell index
//     inside the grid, 4 pi/(2l+1) Q_lm / d^(l+1) beyond the last shell,
//     V(r_0) (d/r_0)^l inside the first) times Y_lm of the direction.
#include "fgi_hartree.h"
#include "fgi_ylm.cuh"

namespace fgi {

namespace {

constexpr int kL = (kHartreeLmax + 1) * (kHartreeLmax + 1);

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
        const double2 g = H.rgrid[a];
        const double dx = P.px[p] - P.atom_xyz[3 * a], dy = P.py[p] - P.atom_xyz[3 * a + 1],
                     dz = P.pz[p] - P.atom_xyz[3 * a + 2];
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        if (!(r > 0.0)) continue;
        const double rk = g.x * exp(g.y * (double)k);
        const double val = P.pw[p] / (rk * rk * rk * g.y) * n[p];
        double Y[L];
        real_ylm_all<LMAX>(dx / r, dy / r, dz / r, Y);
        double *dst = rho + (H.rad_off[a] + k) * kL;
#pragma unroll
        for (int q = 0; q < L; q++) atomicAdd(dst + q, val * Y[q]);
    }
}

// one thread per (atom, lm)
__global__ void k_hartree_radial(HartreeDev H, int l_max, const double *rho, double *V, double *Q)
{
    const int L = (l_max + 1) * (l_max + 1);
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)H.n_atoms * L) return;
    const int a = (int)(t / L), lm = (int)(t % L);
    int l = 0;
    while ((l + 1) * (l + 1) <= lm) l++;
    const double2 g = H.rgrid[a];
    const int n = H.nrad[a];
    const long long o = H.rad_off[a];
    const double h = g.y;
    auto rk = [&](int k) { return g.x * exp(h * (double)k); };
    auto f = [&](int k) { const double r = rk(k); return rho[(o + k) * kL + lm] * pow(r, (double)(l + 3)); };
    auto gg = [&](int k) { const double r = rk(k); return rho[(o + k) * kL + lm] * pow(r, (double)(2 - l)); };
    // integral over interval [k, k+1] of the cubic through the nearest four samples
    auto seg = [&](auto fn, int k) {
        if (n < 4) return 0.5 * h * (fn(k) + fn(k + 1));
        if (k == 0) return h * (9.0 * fn(0) + 19.0 * fn(1) - 5.0 * fn(2) + fn(3)) / 24.0;
        if (k == n - 2) return h * (fn(n - 4) - 5.0 * fn(n - 3) + 19.0 * fn(n - 2) + 9.0 * fn(n - 1)) / 24.0;
        return h * (-fn(k - 1) + 13.0 * fn(k) + 13.0 * fn(k + 1) - fn(k + 2)) / 24.0;
    };
    const double pref = 4.0 * 3.14159265358979323846 / (2.0 * l + 1.0);
    // inner integrals, forward; V gets the inner part first
    double iin = f(0) / (double)(l + 3);
    for (int k = 0; k < n; k++) {
        if (k > 0) iin += seg(f, k - 1);
        V[(o + k) * kL + lm] = pref * iin / pow(rk(k), (double)(l + 1));
    }
    Q[(long long)a * kL + lm] = iin;
    // outer integrals, backward
    double iout = 0.0;
    for (int k = n - 1; k >= 0; k--) {
        if (k < n - 1) iout += seg(gg, k);
        V[(o + k) * kL + lm] += pref * iout * pow(rk(k), (double)l);
    }
}

// CTA per batch, thread per point; the atoms of the batch's system
template <int LMAX>
__global__ void __launch_bounds__(128) k_hartree_eval(DevPlan P, HartreeDev H, const double *V, const double *Q,
                                                      double *vh)
{
    constexpr int L = (LMAX + 1) * (LMAX + 1);
    const DevBatch B = P.batches[blockIdx.x];
    const long long a0 = H.sys_atom0[B.sys], a1 = H.sys_atom0[B.sys + 1];
    for (int i = threadIdx.x; i < B.np; i += blockDim.x) {
        const long long p = B.pt0 + i;
        const double px = P.px[p], py = P.py[p], pz = P.pz[p];
        double acc = 0.0;
        for (long long a = a0; a < a1; a++) {
            const double dx = px - P.atom_xyz[3 * a], dy = py - P.atom_xyz[3 * a + 1], dz = pz - P.atom_xyz[3 * a + 2];
            const double d = sqrt(dx * dx + dy * dy + dz * dz);
            double Y[L];
            if (d > 1e-12) {
                real_ylm_all<LMAX>(dx / d, dy / d, dz / d, Y);
            } else {
#pragma unroll
                for (int q = 0; q < L; q++) Y[q] = 0.0;
                Y[0] = 0.28209479177387814;
            }
            const double2 g = H.rgrid[a];
            const int n = H.nrad[a];
            const double r0 = g.x, rmax = g.x * exp(g.y * (double)(n - 1));
            const double *Va = V + H.rad_off[a] * kL;
            if (d >= rmax) {
                // exterior multipole field
                const double inv = 1.0 / d;
                double dl = inv;                           // 1/d^(l+1)
#pragma unroll
                for (int l = 0; l <= LMAX; l++) {
                    const double pref = 4.0 * 3.14159265358979323846 / (2.0 * l + 1.0) * dl;
                    for (int m = -l; m <= l; m++) acc += pref * Q[a * kL + l * l + l + m] * Y[l * l + l + m];
                    dl *= inv;
                }
            } else if (d <= r0) {
                const double s = d / r0;
                double sl = 1.0;
#pragma unroll
                for (int l = 0; l <= LMAX; l++) {
                    for (int m = -l; m <= l; m++) acc += Va[l * l + l + m] * sl * Y[l * l + l + m];
                    sl *= s;
                }
            } else {
                const double x = log(d / r0) / g.y;
                int i0 = (int)floor(x) - 1;
                i0 = i0 < 0 ? 0 : (i0 > n - 4 ? n - 4 : i0);
                const double t = x - (double)i0;
                // Lagrange weights at nodes t = 0, 1, 2, 3
                const double w0 = -(t - 1.0) * (t - 2.0) * (t - 3.0) / 6.0;
                const double w1 = t * (t - 2.0) * (t - 3.0) / 2.0;
                const double w2 = -t * (t - 1.0) * (t - 3.0) / 2.0;
                const double w3 = t * (t - 1.0) * (t - 2.0) / 6.0;
                const double *v0 = Va + (long long)i0 * kL;
#pragma unroll
                for (int q = 0; q < L; q++)
                    acc += (w0 * v0[q] + w1 * v0[kL + q] + w2 * v0[2 * kL + q] + w3 * v0[3 * kL + q]) * Y[q];
            }
        }
        vh[p] = acc;
    }
}

}  // namespace

size_t hartree_ws_bytes(const HartreeDev &H)
{
    return (size_t)(2 * H.n_shells + H.n_atoms) * kL * sizeof(double);
}

cudaError_t launch_hartree(const DevPlan &P, const HartreeDev &H, int n_batch, long long n_pts, int l_max,
                           const double *n, double *vh, double *ws, cudaStream_t s)
{
    double *rho = ws, *V = ws + H.n_shells * kL, *Q = ws + 2 * H.n_shells * kL;
    cudaError_t e = cudaMemsetAsync(rho, 0, (size_t)H.n_shells * kL * sizeof(double), s);
    if (e != cudaSuccess) return e;
    if (n_pts > 0) {
        const unsigned grid = (unsigned)std::min<long long>((n_pts + 255) / 256, 4864);
        switch (l_max) {
        case 0: k_hartree_moments<0><<<grid, 256, 0, s>>>(P, H, n_pts, n, rho); break;
        case 1: k_hartree_moments<1><<<grid, 256, 0, s>>>(P, H, n_pts, n, rho); break;
        case 2: k_hartree_moments<2><<<grid, 256, 0, s>>>(P, H, n_pts, n, rho); break;
        case 3: k_hartree_moments<3><<<grid, 256, 0, s>>>(P, H, n_pts, n, rho); break;
        case 4: k_hartree_moments<4><<<grid, 256, 0, s>>>(P, H, n_pts, n, rho); break;
        case 5: k_hartree_moments<5><<<grid, 256, 0, s>>>(P, H, n_pts, n, rho); break;
        default: k_hartree_moments<6><<<grid, 256, 0, s>>>(P, H, n_pts, n, rho); break;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const long long nt = (long long)H.n_atoms * (l_max + 1) * (l_max + 1);
    if (nt > 0) {
        k_hartree_radial<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(H, l_max, rho, V, Q);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (n_batch > 0) {
        switch (l_max) {
        case 0: k_hartree_eval<0><<<n_batch, 128, 0, s>>>(P, H, V, Q, vh); break;
        case 1: k_hartree_eval<1><<<n_batch, 128, 0, s>>>(P, H, V, Q, vh); break;
        case 2: k_hartree_eval<2><<<n_batch, 128, 0, s>>>(P, H, V, Q, vh); break;
        case 3: k_hartree_eval<3><<<n_batch, 128, 0, s>>>(P, H, V, Q, vh); break;
        case 4: k_hartree_eval<4><<<n_batch, 128, 0, s>>>(P, H, V, Q, vh); break;
        case 5: k_hartree_eval<5><<<n_batch, 128, 0, s>>>(P, H, V, Q, vh); break;
        default: k_hartree_eval<6><<<n_batch, 128, 0, s>>>(P, H, V, Q, vh); break;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace fgi
