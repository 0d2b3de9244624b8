// The Hartree potential from the density on the grid (multipole method):
// device tables and launcher.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>

#include "fgi_internal.h"

namespace fgi {

// one atom's radial grid, with what the evaluation needs precomputed
struct HartreeRad {
    double r0, lnq;                      // r_k = r0 exp(k ln q)
    double inv_lnq, ln_r0;
    float rmax2_hi, rmax2_lo;            // (last shell radius)^2 as a double-float
    float inv_r0;
    int nrad;
    float inv_lnq_hi, inv_lnq_lo;        // 1/ln q as a double-float
    float ln_r0_f, inv_lnq_f;            // FP32 copies for the interval estimate
    int df_log;                          // ln q small enough for the double-float logarithm
    int pad[3];
};

// the grid's atom-centred structure on the device
struct HartreeDev {
    const int *owner = nullptr;          // [n_pts] owner atom (global index, -1: none)
    const int *shell = nullptr;          // [n_pts] radial shell on the owner's grid
    const long long *rad_off = nullptr;  // [n_atoms + 1] first shell of each atom in the shell tables
    const HartreeRad *rad = nullptr;     // [n_atoms]
    const long long *sys_atom0 = nullptr;  // [n_sys + 1] first atom of each system
    int n_atoms = 0;
    long long n_shells = 0;
};

// radial grid record of one atom (host)
HartreeRad hartree_rad(double r_min, double ln_q, int n_rad);

// scratch of one call: multipoles and potentials on the shells, exterior moments
size_t hartree_ws_bytes(const HartreeDev &H);

// v_H at every point of the grid from n (both device, caller's point order)
cudaError_t launch_hartree(const DevPlan &P, const HartreeDev &H, int n_batch, long long n_pts, int l_max,
                           const double *n, double *vh, double *ws, cudaStream_t s);

}  // namespace fgi
