// Tensor-core (tcgen05) path: operand images, work lists, waves, launchers.
//
// Per batch b (P_b points, n_b active functions) the basis values are
// written once per call into "operand images": BF16 planes of the 3-term
// split phi = x0 + x1 + x2, laid out exactly as the tcgen05 shared-memory
// operand (128-byte swizzled, K-major rows of 64 points, 1 KB atoms of 8
// rows, 16 KB chunks of 128 rows), so that one bulk copy moves one operand
// chunk.  Batches are processed in waves whose images fit a bounded
// workspace (and stay in L2 when the wave is small).
#pragma once
#include <cstddef>
#include <string>
#include <vector>

#include "fgi_internal.h"

namespace fgi {

constexpr int kChunkBytes = 16384;       // 128 rows x 64 columns x 2 bytes

struct TcBatch {
    long long img_phi;     // byte offset (in the wave's workspace) of the phi image
    long long img_aux;     // byte offset of the w v phi image (H) or the D image (density)
    long long plane_phi;   // bytes per plane of the phi / w v phi images
    long long plane_d;     // bytes per plane of the D image
    int nrb;               // 128-row blocks (functions)
    int nc;                // 64-point chunks holding points
    int nc_alloc;          // allocated 64-point chunks (even)
    int nkc;               // 64-function chunks (density contraction depth)
    long long part0;       // first partial-density row of the batch in its wave (128 doubles each)
    long long img_e;       // byte offset of E = G Phi (FP32 [row][point], rows of 64 nc_alloc points)
                           // for the adjoint, -1 when the plan keeps no room for it
};

struct TcWave {
    int b0 = 0, nb = 0;
    long long phi0 = 0, nphi = 0;    // items: (batch, row block)
    long long h0 = 0, nh = 0;        // items: (batch, I, J), I <= J
    long long g0 = 0, ng = 0;        // items: (batch, J) of the D gather
    long long pc0 = 0, npc = 0;      // items: (batch, 64-point chunk) of the density's phi image
    long long d0 = 0, nd = 0;        // items: (batch, point tile of 128): the final sums
    long long e0 = 0, ne = 0;        // items: (batch, point tile, function block J) of the density MMA
    size_t part_off = 0;             // workspace offset (after img_base) of the wave's partial densities
    double phi_flops = 0, phi_bytes = 0, h_flops = 0, h_bytes = 0, n_flops = 0, n_bytes = 0;
    double g_bytes = 0;
};

struct TcPlanInput {
    int n_batch = 0;
    const DevBatch *batches = nullptr;   // FP64-path batch table (points, actives)
    const DevAct *act = nullptr;
    const int *atom_nfn = nullptr;
    const char *tune_path = nullptr;
    long long nnz = 0;                   // stored values of H (scratch sizing)
    int sb_points = 0;                   // super-batch point limit (0: keep the batches)
    double sb_growth = 1.0;              // limit on the union's functions / largest member's
    long long n_fn = 0;                  // functions (all systems)
    bool host_only = false;              // build host tables only (no device copies)
    long long wave_mb = 0;               // operand images per wave, MiB (0: default)
    int bound_grids = 0;                 // leading-digit grids from table bounds: 1 density, 2 also H
    bool with_e = false;                 // room for E = G Phi per batch (the adjoint's tiles)
};

struct TcPlan {
    bool built = false;
    size_t ws_bytes = 0;
    size_t wave_cap = 0;
    size_t img_base = 0;                 // workspace offset of the wave images (scratch below)
    size_t bound_off = 0;                // workspace offset of the per-function bounds of D
    size_t sign_off = 0;                 // workspace offset of the per-batch sign of w v (H images)
    long long nnz = 0, n_fn = 0;
    int num_sms = 1;                     // persistent grids: one CTA per SM
    int bound_grids = 0;                 // see TcPlanInput
    std::vector<DevBatch> sb;            // super-batches (points, union of active atoms)
    std::vector<DevAct> sact;            // their active-atom entries
    std::vector<int> sb_first;           // first input batch of each super-batch (+ n_batch at the end)
    std::vector<int> sb_rank;            // position in its wave's tile lists (-1: no tiles)
    const DevBatch *d_sb = nullptr;
    const DevAct *d_sact = nullptr;
    std::vector<TcBatch> batches;        // per super-batch image geometry
    std::vector<WorkItem> items;
    std::vector<TcWave> waves;
    void *d_mem = nullptr;               // device copies of batches + items
    const TcBatch *d_batches = nullptr;
    const WorkItem *d_items = nullptr;
};

int tc_build(TcPlan &t, const TcPlanInput &in, std::string *err);
void tc_free(TcPlan &t);
size_t tc_workspace_bytes(const TcPlan &t);

// launchers (one wave each); n_split = 3 (split BF16) or 1 (plain BF16)
cudaError_t tc_launch_phi(const TcPlan &t, const DevPlan &P, const TcWave &w, const double *v,
                          void *ws, int n_split, cudaStream_t s);
cudaError_t tc_launch_phi_cols(const TcPlan &t, const DevPlan &P, const TcWave &w, void *ws, int n_split,
                               cudaStream_t s);
// H: accumulates into the 2^-40 fixed-point scratch at the workspace start
cudaError_t tc_launch_h(const TcPlan &t, const DevPlan &P, const TcWave &w, const void *ws, int n_split,
                        cudaStream_t s);
cudaError_t tc_launch_fix_to_h(const TcPlan &t, const void *ws, double *h, long long nnz, int accumulate,
                               cudaStream_t s);
// density: D converted once to double-floats in the scratch (with per-function
// bounds of |D|), then gathered per batch
cudaError_t tc_launch_to_df(const TcPlan &t, const DevPlan &P, const double *x, void *ws, const long long *sys_val0,
                            const long long *sys_nnz, const int *fn_sys, cudaStream_t s);
cudaError_t tc_launch_gather_d(const TcPlan &t, const DevPlan &P, const TcWave &w, double offdiag_scale,
                               void *ws, int n_split, cudaStream_t s, bool full = false);
cudaError_t tc_launch_density(const TcPlan &t, const DevPlan &P, const TcWave &w, const void *ws,
                              double *n, int n_split, cudaStream_t s);
// adjoint of one wave (images and G gathered in full as above): E = G Phi on
// tcgen05 over every function block, dv_p = sum_j phi_j E_j (unweighted) into
// dv, E kept as FP32, then dR_a += -2 sum_p w_p v_p sum_{i on a} grad phi_i . E_i
cudaError_t tc_launch_adjoint(const TcPlan &t, const DevPlan &P, const TcWave &w, const void *ws, const double *v,
                              double *dv, double *dR, int n_split, cudaStream_t s);

// failure-path self-test: a bounded wait that runs out (status time-out)
cudaError_t tc_launch_wait_selftest(int *status, cudaStream_t s);

}  // namespace fgi
