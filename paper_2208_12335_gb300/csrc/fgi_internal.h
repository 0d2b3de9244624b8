// Internal plan structures shared by the host runtime and the CUDA kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fgi {

constexpr int kMaxL = 3;
constexpr int kMaxBatchPoints = 1024;
constexpr int kMaxBatchFns = 8192;       // per-batch local-function tables live in shared memory
constexpr int kImgRows = 128;            // tcgen05 operand image: rows (functions) per tile
constexpr int kImgCols = 64;             // points per 128-byte swizzle row

// status word bits (device)
constexpr int kStatusTimeout = 1;
constexpr int kStatusNonFinite = 2;
constexpr int kStatusBadIndex = 4;

struct DevRadial {
    double h, inv_h, rcut;
    long long coef_off;   // in units of 4 coefficients (one interval)
    int nk, l;
    float inv_h_hi, inv_h_lo;   // 1/h as a double-float
    float rcut_f;               // cutoff rounded to FP32
    int pad;
    long long bound_off;        // first entry of its suffix bounds of |u(r)/r| in DevPlan::rbound
};

struct DevSpecies {
    int shell0;           // first entry in shell_rad[]
    int n_shell;
    int n_fn;
    int shared_grid;      // 1: every shell's spline uses the same knots (scoef holds them interleaved)
    double rcut;          // largest cutoff of the species' radials
    long long scoef_off;  // shared grid: first float4 of the species in scoef
    int nk;               // shared grid: knots
    float inv_h_hi, inv_h_lo;   // shared grid: 1/h as a double-float
    int lmax;             // largest angular momentum of its shells
    int nl[4];            // shells of each l (DevPlan::shells holds them grouped by l)
};

// One radial shell of a species (index shell0 + sh), the fields the
// tensor-core basis kernels read, packed in 32 bytes.  Within a species the
// entries are grouped by l (ascending, otherwise in input order); fn0 gives
// each shell's place among the species' functions, so that the order of
// evaluation does not change which row a value lands in.
struct DevShell {
    int coef_off;         // first interval of the radial in coef_dd (units of 4 coefficients)
    int nk;               // knots
    int l;
    float rcut_f;         // cutoff rounded to FP32
    float inv_h_hi, inv_h_lo;   // 1/h as a double-float
    int bound_off;        // first entry of its suffix bounds of |u(r)/r| in DevPlan::rbound
    int fn0;              // first function of the shell within its species
};

struct DevBatch {
    long long pt0;        // first point (global)
    int np;               // points in the batch
    int sys;              // system
    int act0;             // first active-atom entry
    int n_act;            // active atoms
    int nfn;              // active functions n_b
    int kpad;             // padded point count used by the operand layouts
    long long ws_off;     // element offset of the batch's operand block in the wave's workspace
};

struct DevAct {
    int atom;             // global atom index
    int fn_loc;           // first local function of this atom in the batch
};

struct WorkItem {         // one tile of a per-batch contraction
    int batch;
    short ti, tj;
};

struct DevPlan {
    // points (SoA) and weights
    const double *px, *py, *pz, *pw;
    // atoms
    const double *atom_xyz;       // [n_atoms][3]
    const int *atom_species;
    const long long *atom_fn0;    // global index of the atom's first function
    const int *atom_loc;          // index of the atom inside its system
    // basis
    const DevSpecies *species;
    const int *shell_rad;         // radial id per species shell
    const DevShell *shells;       // the same shells, packed for the tensor-core basis kernels
    int n_shells;                 // entries of shell_rad / shells
    const DevRadial *radials;
    const double *coef;           // [sum intervals][4] FP64
    const float4 *coef_dd;        // [sum intervals][2]: the four coefficients as double-floats (hi, lo)
    const float4 *scoef;          // species on one knot grid: [interval][shell][2], the same double-floats
    // the same two tables with every coefficient times the first
    // normalisation constant of the radial's l (C_0 = 1/(2 sqrt pi), C_1, the
    // xy constant of l = 2, the y(3x^2 - y^2) constant of l = 3), rounded
    // from FP64: the lane-per-point basis kernels.  scoefn interleaves the
    // shells in the order of DevPlan::shells (grouped by l).
    const float4 *coef_ddn;
    const float4 *scoefn;
    const float *pts_dd;          // [n_pts][6]: x, y, z as double-floats (xh, xl, yh, yl, zh, zl)
    const float *atom_dd;         // [n_atoms][6]: the same for atom positions
    // systems
    const int *sys_nat;           // atoms per system
    const long long *sys_pair_off;// offset of the system's pairpos table
    const int *pairpos;           // [nat*nat] per system: position of atom b's run in atom a's row, -1 absent
    const long long *rowptr;      // per global function: index of its first stored value
    const int *col_glob;          // per stored value: global column function, -1 on the diagonal
    // batches
    const DevBatch *batches;
    const DevAct *act;
    int *status;
    // bounds of |phi| (leading-digit grids without a pass over the points):
    // [16] max |Y_lm| (index l*l + l + m), then per radial, per knot
    // interval k, a bound of |u(r)/r| over r >= k h
    const float *rbound;
};

// ---- launchers (return the launch status) ----
// FP64 path
cudaError_t launch_phi_f64(const DevPlan &P, int b0, int nb, double *ws, cudaStream_t s);
cudaError_t launch_h_f64(const DevPlan &P, const WorkItem *items, int n_items, const double *ws,
                         const double *v, double *h, cudaStream_t s);
cudaError_t launch_density_f64(const DevPlan &P, const WorkItem *items, int n_items,
                               const double *ws, const double *d, double offdiag_scale,
                               double *n_out, double *e_out, cudaStream_t s);
cudaError_t launch_adjoint_grad(const DevPlan &P, int b0, int nb, const double *e_ws,
                                const double *v, double *dR, cudaStream_t s);
// shared helpers
cudaError_t launch_scale_by_weight(const DevPlan &P, long long n_pts, double *x, cudaStream_t s);
cudaError_t launch_point_traces(const DevPlan &P, int n_batch, const double *n, double *traces,
                                cudaStream_t s);
cudaError_t launch_matrix_trace(const DevPlan &P, int n_sys, const long long *sys_fn0,
                                const long long *sys_val0, long long n_fn_total,
                                long long nnz_total, const int *fn_sys, const double *a,
                                const double *b, double *out, cudaStream_t s);
cudaError_t launch_check_finite(const DevPlan &P, const double *x, long long n, cudaStream_t s);

}  // namespace fgi

struct fgi_ctx;
namespace fgi {
// host-side helpers shared between the runtime's translation units
int internal_device(const fgi_ctx *c);
int internal_error(fgi_ctx *c, int code, const char *msg);
int internal_integrate_h(fgi_ctx *c, const double *v, double *h, int accumulate, void *ws, size_t ws_bytes,
                         void *stream, bool allow_profile);
}  // namespace fgi
