/*
 * fgi.h -- C ABI of the GB300 library for batched real-space grid
 * integration with numeric atom-centred orbitals (NAO).
 *
 * The paper (FHI-aims, "Development Priorities") names NAO basis sets on
 * real-space integration grids as the numerical core of the method, and
 * ("Meeting the Exascale Challenges") GPU offloading of its computational
 * hotspots, batched matrix-matrix multiplications, sparse matrix operations
 * and data rearrangement as what large systems need.  This library computes,
 * for every batch b of grid points and the basis functions that are non-zero
 * on it,
 *
 *   phi_i(r) = u_i(d)/d * Y_lm(d/|d|),   d = r - R_atom(i)              (basis)
 *   H_ij    += sum_{p in b} w_p v_p phi_i(r_p) phi_j(r_p)  -> sparse H    (integration)
 *   n(r_p)   = sum_ij phi_i(r_p) D_ij phi_j(r_p)                          (density)
 *
 * and the adjoint of L = sum_ij G_ij H_ij.
 *
 * Conventions
 *   - Units: Bohr and Hartree.
 *   - Every function returns an int status: FGI_OK (0) or a negative error
 *     code.  fgi_last_error() gives a message owned by the context.  Nothing
 *     throws across the ABI.
 *   - Host arrays are read during the call and not retained (the library
 *     copies what it needs).
 *   - Device arrays passed to the compute calls are owned by the caller.
 *     The compute calls allocate nothing: scratch space is a caller-owned
 *     device buffer of at least fgi_workspace_size() bytes.
 *   - Compute calls only enqueue work on the caller's CUDA stream (a
 *     cudaStream_t passed as void*; NULL is the legacy default stream) and
 *     return; results are ready when the stream is.  Device-side errors
 *     (bounded waits that ran out, non-finite inputs) are recorded in a
 *     device status word that fgi_sync() reads.
 *   - A context serves one CUDA device; calls on one context must not
 *     overlap in host threads.
 *
 * Basis-function numbering: per system, atom by atom; within an atom, the
 * species' radial shells in order; within a shell of angular momentum l,
 * m = -l..l (real spherical harmonics without the Condon-Shortley phase).
 * Systems follow each other: the functions of system s are
 * fn0(s) .. fn0(s)+n_fn(s)-1.
 *
 * Sparse matrices (H, D, adjoint seeds): upper triangle (i <= j) of each
 * system's matrix in CSR order.  Entry (i, j) is stored when the atoms of i
 * and j are closer than the sum of their largest cutoffs (a superset of the
 * pairs whose functions overlap; the others are exactly zero).  Values of
 * system s occupy [val0(s), val0(s)+nnz(s)) of one array.
 */
#ifndef FGI_H
#define FGI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fgi_ctx fgi_ctx;

enum {
    FGI_OK = 0,
    FGI_ERR_ARG = -1,          /* bad argument (NULL, negative size, out of range) */
    FGI_ERR_STATE = -2,        /* call out of order (e.g. compute before fgi_plan) */
    FGI_ERR_CUDA = -3,         /* a CUDA runtime call failed */
    FGI_ERR_WORKSPACE = -4,    /* workspace NULL, misaligned or too small */
    FGI_ERR_TIMEOUT = -5,      /* a bounded device-side wait ran out */
    FGI_ERR_NONFINITE = -6,    /* NaN or Inf met in an input */
    FGI_ERR_UNSUPPORTED = -7,  /* l > 3, no sm_103 device, ... */
    FGI_ERR_NOMEM = -8         /* host or plan-time device allocation failed */
};

typedef enum {
    FGI_FP64 = 0,        /* every step in FP64 on CUDA cores */
    FGI_SPLIT_BF16 = 1,  /* contractions as 3-term split BF16 on tcgen05, FP32 accumulate,
                            FP64 across batches */
    FGI_BF16 = 2         /* contractions in plain BF16 on tcgen05, FP32 accumulate */
} fgi_precision;

/* Create a context on CUDA device `cuda_device`.  FGI_ERR_UNSUPPORTED if the
   device is not compute capability 10.3, FGI_ERR_CUDA if the CUDA runtime
   finds no driver or device, FGI_ERR_ARG for an index beyond the devices
   present.  There is no CPU fallback.  cuda_device = -1 creates a
   host-only context: inputs, plan tables, pattern and workspace queries
   work; the compute calls return FGI_ERR_STATE. */
int fgi_create(fgi_ctx **out, int cuda_device);
/* Free the context and every device buffer it owns.  NULL is accepted. */
int fgi_destroy(fgi_ctx *ctx);
/* Message of the last error on this context ("" if none). */
const char *fgi_last_error(const fgi_ctx *ctx);

/* Radial function u(r) (= r R(r)) as a uniform cubic spline on r_k = k h,
   k = 0..n_knots-1, with cutoff r_cut = (n_knots-1) h and u = 0 beyond it.
   coef: host [n_knots-1][4] doubles; on [r_k, r_k+1],
   u(r) = c0 + t (c1 + t (c2 + t c3)), t = (r - r_k)/h.  0 <= l <= 3.
   The basis function is phi = u(d)/d * Y_lm (the paper's NAO basis,
   "Development Priorities"). */
int fgi_add_radial(fgi_ctx *ctx, int l, double h, int n_knots, const double *coef,
                   int *radial_id_out);

/* Species with nuclear charge Z and n_shell radial shells (radial ids from
   fgi_add_radial); each shell of angular momentum l gives 2l+1 functions. */
int fgi_add_species(fgi_ctx *ctx, double Z, int n_shell, const int *radial_id,
                    int *species_id_out);

/* n_sys independent systems (the paper's ensemble runs, "Concluding
   Remarks"); atom_off[n_sys+1] (host, int64) splits the atom arrays;
   species[n_atoms] (host); xyz[n_atoms][3] (host, Bohr).  Replaces any
   previous systems and invalidates the plan. */
int fgi_set_systems(fgi_ctx *ctx, int n_sys, const int64_t *atom_off, const int *species,
                    const double *xyz);

/* Integration grid: n_pts points xyz[n_pts][3] and weights w[n_pts] (host),
   grouped into n_batch batches of consecutive points, batch b being
   [batch_off[b], batch_off[b+1]) and belonging to system batch_sys[b].
   A batch may hold at most 1024 points.  Invalidates the plan. */
int fgi_set_grid(fgi_ctx *ctx, int64_t n_pts, const double *xyz, const double *w,
                 int64_t n_batch, const int64_t *batch_off, const int *batch_sys);

/* Build the plan (host, once per geometry and grid): the functions active
   on each batch, the sparsity pattern of H, the tile work lists, and the
   device copies of the inputs.  tune_cache_path: NULL for the defaults, or a
   text file of "key value" lines written by the autotuner
   (paper_2208_12335_gb300/tune.py): density_sb_points (points per density
   super-batch, 0..1024; 0 keeps the given batches), density_sb_growth (limit
   on a super-batch's active functions relative to its largest member,
   1..16), wave_mb (operand-image workspace per wave, MiB, default 8192),
   h_sb_points and
   h_sb_growth (the same two limits for the H path; defaults 512 points and
   1.25: deeper H contractions accumulate more FP32 truncation in the
   remainder products), bound_grids (0, 1 or 2, default 2: the split images'
   leading-digit grids from table bounds of |phi| -- max |Y_lm| and
   per-interval suffix bounds of |u(r)/r| -- for the density images (1) and
   the H images too (2), instead of an FP32 pass over the points (0); the
   bounds apply only when every radial has u(0) = 0).  A missing file
   means the defaults; a malformed or out-of-range value is FGI_ERR_ARG.
   For experiments, the environment variables FGI_SB_POINTS,
   FGI_SB_GROWTH, FGI_H_SB_POINTS, FGI_H_SB_GROWTH, FGI_BOUND_GRIDS and FGI_TC_WAVE_MB
   override the file's values when set.
   The paper has no counterpart for the settings (it prints no kernel). */
int fgi_plan(fgi_ctx *ctx, fgi_precision precision, const char *tune_cache_path);

/* Change the precision of later compute calls without re-planning. */
int fgi_set_precision(fgi_ctx *ctx, fgi_precision precision);

/* Sizes after fgi_plan: total functions, total stored values (all
   systems), total points and atoms. */
int fgi_get_sizes(fgi_ctx *ctx, int64_t *n_fn, int64_t *nnz, int64_t *n_pts, int64_t *n_atoms);

/* Per-system layout: first function, function count, first value, value count. */
int fgi_get_system(fgi_ctx *ctx, int sys, int64_t *fn0, int64_t *n_fn, int64_t *val0,
                   int64_t *nnz);

/* Per-batch work after fgi_plan (host arrays of n_batch entries, written by
   the library): points P_b and active functions n_b of every batch, in the
   order fgi_set_grid gave the batches.  The contractions cost about
   P_b n_b^2; a caller that distributes one system over several processes
   (the paper's process-first parallelisation, "Meeting the Exascale
   Challenges") splits the batches across ranks by this cost.  Either
   pointer may be NULL.  The paper has no counterpart for the call itself.
   FGI_ERR_ARG if n_batch differs from the planned batch count. */
int fgi_get_batch_work(fgi_ctx *ctx, int64_t n_batch, int64_t *points, int32_t *n_active_fns);

/* The tensor-core schedule (host, after fgi_plan) of the H integration
   (which = 0) or of the density (which = 1).  Consecutive batches of one
   system are merged into super-batches: a batch joins while the merged
   points stay within the point limit and the union of active functions
   within the growth limit times the largest member's (the tune-file keys
   h_sb_points / h_sb_growth and density_sb_points / density_sb_growth).
   Consecutive super-batches form waves whose operand images fit the wave
   budget (wave_mb); each wave's tile lists take its super-batches longest
   first by P n^2 (stable for ties), and those without points or functions
   get no tiles.  Outputs (every pointer may be NULL; query the counts
   first):
     *n_super, *n_waves                 counts
     sb_first_batch[n_super + 1]        super-batch s = batches [first[s], first[s+1])
     sb_points[n_super], sb_fns[n_super]  its points and active functions
     wave_first_sb[n_waves + 1]         wave k = super-batches [first[k], first[k+1])
     sb_rank[n_super]                   position in its wave's tile lists, -1 if none
   The paper has no counterpart (it prints no kernel or schedule).
   FGI_ERR_ARG for another `which`. */
int fgi_get_schedule(fgi_ctx *ctx, int which, int64_t *n_super, int64_t *n_waves, int64_t *sb_first_batch,
                     int32_t *sb_points, int32_t *sb_fns, int64_t *wave_first_sb, int32_t *sb_rank);

/* CSR pattern of system `sys` (host arrays owned by the context, valid until
   the next fgi_plan/fgi_set_*): rowptr[n_fn(sys)+1] (relative to val0(sys))
   and col[nnz(sys)] (function index within the system). */
int fgi_get_pattern(fgi_ctx *ctx, int sys, int64_t *nnz, const int64_t **rowptr,
                    const int **col);

/* Bytes of device scratch space the compute calls need (for every
   precision). */
int fgi_workspace_size(fgi_ctx *ctx, size_t *bytes);

/* H integration: h[val] (+)= sum_b sum_{p in b} w_p v_p phi_i phi_j for every
   stored (i, j).  v_dev: device [n_pts] FP64; h_dev: device [nnz] FP64,
   overwritten (accumulate = 0) or added to (accumulate = 1).  Cross-batch
   accumulation: FP64 on the FP64 path; on the split-BF16 and BF16 paths an
   exact 64-bit fixed-point sum with unit 2^-40 Ha (bitwise reproducible,
   the FP32 tile results rounded to the unit), converted to FP64 once at the
   end.  Limits of that sum: one super-batch's contribution to an entry
   must stay below 2^22 Ha (beyond it the status word reports
   FGI_ERR_NONFINITE at the next fgi_sync), and every entry's running sum
   below 2^23 Ha (beyond it the 64-bit sum would wrap; this is not checked,
   and no Hamiltonian of the method comes near it). */
int fgi_integrate_h(fgi_ctx *ctx, const double *v_dev, double *h_dev, int accumulate,
                    void *ws, size_t ws_bytes, void *stream);

/* H integration for callers that cannot allocate device memory (a Fortran
   SCF driver without a CUDA allocator, a plug-in confined to another
   framework's memory pool, code that must not allocate inside its loop).
   The paper has no counterpart: this is a packaging of fgi_integrate_h.
   Same arguments and results as fgi_integrate_h, but the scratch space is a
   static device array of FGI_STATIC_SCRATCH_BYTES inside the library, which
   every GPU holding the library's device code keeps until the process
   exits; the call itself allocates nothing (no cudaMalloc, cudaFree or
   library allocation).
   - The first call on a device looks up the array's device address (once,
     with that device current); make that first call before any stream
     capture.  With CUDA's lazy module loading (the default in recent CUDA
     releases) that first look-up may be what loads this part of the library
     onto the device and reserves the array there: the first call can then
     fail for lack of device memory (reported as FGI_ERR_CUDA), and only
     devices on which the call has run hold the array.
   - A plan whose fgi_workspace_size() exceeds FGI_STATIC_SCRATCH_BYTES is
     rejected with FGI_ERR_WORKSPACE and a message giving both sizes.
   - All calls on a device share the one array, which keeps the last call's
     contents (what must start at zero is cleared on the device by each
     call); calls whose GPU work overlaps (other streams, other host
     threads, other contexts on the same device) race and must be
     serialised by the caller.
   - The launch profile (fgi_profile) does not record this call. */
#define FGI_STATIC_SCRATCH_BYTES ((size_t)64 << 20)
int fgi_integrate_h_static(fgi_ctx *ctx, const double *v_dev, double *h_dev, int accumulate,
                           void *stream);

/* Density: n_dev[p] = sum_ij phi_i(r_p) D_ij phi_j(r_p), in the caller's
   point order, D the symmetric matrix whose upper triangle d_dev[nnz]
   (device FP64) stores.  traces_dev (device [n_sys] FP64, may be NULL)
   receives N_el(s) = sum_{p in s} w_p n_p. */
int fgi_density(fgi_ctx *ctx, const double *d_dev, double *n_dev, double *traces_dev,
                void *ws, size_t ws_bytes, void *stream);

/* Adjoint of L = sum_stored g_k h_k (g_dev: device [nnz], the gradient of L
   with respect to the stored values of H): with G the symmetric matrix
   G_ii = g_ii, G_ij = G_ji = g_ij/2, and the grid held fixed while atoms move,
     dv_dev[p]   = w_p sum_ij G_ij phi_i phi_j                      [n_pts]
     dR_dev[a,:] = -2 sum_p w_p v_p sum_{i on a} grad phi_i . (G phi)_i  [n_atoms][3]
   v_dev is the potential of the forward call.  All device FP64.  The basis
   and its gradient are recomputed per batch (nothing is kept from the
   forward call).  FP64 contexts compute everything in FP64.  Split-BF16
   (and plain BF16) contexts use the density's tensor-core tiles: G is
   gathered per batch in full, E = G Phi is contracted on tcgen05 with the
   context's split, dv_dev = w . sum_j phi_j E_j in double-float, and dR_dev
   from E (kept in FP32) and FP32 basis gradients on CUDA cores; dR_dev is
   summed with FP64 atomics (not bitwise reproducible).  Errors against the
   FP64 oracle: max |d dv| / max |dv| <= 1e-7 and max |d dR| / max |dR| <= 1e-6
   on the tested workloads (split).  The reading of the method behind the
   adjoint (grid points, weights and v held fixed while atoms move, "a
   Pulay-force-like term") is the one the forward integration fixes; the
   paper prints no formula for it. */
int fgi_adjoint(fgi_ctx *ctx, const double *g_dev, const double *v_dev, double *dv_dev,
                double *dR_dev, void *ws, size_t ws_bytes, void *stream);

/* The grid's atom-centred structure, for fgi_hartree: owner[n_pts] (host,
   int32) the atom whose grid each point came from (global atom index, in the
   point's own system; -1 for a point of no atom grid), shell[n_pts] its
   radial shell on that grid, and per atom (host, n_atoms entries) the radial
   grid r_k = r_min[a] exp(k ln_q[a]), k = 0 .. n_rad[a]-1 (n_rad >= 4).  The point weights
   given to fgi_set_grid are then read as (partition weight) x r_k^3 ln q x
   (angular weight).  Call after fgi_set_grid; fgi_set_systems or
   fgi_set_grid discard it.  Copies the tables to the device (a setup call:
   it allocates).  FGI_ERR_ARG for an owner outside the point's system or a
   shell beyond its grid. */
int fgi_set_atom_grids(fgi_ctx *ctx, const int32_t *owner, const int32_t *shell, const double *r_min,
                       const double *ln_q, const int32_t *n_rad);

/* Bytes of device scratch fgi_hartree needs (any l_max). */
int fgi_hartree_workspace_size(fgi_ctx *ctx, size_t *bytes);

/* The step upstream of the integration: the Hartree potential of the density
   on the grid, vh_dev[p] = int n(r') / |r_p - r'| dr' (Hartree, Bohr), by the
   multipole method of Becke & Dickson (J. Chem. Phys. 89, 2993 (1988)) and
   Delley (J. Chem. Phys. 92, 508 (1990)) -- the electrostatic potential that
   the paper's Fig. 4 caption lists as not yet accelerated on GPUs:
     1. rho_a,lm(r_k) = sum over the points of atom a's shell k of
        w_p / (r_k^3 ln q) n_p Y_lm (the partitioned angular quadrature);
     2. per (a, l, m) the radial Poisson equation,
        V(r) = 4 pi/(2l+1) [r^-(l+1) int_0^r rho r'^(l+2) dr' + r^l int_r^inf rho r'^(1-l) dr'],
        the partial integrals in ln r interval by interval by the integral
        of the cubic through the four nearest shells (plus rho(r_0)
        r_0^(l+3)/(l+3) inside the first shell);
     3. vh(r) = sum over the atoms of the point's system and l <= l_max of
        V_a,lm(|r - R_a|) Y_lm, with V between shells by 4-point Lagrange
        interpolation in the fractional shell index, 4 pi/(2l+1) Q_lm /
        d^(l+1) beyond the last shell, V(r_0) (d/r_0)^l inside the first.
   n_dev, vh_dev: device [n_pts] FP64 in the caller's point order;
   0 <= l_max <= 6 (FGI_ERR_UNSUPPORTED otherwise).  Moments and the radial
   solve in FP64; the evaluation (every (point, atom) pair of a system) takes
   the l = 0 terms as double-floats (~1e-12 relative; FP64 interpolation for
   radial grids with ln q > 0.6) and the l >= 1 terms in FP32 (a few FP32
   roundings of the l >= 1 part).  The moments are summed with FP64 atomics:
   not bitwise reproducible.  Needs a plan and fgi_set_atom_grids;
   ws: device, 256-byte aligned, at least fgi_hartree_workspace_size bytes
   (FGI_ERR_WORKSPACE otherwise).  Enqueued on stream, no allocation, no host
   synchronisation (graph-capturable). */
int fgi_hartree(fgi_ctx *ctx, const double *n_dev, double *vh_dev, int l_max, void *ws, size_t ws_bytes,
                void *stream);

/* out_dev[s] = sum_ij A_ij B_ij over system s's full symmetric matrices
   stored as upper triangles a_dev, b_dev (device [nnz] FP64): tr(DS) with
   A = D, B = S, or the band energy with B = H.  FP64. */
int fgi_trace(fgi_ctx *ctx, const double *a_dev, const double *b_dev, double *out_dev,
              void *stream);

/* Wait for the stream and read the device status word: FGI_OK,
   FGI_ERR_TIMEOUT or FGI_ERR_NONFINITE (the word is cleared after reading). */
int fgi_sync(fgi_ctx *ctx, void *stream);

/* Kernel classes for the launch profile. */
enum {
    FGI_KERNEL_BASIS = 0,     /* basis evaluation (and operand images) */
    FGI_KERNEL_H = 1,         /* H contraction + sparse scatter */
    FGI_KERNEL_DENSITY = 2,   /* density contraction */
    FGI_KERNEL_ADJOINT = 3,   /* adjoint position gradient */
    FGI_KERNEL_OTHER = 4      /* reductions and traces */
};

/* Failure-path self-test: enqueues one small kernel whose bounded wait on
   a barrier that nothing completes runs out after about 2 s, as the
   pipelined kernels' waits do when a stage never arrives.  The device status
   word records the time-out; the next fgi_sync reports FGI_ERR_TIMEOUT and
   clears it, and the context stays usable.  No fault and no hang: for
   testing error handling.  Needs a planned context.  The paper has no
   counterpart (it describes no kernels). */
int fgi_selftest_wait_timeout(fgi_ctx *ctx, void *stream);

/* Launch profile: enable = 1 clears the record and starts timing every
   launch of the library's kernels with CUDA events on the call's stream;
   enable = 0 stops.  Not for use inside stream capture. */
int fgi_profile(fgi_ctx *ctx, int enable);

/* Totals over the recorded launches of one kernel class: number of kernel
   launches, summed event time (ms), and the algorithmic FLOPs and bytes
   those launches had to process (per batch, with P points and n active
   functions: H P n (n+1) for the upper triangle; density P n (n+1) + 2 P n
   on the tensor-core paths, which use the upper block triangle of the
   symmetric D, and 2 P n^2 + 2 P n on the FP64 path; scatter 16 bytes per
   stored upper entry).  Waits for the recorded events. */
int fgi_profile_read(fgi_ctx *ctx, int kind, int64_t *launches, double *ms, double *flops,
                     double *bytes);

#ifdef __cplusplus
}
#endif
#endif /* FGI_H */
