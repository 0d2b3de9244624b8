// FP64 CUDA-core path: basis evaluation, H contraction + sparse scatter,
// density contraction, adjoint gradient, and the small reductions.
//
// This path computes every step in FP64.  It is the accuracy reference on
// the GPU and the comparator for the tensor-core path (GB300's FP64 rate is
// far below its BF16 tensor rate).
#include "fgi_basis.cuh"
#include "fgi_index.cuh"
#include "fgi_internal.h"

namespace fgi {

namespace {

// ---------------------------------------------------------------- basis (FP64)
// ws block of batch b: Phi[nfn][kpad], zero for padded points.
__global__ void k_phi_f64(DevPlan P, int b0, double *ws)
{
    const DevBatch B = P.batches[b0 + blockIdx.x];
    double *out = ws + B.ws_off;
    const int total = B.n_act * B.kpad;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int e = idx / B.kpad;
        const int p = idx - e * B.kpad;
        const DevAct A = P.act[B.act0 + e];
        const DevSpecies S = P.species[P.atom_species[A.atom]];
        double *col = out + (long long)A.fn_loc * B.kpad + p;
        if (p >= B.np) {
            for (int f = 0; f < S.n_fn; f++) col[(long long)f * B.kpad] = 0.0;
            continue;
        }
        const long long g = B.pt0 + p;
        const double x = P.px[g] - P.atom_xyz[3 * A.atom + 0];
        const double y = P.py[g] - P.atom_xyz[3 * A.atom + 1];
        const double z = P.pz[g] - P.atom_xyz[3 * A.atom + 2];
        const double d = sqrt(x * x + y * y + z * z);
        const double inv = d > 1e-12 ? 1.0 / d : 0.0;
        const double nx = x * inv, ny = y * inv, nz = z * inv;
        int f = 0;
        for (int sh = 0; sh < S.n_shell; sh++) {
            const DevRadial R = P.radials[P.shell_rad[S.shell0 + sh]];
            const double ud = radial_over_d_f64(R, P.coef, d);
            double Y[7];
            ylm_unit<double>(R.l, nx, ny, nz, Y);
            for (int m = 0; m < 2 * R.l + 1; m++, f++) col[(long long)f * B.kpad] = ud * Y[m];
        }
    }
}

// ------------------------------------------------------- H contraction (FP64)
// One 64x64 tile (ti <= tj) of h_b = Phi_b diag(w v) Phi_b^T, then FP64
// atomic scatter of the upper triangle into the stored values.
constexpr int TF = 64;     // tile edge
constexpr int TK = 16;     // points per step

__global__ void __launch_bounds__(256) k_h_f64(DevPlan P, const WorkItem *items, const double *ws,
                                               const double *v, double *h)
{
    const WorkItem it = items[blockIdx.x];
    const DevBatch B = P.batches[it.batch];
    const double *phi = ws + B.ws_off;
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int i0 = it.ti * TF, j0 = it.tj * TF;
    __shared__ double As[TK][TF + 1];
    __shared__ double Bs[TK][TF + 1];
    __shared__ double wv[TK];
    __shared__ FnRef rowref[TF], colref[TF];
    const DevAct *act = P.act + B.act0;
    if (t < TF && i0 + t < B.nfn) rowref[t] = fn_ref(P, act, find_act(act, B.n_act, i0 + t), i0 + t);
    if (t >= TF && t < 2 * TF && j0 + t - TF < B.nfn)
        colref[t - TF] = fn_ref(P, act, find_act(act, B.n_act, j0 + t - TF), j0 + t - TF);

    double acc[4][4] = {};
    for (int k0 = 0; k0 < B.np; k0 += TK) {
        if (t < TK) {
            const int k = k0 + t;
            double wvk = 0.0;
            if (k < B.np) {
                const double vv = v[B.pt0 + k];
                if (!isfinite(vv)) atomicOr(P.status, kStatusNonFinite);
                wvk = P.pw[B.pt0 + k] * vv;
            }
            wv[t] = wvk;
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const int idx = t + 256 * e;
            const int r = idx >> 4, kk = idx & 15;
            const int k = k0 + kk;
            const bool kin = k < B.kpad;
            As[kk][r] = (i0 + r < B.nfn && kin) ? phi[(long long)(i0 + r) * B.kpad + k] * wv[kk] : 0.0;
            Bs[kk][r] = (j0 + r < B.nfn && kin) ? phi[(long long)(j0 + r) * B.kpad + k] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; kk++) {
            double a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; q++) { a[q] = As[kk][ty * 4 + q]; b[q] = Bs[kk][tx * 4 + q]; }
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const int il = ty * 4 + r;
        if (i0 + il >= B.nfn) continue;
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int jl = tx * 4 + c;
            if (j0 + jl >= B.nfn || i0 + il > j0 + jl) continue;
            const long long k = value_index(P, B.sys, rowref[il], colref[jl]);
            if (k >= 0) atomicAdd(h + k, acc[r][c]);
        }
    }
}

// ------------------------------------------------------------ density (FP64)
// One 64-point tile of batch b: n_p = sum_j (sum_i phi_i(p) D_ij) phi_j(p),
// D gathered from the stored upper triangle (off-diagonal values scaled by
// offdiag_scale: 1 for a matrix, 1/2 for a gradient with respect to stored
// values).  Optionally writes E[j][p] = sum_i phi_i(p) D_ij (adjoint).
__global__ void __launch_bounds__(256) k_density_f64(DevPlan P, const WorkItem *items,
                                                     const double *ws, const double *dval,
                                                     double offdiag_scale, double *n_out,
                                                     double *e_out)
{
    const WorkItem it = items[blockIdx.x];
    const DevBatch B = P.batches[it.batch];
    const double *phi = ws + B.ws_off;
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int p0 = it.ti * TF;
    extern __shared__ unsigned short fnact[];          // local function -> active entry
    __shared__ double As[TK][TF + 1];                  // phi[i][p]
    __shared__ double Bs[TK][TF + 1];                  // D[i][j]
    const DevAct *act = P.act + B.act0;
    for (int l = t; l < B.nfn; l += 256) fnact[l] = (unsigned short)find_act(act, B.n_act, l);
    __syncthreads();

    double part[4] = {0, 0, 0, 0};
    for (int j0 = 0; j0 < B.nfn; j0 += TF) {
        double acc[4][4] = {};
        for (int k0 = 0; k0 < B.nfn; k0 += TK) {
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int idx = t + 256 * e;
                const int kk = idx >> 6, c = idx & 63;
                const int i = k0 + kk;
                As[kk][c] = (i < B.nfn && p0 + c < B.kpad) ? phi[(long long)i * B.kpad + p0 + c] : 0.0;
                const int j = j0 + c;
                double dv = 0.0;
                if (i < B.nfn && j < B.nfn) {
                    const int lo = i < j ? i : j, hi = i < j ? j : i;
                    const FnRef a = fn_ref(P, act, fnact[lo], lo);
                    const FnRef b = fn_ref(P, act, fnact[hi], hi);
                    const long long k = value_index(P, B.sys, a, b);
                    if (k >= 0) dv = dval[k] * (lo == hi ? 1.0 : offdiag_scale);
                }
                Bs[kk][c] = dv;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < TK; kk++) {
                double a[4], b[4];
#pragma unroll
                for (int q = 0; q < 4; q++) { a[q] = As[kk][ty * 4 + q]; b[q] = Bs[kk][tx * 4 + q]; }
#pragma unroll
                for (int r = 0; r < 4; r++)
#pragma unroll
                    for (int c = 0; c < 4; c++) acc[r][c] = fma(a[r], b[c], acc[r][c]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int p = p0 + ty * 4 + r;
            if (p >= B.np) continue;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const int j = j0 + tx * 4 + c;
                if (j >= B.nfn) continue;
                part[r] = fma(acc[r][c], phi[(long long)j * B.kpad + p], part[r]);
                if (e_out) e_out[B.ws_off + (long long)j * B.kpad + p] = acc[r][c];
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 4; r++) {
        double s = part[r];
        for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        part[r] = s;
    }
    if (tx == 0) {
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int p = p0 + ty * 4 + r;
            if (p < B.np) n_out[B.pt0 + p] = part[r];
        }
    }
}

// -------------------------------------------------- adjoint position gradient
// dR[a] += -2 sum_p w_p v_p sum_{i on a} grad phi_i(r_p) . E[i][p]
__global__ void k_adjoint_grad(DevPlan P, int b0, const double *e_ws, const double *v, double *dR)
{
    const DevBatch B = P.batches[b0 + blockIdx.x];
    const double *E = e_ws + B.ws_off;
    const int total = B.n_act * B.kpad;              // kpad is a multiple of 32
    for (int idx0 = 0; idx0 < total; idx0 += blockDim.x) {
        const int idx = idx0 + threadIdx.x;
        double gx = 0.0, gy = 0.0, gz = 0.0;
        int atom = -1;
        if (idx < total) {
            const int e = idx / B.kpad;
            const int p = idx - e * B.kpad;
            const DevAct A = P.act[B.act0 + e];
            atom = A.atom;
            if (p < B.np) {
                const long long g = B.pt0 + p;
                const double x = P.px[g] - P.atom_xyz[3 * A.atom + 0];
                const double y = P.py[g] - P.atom_xyz[3 * A.atom + 1];
                const double z = P.pz[g] - P.atom_xyz[3 * A.atom + 2];
                const double d = sqrt(x * x + y * y + z * z);
                const DevSpecies S = P.species[P.atom_species[A.atom]];
                const double pref = -2.0 * P.pw[g] * v[g];
                if (d > 1e-12 && pref != 0.0) {
                    const double inv = 1.0 / d;
                    const double nx = x * inv, ny = y * inv, nz = z * inv;
                    int f = 0;
                    for (int sh = 0; sh < S.n_shell; sh++) {
                        const DevRadial R = P.radials[P.shell_rad[S.shell0 + sh]];
                        double du;
                        const double ud = radial_over_d_f64(R, P.coef, d, &du);
                        const int nm = 2 * R.l + 1;
                        if (ud == 0.0 && du == 0.0) { f += nm; continue; }
                        double Y[7], G[7][3];
                        ylm_unit<double>(R.l, nx, ny, nz, Y);
                        ylm_poly_grad<double>(R.l, nx, ny, nz, G);
                        // grad phi = n Y (u' - (l+1) u/d)/d + (u/d^2) grad P(n)
                        const double radial = (du - (R.l + 1) * ud) * inv;
                        const double tang = ud * inv;
                        for (int m = 0; m < nm; m++, f++) {
                            const double ev = E[(long long)(A.fn_loc + f) * B.kpad + p];
                            const double a = radial * Y[m];
                            gx = fma(ev, a * nx + tang * G[m][0], gx);
                            gy = fma(ev, a * ny + tang * G[m][1], gy);
                            gz = fma(ev, a * nz + tang * G[m][2], gz);
                        }
                    }
                    gx *= pref; gy *= pref; gz *= pref;
                }
            }
        }
        // a warp covers 32 consecutive points of one atom (kpad % 32 == 0)
        for (int o = 16; o > 0; o >>= 1) {
            gx += __shfl_xor_sync(0xffffffffu, gx, o);
            gy += __shfl_xor_sync(0xffffffffu, gy, o);
            gz += __shfl_xor_sync(0xffffffffu, gz, o);
        }
        if ((threadIdx.x & 31) == 0 && atom >= 0) {
            atomicAdd(dR + 3 * atom + 0, gx);
            atomicAdd(dR + 3 * atom + 1, gy);
            atomicAdd(dR + 3 * atom + 2, gz);
        }
    }
}

// ------------------------------------------------------------- small kernels
__global__ void k_scale_by_weight(DevPlan P, long long n, double *x)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        x[i] *= P.pw[i];
}

__global__ void k_point_traces(DevPlan P, int n_batch, const double *n, double *traces)
{
    for (int b = blockIdx.x; b < n_batch; b += gridDim.x) {
        const DevBatch B = P.batches[b];
        double s = 0.0;
        for (int p = threadIdx.x; p < B.np; p += blockDim.x) s += P.pw[B.pt0 + p] * n[B.pt0 + p];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        __shared__ double red[32];
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x < 32) {
            s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (threadIdx.x == 0) atomicAdd(traces + B.sys, s);
        }
        __syncthreads();
    }
}

// out[s] = 2 sum_k a_k b_k - sum_diag a b  (full symmetric product from upper storage)
__global__ void k_matrix_trace(int n_sys, const long long *sys_val0, const long long *sys_fn0,
                               const long long *rowptr, long long nnz, long long n_fn,
                               const int *fn_sys, const double *a, const double *b, double *out)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    // values: contiguous chunk per thread so the system changes rarely
    const long long chunk = (nnz + stride - 1) / stride;
    long long k0 = tid * chunk, k1 = k0 + chunk < nnz ? k0 + chunk : nnz;
    if (k0 < k1) {
        int lo = 0, hi = n_sys - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (sys_val0[mid] <= k0) lo = mid; else hi = mid - 1;
        }
        int s = lo;
        double acc = 0.0;
        for (long long k = k0; k < k1; k++) {
            while (s + 1 < n_sys && sys_val0[s + 1] <= k) {
                atomicAdd(out + s, 2.0 * acc);
                acc = 0.0;
                s++;
            }
            acc = fma(a[k], b[k], acc);
        }
        atomicAdd(out + s, 2.0 * acc);
    }
    for (long long i = tid; i < n_fn; i += stride) {
        const long long k = rowptr[i];
        atomicAdd(out + fn_sys[i], -a[k] * b[k]);
    }
}

__global__ void k_check_finite(DevPlan P, const double *x, long long n)
{
    bool bad = false;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        bad |= !isfinite(x[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(P.status, kStatusNonFinite);
}

}  // namespace

cudaError_t launch_phi_f64(const DevPlan &P, int b0, int nb, double *ws, cudaStream_t s)
{
    if (nb <= 0) return cudaSuccess;
    k_phi_f64<<<nb, 256, 0, s>>>(P, b0, ws);
    return cudaGetLastError();
}

cudaError_t launch_h_f64(const DevPlan &P, const WorkItem *items, int n_items, const double *ws,
                         const double *v, double *h, cudaStream_t s)
{
    if (n_items <= 0) return cudaSuccess;
    k_h_f64<<<n_items, 256, 0, s>>>(P, items, ws, v, h);
    return cudaGetLastError();
}

cudaError_t launch_density_f64(const DevPlan &P, const WorkItem *items, int n_items,
                               const double *ws, const double *d, double offdiag_scale,
                               double *n_out, double *e_out, cudaStream_t s)
{
    if (n_items <= 0) return cudaSuccess;
    k_density_f64<<<n_items, 256, kMaxBatchFns * sizeof(unsigned short), s>>>(
        P, items, ws, d, offdiag_scale, n_out, e_out);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_grad(const DevPlan &P, int b0, int nb, const double *e_ws,
                                const double *v, double *dR, cudaStream_t s)
{
    if (nb <= 0) return cudaSuccess;
    k_adjoint_grad<<<nb, 256, 0, s>>>(P, b0, e_ws, v, dR);
    return cudaGetLastError();
}

cudaError_t launch_scale_by_weight(const DevPlan &P, long long n_pts, double *x, cudaStream_t s)
{
    if (n_pts <= 0) return cudaSuccess;
    k_scale_by_weight<<<1216, 256, 0, s>>>(P, n_pts, x);
    return cudaGetLastError();
}

cudaError_t launch_point_traces(const DevPlan &P, int n_batch, const double *n, double *traces,
                                cudaStream_t s)
{
    if (n_batch <= 0) return cudaSuccess;
    k_point_traces<<<n_batch < 4864 ? n_batch : 4864, 256, 0, s>>>(P, n_batch, n, traces);
    return cudaGetLastError();
}

cudaError_t launch_matrix_trace(const DevPlan &P, int n_sys, const long long *sys_fn0,
                                const long long *sys_val0, long long n_fn_total,
                                long long nnz_total, const int *fn_sys, const double *a,
                                const double *b, double *out, cudaStream_t s)
{
    (void)sys_fn0;
    k_matrix_trace<<<1216, 256, 0, s>>>(n_sys, sys_val0, sys_fn0, P.rowptr, nnz_total, n_fn_total,
                                        fn_sys, a, b, out);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const DevPlan &P, const double *x, long long n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_check_finite<<<1216, 256, 0, s>>>(P, x, n);
    return cudaGetLastError();
}

}  // namespace fgi
