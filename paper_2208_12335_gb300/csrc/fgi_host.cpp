// Host runtime of the C ABI: input tables, the plan (active functions per
// batch, sparsity pattern, tile work lists, waves), device storage, and the
// call sequences of the compute entry points.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "fgi_bounds.h"
#include "fgi_hartree.h"
#include "fgi_ylm.cuh"
#include "fgi_internal.h"
#include "fgi_tc.h"
#include "../../include/fgi.h"

using namespace fgi;

namespace {

struct RadialH {
    int l;
    double h;
    int nk;
    std::vector<double> coef;
};

struct SpeciesH {
    double Z;
    std::vector<int> shells;
    int n_fn;
    double rcut;
};

struct ProfRec {
    int kind;
    cudaEvent_t a, b;
    double flops, bytes;
    int kernels;                 // kernel launches inside the timed scope
};

struct Wave {
    double phi_flops = 0, phi_bytes = 0, h_flops = 0, h_bytes = 0, n_flops = 0, n_bytes = 0;
    int b0 = 0, nb = 0;            // batch range
    long long it0 = 0, nit = 0;    // items range (H tiles, FP64)
    long long dt0 = 0, ndt = 0;    // items range (density tiles, FP64)
    size_t ws_elems = 0;           // FP64 elements of the Phi block
};

// Allocator whose value-less construct leaves the element uninitialised, so
// that resize() of a large buffer does not zero it on one thread before a
// parallel loop fills it (the fill is then also the pages' first touch).
template <typename T>
struct NoInitAlloc : std::allocator<T> {
    template <typename U>
    struct rebind {
        using other = NoInitAlloc<U>;
    };
    NoInitAlloc() = default;
    template <typename U>
    NoInitAlloc(const NoInitAlloc<U> &) noexcept {}
    template <typename U>
    void construct(U *p) noexcept
    {
        ::new ((void *)p) U;
    }
    template <typename U, typename... A>
    void construct(U *p, A &&...a)
    {
        ::new ((void *)p) U(std::forward<A>(a)...);
    }
};

template <typename T>
using BigVec = std::vector<T, NoInitAlloc<T>>;

// dst[0..n) = src[0..n), in parallel chunks
template <typename T>
void par_copy(T *dst, const T *src, int64_t n)
{
    const int64_t chunk = 1 << 16;
#pragma omp parallel for schedule(static)
    for (int64_t c0 = 0; c0 < n; c0 += chunk)
        std::memcpy(dst + c0, src + c0, sizeof(T) * (size_t)std::min(chunk, n - c0));
}

}  // namespace

struct fgi_ctx {
    int device = 0;
    std::string err;
    std::vector<RadialH> radials;
    std::vector<SpeciesH> species;
    // systems
    int n_sys = 0;
    std::vector<int64_t> atom_off;
    std::vector<int> atom_species;
    std::vector<double> atom_xyz;
    bool have_systems = false;
    // grid
    int64_t n_pts = 0;
    BigVec<double> pts, w;
    std::vector<int64_t> batch_off;
    std::vector<int> batch_sys;
    bool have_grid = false;
    // plan
    bool planned = false;
    fgi_precision precision = FGI_FP64;
    int64_t n_fn = 0, nnz = 0;
    std::vector<long long> atom_fn0;
    std::vector<int> atom_loc, atom_nfn, atom_sys;
    std::vector<int64_t> sys_fn0, sys_nfn, sys_val0, sys_nnz;
    std::vector<long long> rowptr;            // global value index per global function
    std::vector<int> fn_sys;
    std::vector<int> pairpos;
    std::vector<long long> sys_pair_off;
    std::vector<std::vector<int>> nbr;        // per atom: neighbour atoms b >= a (global)
    std::vector<DevBatch> batches_f64;
    std::vector<DevAct> act;
    std::vector<Wave> waves;
    std::vector<WorkItem> items;
    size_t ws_f64_bytes = 0;
    // pattern cache for fgi_get_pattern
    int pattern_sys = -1;
    std::vector<int64_t> pat_rowptr;
    std::vector<int> pat_col;
    // device
    char *d_arena = nullptr;
    size_t arena_bytes = 0;
    DevPlan dp{};
    DevBatch *d_batches_f64 = nullptr;
    WorkItem *d_items = nullptr;
    long long *d_sys_val0 = nullptr, *d_sys_fn0 = nullptr, *d_sys_nnz = nullptr;
    int *d_fn_sys = nullptr;
    int *d_status = nullptr;
    TcPlan tc;                                // tensor-core plan of the H integration (the batches as given)
    TcPlan tcd;                               // tensor-core plan of the density (super-batches)
    TcPlan tca;                               // the density's super-batches with room for E (the adjoint)
    // atom-centred structure of the grid (the Hartree potential)
    bool have_atom_grids = false;
    std::vector<int> hg_owner, hg_shell, hg_nrad;
    std::vector<double> hg_rmin, hg_lnq;
    char *d_hartree = nullptr;
    HartreeDev hd{};
    // per-kernel CUDA-event profile
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<ProfRec> recs;
    long long prof_dropped = 0;
};

namespace {

int set_err(fgi_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

#define CUDA_TRY(c, expr)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return set_err(c, FGI_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_));       \
    } while (0)

void free_atom_grids(fgi_ctx *c)
{
    if (c->d_hartree) cudaFree(c->d_hartree);
    c->d_hartree = nullptr;
    c->hd = HartreeDev{};
    c->have_atom_grids = false;
}

void free_device(fgi_ctx *c)
{
    if (c->d_arena) cudaFree(c->d_arena);
    c->d_arena = nullptr;
    c->arena_bytes = 0;
    tc_free(c->tc);
    tc_free(c->tcd);
    tc_free(c->tca);
    c->planned = false;
}

void invalidate(fgi_ctx *c)
{
    c->planned = false;
    c->pattern_sys = -1;
    c->pat_rowptr.clear();
    c->pat_col.clear();
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

void wave_work(fgi_ctx *c);

// Two tensor-core plans: H keeps the batches as given (its split accuracy
// depends on the points per contraction), the density merges neighbouring
// batches into super-batches of up to 1024 points (its accuracy does not).
// Tuned settings: a text file of "key value" lines (the autotuner writes it):
//   density_sb_points  super-batch point limit of the density path (0: none, <= 1024)
//   density_sb_growth  limit on a super-batch's functions / its largest member's
//   wave_mb            operand-image workspace per wave, MiB
//   h_sb_points        super-batch point limit of the H path (0: none, <= 1024)
//   h_sb_growth        the H path's limit on the union's functions / largest member's
//   bound_grids        leading-digit grids of the split images from table
//                      bounds of |phi| instead of a pass over the points:
//                      0 none, 1 the density images, 2 also the H images
// Unknown keys are ignored; a malformed value is an argument error.
struct TuneSettings {
    int sb_points = 1024;
    double sb_growth = 1.35;
    // operand images per wave: 8 GiB.  The persistent contraction kernels
    // walk a wave's tile list with a fixed stride, so CTAs drift apart over
    // a long wave and the tiles in flight outgrow L2; shorter waves re-align
    // them (1000-atom step: density 163.8 -> 155.0 ms, step 593.1 -> 588.5 ms
    // against 24 GiB waves) until the extra launches cost more (3 GiB: 603 ms)
    long long wave_mb = 8192;
    // merges neighbouring batches (fewer tiles and scatter atomics); 512
    // points keep the FP32 accumulation of the remainder products (one
    // truncation per 16-point MMA step) within the H tolerance
    int h_sb_points = 512;
    double h_sb_growth = 1.25;
    int bound_grids = 2;        // table-bound digit grids for the H and density images
};

int read_tune_file(const char *path, TuneSettings &t, std::string *err)
{
    FILE *f = fopen(path, "r");
    if (!f) return FGI_OK;      // no file yet: the defaults
    char key[64];
    double val;
    int rc = FGI_OK;
    while (true) {
        const int n = fscanf(f, "%63s %lf", key, &val);
        if (n == EOF) break;
        if (n != 2) {
            *err = std::string("tune file ") + path + ": expected 'key value' lines";
            rc = FGI_ERR_ARG;
            break;
        }
        const std::string k(key);
        if (k == "density_sb_points") {
            if (!(val >= 0 && val <= kMaxBatchPoints)) {
                *err = "tune file: density_sb_points out of range";
                rc = FGI_ERR_ARG;
                break;
            }
            t.sb_points = (int)val;
        } else if (k == "density_sb_growth") {
            if (!(val >= 1.0 && val <= 16.0)) {
                *err = "tune file: density_sb_growth out of range";
                rc = FGI_ERR_ARG;
                break;
            }
            t.sb_growth = val;
        } else if (k == "h_sb_points") {
            if (!(val >= 0 && val <= kMaxBatchPoints)) {
                *err = "tune file: h_sb_points out of range";
                rc = FGI_ERR_ARG;
                break;
            }
            t.h_sb_points = (int)val;
        } else if (k == "h_sb_growth") {
            if (!(val >= 1.0 && val <= 16.0)) {
                *err = "tune file: h_sb_growth out of range";
                rc = FGI_ERR_ARG;
                break;
            }
            t.h_sb_growth = val;
        } else if (k == "wave_mb") {
            if (!(val >= 1.0)) {
                *err = "tune file: wave_mb out of range";
                rc = FGI_ERR_ARG;
                break;
            }
            t.wave_mb = (long long)val;
        } else if (k == "bound_grids") {
            if (!(val == 0.0 || val == 1.0 || val == 2.0)) {
                *err = "tune file: bound_grids must be 0, 1 or 2";
                rc = FGI_ERR_ARG;
                break;
            }
            t.bound_grids = (int)val;
        }
    }
    fclose(f);
    return rc;
}

int build_tc_plans(fgi_ctx *c, TcPlanInput tin, std::string *err)
{
    TuneSettings ts;
    if (tin.tune_path) {
        const int rc = read_tune_file(tin.tune_path, ts, err);
        if (rc != FGI_OK) return rc;
    }
    // environment overrides for experiments
    if (const char *e = getenv("FGI_SB_POINTS")) ts.sb_points = atoi(e);
    if (const char *e = getenv("FGI_SB_GROWTH")) ts.sb_growth = atof(e);
    if (const char *e = getenv("FGI_H_SB_POINTS")) ts.h_sb_points = atoi(e);
    if (const char *e = getenv("FGI_H_SB_GROWTH")) ts.h_sb_growth = atof(e);
    if (const char *e = getenv("FGI_BOUND_GRIDS")) ts.bound_grids = std::min(std::max(atoi(e), 0), 2);
    tin.wave_mb = ts.wave_mb;
    // the table bounds need u(0) = 0 for every radial (u(r)/r bounded at 0)
    bool bounded = true;
    for (const RadialH &r : c->radials) bounded = bounded && !r.coef.empty() && r.coef[0] == 0.0;
    tin.bound_grids = bounded ? ts.bound_grids : 0;
    tin.sb_points = ts.h_sb_points;
    tin.sb_growth = ts.h_sb_growth;
    int rc = tc_build(c->tc, tin, err);
    if (rc != FGI_OK) return rc;
    tin.sb_points = ts.sb_points;
    tin.sb_growth = ts.sb_growth;
    rc = tc_build(c->tcd, tin, err);
    if (rc != FGI_OK) return rc;
    tin.with_e = true;                   // the adjoint: the density's tiles plus room for E = G Phi
    return tc_build(c->tca, tin, err);
}

// ------------------------------------------------------------ plan building
int build_plan(fgi_ctx *c, const char *tune_path)
{
    const int n_at = (int)c->atom_species.size();
    // atoms
    c->atom_fn0.assign(n_at, 0);
    c->atom_loc.assign(n_at, 0);
    c->atom_nfn.assign(n_at, 0);
    c->atom_sys.assign(n_at, 0);
    c->sys_fn0.assign(c->n_sys, 0);
    c->sys_nfn.assign(c->n_sys, 0);
    long long fn = 0;
    for (int s = 0; s < c->n_sys; s++) {
        c->sys_fn0[s] = fn;
        for (int64_t a = c->atom_off[s]; a < c->atom_off[s + 1]; a++) {
            c->atom_fn0[a] = fn;
            c->atom_loc[a] = (int)(a - c->atom_off[s]);
            c->atom_nfn[a] = c->species[c->atom_species[a]].n_fn;
            c->atom_sys[a] = s;
            fn += c->atom_nfn[a];
        }
        c->sys_nfn[s] = fn - c->sys_fn0[s];
    }
    c->n_fn = fn;
    // pattern: neighbour lists, row pointers, pair positions
    c->nbr.assign(n_at, {});
    c->rowptr.assign(c->n_fn, 0);
    c->fn_sys.assign(c->n_fn, 0);
    c->sys_val0.assign(c->n_sys, 0);
    c->sys_nnz.assign(c->n_sys, 0);
    c->sys_pair_off.assign(c->n_sys, 0);
    long long pair_total = 0;
    for (int s = 0; s < c->n_sys; s++) {
        long long nat = c->atom_off[s + 1] - c->atom_off[s];
        c->sys_pair_off[s] = pair_total;
        pair_total += nat * nat;
    }
    c->pairpos.assign(pair_total, -1);
    long long cursor = 0;
    for (int s = 0; s < c->n_sys; s++) {
        c->sys_val0[s] = cursor;
        const int64_t a0 = c->atom_off[s], a1 = c->atom_off[s + 1];
        const long long nat = a1 - a0;
        for (int64_t a = a0; a < a1; a++) {
            const double ra = c->species[c->atom_species[a]].rcut;
            const double *xa = &c->atom_xyz[3 * a];
            long long pos = 0;
            for (int64_t b = a; b < a1; b++) {
                const double rb = c->species[c->atom_species[b]].rcut;
                const double *xb = &c->atom_xyz[3 * b];
                const double dx = xa[0] - xb[0], dy = xa[1] - xb[1], dz = xa[2] - xb[2];
                if (b == a || std::sqrt(dx * dx + dy * dy + dz * dz) < ra + rb) {
                    c->nbr[a].push_back((int)b);
                    c->pairpos[c->sys_pair_off[s] + (a - a0) * nat + (b - a0)] = (int)pos;
                    pos += c->atom_nfn[b];
                }
            }
            const long long RL = pos;
            for (int li = 0; li < c->atom_nfn[a]; li++) {
                c->rowptr[c->atom_fn0[a] + li] = cursor;
                c->fn_sys[c->atom_fn0[a] + li] = s;
                cursor += RL - li;
            }
        }
        c->sys_nnz[s] = cursor - c->sys_val0[s];
    }
    c->nnz = cursor;
    if (c->nnz > (long long)1 << 40) return set_err(c, FGI_ERR_UNSUPPORTED, "pattern too large");

    // active atoms per batch
    const int64_t nb = (int64_t)c->batch_sys.size();
    std::vector<std::vector<int>> active(nb);
    int too_many = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(max : too_many)
    for (int64_t b = 0; b < nb; b++) {
        const int64_t p0 = c->batch_off[b], p1 = c->batch_off[b + 1];
        if (p1 == p0) continue;   // an empty batch has no active atoms
        const int s = c->batch_sys[b];
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int64_t p = p0; p < p1; p++)
            for (int k = 0; k < 3; k++) {
                lo[k] = std::min(lo[k], c->pts[3 * p + k]);
                hi[k] = std::max(hi[k], c->pts[3 * p + k]);
            }
        double cen[3], rad2 = 0.0;
        for (int k = 0; k < 3; k++) cen[k] = 0.5 * (lo[k] + hi[k]);
        for (int64_t p = p0; p < p1; p++) {
            double d2 = 0.0;
            for (int k = 0; k < 3; k++) d2 += (c->pts[3 * p + k] - cen[k]) * (c->pts[3 * p + k] - cen[k]);
            rad2 = std::max(rad2, d2);
        }
        const double rad = std::sqrt(rad2);
        int nfn_b = 0;
        for (int64_t a = c->atom_off[s]; a < c->atom_off[s + 1]; a++) {
            const double rc = c->species[c->atom_species[a]].rcut;
            const double *xa = &c->atom_xyz[3 * a];
            double dc = 0.0;
            for (int k = 0; k < 3; k++) dc += (xa[k] - cen[k]) * (xa[k] - cen[k]);
            dc = std::sqrt(dc);
            if (dc >= rad + rc) continue;
            bool on = dc + rad < rc;
            for (int64_t p = p0; p < p1 && !on; p++) {
                double d2 = 0.0;
                for (int k = 0; k < 3; k++) d2 += (c->pts[3 * p + k] - xa[k]) * (c->pts[3 * p + k] - xa[k]);
                on = d2 < rc * rc;
            }
            if (on) {
                active[b].push_back((int)a);
                nfn_b += c->atom_nfn[a];
            }
        }
        if (nfn_b > kMaxBatchFns) too_many = 1;
    }
    if (too_many)
        return set_err(c, FGI_ERR_UNSUPPORTED, "a batch has more than %d active functions; use smaller batches",
                       kMaxBatchFns);

    // batches, active entries, FP64 waves and work items
    c->act.clear();
    {
        size_t n_act = 0;
        for (int64_t b = 0; b < nb; b++) n_act += active[b].size();
        c->act.reserve(n_act);
    }
    c->batches_f64.assign(nb, DevBatch{});
    for (int64_t b = 0; b < nb; b++) {
        DevBatch &B = c->batches_f64[b];
        B.pt0 = c->batch_off[b];
        B.np = (int)(c->batch_off[b + 1] - c->batch_off[b]);
        B.sys = c->batch_sys[b];
        B.act0 = (int)c->act.size();
        B.n_act = (int)active[b].size();
        int fl = 0;
        for (int a : active[b]) {
            c->act.push_back(DevAct{a, fl});
            fl += c->atom_nfn[a];
        }
        B.nfn = fl;
        B.kpad = (B.np + 31) / 32 * 32;
    }
    const size_t wave_cap = (size_t)1 << 27;   // FP64 elements (1 GiB) of Phi per wave
    c->waves.clear();
    c->items.clear();
    {
        Wave wv;
        size_t off = 0;
        for (int64_t b = 0; b < nb; b++) {
            DevBatch &B = c->batches_f64[b];
            const size_t need = (size_t)B.nfn * B.kpad;
            if (wv.nb > 0 && off + need > wave_cap) {
                wv.ws_elems = off;
                c->waves.push_back(wv);
                wv = Wave{};
                wv.b0 = (int)b;
                off = 0;
            }
            if (wv.nb == 0) wv.b0 = (int)b;
            B.ws_off = (long long)off;
            off += align_up(need, 32);
            wv.nb++;
        }
        if (wv.nb > 0) {
            wv.ws_elems = off;
            c->waves.push_back(wv);
        }
        size_t max_elems = 0;
        size_t n_items = 0;
        for (int64_t b = 0; b < nb; b++) {
            const long long nt = (c->batches_f64[b].nfn + 63) / 64;
            n_items += (size_t)(nt * (nt + 1) / 2);
            if (c->batches_f64[b].nfn > 0) n_items += (size_t)((c->batches_f64[b].np + 63) / 64);
        }
        c->items.reserve(n_items);
        for (Wave &w : c->waves) {
            w.it0 = (long long)c->items.size();
            for (int b = w.b0; b < w.b0 + w.nb; b++) {
                const int nt = (c->batches_f64[b].nfn + 63) / 64;
                for (int i = 0; i < nt; i++)
                    for (int j = i; j < nt; j++) c->items.push_back(WorkItem{b, (short)i, (short)j});
            }
            w.nit = (long long)c->items.size() - w.it0;
            w.dt0 = (long long)c->items.size();
            for (int b = w.b0; b < w.b0 + w.nb; b++) {
                if (c->batches_f64[b].nfn == 0) continue;
                const int nt = (c->batches_f64[b].np + 63) / 64;
                for (int i = 0; i < nt; i++) c->items.push_back(WorkItem{b, (short)i, 0});
            }
            w.ndt = (long long)c->items.size() - w.dt0;
            max_elems = std::max(max_elems, w.ws_elems);
        }
        c->ws_f64_bytes = 2 * max_elems * sizeof(double) + 256;   // Phi + E (adjoint)
    }
    wave_work(c);

    // ---- device arena
    free_device(c);
    if (c->device < 0) {
        TcPlanInput tin;
        tin.n_batch = (int)nb;
        tin.batches = c->batches_f64.data();
        tin.act = c->act.data();
        tin.atom_nfn = c->atom_nfn.data();
        tin.tune_path = tune_path;
        tin.nnz = c->nnz;
        tin.n_fn = c->n_fn;
        tin.host_only = true;
        std::string terr;
        int rc = build_tc_plans(c, tin, &terr);
        if (rc != FGI_OK) return set_err(c, rc, "%s", terr.c_str());
        c->planned = true;
        return FGI_OK;
    }
    std::vector<DevRadial> drad;
    std::vector<double> coef;
    for (const RadialH &r : c->radials) {
        DevRadial d;
        d.h = r.h;
        d.inv_h = 1.0 / r.h;
        d.rcut = r.h * (r.nk - 1);
        d.coef_off = (long long)(coef.size() / 4);
        d.nk = r.nk;
        d.l = r.l;
        d.inv_h_hi = (float)d.inv_h;
        d.inv_h_lo = (float)(d.inv_h - (double)d.inv_h_hi);
        d.rcut_f = (float)d.rcut;
        d.pad = 0;
        d.bound_off = 0;
        coef.insert(coef.end(), r.coef.begin(), r.coef.end());
        drad.push_back(d);
    }
    // bounds of |phi|: max |Y_lm|, then per radial the suffix bounds of |u(r)/r|
    std::vector<float> rbound(kYlmMaxEntries);
    ylm_abs_max(rbound.data());
    for (size_t i = 0; i < c->radials.size(); i++) {
        const RadialH &r = c->radials[i];
        drad[i].bound_off = (long long)rbound.size();
        rbound.resize(rbound.size() + (size_t)(r.nk - 1));
        radial_over_r_bounds(r.coef.data(), r.nk - 1, r.h, rbound.data() + drad[i].bound_off);
    }
    // coefficients as double-floats: per interval (hi0..hi3), (lo0..lo3)
    std::vector<float> coef_dd(coef.size() * 2);
    for (size_t k = 0; k < coef.size() / 4; k++)
        for (int q = 0; q < 4; q++) {
            const float hi = (float)coef[4 * k + q];
            coef_dd[8 * k + q] = hi;
            coef_dd[8 * k + 4 + q] = (float)(coef[4 * k + q] - (double)hi);
        }
    // the same with every coefficient times the first normalisation constant
    // of the radial's l (real harmonics, no Condon-Shortley phase): the
    // lane-per-point basis kernels evaluate C_l u(r) directly
    static const double kFirstYlmC[4] = {0.28209479177387814,   // 1/(2 sqrt pi)
                                         0.4886025119029199,    // sqrt(3/(4 pi))
                                         1.0925484305920792,    // (1/2) sqrt(15/pi), xy
                                         0.5900435899266435};   // (1/4) sqrt(35/(2 pi)), y(3x^2 - y^2)
    std::vector<float> coef_ddn(coef.size() * 2);
    for (size_t i = 0; i < c->radials.size(); i++) {
        const double cl = kFirstYlmC[std::min(std::max(c->radials[i].l, 0), 3)];
        for (long long k = drad[i].coef_off; k < drad[i].coef_off + (long long)(c->radials[i].coef.size() / 4); k++)
            for (int q = 0; q < 4; q++) {
                const double v = coef[4 * k + q] * cl;
                const float hi = (float)v;
                coef_ddn[8 * k + q] = hi;
                coef_ddn[8 * k + 4 + q] = (float)(v - (double)hi);
            }
    }
    // coordinates as double-floats: per point (x_hi, x_lo, y_hi, y_lo, z_hi, z_lo)
    auto to_dd = [](const double *xyz, int64_t n) {
        BigVec<float> out(6 * (size_t)n);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++)
            for (int k = 0; k < 3; k++) {
                const float hi = (float)xyz[3 * i + k];
                out[6 * i + 2 * k] = hi;
                out[6 * i + 2 * k + 1] = (float)(xyz[3 * i + k] - (double)hi);
            }
        return out;
    };
    BigVec<float> pts_dd = to_dd(c->pts.data(), c->n_pts);
    BigVec<float> atom_dd = to_dd(c->atom_xyz.data(), (int64_t)(c->atom_xyz.size() / 3));
    std::vector<DevSpecies> dsp;
    std::vector<int> shell_rad;
    // species whose shells share one knot grid also get their coefficients
    // interleaved by interval, so that one point's shells read neighbouring
    // cache lines
    std::vector<float> scoef, scoefn;
    std::vector<int> shell_fn0, shell_by_l;     // per species slot: first function, radial (grouped by l)
    for (const SpeciesH &s : c->species) {
        DevSpecies d{};
        d.shell0 = (int)shell_rad.size();
        d.n_shell = (int)s.shells.size();
        d.n_fn = s.n_fn;
        d.rcut = s.rcut;
        bool shared = !s.shells.empty();
        for (int sh : s.shells)
            shared = shared && c->radials[sh].h == c->radials[s.shells[0]].h &&
                     c->radials[sh].nk == c->radials[s.shells[0]].nk;
        d.shared_grid = shared ? 1 : 0;
        // the shells grouped by l (stable), with each one's first function
        std::vector<int> first(s.shells.size()), lord;
        {
            int fn = 0;
            for (size_t i = 0; i < s.shells.size(); i++) {
                first[i] = fn;
                fn += 2 * c->radials[s.shells[i]].l + 1;
            }
            for (int l = 0; l <= 3; l++)
                for (size_t i = 0; i < s.shells.size(); i++)
                    if (c->radials[s.shells[i]].l == l) {
                        lord.push_back((int)i);
                        d.nl[l]++;
                    }
        }
        if (shared) {
            const RadialH &r0 = c->radials[s.shells[0]];
            d.nk = r0.nk;
            d.inv_h_hi = (float)(1.0 / r0.h);
            d.inv_h_lo = (float)(1.0 / r0.h - (double)d.inv_h_hi);
            d.scoef_off = (long long)(scoef.size() / 4);
            for (int k = 0; k < r0.nk - 1; k++)
                for (int sh : s.shells) {
                    const size_t src = 8 * ((size_t)drad[sh].coef_off + k);
                    scoef.insert(scoef.end(), coef_dd.begin() + src, coef_dd.begin() + src + 8);
                }
            for (int k = 0; k < r0.nk - 1; k++)
                for (int i : lord) {
                    const size_t src = 8 * ((size_t)drad[s.shells[i]].coef_off + k);
                    scoefn.insert(scoefn.end(), coef_ddn.begin() + src, coef_ddn.begin() + src + 8);
                }
        }
        shell_rad.insert(shell_rad.end(), s.shells.begin(), s.shells.end());
        for (int i : lord) {
            shell_fn0.push_back(first[i]);
            shell_by_l.push_back(s.shells[i]);
        }
        d.lmax = 0;
        for (int sh : s.shells) d.lmax = std::max(d.lmax, c->radials[sh].l);
        dsp.push_back(d);
    }
    std::vector<DevShell> dshell;
    for (size_t i = 0; i < shell_by_l.size(); i++) {
        const DevRadial &R = drad[shell_by_l[i]];
        DevShell q{};
        q.coef_off = (int)R.coef_off;
        q.nk = R.nk;
        q.l = R.l;
        q.rcut_f = R.rcut_f;
        q.inv_h_hi = R.inv_h_hi;
        q.inv_h_lo = R.inv_h_lo;
        q.bound_off = (int)R.bound_off;
        q.fn0 = shell_fn0[i];
        dshell.push_back(q);
    }
    if (scoef.empty()) scoef.assign(8, 0.f);
    if (scoefn.empty()) scoefn.assign(8, 0.f);
    BigVec<double> px(c->n_pts), py(c->n_pts), pz(c->n_pts);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < c->n_pts; p++) {
        px[p] = c->pts[3 * p];
        py[p] = c->pts[3 * p + 1];
        pz[p] = c->pts[3 * p + 2];
    }
    std::vector<int> sys_nat(c->n_sys);
    for (int s = 0; s < c->n_sys; s++) sys_nat[s] = (int)(c->atom_off[s + 1] - c->atom_off[s]);
    std::vector<long long> sys_val0(c->sys_val0.begin(), c->sys_val0.end());
    std::vector<long long> sys_fn0(c->sys_fn0.begin(), c->sys_fn0.end());
    std::vector<long long> sys_nnz(c->sys_nnz.begin(), c->sys_nnz.end());
    // global column function of every stored value (-1 on the diagonal)
    std::vector<int> col_glob((size_t)c->nnz);
    for (int s = 0; s < c->n_sys; s++)
        for (int64_t a = c->atom_off[s]; a < c->atom_off[s + 1]; a++)
            for (int li = 0; li < c->atom_nfn[a]; li++) {
                const long long gi = c->atom_fn0[a] + li;
                long long k = c->rowptr[gi];
                for (long long j = gi; j < c->atom_fn0[a] + c->atom_nfn[a]; j++) col_glob[k++] = j == gi ? -1 : (int)j;
                for (int b : c->nbr[a]) {
                    if (b == a) continue;
                    for (int lj = 0; lj < c->atom_nfn[b]; lj++) col_glob[k++] = (int)(c->atom_fn0[b] + lj);
                }
            }

    struct Blob {
        const void *src;
        size_t bytes;
        size_t off;
    };
    std::vector<Blob> blobs;
    size_t total = 0;
    auto add = [&](const void *src, size_t bytes) {
        Blob b{src, bytes, total};
        total = align_up(total + std::max<size_t>(bytes, 1), 256);
        blobs.push_back(b);
        return blobs.size() - 1;
    };
    size_t i_px = add(px.data(), px.size() * 8), i_py = add(py.data(), py.size() * 8),
           i_pz = add(pz.data(), pz.size() * 8), i_pw = add(c->w.data(), c->w.size() * 8),
           i_axyz = add(c->atom_xyz.data(), c->atom_xyz.size() * 8),
           i_asp = add(c->atom_species.data(), c->atom_species.size() * 4),
           i_afn0 = add(c->atom_fn0.data(), c->atom_fn0.size() * 8),
           i_aloc = add(c->atom_loc.data(), c->atom_loc.size() * 4),
           i_sp = add(dsp.data(), dsp.size() * sizeof(DevSpecies)),
           i_shr = add(shell_rad.data(), shell_rad.size() * 4),
           i_dsh = add(dshell.data(), dshell.size() * sizeof(DevShell)),
           i_rad = add(drad.data(), drad.size() * sizeof(DevRadial)),
           i_coef = add(coef.data(), coef.size() * 8), i_coefdd = add(coef_dd.data(), coef_dd.size() * 4),
           i_scoef = add(scoef.data(), scoef.size() * 4),
           i_coefddn = add(coef_ddn.data(), coef_ddn.size() * 4), i_scoefn = add(scoefn.data(), scoefn.size() * 4),
           i_ptsdd = add(pts_dd.data(), pts_dd.size() * 4), i_atdd = add(atom_dd.data(), atom_dd.size() * 4),
           i_snat = add(sys_nat.data(), sys_nat.size() * 4),
           i_spo = add(c->sys_pair_off.data(), c->sys_pair_off.size() * 8),
           i_pp = add(c->pairpos.data(), c->pairpos.size() * 4),
           i_rp = add(c->rowptr.data(), c->rowptr.size() * 8),
           i_bf = add(c->batches_f64.data(), c->batches_f64.size() * sizeof(DevBatch)),
           i_act = add(c->act.data(), c->act.size() * sizeof(DevAct)),
           i_items = add(c->items.data(), c->items.size() * sizeof(WorkItem)),
           i_sv0 = add(sys_val0.data(), sys_val0.size() * 8), i_sf0 = add(sys_fn0.data(), sys_fn0.size() * 8),
           i_fsys = add(c->fn_sys.data(), c->fn_sys.size() * 4), i_status = add(nullptr, 64),
           i_snnz = add(sys_nnz.data(), sys_nnz.size() * 8), i_colg = add(col_glob.data(), col_glob.size() * 4),
           i_rbnd = add(rbound.data(), rbound.size() * 4);
    cudaError_t e = cudaMalloc((void **)&c->d_arena, total);
    if (e != cudaSuccess) {
        c->d_arena = nullptr;
        return set_err(c, FGI_ERR_NOMEM, "plan: cudaMalloc(%zu) failed: %s", total, cudaGetErrorString(e));
    }
    c->arena_bytes = total;
    for (const Blob &b : blobs) {
        if (b.src && b.bytes) CUDA_TRY(c, cudaMemcpy(c->d_arena + b.off, b.src, b.bytes, cudaMemcpyHostToDevice));
    }
    CUDA_TRY(c, cudaMemset(c->d_arena + blobs[i_status].off, 0, 64));
    auto at = [&](size_t i) { return (void *)(c->d_arena + blobs[i].off); };
    DevPlan &P = c->dp;
    P.px = (const double *)at(i_px);
    P.py = (const double *)at(i_py);
    P.pz = (const double *)at(i_pz);
    P.pw = (const double *)at(i_pw);
    P.atom_xyz = (const double *)at(i_axyz);
    P.atom_species = (const int *)at(i_asp);
    P.atom_fn0 = (const long long *)at(i_afn0);
    P.atom_loc = (const int *)at(i_aloc);
    P.species = (const DevSpecies *)at(i_sp);
    P.shell_rad = (const int *)at(i_shr);
    P.shells = (const DevShell *)at(i_dsh);
    P.n_shells = (int)shell_rad.size();
    P.radials = (const DevRadial *)at(i_rad);
    P.coef = (const double *)at(i_coef);
    P.coef_dd = (const float4 *)at(i_coefdd);
    P.scoef = (const float4 *)at(i_scoef);
    P.coef_ddn = (const float4 *)at(i_coefddn);
    P.scoefn = (const float4 *)at(i_scoefn);
    P.pts_dd = (const float *)at(i_ptsdd);
    P.atom_dd = (const float *)at(i_atdd);
    P.sys_nat = (const int *)at(i_snat);
    P.sys_pair_off = (const long long *)at(i_spo);
    P.pairpos = (const int *)at(i_pp);
    P.rowptr = (const long long *)at(i_rp);
    P.batches = (const DevBatch *)at(i_bf);
    P.act = (const DevAct *)at(i_act);
    P.status = (int *)at(i_status);
    c->d_batches_f64 = (DevBatch *)at(i_bf);
    c->d_items = (WorkItem *)at(i_items);
    c->d_sys_val0 = (long long *)at(i_sv0);
    c->d_sys_fn0 = (long long *)at(i_sf0);
    c->d_fn_sys = (int *)at(i_fsys);
    c->d_sys_nnz = (long long *)at(i_snnz);
    P.col_glob = (const int *)at(i_colg);
    P.rbound = (const float *)at(i_rbnd);
    c->d_status = (int *)at(i_status);

    // tensor-core path plan (operand images, tiles, waves)
    TcPlanInput tin;
    tin.n_batch = (int)nb;
    tin.batches = c->batches_f64.data();
    tin.act = c->act.data();
    tin.atom_nfn = c->atom_nfn.data();
    tin.tune_path = tune_path;
    tin.nnz = c->nnz;
    tin.n_fn = c->n_fn;
    std::string terr;
    int rc = build_tc_plans(c, tin, &terr);
    if (rc != FGI_OK) return set_err(c, rc, "%s", terr.c_str());
    c->planned = true;
    return FGI_OK;
}

int check_ready(fgi_ctx *c)
{
    if (!c) return FGI_ERR_ARG;
    if (!c->planned) return set_err(c, FGI_ERR_STATE, "call fgi_plan first");
    return FGI_OK;
}

int check_compute(fgi_ctx *c)
{
    int rc = check_ready(c);
    if (rc) return rc;
    if (c->device < 0) return set_err(c, FGI_ERR_STATE, "host-only context (device -1) cannot compute");
    return FGI_OK;
}

size_t workspace_need(fgi_ctx *c)
{
    return std::max(std::max(c->ws_f64_bytes, tc_workspace_bytes(c->tca)),
                    std::max(tc_workspace_bytes(c->tc), tc_workspace_bytes(c->tcd)));
}

int check_ws(fgi_ctx *c, void *ws, size_t bytes)
{
    if (!ws || ((uintptr_t)ws & 255)) return set_err(c, FGI_ERR_WORKSPACE, "workspace NULL or not 256-byte aligned");
    if (bytes < workspace_need(c))
        return set_err(c, FGI_ERR_WORKSPACE, "workspace of %zu bytes, need %zu", bytes, workspace_need(c));
    return FGI_OK;
}

// Launch-profiling scope: events around one launch on the call's stream.
bool known_precision(int p)
{
    return p == FGI_FP64 || p == FGI_SPLIT_BF16 || p == FGI_BF16;
}

// BF16 terms per operand value on the tensor-core paths: 3 (split BF16, 8
// products) or 1 (plain BF16)
int split_terms(int p) { return p == FGI_SPLIT_BF16 ? 3 : 1; }

struct ProfScope {
    fgi_ctx *c;
    cudaStream_t s;
    int kind;
    double flops, bytes;
    cudaEvent_t a = nullptr, b = nullptr;
    int kernels;
    ProfScope(fgi_ctx *c_, cudaStream_t s_, int kind_, double f, double by, int kernels_ = 1)
        : c(c_), s(s_), kind(kind_), flops(f), bytes(by), kernels(kernels_)
    {
        if (!c->prof_on) return;
        while (c->ev_used + 2 > c->ev_pool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) {
                c->prof_dropped++;
                return;
            }
            c->ev_pool.push_back(e);
        }
        a = c->ev_pool[c->ev_used++];
        b = c->ev_pool[c->ev_used++];
        cudaEventRecord(a, s);
    }
    ~ProfScope()
    {
        if (!a) return;
        cudaEventRecord(b, s);
        c->recs.push_back(ProfRec{kind, a, b, flops, bytes, kernels});
    }
};

void wave_work(fgi_ctx *c)
{
    for (Wave &w : c->waves) {
        for (int b = w.b0; b < w.b0 + w.nb; b++) {
            const DevBatch &B = c->batches_f64[b];
            const double P = B.np, n = B.nfn;
            w.phi_flops += 30.0 * P * n;
            w.phi_bytes += 32.0 * P + 8.0 * P * n;
            w.h_flops += P * n * (n + 1.0);          // upper triangle incl. diagonal
            w.h_bytes += 16.0 * n * (n + 1) / 2 + 16.0 * P;
            w.n_flops += 2.0 * P * n * n + 2.0 * P * n;
            w.n_bytes += 8.0 * n * n + 16.0 * P;
        }
    }
}

}  // namespace

// ========================================================= internal entry points
namespace fgi {

int internal_device(const fgi_ctx *c) { return c ? c->device : -1; }

int internal_error(fgi_ctx *c, int code, const char *msg)
{
    if (c) c->err = msg;
    return code;
}

int internal_integrate_h(fgi_ctx *c, const double *v, double *h, int accumulate, void *ws, size_t ws_bytes,
                         void *stream, bool allow_profile)
{
    struct ProfMute {
        fgi_ctx *c;
        bool saved;
        ProfMute(fgi_ctx *c_, bool allow) : c(c_), saved(c_ ? c_->prof_on : false)
        {
            if (c && !allow) c->prof_on = false;
        }
        ~ProfMute()
        {
            if (c) c->prof_on = saved;
        }
    } mute(c, allow_profile);
    int rc = check_compute(c);
    if (rc) return rc;
    if (!v || !h) return set_err(c, FGI_ERR_ARG, "v or h is NULL");
    if ((rc = check_ws(c, ws, ws_bytes))) return rc;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (c->precision == FGI_FP64) {
        if (!accumulate) CUDA_TRY(c, cudaMemsetAsync(h, 0, (size_t)c->nnz * sizeof(double), s));
        DevPlan P = c->dp;
        P.batches = c->d_batches_f64;
        for (const Wave &w : c->waves) {
            {
                ProfScope ps(c, s, 0, w.phi_flops, w.phi_bytes);
                CUDA_TRY(c, launch_phi_f64(P, w.b0, w.nb, (double *)ws, s));
            }
            ProfScope ps(c, s, 1, w.h_flops, w.h_bytes);
            CUDA_TRY(c, launch_h_f64(P, c->d_items + w.it0, (int)w.nit, (const double *)ws, v, h, s));
        }
        return FGI_OK;
    }
    const int n_split = split_terms(c->precision);
    DevPlan P = c->dp;
    P.batches = c->tc.d_sb;
    P.act = c->tc.d_sact;
    CUDA_TRY(c, cudaMemsetAsync(ws, 0, (size_t)c->nnz * 8, s));       // fixed-point accumulator
    for (const TcWave &w : c->tc.waves) {
        {
            ProfScope ps(c, s, 0, w.phi_flops, w.phi_bytes);
            CUDA_TRY(c, tc_launch_phi(c->tc, P, w, v, ws, n_split, s));
        }
        ProfScope ps(c, s, 1, w.h_flops, w.h_bytes);
        CUDA_TRY(c, tc_launch_h(c->tc, P, w, ws, n_split, s));
    }
    {
        ProfScope ps(c, s, 4, 2.0 * c->nnz, 24.0 * c->nnz);
        CUDA_TRY(c, tc_launch_fix_to_h(c->tc, ws, h, c->nnz, accumulate, s));
    }
    return FGI_OK;
}


}  // namespace fgi

// ================================================================== the ABI
extern "C" {

int fgi_create(fgi_ctx **out, int cuda_device)
{
    if (!out) return FGI_ERR_ARG;
    *out = nullptr;
    if (cuda_device == -1) {            // host-only context: inputs and plan tables, no compute
        fgi_ctx *c = new (std::nothrow) fgi_ctx();
        if (!c) return FGI_ERR_NOMEM;
        c->device = -1;
        *out = c;
        return FGI_OK;
    }
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) return FGI_ERR_CUDA;   // no driver or no device
    if (cuda_device < 0 || cuda_device >= n) return FGI_ERR_ARG;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, cuda_device) != cudaSuccess) return FGI_ERR_CUDA;
    if (!(prop.major == 10 && prop.minor == 3)) return FGI_ERR_UNSUPPORTED;
    fgi_ctx *c = new (std::nothrow) fgi_ctx();
    if (!c) return FGI_ERR_NOMEM;
    c->device = cuda_device;
    *out = c;
    return FGI_OK;
}

int fgi_destroy(fgi_ctx *c)
{
    if (!c) return FGI_OK;
    if (c->device >= 0) {
        DeviceGuard g(c->device);
        free_device(c);
        free_atom_grids(c);
        for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    }
    delete c;
    return FGI_OK;
}

const char *fgi_last_error(const fgi_ctx *c) { return c ? c->err.c_str() : "null context"; }

int fgi_add_radial(fgi_ctx *c, int l, double h, int n_knots, const double *coef, int *id_out)
{
    if (!c) return FGI_ERR_ARG;
    if (l < 0 || l > kMaxL) return set_err(c, FGI_ERR_UNSUPPORTED, "l = %d; 0 <= l <= %d supported", l, kMaxL);
    if (!(h > 0.0) || !std::isfinite(h) || n_knots < 2 || !coef)
        return set_err(c, FGI_ERR_ARG, "radial: need h > 0, n_knots >= 2, coef");
    RadialH r;
    r.l = l;
    r.h = h;
    r.nk = n_knots;
    r.coef.assign(coef, coef + 4 * (size_t)(n_knots - 1));
    for (double x : r.coef)
        if (!std::isfinite(x)) return set_err(c, FGI_ERR_NONFINITE, "radial coefficients not finite");
    c->radials.push_back(std::move(r));
    if (id_out) *id_out = (int)c->radials.size() - 1;
    invalidate(c);
    return FGI_OK;
}

int fgi_add_species(fgi_ctx *c, double Z, int n_shell, const int *radial_id, int *id_out)
{
    if (!c) return FGI_ERR_ARG;
    if (n_shell < 1 || !radial_id) return set_err(c, FGI_ERR_ARG, "species: need n_shell >= 1");
    SpeciesH s;
    s.Z = Z;
    s.n_fn = 0;
    s.rcut = 0.0;
    for (int k = 0; k < n_shell; k++) {
        int r = radial_id[k];
        if (r < 0 || r >= (int)c->radials.size()) return set_err(c, FGI_ERR_ARG, "species: bad radial id %d", r);
        s.shells.push_back(r);
        s.n_fn += 2 * c->radials[r].l + 1;
        s.rcut = std::max(s.rcut, c->radials[r].h * (c->radials[r].nk - 1));
    }
    c->species.push_back(std::move(s));
    if (id_out) *id_out = (int)c->species.size() - 1;
    invalidate(c);
    return FGI_OK;
}

int fgi_set_systems(fgi_ctx *c, int n_sys, const int64_t *atom_off, const int *species,
                    const double *xyz)
{
    if (!c) return FGI_ERR_ARG;
    if (n_sys < 1 || !atom_off || atom_off[0] != 0) return set_err(c, FGI_ERR_ARG, "systems: bad atom_off");
    for (int s = 0; s < n_sys; s++)
        if (atom_off[s + 1] < atom_off[s]) return set_err(c, FGI_ERR_ARG, "systems: atom_off not ascending");
    const int64_t na = atom_off[n_sys];
    if (na > 0 && (!species || !xyz)) return set_err(c, FGI_ERR_ARG, "systems: NULL arrays");
    for (int64_t a = 0; a < na; a++) {
        if (species[a] < 0 || species[a] >= (int)c->species.size())
            return set_err(c, FGI_ERR_ARG, "systems: bad species id at atom %lld", (long long)a);
        for (int k = 0; k < 3; k++)
            if (!std::isfinite(xyz[3 * a + k])) return set_err(c, FGI_ERR_NONFINITE, "systems: xyz not finite");
    }
    c->n_sys = n_sys;
    c->atom_off.assign(atom_off, atom_off + n_sys + 1);
    c->atom_species.assign(species, species + na);
    c->atom_xyz.assign(xyz, xyz + 3 * na);
    c->have_systems = true;
    invalidate(c);
    if (c->have_atom_grids) {
        DeviceGuard g(c->device >= 0 ? c->device : 0);
        free_atom_grids(c);
    }
    return FGI_OK;
}

int fgi_set_grid(fgi_ctx *c, int64_t n_pts, const double *xyz, const double *w, int64_t n_batch,
                 const int64_t *batch_off, const int *batch_sys)
{
    if (!c) return FGI_ERR_ARG;
    if (n_pts < 0 || n_batch < 0 || (n_pts > 0 && (!xyz || !w)) || !batch_off || (n_batch > 0 && !batch_sys))
        return set_err(c, FGI_ERR_ARG, "grid: bad arguments");
    if (batch_off[0] != 0 || batch_off[n_batch] != n_pts) return set_err(c, FGI_ERR_ARG, "grid: batch_off must span [0, n_pts]");
    for (int64_t b = 0; b < n_batch; b++) {
        const int64_t np = batch_off[b + 1] - batch_off[b];
        if (np < 0 || np > kMaxBatchPoints)
            return set_err(c, FGI_ERR_ARG, "grid: batch %lld has %lld points (0..%d allowed)", (long long)b,
                           (long long)np, kMaxBatchPoints);
        if (batch_sys[b] < 0) return set_err(c, FGI_ERR_ARG, "grid: bad batch_sys");
    }
    int64_t first_bad = n_pts;   // the lowest index of a non-finite point
#pragma omp parallel for schedule(static) reduction(min : first_bad)
    for (int64_t p = 0; p < n_pts; p++)
        if (!std::isfinite(w[p]) || !std::isfinite(xyz[3 * p]) || !std::isfinite(xyz[3 * p + 1]) ||
            !std::isfinite(xyz[3 * p + 2]))
            first_bad = std::min(first_bad, p);
    if (first_bad < n_pts)
        return set_err(c, FGI_ERR_NONFINITE, "grid: point %lld not finite", (long long)first_bad);
    c->n_pts = n_pts;
    c->pts.resize(3 * (size_t)n_pts);
    c->w.resize((size_t)n_pts);
    par_copy(c->pts.data(), xyz, 3 * n_pts);
    par_copy(c->w.data(), w, n_pts);
    c->batch_off.assign(batch_off, batch_off + n_batch + 1);
    c->batch_sys.assign(batch_sys, batch_sys + n_batch);
    c->have_grid = true;
    invalidate(c);
    if (c->have_atom_grids) {
        DeviceGuard g(c->device >= 0 ? c->device : 0);
        free_atom_grids(c);
    }
    return FGI_OK;
}

int fgi_plan(fgi_ctx *c, fgi_precision precision, const char *tune_cache_path)
{
    if (!c) return FGI_ERR_ARG;
    if (!c->have_systems || !c->have_grid) return set_err(c, FGI_ERR_STATE, "set systems and grid before fgi_plan");
    if (!known_precision(precision))
        return set_err(c, FGI_ERR_ARG, "unknown precision %d", (int)precision);
    for (int b : c->batch_sys)
        if (b >= c->n_sys) return set_err(c, FGI_ERR_ARG, "grid: batch_sys out of range");
    invalidate(c);
    if (c->device < 0) {
        c->precision = precision;
        try {
            return build_plan(c, tune_cache_path);
        } catch (const std::bad_alloc &) {
            return set_err(c, FGI_ERR_NOMEM, "plan: host allocation failed");
        }
    }
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(c, FGI_ERR_CUDA, "cudaSetDevice failed");
    c->precision = precision;
    try {
        return build_plan(c, tune_cache_path);
    } catch (const std::bad_alloc &) {
        return set_err(c, FGI_ERR_NOMEM, "plan: host allocation failed");
    }
}

int fgi_set_precision(fgi_ctx *c, fgi_precision precision)
{
    int rc = check_ready(c);
    if (rc) return rc;
    if (!known_precision(precision))
        return set_err(c, FGI_ERR_ARG, "unknown precision %d", (int)precision);
    c->precision = precision;
    return FGI_OK;
}

int fgi_get_sizes(fgi_ctx *c, int64_t *n_fn, int64_t *nnz, int64_t *n_pts, int64_t *n_atoms)
{
    int rc = check_ready(c);
    if (rc) return rc;
    if (n_fn) *n_fn = c->n_fn;
    if (nnz) *nnz = c->nnz;
    if (n_pts) *n_pts = c->n_pts;
    if (n_atoms) *n_atoms = (int64_t)c->atom_species.size();
    return FGI_OK;
}

int fgi_get_system(fgi_ctx *c, int sys, int64_t *fn0, int64_t *n_fn, int64_t *val0, int64_t *nnz)
{
    int rc = check_ready(c);
    if (rc) return rc;
    if (sys < 0 || sys >= c->n_sys) return set_err(c, FGI_ERR_ARG, "system %d out of range", sys);
    if (fn0) *fn0 = c->sys_fn0[sys];
    if (n_fn) *n_fn = c->sys_nfn[sys];
    if (val0) *val0 = c->sys_val0[sys];
    if (nnz) *nnz = c->sys_nnz[sys];
    return FGI_OK;
}

int fgi_get_batch_work(fgi_ctx *c, int64_t n_batch, int64_t *points, int32_t *n_active_fns)
{
    int rc = check_ready(c);
    if (rc) return rc;
    if (n_batch != (int64_t)c->batches_f64.size())
        return set_err(c, FGI_ERR_ARG, "n_batch %lld differs from the planned %lld batches", (long long)n_batch,
                       (long long)c->batches_f64.size());
    for (int64_t b = 0; b < n_batch; b++) {
        if (points) points[b] = c->batches_f64[b].np;
        if (n_active_fns) n_active_fns[b] = c->batches_f64[b].nfn;
    }
    return FGI_OK;
}

int fgi_get_schedule(fgi_ctx *c, int which, int64_t *n_super, int64_t *n_waves, int64_t *sb_first_batch,
                     int32_t *sb_points, int32_t *sb_fns, int64_t *wave_first_sb, int32_t *sb_rank)
{
    int rc = check_ready(c);
    if (rc) return rc;
    if (which != 0 && which != 1) return set_err(c, FGI_ERR_ARG, "which must be 0 (H) or 1 (density)");
    const TcPlan &t = which == 0 ? c->tc : c->tcd;
    const int64_t ns = (int64_t)t.sb.size(), nw = (int64_t)t.waves.size();
    if (n_super) *n_super = ns;
    if (n_waves) *n_waves = nw;
    for (int64_t s = 0; s < ns; s++) {
        if (sb_points) sb_points[s] = t.sb[s].np;
        if (sb_fns) sb_fns[s] = t.sb[s].nfn;
        if (sb_rank) sb_rank[s] = t.sb_rank[s];
    }
    if (sb_first_batch)
        for (int64_t s = 0; s <= ns; s++) sb_first_batch[s] = t.sb_first[s];
    if (wave_first_sb) {
        for (int64_t k = 0; k < nw; k++) wave_first_sb[k] = t.waves[k].b0;
        wave_first_sb[nw] = ns;
    }
    return FGI_OK;
}

int fgi_get_pattern(fgi_ctx *c, int sys, int64_t *nnz, const int64_t **rowptr, const int **col)
{
    int rc = check_ready(c);
    if (rc) return rc;
    if (sys < 0 || sys >= c->n_sys) return set_err(c, FGI_ERR_ARG, "system %d out of range", sys);
    if (c->pattern_sys != sys) {
        try {
            const int64_t nf = c->sys_nfn[sys], f0 = c->sys_fn0[sys], v0 = c->sys_val0[sys];
            c->pat_rowptr.assign(nf + 1, 0);
            c->pat_col.assign(c->sys_nnz[sys], 0);
            for (int64_t a = c->atom_off[sys]; a < c->atom_off[sys + 1]; a++) {
                for (int li = 0; li < c->atom_nfn[a]; li++) {
                    const long long gi = c->atom_fn0[a] + li;
                    long long k = c->rowptr[gi] - v0;
                    c->pat_rowptr[gi - f0] = k;
                    for (long long j = gi; j < c->atom_fn0[a] + c->atom_nfn[a]; j++) c->pat_col[k++] = (int)(j - f0);
                    for (int b : c->nbr[a]) {
                        if (b == a) continue;
                        for (int lj = 0; lj < c->atom_nfn[b]; lj++) c->pat_col[k++] = (int)(c->atom_fn0[b] + lj - f0);
                    }
                }
            }
            c->pat_rowptr[nf] = c->sys_nnz[sys];
            c->pattern_sys = sys;
        } catch (const std::bad_alloc &) {
            c->pattern_sys = -1;
            return set_err(c, FGI_ERR_NOMEM, "pattern: host allocation failed");
        }
    }
    if (nnz) *nnz = c->sys_nnz[sys];
    if (rowptr) *rowptr = c->pat_rowptr.data();
    if (col) *col = c->pat_col.data();
    return FGI_OK;
}

int fgi_workspace_size(fgi_ctx *c, size_t *bytes)
{
    int rc = check_ready(c);
    if (rc) return rc;
    if (!bytes) return set_err(c, FGI_ERR_ARG, "bytes is NULL");
    *bytes = workspace_need(c);
    return FGI_OK;
}

int fgi_integrate_h(fgi_ctx *c, const double *v, double *h, int accumulate, void *ws, size_t ws_bytes,
                    void *stream)
{
    return fgi::internal_integrate_h(c, v, h, accumulate, ws, ws_bytes, stream, true);
}

int fgi_density(fgi_ctx *c, const double *d, double *n, double *traces, void *ws, size_t ws_bytes,
                void *stream)
{
    int rc = check_compute(c);
    if (rc) return rc;
    if (!d || !n) return set_err(c, FGI_ERR_ARG, "d or n is NULL");
    if ((rc = check_ws(c, ws, ws_bytes))) return rc;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(c, cudaMemsetAsync(n, 0, (size_t)c->n_pts * sizeof(double), s));
    DevPlan P = c->dp;
    P.batches = c->d_batches_f64;
    if (c->precision == FGI_FP64) {
        for (const Wave &w : c->waves) {
            {
                ProfScope ps(c, s, 0, w.phi_flops, w.phi_bytes);
                CUDA_TRY(c, launch_phi_f64(P, w.b0, w.nb, (double *)ws, s));
            }
            ProfScope ps(c, s, 2, w.n_flops, w.n_bytes);
            CUDA_TRY(c, launch_density_f64(P, c->d_items + w.dt0, (int)w.ndt, (const double *)ws, d, 1.0, n,
                                           nullptr, s));
        }
    } else {
        const int n_split = split_terms(c->precision);
        DevPlan Q = c->dp;
        Q.batches = c->tcd.d_sb;
        Q.act = c->tcd.d_sact;
        {
            ProfScope ps(c, s, 4, 0.0, 16.0 * c->nnz, 2);          // conversion of D and its bounds
            CUDA_TRY(c, tc_launch_to_df(c->tcd, Q, d, ws, c->d_sys_val0, c->d_sys_nnz, c->d_fn_sys, s));
        }
        for (const TcWave &w : c->tcd.waves) {
            {
                ProfScope ps(c, s, 0, w.phi_flops, w.phi_bytes);
                CUDA_TRY(c, tc_launch_phi_cols(c->tcd, Q, w, ws, n_split, s));
            }
            {
                ProfScope ps(c, s, 4, 0.0, w.g_bytes);
                CUDA_TRY(c, tc_launch_gather_d(c->tcd, Q, w, 1.0, ws, n_split, s));
            }
            ProfScope ps(c, s, 2, w.n_flops, w.n_bytes, 2);        // contraction + per-block sums
            CUDA_TRY(c, tc_launch_density(c->tcd, Q, w, ws, n, n_split, s));
        }
    }
    if (traces) {
        CUDA_TRY(c, cudaMemsetAsync(traces, 0, (size_t)c->n_sys * sizeof(double), s));
        ProfScope ps(c, s, 4, 2.0 * c->n_pts, 16.0 * c->n_pts);
        CUDA_TRY(c, launch_point_traces(P, (int)c->batch_sys.size(), n, traces, s));
    }
    return FGI_OK;
}

int fgi_adjoint(fgi_ctx *c, const double *gv, const double *v, double *dv, double *dR, void *ws,
                size_t ws_bytes, void *stream)
{
    int rc = check_compute(c);
    if (rc) return rc;
    if (!gv || !v || !dv || !dR) return set_err(c, FGI_ERR_ARG, "NULL argument");
    if ((rc = check_ws(c, ws, ws_bytes))) return rc;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(c, cudaMemsetAsync(dv, 0, (size_t)c->n_pts * sizeof(double), s));
    CUDA_TRY(c, cudaMemsetAsync(dR, 0, c->atom_species.size() * 3 * sizeof(double), s));
    DevPlan P = c->dp;
    P.batches = c->d_batches_f64;
    if (c->precision != FGI_FP64) {
        // tensor-core adjoint on the density's tiles: G gathered in full (its
        // off-diagonal stored values halved), E = G Phi on tcgen05, dv from
        // the contraction's epilogue, dR from E and the basis gradients
        const int n_split = split_terms(c->precision);
        DevPlan Q = c->dp;
        Q.batches = c->tca.d_sb;
        Q.act = c->tca.d_sact;
        {
            ProfScope ps(c, s, 4, 0.0, 16.0 * c->nnz, 2);          // conversion of G and its bounds
            CUDA_TRY(c, tc_launch_to_df(c->tca, Q, gv, ws, c->d_sys_val0, c->d_sys_nnz, c->d_fn_sys, s));
        }
        for (const TcWave &w : c->tca.waves) {
            {
                ProfScope ps(c, s, 0, w.phi_flops, w.phi_bytes);
                CUDA_TRY(c, tc_launch_phi_cols(c->tca, Q, w, ws, n_split, s));
            }
            {
                ProfScope ps(c, s, 4, 0.0, 2.0 * w.g_bytes);
                CUDA_TRY(c, tc_launch_gather_d(c->tca, Q, w, 0.5, ws, n_split, s, true));
            }
            // full G: twice the density's upper-block-triangle work, plus the gradient
            ProfScope ps(c, s, 3, 2.0 * w.n_flops + 40.0 * w.phi_flops / 30.0, w.n_bytes, 3);
            CUDA_TRY(c, tc_launch_adjoint(c->tca, Q, w, ws, v, dv, dR, n_split, s));
        }
        CUDA_TRY(c, launch_scale_by_weight(P, c->n_pts, dv, s));
        return FGI_OK;
    }
    size_t max_elems = 0;
    for (const Wave &w : c->waves) max_elems = std::max(max_elems, w.ws_elems);
    double *phi_ws = (double *)ws;
    double *e_ws = phi_ws + max_elems;
    for (const Wave &w : c->waves) {
        {
            ProfScope ps(c, s, 0, w.phi_flops, w.phi_bytes);
            CUDA_TRY(c, launch_phi_f64(P, w.b0, w.nb, phi_ws, s));
        }
        {
            ProfScope ps(c, s, 2, w.n_flops, w.n_bytes);
            CUDA_TRY(c, launch_density_f64(P, c->d_items + w.dt0, (int)w.ndt, phi_ws, gv, 0.5, dv, e_ws, s));
        }
        ProfScope ps(c, s, 3, 40.0 * w.phi_flops / 30.0, w.phi_bytes);
        CUDA_TRY(c, launch_adjoint_grad(P, w.b0, w.nb, e_ws, v, dR, s));
    }
    CUDA_TRY(c, launch_scale_by_weight(P, c->n_pts, dv, s));
    return FGI_OK;
}

int fgi_set_atom_grids(fgi_ctx *c, const int32_t *owner, const int32_t *shell, const double *r_min,
                       const double *ln_q, const int32_t *n_rad)
{
    if (!c) return FGI_ERR_ARG;
    if (!c->have_systems || !c->have_grid) return set_err(c, FGI_ERR_STATE, "set systems and grid first");
    const int n_at = (int)c->atom_species.size();
    if ((c->n_pts > 0 && (!owner || !shell)) || (n_at > 0 && (!r_min || !ln_q || !n_rad)))
        return set_err(c, FGI_ERR_ARG, "atom grids: NULL argument");
    for (int a = 0; a < n_at; a++)
        if (!(r_min[a] > 0.0) || !(ln_q[a] > 0.0) || !std::isfinite(r_min[a]) || !std::isfinite(ln_q[a]) || n_rad[a] < 4)
            return set_err(c, FGI_ERR_ARG, "atom grids: atom %d needs r_min > 0, ln q > 0, n_rad >= 4", a);
    // every point's owner lies in the point's own system, its shell on the owner's grid
    std::vector<int> pt_sys((size_t)c->n_pts);
    for (size_t b = 0; b + 1 < c->batch_off.size(); b++)
        for (int64_t p = c->batch_off[b]; p < c->batch_off[b + 1]; p++) pt_sys[(size_t)p] = c->batch_sys[b];
    for (int64_t p = 0; p < c->n_pts; p++) {
        const int a = owner[p];
        if (a == -1) continue;
        if (a < 0 || a >= n_at || shell[p] < 0 || shell[p] >= n_rad[a])
            return set_err(c, FGI_ERR_ARG, "atom grids: point %lld has owner %d, shell %d", (long long)p, a,
                           (int)shell[p]);
        if (a < c->atom_off[pt_sys[(size_t)p]] || a >= c->atom_off[pt_sys[(size_t)p] + 1])
            return set_err(c, FGI_ERR_ARG, "atom grids: point %lld belongs to another system than its owner",
                           (long long)p);
    }
    if (c->device >= 0) {
        DeviceGuard g(c->device);
        free_atom_grids(c);
    }
    c->hg_owner.assign(owner, owner + c->n_pts);
    c->hg_shell.assign(shell, shell + c->n_pts);
    c->hg_rmin.assign(r_min, r_min + n_at);
    c->hg_lnq.assign(ln_q, ln_q + n_at);
    c->hg_nrad.assign(n_rad, n_rad + n_at);
    std::vector<long long> rad_off(n_at + 1, 0);
    for (int a = 0; a < n_at; a++) rad_off[a + 1] = rad_off[a] + n_rad[a];
    std::vector<HartreeRad> rgrid(n_at);
    for (int a = 0; a < n_at; a++) rgrid[a] = hartree_rad(r_min[a], ln_q[a], n_rad[a]);
    std::vector<long long> sys_atom0(c->atom_off.begin(), c->atom_off.end());
    c->hd.n_atoms = n_at;
    c->hd.n_shells = rad_off[n_at];
    if (c->device >= 0) {
        DeviceGuard g(c->device);
        const size_t s_own = align_up(4 * (size_t)c->n_pts + 4, 256), s_off = align_up(8 * (size_t)(n_at + 1), 256),
                     s_rg = align_up(sizeof(HartreeRad) * (size_t)(n_at + 1), 256),
                     s_sys = align_up(8 * sys_atom0.size(), 256);
        const size_t tot = 2 * s_own + s_off + s_rg + s_sys;
        CUDA_TRY(c, cudaMalloc((void **)&c->d_hartree, tot));
        char *b = c->d_hartree;
        CUDA_TRY(c, cudaMemcpy(b, owner, 4 * (size_t)c->n_pts, cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(b + s_own, shell, 4 * (size_t)c->n_pts, cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(b + 2 * s_own, rad_off.data(), 8 * rad_off.size(), cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(b + 2 * s_own + s_off, rgrid.data(), sizeof(HartreeRad) * (size_t)n_at,
                               cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(b + 2 * s_own + s_off + s_rg, sys_atom0.data(), 8 * sys_atom0.size(),
                               cudaMemcpyHostToDevice));
        c->hd.owner = (const int *)b;
        c->hd.shell = (const int *)(b + s_own);
        c->hd.rad_off = (const long long *)(b + 2 * s_own);
        c->hd.rad = (const HartreeRad *)(b + 2 * s_own + s_off);
        c->hd.sys_atom0 = (const long long *)(b + 2 * s_own + s_off + s_rg);
    }
    c->have_atom_grids = true;
    return FGI_OK;
}

int fgi_hartree_workspace_size(fgi_ctx *c, size_t *bytes)
{
    if (!c || !bytes) return FGI_ERR_ARG;
    if (!c->have_atom_grids) return set_err(c, FGI_ERR_STATE, "call fgi_set_atom_grids first");
    *bytes = hartree_ws_bytes(c->hd);
    return FGI_OK;
}

int fgi_hartree(fgi_ctx *c, const double *n, double *vh, int l_max, void *ws, size_t ws_bytes, void *stream)
{
    int rc = check_compute(c);
    if (rc) return rc;
    if (!c->have_atom_grids) return set_err(c, FGI_ERR_STATE, "call fgi_set_atom_grids first");
    if (!n || !vh) return set_err(c, FGI_ERR_ARG, "n or vh is NULL");
    if (l_max < 0 || l_max > kHartreeLmax)
        return set_err(c, FGI_ERR_UNSUPPORTED, "l_max = %d; 0 <= l_max <= %d supported", l_max, kHartreeLmax);
    if (!ws || ((uintptr_t)ws & 255)) return set_err(c, FGI_ERR_WORKSPACE, "workspace NULL or not 256-byte aligned");
    if (ws_bytes < hartree_ws_bytes(c->hd))
        return set_err(c, FGI_ERR_WORKSPACE, "workspace of %zu bytes, need %zu", ws_bytes, hartree_ws_bytes(c->hd));
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    DevPlan P = c->dp;
    P.batches = c->d_batches_f64;
    ProfScope ps(c, s, 4, 0.0, 8.0 * (double)c->n_pts, 3);
    CUDA_TRY(c, launch_hartree(P, c->hd, (int)c->batch_sys.size(), c->n_pts, l_max, n, vh, (double *)ws, s));
    return FGI_OK;
}

int fgi_trace(fgi_ctx *c, const double *a, const double *b, double *out, void *stream)
{
    int rc = check_compute(c);
    if (rc) return rc;
    if (!a || !b || !out) return set_err(c, FGI_ERR_ARG, "NULL argument");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(c, cudaMemsetAsync(out, 0, (size_t)c->n_sys * sizeof(double), s));
    if (c->n_fn > 0)
        CUDA_TRY(c, launch_matrix_trace(c->dp, c->n_sys, c->d_sys_fn0, c->d_sys_val0, c->n_fn, c->nnz, c->d_fn_sys,
                                        a, b, out, s));
    return FGI_OK;
}

int fgi_sync(fgi_ctx *c, void *stream)
{
    int rc = check_compute(c);
    if (rc) return rc;
    DeviceGuard g(c->device);
    CUDA_TRY(c, cudaStreamSynchronize((cudaStream_t)stream));
    int st = 0;
    CUDA_TRY(c, cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st) CUDA_TRY(c, cudaMemset(c->d_status, 0, sizeof(int)));
    if (st & kStatusTimeout) return set_err(c, FGI_ERR_TIMEOUT, "a bounded device wait ran out");
    if (st & kStatusNonFinite) return set_err(c, FGI_ERR_NONFINITE, "non-finite value in an input");
    if (st & kStatusBadIndex) return set_err(c, FGI_ERR_CUDA, "device index check failed");
    return FGI_OK;
}

int fgi_selftest_wait_timeout(fgi_ctx *c, void *stream)
{
    int rc = check_compute(c);
    if (rc) return rc;
    DeviceGuard g(c->device);
    CUDA_TRY(c, tc_launch_wait_selftest(c->d_status, (cudaStream_t)stream));
    return FGI_OK;
}

int fgi_profile(fgi_ctx *c, int enable)
{
    int rc = check_compute(c);
    if (rc) return rc;
    DeviceGuard g(c->device);
    if (enable) {
        while (c->ev_pool.size() < 1024) {
            cudaEvent_t e;
            CUDA_TRY(c, cudaEventCreate(&e));
            c->ev_pool.push_back(e);
        }
    }
    c->prof_on = enable != 0;
    c->ev_used = 0;
    c->recs.clear();
    c->prof_dropped = 0;
    return FGI_OK;
}

int fgi_profile_read(fgi_ctx *c, int kind, int64_t *launches, double *ms, double *flops, double *bytes)
{
    int rc = check_compute(c);
    if (rc) return rc;
    if (kind < 0 || kind > 4) return set_err(c, FGI_ERR_ARG, "kernel kind %d out of range", kind);
    DeviceGuard g(c->device);
    long long n = 0;
    double t = 0, f = 0, by = 0;
    for (const ProfRec &r : c->recs) {
        if (r.kind != kind) continue;
        CUDA_TRY(c, cudaEventSynchronize(r.b));
        float e = 0.f;
        CUDA_TRY(c, cudaEventElapsedTime(&e, r.a, r.b));
        n += r.kernels;
        t += e;
        f += r.flops;
        by += r.bytes;
    }
    if (launches) *launches = n;
    if (ms) *ms = t;
    if (flops) *flops = f;
    if (bytes) *bytes = by;
    if (c->prof_dropped) return set_err(c, FGI_ERR_ARG, "profile event pool exhausted (%lld launches not timed)",
                                        c->prof_dropped);
    return FGI_OK;
}

}  // extern "C"
